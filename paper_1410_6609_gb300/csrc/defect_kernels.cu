// defect_kernels.cu -- the outer step of the mixed-precision defect correction with its residual
// updated by recurrence (not in the paper; the paper's solver is FP64 throughout).
//
// An outer step adds s e (e: the single-precision inner cycles' correction, s: a power of two) to
// the FP64 iterate, so its residual changes by exactly -s A e: r~' = r~ + s (sum of e's six
// neighbours - (6 + d) e_c) in the scaled units of the level (r~ = g + sum - D x, Sec. 2.4 and
// Sec. 3). This file forms that change exactly enough to carry the residual from step to step
// without reading the iterate's stencil:
//  - A e of seven floats with small integer weights is summed by three cascades of error-free
//    additions (Knuth's TwoSum; the diagonal product's rounding error recovered by one FMA): the
//    terms, their rounding errors, and those errors' errors, so that only the last, third-order
//    sum rounds (Ogita, Rump and Oishi, "Accurate sum and dot product", 2005, the K = 3 case of
//    SumK). Its error is below 2^-60 of the sum of the terms' magnitudes.
//  - The residual is held as a pair of floats hi + lo in units of the current scale s: hi is the
//    single-precision right-hand side the next inner cycles solve for, lo (|lo| <= ulp(hi)/2) the
//    rest, so the pair carries about 48 bits. New pair = old pair - A e in error-free steps, one
//    rounding of the small remainders (below 2^-45 of the old and new residuals), then a
//    power-of-two rescaling to the next step's scale (exact).
//  - The iterate update phi' = phi + s e is the single rounded FP64 add of the plain update.
// Single precision is the right tool here: the error-free transformations run on the FP32 pipe,
// the whole step reads e, phi and the pair once and writes phi and the pair once (36 B per cell,
// against 40 B for the plain update followed by the FP64 residual walk, which is bound by its
// integer work), and only the iterate update uses the FP64 pipe. The solver still evaluates the
// residual directly (the fixed-point walk) before it accepts convergence. The batched launch runs
// the same per-item body over many systems, each exactly as its single-system launch would.
#include "level_ops.cuh"

namespace ccmg {
namespace {

using namespace ops;

// a + b = s + t exactly (round to nearest; no overflow).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& t) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  t = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// The three leading components of xm + xp + ym + yp + zm + zp + nd c (nd = -(6 + d)): the
// exact value minus the rounding of the third component, which is below 2^-60 of the terms'
// magnitudes.
struct F3 {
  float a, b, c;
};
__device__ __forceinline__ F3 stencil_sum(float xm, float xp, float ym, float yp, float zm, float zp, float nd,
                                          float c) {
  const float p = __fmul_rn(nd, c);
  const float q = __fmaf_rn(nd, c, -p);  // nd c = p + q exactly
  float s, e1, e2, e3, e4, e5, e6;
  two_sum(xm, xp, s, e1);
  two_sum(s, ym, s, e2);
  two_sum(s, yp, s, e3);
  two_sum(s, zm, s, e4);
  two_sum(s, zp, s, e5);
  two_sum(s, p, s, e6);
  float t, f1, f2, f3, f4, f5, f6;
  two_sum(e1, e2, t, f1);
  two_sum(t, e3, t, f2);
  two_sum(t, e4, t, f3);
  two_sum(t, e5, t, f4);
  two_sum(t, e6, t, f5);
  two_sum(t, q, t, f6);
  const float u = __fadd_rn(__fadd_rn(__fadd_rn(__fadd_rn(__fadd_rn(f1, f2), f3), f4), f5), f6);
  return {s, t, u};
}

// (hi, lo) = (qh + ql) + (T.a + T.b + T.c) as a normalised float pair (hi = the sum rounded to
// float, |lo| <= ulp(hi)/2): the leading parts cancel without error, the rest is rounded once.
__device__ __forceinline__ void add_pair(float qh, float ql, const F3& T, float& hi, float& lo) {
  float u, eu, v, ev, h1, e1;
  two_sum(qh, T.a, u, eu);
  two_sum(ql, T.b, v, ev);
  two_sum(u, v, h1, e1);
  const float rest = __fadd_rn(__fadd_rn(__fadd_rn(eu, ev), e1), T.c);
  two_sum(h1, rest, hi, lo);
}

// split_scaled for the rare operands (subnormal, infinite or NaN x, or x 2^q outside the range
// where hi and lo are normal floats), out of line so that its FP64 operations are never issued
// for the common ones.
static __device__ __noinline__ float2 split_scaled_general(double x, int q) {
  const float hi = f32_of_scaled(x, q);
  const double xs = ldexp_rne(x, q);
  return make_float2(hi, (isfinite(hi) && hi != 0.0f) ? __double2float_rn(__dsub_rn(xs, (double)hi)) : 0.0f);
}

// x 2^q as a float pair: hi = float(x 2^q) rounded to nearest even, lo = the remainder rounded to
// nearest (x's 53-bit significand split into its top 24 bits and the 29 below). Zeros and the
// common case (normal x, hi and lo both normal floats) in integer operations.
__device__ __forceinline__ void split_scaled(double x, int q, float& hi, float& lo) {
  const unsigned xh = (unsigned)__double2hiint(x), xl = (unsigned)__double2loint(x);
  const int E = (int)((xh >> 20) & 0x7ffu);
  const int eL = E - 1023 + q;  // x 2^q lies in [2^eL, 2^(eL+1))
  if (E != 0 && E != 0x7ff && eL >= -74 && eL <= 126) {
    const unsigned m23 = ((xh & 0xfffffu) << 3) | (xl >> 29);
    const unsigned rest = xl & 0x1fffffffu;
    const unsigned up = (rest > 0x10000000u || (rest == 0x10000000u && (m23 & 1u))) ? 1u : 0u;
    hi = __uint_as_float((xh & 0x80000000u) | ((((unsigned)(eL + 127) << 23) | m23) + up));
    // remainder (rest - up 2^29) 2^(eL - 52), |rest - up 2^29| <= 2^28, with x's sign
    const float r = __fmul_rn(__int2float_rn((int)rest - (int)(up << 29)), __uint_as_float((unsigned)(eL + 75) << 23));
    lo = (xh & 0x80000000u) ? -r : r;
    return;
  }
  if (((xh & 0x7fffffffu) | xl) == 0u) {  // +-0
    hi = __uint_as_float(xh & 0x80000000u);
    lo = 0.0f;
    return;
  }
  const float2 hl = split_scaled_general(x, q);
  hi = hl.x;
  lo = hl.y;
}

// Division of n < 2^31 by an invariant d >= 1 as a multiply-high, an add and a shift (Granlund and
// Montgomery, "Division by invariant integers using multiplication", 1994): with l = ceil(log2 d)
// and m = floor(2^32 (2^l - d) / d) + 1, n / d = (mulhi(m, n) + n) >> l; the sum stays below 2^32.
struct FastDiv {
  unsigned m;
  int l;
};
__host__ __device__ inline FastDiv make_fastdiv(unsigned d) {
  int l = 0;
  while ((1ull << l) < d) ++l;
  return {(unsigned)(((1ull << 32) * ((1ull << l) - d)) / d + 1), l};
}
__device__ __forceinline__ unsigned fdiv(unsigned n, const FastDiv& f) { return (__umulhi(f.m, n) + n) >> f.l; }


// One outer step over the finest level (packed, rows of whole 4-float vectors), four packed
// columns of one colour's row per item (the other colour's segment is read for the x-neighbours;
// both colours of a row in one item held twice the registers, two CTAs per SM instead of three,
// and took 1.04 against 0.93 ms at 512^3). ZERO: the iterate is zero and unwritten (the
// first step of a solve from zero): phi' = s e, and the residual pair is formed from g.
// Otherwise phi' = phi + s e and the pair is read from (qh, ql). Writes phi', the new pair in
// units of the next scale, and adds the squares of the new hi values to the thread's compensated
// float sum (ss, sc2). FAST: the scale is a power of two with s e exact and the rescaling factor a
// normal float (always, for the solver's scales); the other case takes ldexpf and the FMA. The
// choice is uniform over the launch and made outside the loop, so that the FP64 operations of the
// rare case are never issued for the common one (if-converted, they kept the FP64 pipe 70-84 %
// busy).
template <bool ZERO, bool PER, bool FAST>
__device__ __forceinline__ void rec_items(double* __restrict__ x, const float* __restrict__ e,
                                          float* __restrict__ qh, float* __restrict__ ql,
                                          const double* __restrict__ g, const Geom& G, const FastDiv& by_nvec,
                                          const FastDiv& by_ny, double sc, int p, int dk, float fac, unsigned blk,
                                          unsigned nblk, float& ss, float& sc2) {
  const int per = PER ? G.per : 0;
  const bool px = (per & 1) != 0;
  const unsigned nvec = (unsigned)G.hx >> 2;
  const unsigned items2 = 2u * nvec * (unsigned)G.ny * (unsigned)G.nz;  // < 2^31 (checked at launch)
  for (unsigned it = blk * blockDim.x + threadIdx.x; it < items2; it += nblk * blockDim.x) {
    const unsigned rowc = fdiv(it, by_nvec);
    const int iv = (int)(it - rowc * nvec);
    const int c = (int)(rowc & 1u);
    const unsigned rowi = rowc >> 1;
    const int k = (int)fdiv(rowi, by_ny), j = (int)rowi - k * G.ny;
    const long long row = (long long)rowi * G.hx;
    const int m0 = iv * 4;
    int dyz = 0;
    if (j == 0) dyz += G.sh[2];
    if (j == G.ny - 1) dyz += G.sh[3];
    if (k == 0) dyz += G.sh[4];
    if (k == G.nz - 1) dyz += G.sh[5];
    float own[4], oth[4];
    load_vec(e + (long long)c * G.csz + row + m0, own);
    const float* yr = e + (long long)(1 - c) * G.csz + row;  // the other colour's row
    load_vec(yr + m0, oth);
    float sq = 0.0f;
    {
      const int s = (c + j + k) & 1;
      float edge;
      if (s == 0) edge = m0 > 0 ? __ldg(yr + m0 - 1) : (px ? __ldg(yr + G.hx - 1) : 0.0f);
      else edge = m0 + 4 < G.hx ? __ldg(yr + m0 + 4) : (px ? __ldg(yr) : 0.0f);
      float ym[4], yp[4], zm[4], zp[4];
      load_nb_vec<0, PER>(yr, G, m0, j, k, ym);
      load_nb_vec<1, PER>(yr, G, m0, j, k, yp);
      load_nb_vec<2, PER>(yr, G, m0, j, k, zm);
      load_nb_vec<3, PER>(yr, G, m0, j, k, zp);
      const long long o = (long long)c * G.csz + row + m0;
      float hv[4], lv[4];
      double xv[4];
      if constexpr (ZERO) {
        double g2[2];
        load_vec(g + o, g2);
        split_scaled(g2[0], -p, hv[0], lv[0]);
        split_scaled(g2[1], -p, hv[1], lv[1]);
        load_vec(g + o + 2, g2);
        split_scaled(g2[0], -p, hv[2], lv[2]);
        split_scaled(g2[1], -p, hv[3], lv[3]);
      } else {
        load_vec(qh + o, hv);
        load_vec(ql + o, lv);
        double x2[2];
        load_vec(x + o, x2);
        xv[0] = x2[0];
        xv[1] = x2[1];
        load_vec(x + o + 2, x2);
        xv[2] = x2[0];
        xv[3] = x2[1];
      }
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const float xm = s == 0 ? (v == 0 ? edge : oth[(v + 3) & 3]) : oth[v];
        const float xp = s == 0 ? oth[v] : (v == 3 ? edge : oth[(v + 1) & 3]);
        int d = dyz;
        if (m0 + v == 0 && s == 0) d += G.sh[0];
        if (m0 + v == G.hx - 1 && s == 1) d += G.sh[1];
        const F3 T = stencil_sum(xm, xp, ym[v], yp[v], zm[v], zp[v], neg_diag<float>(d), own[v]);
        float hi, lo;
        add_pair(hv[v], lv[v], T, hi, lo);
        hv[v] = FAST ? __fmul_rn(hi, fac) : ldexpf(hi, dk);
        lv[v] = FAST ? __fmul_rn(lo, fac) : ldexpf(lo, dk);
        sq = __fmaf_rn(hv[v], hv[v], sq);
        if constexpr (ZERO) {
          if constexpr (FAST) {
            const double w = f64_of_scaled(own[v], p);
            xv[v] = (__double_as_longlong(w) == (long long)0x8000000000000000ULL) ? 0.0 : w;
          } else {
            xv[v] = fma(sc, (double)own[v], 0.0);
          }
        } else {
          xv[v] = FAST ? xv[v] + f64_of_scaled(own[v], p) : fma(sc, (double)own[v], xv[v]);
        }
      }
      store_vec(qh + o, hv);
      store_vec(ql + o, lv);
      double x2[2] = {xv[0], xv[1]};
      store_vec(x + o, x2);
      x2[0] = xv[2];
      x2[1] = xv[3];
      store_vec(x + o + 2, x2);
    }
    float t;
    two_sum(ss, sq, ss, t);
    sc2 = __fadd_rn(sc2, t);
  }
}

template <bool ZERO, bool PER>
__global__ void __launch_bounds__(256) k_defect_rec(double* __restrict__ x, const float* __restrict__ e,
                                                    float* __restrict__ qh, float* __restrict__ ql,
                                                    const double* __restrict__ g, Geom G, FastDiv by_nvec,
                                                    FastDiv by_ny, const double* __restrict__ scal, int slot,
                                                    int slot_next, double* __restrict__ partials) {
  __shared__ double red[33];
  const double sc = scal[slot];
  const int p = pow2_exponent(sc), pn = pow2_exponent(scal[slot_next]);
  const int dk = p - pn;  // new pair = (pair + A e) 2^(p - pn)
  const bool f_ok = dk >= -126 && dk <= 127;
  const float fac = f_ok ? __uint_as_float((unsigned)(dk + 127) << 23) : 1.0f;
  const bool p_ok = p != kBadPow2 && p >= -kScaleExpLimit && p <= kScaleExpLimit;
  float ss = 0.0f, sc2 = 0.0f;
  if (p_ok && f_ok)
    rec_items<ZERO, PER, true>(x, e, qh, ql, g, G, by_nvec, by_ny, sc, p, dk, fac, blockIdx.x, gridDim.x, ss, sc2);
  else
    rec_items<ZERO, PER, false>(x, e, qh, ql, g, G, by_nvec, by_ny, sc, p, dk, fac, blockIdx.x, gridDim.x, ss, sc2);
  const double acc = block_sum((double)ss + (double)sc2, red);
  if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

// The step's scalars: ||r~'||^2 = (fixed-order sum of the partials) s'^2 into scal[slot_rsum],
// ||r~'|| / ||g|| into scal[slot_rel], and the next scale (scal[slot_next], its inverse) becomes
// the current one (scal[slot_scale], scal[slot_scale + 1]).
__global__ void __launch_bounds__(256) k_defect_finalize(const double* __restrict__ partials, int n, double* scal,
                                                         int slot_rsum, int slot_rel, int slot_gsum, int slot_scale,
                                                         int slot_next) {
  __shared__ double red[33];
  const double acc = sum_partials(partials, n, red);
  if (threadIdx.x == 0) {
    const double sn = scal[slot_next];
    const double rs = (acc * sn) * sn;
    scal[slot_rsum] = rs;
    const double gs = scal[slot_gsum];
    scal[slot_rel] = gs > 0.0 ? sqrt(rs) / sqrt(gs) : sqrt(rs);
    scal[slot_scale] = sn;
    scal[slot_scale + 1] = scal[slot_next + 1];
  }
}

// Natural-order double field -> the packed residual pair in units of 2^-q (for verification).
__global__ void __launch_bounds__(256) k_pack_pair(float* __restrict__ qh, float* __restrict__ ql, Geom G,
                                                   const double* __restrict__ src, int q) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= G.nx || j >= G.ny) return;
  const long long pidx = (long long)i + (long long)G.nx * ((long long)j + (long long)G.ny * k);
  const long long o = (long long)((i + j + k) & 1) * G.csz + ((long long)k * G.ny + j) * G.hx + (i >> 1);
  float hi, lo;
  split_scaled(src[pidx], q, hi, lo);
  qh[o] = hi;
  ql[o] = lo;
}

// The same step over the finest levels of many systems (batched solves). Entry e of the table is
// one system's level 0 (x: phi, g: g, xc: the correction e, gc: the pair's hi, aux: its lo), split
// into exactly the gx CTAs that the single-system launch takes for it; virtual block lb runs that
// CTA's grid-stride items and writes its partial at the same position, so every system's values
// and norm are bit-identical to those of its single-system step. Systems that are not active, or
// do not step by recurrence this cycle (rec[sys] == 0), are skipped, a whole entry at a time. ZERO:
// the launch for the systems whose iterate is zero and unwritten (zero[sys], the first-step form);
// the other launch takes the rest (one kernel for both held 117 registers, two CTAs per SM, and
// took 2.3 ms for the 64-system batch). A persistent grid walks the virtual blocks in order.
template <bool PER, bool ZERO>
__global__ void __launch_bounds__(256, 3) kb_defect_rec(const BEntry* __restrict__ E, const int* __restrict__ start,
                                                     int count, int total, const int* __restrict__ active,
                                                     const int* __restrict__ rec, const int* __restrict__ zero,
                                                     const double* __restrict__ scal, double* __restrict__ partials) {
  __shared__ double red[33];
  if ((int)blockIdx.x >= total) return;
  int lo = 0, hi = count - 1;  // the entry of the first virtual block (offsets ascend)
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(start + mid) <= (int)blockIdx.x) lo = mid;
    else hi = mid - 1;
  }
  int e = lo;
  for (int b = blockIdx.x; b < total; b += gridDim.x) {
    while (__ldg(start + e + 1) <= b) ++e;
    const BEntry& en = E[e];
    const int sys = en.sys;
    if (!active[sys] || !rec[sys] || (zero[sys] != 0) != ZERO) {  // to this CTA's first block of the next entry
      const int next = __ldg(start + e + 1);
      if (next > b) b += ((next - b - 1) / (int)gridDim.x) * (int)gridDim.x;
      continue;
    }
    const unsigned lb = (unsigned)(b - __ldg(start + e)), nb = (unsigned)(__ldg(start + e + 1) - __ldg(start + e));
    const Geom G = en.G;
    const double* sp = scal + kScalStride * sys;
    const double sc = sp[kSlotScale];
    const int p = pow2_exponent(sc), pn = pow2_exponent(sp[kSlotNext]);
    const int dk = p - pn;
    const bool f_ok = dk >= -126 && dk <= 127;
    const float fac = f_ok ? __uint_as_float((unsigned)(dk + 127) << 23) : 1.0f;
    const bool fast = f_ok && p != kBadPow2 && p >= -kScaleExpLimit && p <= kScaleExpLimit;
    const FastDiv by_nvec = make_fastdiv((unsigned)(G.hx / 4)), by_ny = make_fastdiv((unsigned)G.ny);
    double* x = (double*)en.x;
    const float* ev = (const float*)en.xc;
    float* qh = (float*)en.gc;
    float* ql = (float*)en.aux;
    const double* g = (const double*)en.g;
    float ss = 0.0f, sc2 = 0.0f;
    if (fast) rec_items<ZERO, PER, true>(x, ev, qh, ql, g, G, by_nvec, by_ny, sc, p, dk, fac, lb, nb, ss, sc2);
    else rec_items<ZERO, PER, false>(x, ev, qh, ql, g, G, by_nvec, by_ny, sc, p, dk, fac, lb, nb, ss, sc2);
    const double acc = block_sum((double)ss + (double)sc2, red);
    if (threadIdx.x == 0) partials[b] = acc;
  }
}

// Per stepping system: the next scale from the last residual norm, as k_set_scale computes it.
__global__ void kb_defect_set_next(const BEntry* __restrict__ E, int count, const int* __restrict__ active,
                                   const int* __restrict__ rec, double* __restrict__ scal) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= count) return;
  const int sys = E[e].sys;
  if (!active[sys] || !rec[sys]) return;
  const Geom G = E[e].G;
  double* sp = scal + kScalStride * sys;
  const double s = pow2_floor(sqrt(sp[kSlotRsum] / (double)(2 * G.csz)));
  sp[kSlotNext] = s;
  sp[kSlotNext + 1] = 1.0 / s;
}

// Per stepping system (one CTA each): k_defect_finalize over its partials.
__global__ void __launch_bounds__(256) kb_defect_finalize(const BEntry* __restrict__ E, const int* __restrict__ start,
                                                          const int* __restrict__ active, const int* __restrict__ rec,
                                                          const double* __restrict__ partials,
                                                          double* __restrict__ scal) {
  __shared__ double red[33];
  const int e = blockIdx.x;
  const int sys = E[e].sys;
  if (!active[sys] || !rec[sys]) return;
  const double acc = sum_partials(partials + start[e], start[e + 1] - start[e], red);
  if (threadIdx.x == 0) {
    double* sp = scal + kScalStride * sys;
    const double sn = sp[kSlotNext];
    const double rs = (acc * sn) * sn;
    sp[kSlotRsum] = rs;
    const double gs = sp[kSlotGsum];
    sp[kSlotRel] = gs > 0.0 ? sqrt(rs) / sqrt(gs) : sqrt(rs);
    sp[kSlotScale] = sn;
    sp[kSlotInvScale] = sp[kSlotNext + 1];
  }
}

// CTAs of the step kernel: the SMs times the CTAs of its largest variant (72-76 registers) that
// fit on one; the same grid for every variant (four CTAs per SM for the 64-register ones took
// 0.88 against 0.87 ms at 512^3)
int g_defect_grid = 0;

cudaError_t defect_grid(int* out) {
  if (g_defect_grid == 0) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err == cudaSuccess) err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (err == cudaSuccess) err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_defect_rec<true, true>, 256, 0);
    if (err != cudaSuccess) return err;
    g_defect_grid = sms * (per_sm > 0 ? per_sm : 1);
    if (g_defect_grid > kMaxPartials) g_defect_grid = kMaxPartials;
  }
  *out = g_defect_grid;
  return cudaSuccess;
}

template <bool ZERO, bool PER>
cudaError_t launch_rec(double* x, const float* e, float* qh, float* ql, const double* g, const Geom& G,
                       const double* scal, int slot, int slot_next, double* partials, long long items, int* nparts,
                       cudaStream_t s) {
  int grid = 0;
  cudaError_t err = defect_grid(&grid);
  if (err != cudaSuccess) return err;
  long long blocks = (items + 255) / 256;
  if (blocks > grid) blocks = grid;
  if (blocks < 1) blocks = 1;
  const FastDiv by_nvec = make_fastdiv((unsigned)(G.hx / 4)), by_ny = make_fastdiv((unsigned)G.ny);
  k_defect_rec<ZERO, PER><<<(int)blocks, 256, 0, s>>>(x, e, qh, ql, g, G, by_nvec, by_ny, scal, slot, slot_next,
                                                      partials);
  *nparts = (int)blocks;
  return cudaGetLastError();
}

}  // namespace

bool defect_rec_applies(const Geom& G) { return G.packed && G.hx >= 4 && (G.hx & 3) == 0; }

cudaError_t launch_defect_rec(double* x, const float* e, float* qh, float* ql, const double* g, const Geom& G,
                              double* scal, int slot, int slot_next, bool zero, double* partials, int* nparts,
                              cudaStream_t s) {
  if (!defect_rec_applies(G)) return cudaErrorInvalidValue;
  const long long items = 2LL * (G.hx / 4) * G.ny * G.nz;
  if (items >= (1LL << 31) - 256LL * kMaxPartials) return cudaErrorInvalidValue;  // 32-bit item indices
  const bool per = G.per != 0;
  if (zero)
    return per ? launch_rec<true, true>(x, e, qh, ql, g, G, scal, slot, slot_next, partials, items, nparts, s)
               : launch_rec<true, false>(x, e, qh, ql, g, G, scal, slot, slot_next, partials, items, nparts, s);
  return per ? launch_rec<false, true>(x, e, qh, ql, g, G, scal, slot, slot_next, partials, items, nparts, s)
             : launch_rec<false, false>(x, e, qh, ql, g, G, scal, slot, slot_next, partials, items, nparts, s);
}

// One batched launch: a persistent grid of the SMs times the CTAs of this variant that fit on one,
// at most one per virtual block.
template <bool PER, bool ZERO>
cudaError_t launch_kb_rec(const BLaunch& L, const int* active, const int* rec, const int* zero, double* scal,
                          double* partials, cudaStream_t s) {
  static int ctas_max = 0;
  if (ctas_max == 0) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err == cudaSuccess) err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (err == cudaSuccess) err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kb_defect_rec<PER, ZERO>, 256, 0);
    if (err != cudaSuccess) return err;
    ctas_max = sms * (per_sm > 0 ? per_sm : 1);
  }
  const int ctas = L.blocks < ctas_max ? L.blocks : ctas_max;
  kb_defect_rec<PER, ZERO><<<ctas, 256, 0, s>>>(L.entries, L.start, L.count, L.blocks, active, rec, zero, scal, partials);
  return cudaGetLastError();
}

int defect_rec_blocks(const Geom& G) {
  int grid = 0;
  if (defect_grid(&grid) != cudaSuccess || grid < 1) return 0;
  const long long items = 2LL * (G.hx / 4) * G.ny * G.nz;
  long long blocks = (items + 255) / 256;
  if (blocks > grid) blocks = grid;
  return (int)(blocks < 1 ? 1 : blocks);
}

cudaError_t launch_b_defect_step(const BLaunch& L, const int* active, const int* rec, const int* zero, double* scal,
                                 double* partials, cudaStream_t s) {
  if (L.count == 0) return cudaSuccess;
  kb_defect_set_next<<<(L.count + 63) / 64, 64, 0, s>>>(L.entries, L.count, active, rec, scal);
  cudaError_t err = cudaSuccess;
  if (L.per) {
    if ((err = launch_kb_rec<true, true>(L, active, rec, zero, scal, partials, s)) != cudaSuccess) return err;
    if ((err = launch_kb_rec<true, false>(L, active, rec, zero, scal, partials, s)) != cudaSuccess) return err;
  } else {
    if ((err = launch_kb_rec<false, true>(L, active, rec, zero, scal, partials, s)) != cudaSuccess) return err;
    if ((err = launch_kb_rec<false, false>(L, active, rec, zero, scal, partials, s)) != cudaSuccess) return err;
  }
  kb_defect_finalize<<<L.count, 256, 0, s>>>(L.entries, L.start, active, rec, partials, scal);
  return cudaGetLastError();
}

cudaError_t launch_defect_finalize(const double* partials, int nparts, double* scal, int slot_rsum, int slot_rel,
                                   int slot_gsum, int slot_scale, int slot_next, cudaStream_t s) {
  k_defect_finalize<<<1, 256, 0, s>>>(partials, nparts, scal, slot_rsum, slot_rel, slot_gsum, slot_scale, slot_next);
  return cudaGetLastError();
}

cudaError_t launch_pack_pair(float* qh, float* ql, const Geom& G, const double* src, int q, cudaStream_t s) {
  const int bx = G.nx >= 128 ? 128 : (G.nx >= 64 ? 64 : 32);
  const int by = 256 / bx;
  dim3 b(bx, by, 1), gr((G.nx + bx - 1) / bx, (G.ny + by - 1) / by, G.nz);
  k_pack_pair<<<gr, b, 0, s>>>(qh, ql, G, src, q);
  return cudaGetLastError();
}

}  // namespace ccmg
