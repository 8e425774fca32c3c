// level_kernels.cu -- per-level multigrid kernels for sm_103a (Sec. 3 and Sec. 5.3 of the paper).
//
// All kernels work on the checkerboard-separated level layout described in ccmg_internal.cuh
// (two colour arrays per field, unit-stride rows) with the scaled right-hand side g = f / c_l.
// Templated on the storage/arithmetic type T (double for the FP64 solver, float for the inner
// cycle of the mixed-precision defect correction). The coarsest-grid CG always computes in
// double. The per-thread arithmetic is in level_ops.cuh; these are single-system launches.
#include "level_ops.cuh"

namespace ccmg {
namespace {

using namespace ops;

template <typename T, bool ZERO>
__global__ void __launch_bounds__(256) k_smooth(T* __restrict__ x, const T* __restrict__ g, Geom G, InvDiag<T> inv,
                                                int colour) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (m >= G.hx || j >= G.ny) return;
  smooth_cell<T, ZERO>(x, g, G, inv, colour, m, j, k);
}

template <typename T, int V, bool ZERO, bool PER>
__global__ void __launch_bounds__(256) k_smooth_vec(T* __restrict__ x, const T* __restrict__ g, Geom G,
                                                    InvDiag<T> inv, int colour) {
  const int mv = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (mv >= G.hx / V || j >= G.ny) return;
  smooth_vec<T, V, ZERO, PER>(x, g, G, inv, colour, mv, j, k);
}

// PER: compiled with periodic-axis support (launched for levels that have a periodic axis; the
// other variant keeps the register footprint of walls alone).
template <typename T, int V, bool PER>
__global__ void __launch_bounds__(256) k_smooth_vec_prolong(T* __restrict__ x, const T* __restrict__ g, Geom G,
                                                            InvDiag<T> inv, const T* __restrict__ ec, Geom Gc,
                                                            T omega) {
  const int mv = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (mv >= G.hx / V || j >= G.ny) return;
  smooth_vec_prolong<T, V, PER>(x, g, G, inv, ec, Gc, omega, mv, j, k);
}

template <typename T, bool RED_ONLY>
__global__ void __launch_bounds__(256) k_resid_restrict(const T* __restrict__ x, const T* __restrict__ g, Geom G,
                                                        T* __restrict__ gc, Geom Gc) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  const int J = blockIdx.y * blockDim.y + threadIdx.y;
  const int K = blockIdx.z;
  if (I >= Gc.nx || J >= Gc.ny) return;
  resid_restrict_cell<T, RED_ONLY>(x, g, G, gc, Gc, I, J, K);
}

template <typename T, int V, bool RED_ONLY, bool PER>
__global__ void __launch_bounds__(256) k_resid_restrict_vec(const T* __restrict__ x, const T* __restrict__ g, Geom G,
                                                            T* __restrict__ gc, Geom Gc) {
  const int iv = blockIdx.x * blockDim.x + threadIdx.x;
  const int J = blockIdx.y * blockDim.y + threadIdx.y;
  const int K = blockIdx.z;
  if (iv >= Gc.nx / V || J >= Gc.ny) return;
  resid_restrict_vec<T, V, RED_ONLY, PER>(x, g, G, gc, Gc, iv, J, K);
}

// FP64 residual and restriction by the residual walk (packed levels): the tiles of block
// blockIdx.x of gridDim.x, every fine residual summed in fixed point per ring row, the eight
// children of each coarse cell added and scaled by 1/4 (resid_tiles_accum, MODE 3).
template <bool PER>
__global__ void __launch_bounds__(256, 3) k_resid_restrict_walk(const double* __restrict__ x,
                                                             const double* __restrict__ g, Geom G,
                                                             double* __restrict__ gc, Geom Gc) {
  resid_tiles_accum<3, PER>(x, g, G, blockIdx.x, gridDim.x, 0.0, nullptr, nullptr, 0.0, kBadPow2, gc, &Gc);
}

template <typename T>
__global__ void __launch_bounds__(256) k_prolong(T* __restrict__ x, Geom G, const T* __restrict__ ec, Geom Gc,
                                                 T omega, int red_only) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  const int J = blockIdx.y * blockDim.y + threadIdx.y;
  const int K = blockIdx.z;
  if (I >= Gc.nx || J >= Gc.ny) return;
  prolong_cell<T>(x, G, ec, Gc, omega, red_only, I, J, K);
}

template <typename T>
__global__ void __launch_bounds__(1024) k_coarse_cg(T* __restrict__ xo, const T* __restrict__ bi, Geom G, double rtol,
                                                    int maxit, int* iters) {
  extern __shared__ double sm[];
  __shared__ double red[33];
  const int it = coarse_cg_block<T>(xo, bi, G, rtol, maxit, sm, red);
  if (threadIdx.x == 0 && iters) *iters = it;
}

// ---------------------------------------------------------------------------------------------
// Scaled residual with per-block partial sums of r~^2 (the termination test of Algorithm 1); the
// row walk and the reduction are in level_ops.cuh (resid_norm_accum), so a batched launch over
// many systems reproduces each system's partial sums exactly.
template <typename T, int MODE, bool PER>
__global__ void __launch_bounds__(256, 3) k_resid_norm(const T* __restrict__ x, const T* __restrict__ g, Geom G,
                                                    double* __restrict__ partials, double c0,
                                                    double* __restrict__ outn, float* __restrict__ outp,
                                                    const double* __restrict__ inv_scale) {
  __shared__ double red[33];
  const double isc = (MODE == 2) ? inv_scale[0] : 0.0;
  double acc = resid_norm_accum<T, MODE, PER>(x, g, G, blockIdx.x, gridDim.x, c0, outn, outp, isc);
  acc = block_sum(acc, red);
  if (threadIdx.x == 0 && threadIdx.y == 0) partials[blockIdx.x] = acc;
}

template <typename T>
__global__ void __launch_bounds__(256) k_sumsq(const T* __restrict__ a, long long n, double* __restrict__ partials) {
  __shared__ double red[33];
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double v = (double)a[i];
    acc = fma(v, v, acc);
  }
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

__global__ void __launch_bounds__(256) k_finalize(const double* __restrict__ partials, int n, double* scal, int slot,
                                                  int slot_rel, int slot_ref) {
  __shared__ double red[33];
  const double acc = sum_partials(partials, n, red);
  if (threadIdx.x == 0) {
    scal[slot] = acc;
    if (slot_rel >= 0) {
      const double ref = scal[slot_ref];
      scal[slot_rel] = ref > 0.0 ? sqrt(acc) / sqrt(ref) : sqrt(acc);
    }
  }
}

// Scale of the next defect-correction step: the largest power of two not above the RMS of the
// residual (exact scaling in both directions).
__global__ void k_set_scale(double* scal, int src, int dst, double n) {
  const double s = pow2_floor(sqrt(scal[src] / n));
  scal[dst] = s;
  scal[dst + 1] = 1.0 / s;
}

// ---------------------------------------------------------------------------------------------
// Right-hand side (Sec. 2.4 and Sec. 5.3: the wall conditions enter the right-hand side once, on
// the finest grid): f = rho/eps + wall terms, stored scaled, g = f * h^2. A face with one value
// has its term precomputed (t[q]); a face with values per cell computes 2 g / h^2 (Dirichlet) or
// g / h (Neumann) per cell with the same operations.
__device__ __forceinline__ double wall_term(const WallTerms& wt, int q, int i, int j, int k, const Geom& G) {
  if (!wt.field[q]) return wt.t[q];
  const double g = __ldg(wt.field[q] + face_index(q, i, j, k, G.nx, G.ny));
  return wt.type[q] == 0 ? 2.0 * g / (wt.h * wt.h) : g / wt.h;
}
// FIELD: some face carries values per cell (the kernels are compiled both ways, so the common
// uniform case keeps its small register footprint).
// A periodic face has no wall term (its neighbour is the cell at the opposite side).
template <bool FIELD>
__device__ __forceinline__ double add_wall_terms(double v, int i, int j, int k, const Geom& G, const WallTerms& wt) {
  const bool px = (G.per & 1) != 0, py = (G.per & 2) != 0, pz = (G.per & 4) != 0;
  if (i == 0 && !px) v = v + (FIELD ? wall_term(wt, 0, i, j, k, G) : wt.t[0]);
  if (i == G.nx - 1 && !px) v = v + (FIELD ? wall_term(wt, 1, i, j, k, G) : wt.t[1]);
  if (j == 0 && !py) v = v + (FIELD ? wall_term(wt, 2, i, j, k, G) : wt.t[2]);
  if (j == G.ny - 1 && !py) v = v + (FIELD ? wall_term(wt, 3, i, j, k, G) : wt.t[3]);
  if (k == 0 && !pz) v = v + (FIELD ? wall_term(wt, 4, i, j, k, G) : wt.t[4]);
  if (k == G.nz - 1 && !pz) v = v + (FIELD ? wall_term(wt, 5, i, j, k, G) : wt.t[5]);
  return v;
}
// POW2: 1/eps = 2^qe and h^2 = 2^qh (lattice units), the products are exponent shifts.
template <typename T, bool POW2, bool FIELD>
__device__ __forceinline__ void set_rhs_cell(T* __restrict__ gout, const Geom& G, const double* __restrict__ rho,
                                             double inv_eps, double hsq, int qe, int qh, const WallTerms& wt, int raw,
                                             int i, int j, int k) {
  const long long p = (long long)i + (long long)G.nx * ((long long)j + (long long)G.ny * k);
  double v = rho[p];
  if (!raw) {
    v = POW2 ? ldexp_rne(v, qe) : v * inv_eps;
    // only warps holding wall cells add wall terms (a warp vote keeps the compiler from turning
    // the rare branches into FP64 adds of zero by every cell)
    const bool wall = i == 0 || i == G.nx - 1 || j == 0 || j == G.ny - 1 || k == 0 || k == G.nz - 1;
    if (__any_sync(__activemask(), wall)) v = add_wall_terms<FIELD>(v, i, j, k, G, wt);
  }
  long long o = p;
  if (G.packed) o = (long long)((i + j + k) & 1) * G.csz + ((long long)k * G.ny + j) * G.hx + (i >> 1);
  gout[o] = (T)(POW2 ? ldexp_rne(v, qh) : v * hsq);
}
template <typename T, bool POW2, bool FIELD>
__global__ void __launch_bounds__(256) k_set_rhs(T* __restrict__ gout, Geom G, const double* __restrict__ rho,
                                                 double inv_eps, double hsq, int qe, int qh, WallTerms wt, int raw) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= G.nx || j >= G.ny) return;
  set_rhs_cell<T, POW2, FIELD>(gout, G, rho, inv_eps, hsq, qe, qh, wt, raw, i, j, k);
}

// The same for a packed level, two cells per thread: cells 2m and 2m+1 of row (j, k) are one
// 16-byte load of rho and land at index m of the two colour arrays, so both the loads and the
// stores of a warp are contiguous.
template <typename T, bool POW2, bool FIELD>
__device__ __forceinline__ void set_rhs_pair(T* __restrict__ gout, const Geom& G, const double* __restrict__ rho,
                                             double inv_eps, double hsq, int qe, int qh, const WallTerms& wt, int raw,
                                             int m, int j, int k) {
  const int i0 = 2 * m;
  const long long p = (long long)i0 + (long long)G.nx * ((long long)j + (long long)G.ny * k);
  const double2 r = __ldg(reinterpret_cast<const double2*>(rho + p));
  double v0 = r.x, v1 = r.y;
  if (!raw) {
    v0 = POW2 ? ldexp_rne(v0, qe) : v0 * inv_eps;
    v1 = POW2 ? ldexp_rne(v1, qe) : v1 * inv_eps;
    const bool wall = i0 == 0 || i0 + 1 == G.nx - 1 || j == 0 || j == G.ny - 1 || k == 0 || k == G.nz - 1;
    if (__any_sync(__activemask(), wall)) {
      v0 = add_wall_terms<FIELD>(v0, i0, j, k, G, wt);
      v1 = add_wall_terms<FIELD>(v1, i0 + 1, j, k, G, wt);
    }
  }
  const int c0 = (i0 + j + k) & 1;
  const long long o = ((long long)k * G.ny + j) * G.hx + m;
  gout[(long long)c0 * G.csz + o] = (T)(POW2 ? ldexp_rne(v0, qh) : v0 * hsq);
  gout[(long long)(c0 ^ 1) * G.csz + o] = (T)(POW2 ? ldexp_rne(v1, qh) : v1 * hsq);
}
template <typename T, bool POW2, bool FIELD>
__global__ void __launch_bounds__(256) k_set_rhs_pair(T* __restrict__ gout, Geom G, const double* __restrict__ rho,
                                                      double inv_eps, double hsq, int qe, int qh, WallTerms wt,
                                                      int raw) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (m >= G.hx || j >= G.ny) return;
  set_rhs_pair<T, POW2, FIELD>(gout, G, rho, inv_eps, hsq, qe, qh, wt, raw, m, j, k);
}

// Batched right-hand sides (mg_batch_set_rhs_all): blocks of 256 items (cell pairs of a packed
// level with aligned rho, else cells) of every system in turn, each item the same per-cell
// operations as the single-system kernels above.
template <bool POW2, bool FIELD>
__device__ __forceinline__ void set_rhs_item(const RhsJob& J, long long q) {
  const Geom& G = J.G;
  if (J.pair) {
    const long long row = q / G.hx;
    const int m = (int)(q - row * G.hx), j = (int)(row % G.ny), k = (int)(row / G.ny);
    if (k < G.nz) set_rhs_pair<double, POW2, FIELD>(J.g, G, J.rho, J.inv_eps, J.hsq, J.qe, J.qh, J.wt, 0, m, j, k);
  } else {
    const long long row = q / G.nx;
    const int i = (int)(q - row * G.nx), j = (int)(row % G.ny), k = (int)(row / G.ny);
    if (k < G.nz) set_rhs_cell<double, POW2, FIELD>(J.g, G, J.rho, J.inv_eps, J.hsq, J.qe, J.qh, J.wt, 0, i, j, k);
  }
}
__global__ void __launch_bounds__(256) k_set_rhs_all(const RhsJob* __restrict__ jobs, int B, long long nblocks) {
  int s = 0;
  for (long long vb = blockIdx.x; vb < nblocks; vb += gridDim.x) {
    while (s + 1 < B && jobs[s + 1].b0 <= vb) ++s;
    const RhsJob& J = jobs[s];
    const long long q = (vb - J.b0) * 256 + threadIdx.x;
    if (J.pow2) {
      if (J.fld) set_rhs_item<true, true>(J, q);
      else set_rhs_item<true, false>(J, q);
    } else {
      if (J.fld) set_rhs_item<false, true>(J, q);
      else set_rhs_item<false, false>(J, q);
    }
  }
}
// Each system's sum of squares of g in the block layout of k_sumsq with its own grid of J.sbn
// blocks (the same partials, hence the same norm as a single context), then per system the fixed
// order sum of its partials (k_finalize) and the scale (k_set_scale).
__global__ void __launch_bounds__(256) k_sumsq_all(const RhsJob* __restrict__ jobs, int B, int nsblocks,
                                                   double* __restrict__ partials) {
  __shared__ double red[33];
  int s = 0;
  for (int vb = blockIdx.x; vb < nsblocks; vb += gridDim.x) {
    while (s + 1 < B && jobs[s + 1].sb0 <= vb) ++s;
    const RhsJob& J = jobs[s];
    const long long n = (long long)J.n, lb = vb - J.sb0;
    double acc = 0.0;
    for (long long i = lb * 256 + threadIdx.x; i < n; i += (long long)J.sbn * 256) {
      const double v = J.g[i];
      acc = fma(v, v, acc);
    }
    acc = block_sum(acc, red);
    if (threadIdx.x == 0) partials[vb] = acc;
  }
}
__global__ void __launch_bounds__(256) k_finalize_all(const RhsJob* __restrict__ jobs, const double* __restrict__ partials,
                                                      int slot_gsum, int slot_scale) {
  __shared__ double red[33];
  const RhsJob& J = jobs[blockIdx.x];
  const double acc = sum_partials(partials + J.sb0, J.sbn, red);
  if (threadIdx.x == 0) {
    J.scal[slot_gsum] = acc;
    const double sc = pow2_floor(sqrt(J.scal[slot_gsum] / J.n));
    J.scal[slot_scale] = sc;
    J.scal[slot_scale + 1] = 1.0 / sc;
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_pack(T* __restrict__ dst, Geom G, const double* __restrict__ src,
                                              double scale) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= G.nx || j >= G.ny) return;
  const long long p = (long long)i + (long long)G.nx * ((long long)j + (long long)G.ny * k);
  long long o = p;
  if (G.packed) o = (long long)((i + j + k) & 1) * G.csz + ((long long)k * G.ny + j) * G.hx + (i >> 1);
  dst[o] = src ? (T)(src[p] * scale) : T(0);
}

template <typename T>
__global__ void __launch_bounds__(256) k_unpack(double* __restrict__ dst, const T* __restrict__ src, Geom G,
                                                double scale) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= G.nx || j >= G.ny) return;
  const long long p = (long long)i + (long long)G.nx * ((long long)j + (long long)G.ny * k);
  long long o = p;
  if (G.packed) o = (long long)((i + j + k) & 1) * G.csz + ((long long)k * G.ny + j) * G.hx + (i >> 1);
  dst[p] = (double)src[o] * scale;
}

// Termination residual of a zero iterate: r = f exactly (g + 0 - (6+d) 0 = g), so ||r|| = ||f||
// and the relative residual is 1 (0 for f = 0). Writes the scalars; with outp also the scaled
// single-precision residual float(g * inv_scale), the values the residual kernel would produce.
__global__ void __launch_bounds__(256) k_resid_zero(const double* __restrict__ g, long long n, float* __restrict__ outp,
                                                    double* __restrict__ scal, int slot_rsum, int slot_rel,
                                                    int slot_gsum, int slot_inv_scale) {
  const double gsum = scal[slot_gsum];
  if (outp) {
    const double isc = scal[slot_inv_scale];
    const int p = pow2_exponent(isc);
    const long long i0 = blockIdx.x * (long long)blockDim.x + threadIdx.x, st = (long long)gridDim.x * blockDim.x;
    if (p != kBadPow2)
      for (long long i = i0; i < n; i += st) outp[i] = f32_of_scaled(g[i], p);
    else
      for (long long i = i0; i < n; i += st) outp[i] = (float)(g[i] * isc);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    scal[slot_rsum] = gsum;
    scal[slot_rel] = gsum > 0.0 ? sqrt(gsum) / sqrt(gsum) : 0.0;
  }
}

__global__ void __launch_bounds__(256) k_update_mixed(double* __restrict__ x, const float* __restrict__ e, long long n,
                                                      const double* __restrict__ scal, int slot) {
  const double sc = scal[slot];
  const int p = pow2_exponent(sc);
  const long long i0 = blockIdx.x * (long long)blockDim.x + threadIdx.x, st = (long long)gridDim.x * blockDim.x;
  // sc = 2^p within the scale bounds: s e is exact, so fma(sc, e, x) = x + s e
  if (p != kBadPow2 && p >= -kScaleExpLimit && p <= kScaleExpLimit)
    for (long long i = i0; i < n; i += st) x[i] = x[i] + f64_of_scaled(e[i], p);
  else
    for (long long i = i0; i < n; i += st) x[i] = fma(sc, (double)e[i], x[i]);
}

// The power-of-two products and conversions on arbitrary data (for verification): xf =
// float(x * isc) as the residual kernels write it, yo = fma(sc, double(e), y) as the update
// applies it, xs = x * sc as the lattice-unit products take it; isc = 1/sc.
__global__ void __launch_bounds__(256) k_scale_convert(const double* __restrict__ x, const float* __restrict__ e,
                                                       const double* __restrict__ y, long long n, double sc,
                                                       double isc, float* __restrict__ xf, double* __restrict__ yo,
                                                       double* __restrict__ xs) {
  const int p = pow2_exponent(sc), q = pow2_exponent(isc);
  const long long i0 = blockIdx.x * (long long)blockDim.x + threadIdx.x, st = (long long)gridDim.x * blockDim.x;
  if (q != kBadPow2)
    for (long long i = i0; i < n; i += st) xf[i] = f32_of_scaled(x[i], q);
  else
    for (long long i = i0; i < n; i += st) xf[i] = (float)(x[i] * isc);
  if (p != kBadPow2 && p >= -kScaleExpLimit && p <= kScaleExpLimit)
    for (long long i = i0; i < n; i += st) yo[i] = y[i] + f64_of_scaled(e[i], p);
  else
    for (long long i = i0; i < n; i += st) yo[i] = fma(sc, (double)e[i], y[i]);
  if (p != kBadPow2)
    for (long long i = i0; i < n; i += st) xs[i] = ldexp_rne(x[i], p);
  else
    for (long long i = i0; i < n; i += st) xs[i] = x[i] * sc;
}

// The update of a zero iterate: x = fma(sc, double(e), +0), i.e. s e with a zero product
// stored as +0; x itself is not read.
__global__ void __launch_bounds__(256) k_set_mixed(double* __restrict__ x, const float* __restrict__ e, long long n,
                                                   const double* __restrict__ scal, int slot) {
  const double sc = scal[slot];
  const int p = pow2_exponent(sc);
  const long long i0 = blockIdx.x * (long long)blockDim.x + threadIdx.x, st = (long long)gridDim.x * blockDim.x;
  if (p != kBadPow2 && p >= -kScaleExpLimit && p <= kScaleExpLimit)
    for (long long i = i0; i < n; i += st) {
      const double v = f64_of_scaled(e[i], p);
      x[i] = (__double_as_longlong(v) == (long long)0x8000000000000000ULL) ? 0.0 : v;
    }
  else
    for (long long i = i0; i < n; i += st) x[i] = fma(sc, (double)e[i], 0.0);
}

// Launch shape for a (w x h x depth) thread grid with 256-thread blocks.
void shape(int w, int h, int depth, dim3& b, dim3& g) {
  const int bx = w >= 128 ? 128 : (w >= 64 ? 64 : 32);
  const int by = 256 / bx;
  b = dim3(bx, by, 1);
  g = dim3((w + bx - 1) / bx, (h + by - 1) / by, depth);
}


}  // namespace

// ================================ launchers ================================================

template <typename T>
cudaError_t launch_smooth(T* x, const T* g, const Geom& G, const InvDiag<T>& inv, int colour, bool zero_start,
                          cudaStream_t s) {
  constexpr int V = 16 / sizeof(T);
  if (G.hx % V == 0) {
    const int nvec = G.hx / V;
    int bx = 1;
    while (bx < nvec && bx < 128) bx *= 2;
    const int by = 256 / bx;
    dim3 b(bx, by, 1), gr((nvec + bx - 1) / bx, (G.ny + by - 1) / by, G.nz);
    if (zero_start)  // no neighbour is read
      k_smooth_vec<T, V, true, false><<<gr, b, 0, s>>>(x, g, G, inv, colour);
    else if (G.per)
      k_smooth_vec<T, V, false, true><<<gr, b, 0, s>>>(x, g, G, inv, colour);
    else
      k_smooth_vec<T, V, false, false><<<gr, b, 0, s>>>(x, g, G, inv, colour);
    return cudaGetLastError();
  }
  dim3 b, gr;
  shape(G.hx, G.ny, G.nz, b, gr);
  if (zero_start)
    k_smooth<T, true><<<gr, b, 0, s>>>(x, g, G, inv, colour);
  else
    k_smooth<T, false><<<gr, b, 0, s>>>(x, g, G, inv, colour);
  return cudaGetLastError();
}

cudaError_t launch_smooth_prolong(float* x, const float* g, const Geom& G, const InvDiag<float>& inv, const float* ec,
                                  const Geom& Gc, float omega, cudaStream_t s) {
  constexpr int V = 4;
  if (G.hx % V != 0) return cudaErrorInvalidValue;
  const int nvec = G.hx / V;
  int bx = 1;
  while (bx < nvec && bx < 128) bx *= 2;
  const int by = 256 / bx;
  dim3 b(bx, by, 1), gr((nvec + bx - 1) / bx, (G.ny + by - 1) / by, G.nz);
  if (G.per)
    k_smooth_vec_prolong<float, V, true><<<gr, b, 0, s>>>(x, g, G, inv, ec, Gc, omega);
  else
    k_smooth_vec_prolong<float, V, false><<<gr, b, 0, s>>>(x, g, G, inv, ec, Gc, omega);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_resid_restrict(const T* x, const T* g, const Geom& G, T* gc, const Geom& Gc, bool red_only,
                                  cudaStream_t s) {
  constexpr int V = 16 / sizeof(T);
  if (G.hx % V == 0) {
    const int nvec = Gc.nx / V;
    int bx = 1;
    while (bx < nvec && bx < 64) bx *= 2;
    const int by = 256 / bx;
    dim3 b(bx, by, 1), gr((nvec + bx - 1) / bx, (Gc.ny + by - 1) / by, Gc.nz);
    if (G.per) {
      if (red_only)
        k_resid_restrict_vec<T, V, true, true><<<gr, b, 0, s>>>(x, g, G, gc, Gc);
      else
        k_resid_restrict_vec<T, V, false, true><<<gr, b, 0, s>>>(x, g, G, gc, Gc);
    } else {
      if (red_only)
        k_resid_restrict_vec<T, V, true, false><<<gr, b, 0, s>>>(x, g, G, gc, Gc);
      else
        k_resid_restrict_vec<T, V, false, false><<<gr, b, 0, s>>>(x, g, G, gc, Gc);
    }
    return cudaGetLastError();
  }
  dim3 b, gr;
  shape(Gc.nx, Gc.ny, Gc.nz, b, gr);
  if (red_only)
    k_resid_restrict<T, true><<<gr, b, 0, s>>>(x, g, G, gc, Gc);
  else
    k_resid_restrict<T, false><<<gr, b, 0, s>>>(x, g, G, gc, Gc);
  return cudaGetLastError();
}

bool resid_restrict_walk_applies(const Geom& G) { return G.packed && G.hx >= kResTM; }

cudaError_t launch_resid_restrict_walk(const double* x, const double* g, const Geom& G, double* gc, const Geom& Gc,
                                       cudaStream_t s) {
  if (!resid_restrict_walk_applies(G)) return cudaErrorInvalidValue;
  const long long tiles = resid_tile_count(G);
  const int grid = (int)(tiles < (1LL << 20) ? tiles : (1LL << 20));
  const dim3 b(kResBX, kResBY, 1);
  if (G.per) k_resid_restrict_walk<true><<<grid, b, 0, s>>>(x, g, G, gc, Gc);
  else k_resid_restrict_walk<false><<<grid, b, 0, s>>>(x, g, G, gc, Gc);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_prolong(T* x, const Geom& G, const T* ec, const Geom& Gc, T omega, bool red_only, cudaStream_t s) {
  dim3 b, gr;
  shape(Gc.nx, Gc.ny, Gc.nz, b, gr);
  k_prolong<T><<<gr, b, 0, s>>>(x, G, ec, Gc, omega, red_only ? 1 : 0);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_coarse_cg(T* x, const T* b, const Geom& Gc, double rtol, int maxit, int* d_iters, cudaStream_t s) {
  const int n = Gc.nx * Gc.ny * Gc.nz;
  int threads = ((n + 31) / 32) * 32;
  if (threads > 256) threads = 256;
  if (threads < 32) threads = 32;
  const size_t smem = (size_t)4 * n * sizeof(double);
  k_coarse_cg<T><<<1, threads, smem, s>>>(x, b, Gc, rtol, maxit, d_iters);
  return cudaGetLastError();
}

// Opt in to the dynamic shared memory the coarse CG needs (four vectors of kMaxCoarseCells
// doubles). Called once per context creation, outside any stream capture.
cudaError_t prepare_coarse_cg() {
  const int bytes = (int)(4 * kMaxCoarseCells * sizeof(double));
  cudaError_t e = cudaFuncSetAttribute(k_coarse_cg<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_coarse_cg<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

template <typename T>
cudaError_t launch_resid_norm(const T* x, const T* g, const Geom& G, double* partials, int* nparts, int mode,
                              double c0, double* out_natural, float* out_packed, const double* inv_scale,
                              cudaStream_t s) {
  const int grid = resid_norm_blocks(G);
  const dim3 b(kResBX, kResBY, 1);
  if (G.per) {
    if (mode == 0) k_resid_norm<T, 0, true><<<grid, b, 0, s>>>(x, g, G, partials, c0, out_natural, out_packed, inv_scale);
    if (mode == 1) k_resid_norm<T, 1, true><<<grid, b, 0, s>>>(x, g, G, partials, c0, out_natural, out_packed, inv_scale);
    if (mode == 2) k_resid_norm<T, 2, true><<<grid, b, 0, s>>>(x, g, G, partials, c0, out_natural, out_packed, inv_scale);
  } else {
    if (mode == 0) k_resid_norm<T, 0, false><<<grid, b, 0, s>>>(x, g, G, partials, c0, out_natural, out_packed, inv_scale);
    if (mode == 1) k_resid_norm<T, 1, false><<<grid, b, 0, s>>>(x, g, G, partials, c0, out_natural, out_packed, inv_scale);
    if (mode == 2) k_resid_norm<T, 2, false><<<grid, b, 0, s>>>(x, g, G, partials, c0, out_natural, out_packed, inv_scale);
  }
  *nparts = grid;
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_sumsq(const T* a, long long n, double* partials, int* nparts, cudaStream_t s) {
  long long blocks = (n + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  if (blocks < 1) blocks = 1;
  k_sumsq<T><<<(int)blocks, 256, 0, s>>>(a, n, partials);
  *nparts = (int)blocks;
  return cudaGetLastError();
}

cudaError_t launch_finalize(const double* partials, int nparts, double* scal, int slot, int slot_rel, int slot_ref,
                            cudaStream_t s) {
  k_finalize<<<1, 256, 0, s>>>(partials, nparts, scal, slot, slot_rel, slot_ref);
  return cudaGetLastError();
}

cudaError_t launch_set_scale(double* scal, int src, int dst, double n, cudaStream_t s) {
  k_set_scale<<<1, 1, 0, s>>>(scal, src, dst, n);
  return cudaGetLastError();
}

WallTerms make_wall_terms(const FaceBC& bc, double h) {
  WallTerms wt;
  for (int q = 0; q < 6; ++q) {
    wt.t[q] = bc.type[q] == 0 ? 2.0 * bc.value[q] / (h * h) : (bc.type[q] == 1 ? bc.value[q] / h : 0.0);
    wt.field[q] = bc.field[q];
    wt.type[q] = bc.type[q];
  }
  wt.h = h;
  return wt;
}

void rhs_job_static(RhsJob& j, const Geom& G, double* g, double inv_eps, double h, const FaceBC& bc, double* scal) {
  j.G = G;
  j.g = g;
  j.rho = nullptr;
  j.inv_eps = inv_eps;
  j.hsq = h * h;
  j.qe = host_pow2_exponent(inv_eps);
  j.qh = host_pow2_exponent(j.hsq);
  j.pow2 = j.qe != kBadPow2 && j.qh != kBadPow2;
  j.fld = has_field(bc) ? 1 : 0;
  j.wt = make_wall_terms(bc, h);
  j.pair = 0;
  j.b0 = 0;
  const long long n = (long long)G.nx * G.ny * G.nz;
  long long blocks = (n + 255) / 256;  // as launch_sumsq
  if (blocks > 152 * 8) blocks = 152 * 8;
  if (blocks < 1) blocks = 1;
  j.sb0 = 0;
  j.sbn = (int)blocks;
  j.scal = scal;
  j.n = (double)n;
}

cudaError_t launch_set_rhs_all(const RhsJob* d_jobs, int B, long long nblocks, int nsblocks, double* partials,
                               int slot_gsum, int slot_scale, cudaStream_t s) {
  if (B < 1) return cudaSuccess;
  const long long g1 = nblocks < 152 * 16 ? nblocks : 152 * 16;
  k_set_rhs_all<<<(int)(g1 > 0 ? g1 : 1), 256, 0, s>>>(d_jobs, B, nblocks);
  const int g2 = nsblocks < 152 * 8 ? nsblocks : 152 * 8;
  k_sumsq_all<<<g2 > 0 ? g2 : 1, 256, 0, s>>>(d_jobs, B, nsblocks, partials);
  k_finalize_all<<<B, 256, 0, s>>>(d_jobs, partials, slot_gsum, slot_scale);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_set_rhs(T* g, const Geom& G, const double* rho, double inv_eps, double h, const FaceBC& bc, int raw,
                           cudaStream_t s) {
  const WallTerms wt = make_wall_terms(bc, h);
  const bool fld = has_field(bc);
  dim3 b, gr;
  const double hsq = h * h;
  const int qe = host_pow2_exponent(inv_eps), qh = host_pow2_exponent(hsq);
  const bool pow2 = qe != kBadPow2 && qh != kBadPow2;
  if (G.packed && reinterpret_cast<uintptr_t>(rho) % 16 == 0) {
    shape(G.hx, G.ny, G.nz, b, gr);
    if (fld) {
      if (pow2) k_set_rhs_pair<T, true, true><<<gr, b, 0, s>>>(g, G, rho, inv_eps, hsq, qe, qh, wt, raw);
      else k_set_rhs_pair<T, false, true><<<gr, b, 0, s>>>(g, G, rho, inv_eps, hsq, qe, qh, wt, raw);
    } else {
      if (pow2) k_set_rhs_pair<T, true, false><<<gr, b, 0, s>>>(g, G, rho, inv_eps, hsq, qe, qh, wt, raw);
      else k_set_rhs_pair<T, false, false><<<gr, b, 0, s>>>(g, G, rho, inv_eps, hsq, qe, qh, wt, raw);
    }
    return cudaGetLastError();
  }
  shape(G.nx, G.ny, G.nz, b, gr);
  if (fld) {
    if (pow2) k_set_rhs<T, true, true><<<gr, b, 0, s>>>(g, G, rho, inv_eps, hsq, qe, qh, wt, raw);
    else k_set_rhs<T, false, true><<<gr, b, 0, s>>>(g, G, rho, inv_eps, hsq, qe, qh, wt, raw);
  } else {
    if (pow2) k_set_rhs<T, true, false><<<gr, b, 0, s>>>(g, G, rho, inv_eps, hsq, qe, qh, wt, raw);
    else k_set_rhs<T, false, false><<<gr, b, 0, s>>>(g, G, rho, inv_eps, hsq, qe, qh, wt, raw);
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_pack(T* dst, const Geom& G, const double* src, double scale, cudaStream_t s) {
  dim3 b, gr;
  shape(G.nx, G.ny, G.nz, b, gr);
  k_pack<T><<<gr, b, 0, s>>>(dst, G, src, scale);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_unpack(double* dst, const T* src, const Geom& G, double scale, cudaStream_t s) {
  dim3 b, gr;
  shape(G.nx, G.ny, G.nz, b, gr);
  k_unpack<T><<<gr, b, 0, s>>>(dst, src, G, scale);
  return cudaGetLastError();
}

cudaError_t launch_resid_zero(const double* g, long long n, float* outp, double* scal, int slot_rsum, int slot_rel,
                              int slot_gsum, int slot_inv_scale, cudaStream_t s) {
  long long blocks = outp ? (n + 255) / 256 : 1;
  if (blocks > 152 * 16) blocks = 152 * 16;
  k_resid_zero<<<(int)blocks, 256, 0, s>>>(g, n, outp, scal, slot_rsum, slot_rel, slot_gsum, slot_inv_scale);
  return cudaGetLastError();
}

cudaError_t launch_scale_convert(const double* x, const float* e, const double* y, long long n, double sc, float* xf,
                                 double* yo, double* xs, cudaStream_t s) {
  long long blocks = (n + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (blocks < 1) blocks = 1;
  k_scale_convert<<<(int)blocks, 256, 0, s>>>(x, e, y, n, sc, 1.0 / sc, xf, yo, xs);
  return cudaGetLastError();
}

cudaError_t launch_set_mixed(double* x, const float* e, long long n, const double* scal, int slot, cudaStream_t s) {
  long long blocks = (n + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (blocks < 1) blocks = 1;
  k_set_mixed<<<(int)blocks, 256, 0, s>>>(x, e, n, scal, slot);
  return cudaGetLastError();
}

cudaError_t launch_update_mixed(double* x, const float* e, long long n, const double* scal, int slot, cudaStream_t s) {
  long long blocks = (n + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (blocks < 1) blocks = 1;
  k_update_mixed<<<(int)blocks, 256, 0, s>>>(x, e, n, scal, slot);
  return cudaGetLastError();
}

#define CCMG_INSTANTIATE(T)                                                                                         \
  template cudaError_t launch_smooth<T>(T*, const T*, const Geom&, const InvDiag<T>&, int, bool, cudaStream_t);     \
  template cudaError_t launch_resid_restrict<T>(const T*, const T*, const Geom&, T*, const Geom&, bool, cudaStream_t);    \
  template cudaError_t launch_prolong<T>(T*, const Geom&, const T*, const Geom&, T, bool, cudaStream_t);            \
  template cudaError_t launch_coarse_cg<T>(T*, const T*, const Geom&, double, int, int*, cudaStream_t);             \
  template cudaError_t launch_resid_norm<T>(const T*, const T*, const Geom&, double*, int*, int, double, double*,   \
                                            float*, const double*, cudaStream_t);                                   \
  template cudaError_t launch_sumsq<T>(const T*, long long, double*, int*, cudaStream_t);                           \
  template cudaError_t launch_set_rhs<T>(T*, const Geom&, const double*, double, double, const FaceBC&, int,        \
                                         cudaStream_t);                                                             \
  template cudaError_t launch_pack<T>(T*, const Geom&, const double*, double, cudaStream_t);                        \
  template cudaError_t launch_unpack<T>(double*, const T*, const Geom&, double, cudaStream_t);

CCMG_INSTANTIATE(double)
CCMG_INSTANTIATE(float)

}  // namespace ccmg
