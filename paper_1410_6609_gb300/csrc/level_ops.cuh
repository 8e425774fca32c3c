// level_ops.cuh -- device-side bodies of the per-level multigrid operations (Sec. 3, Sec. 5.3).
//
// Shared by the single-system kernels (level_kernels.cu) and the batched kernels over many
// systems of different sizes (batch_kernels.cu): each body works on one thread's cell (or vector
// of cells) at explicit coordinates, so both launch schemes perform bit-identical arithmetic.
// Layout and scaling conventions are those of ccmg_internal.cuh.
#pragma once
#include <type_traits>
#include <cstring>

#include "ccmg_internal.cuh"

namespace ccmg {
namespace ops {

__device__ __forceinline__ double fmat(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float fmat(float a, float b, float c) { return __fmaf_rn(a, b, c); }
// A product and a sum that the compiler may not fuse into one FMA (kernels that must agree bit
// for bit round both).
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }

// Diagonal shift d of the folded boundary stencil for packed-row coordinates (m, s, j, k):
// +1 per Dirichlet face, -1 per Neumann face the cell touches (Sec. 2.4, Boundary conditions).
__device__ __forceinline__ int diag_shift_packed(const Geom& G, int m, int s, int j, int k) {
  int d = 0;
  if (m == 0 && s == 0) d += G.sh[0];
  if (m == G.hx - 1 && s == 1) d += G.sh[1];
  if (j == 0) d += G.sh[2];
  if (j == G.ny - 1) d += G.sh[3];
  if (k == 0) d += G.sh[4];
  if (k == G.nz - 1) d += G.sh[5];
  return d;
}

// 1/(6+d) from the per-type table without dynamic indexing (keeps the table in registers).
template <typename T>
__device__ __forceinline__ T inv_of(const InvDiag<T>& inv, int d) {
  T r = inv.v[3];
  r = (d == -3) ? inv.v[0] : r;
  r = (d == -2) ? inv.v[1] : r;
  r = (d == -1) ? inv.v[2] : r;
  r = (d == 1) ? inv.v[4] : r;
  r = (d == 2) ? inv.v[5] : r;
  r = (d == 3) ? inv.v[6] : r;
  return r;
}

// -(6 + d) as a floating-point constant chosen by selects (an int->double conversion would run
// on the FP64 pipe, which is the bottleneck of the FP64 kernels).
template <typename T>
__device__ __forceinline__ T neg_diag(int d) {
  T r = T(-6);
  r = (d == -3) ? T(-3) : r;
  r = (d == -2) ? T(-4) : r;
  r = (d == -1) ? T(-5) : r;
  r = (d == 1) ? T(-7) : r;
  r = (d == 2) ? T(-8) : r;
  r = (d == 3) ? T(-9) : r;
  return r;
}

// 1/(6 + d) for the V cells m0 .. m0+V-1 of packed row (s, j, k). Cells away from every wall
// (the bulk) take 1/6 without evaluating the per-cell shift; the branch is taken by the few
// threads at a wall.
template <typename T, int V>
__device__ __forceinline__ void inv_diag_vec(const Geom& G, const InvDiag<T>& inv, int m0, int s, int j, int k,
                                             T (&invd)[V]) {
  if (j == 0 || j == G.ny - 1 || k == 0 || k == G.nz - 1 || m0 == 0 || m0 + V >= G.hx) {
    int dbase = 0;
    if (j == 0) dbase += G.sh[2];
    if (j == G.ny - 1) dbase += G.sh[3];
    if (k == 0) dbase += G.sh[4];
    if (k == G.nz - 1) dbase += G.sh[5];
#pragma unroll
    for (int v = 0; v < V; ++v) {
      int d = dbase;
      if (m0 + v == 0 && s == 0) d += G.sh[0];
      if (m0 + v == G.hx - 1 && s == 1) d += G.sh[1];
      invd[v] = inv_of(inv, d);
    }
  } else {
#pragma unroll
    for (int v = 0; v < V; ++v) invd[v] = inv.v[3];
  }
}

// ---------------------------------------------------------------------------------------------
// Power-of-two scaling. The defect-correction scale is a power of two, and so are the 1/(2h),
// 1/eps and h^2 factors of the lattice-unit workloads. Multiplying by 2^q and the conversions
// float(x 2^q) and double(e) 2^p then reduce to exponent arithmetic and one round-to-nearest-even
// of the significand, done here in integer operations: on GB300 the FP64 pipe runs at 1/64 of
// the FP32 rate and the FP64 multiply and the conversion instructions would occupy it. The
// routines are total (zeros, subnormal inputs and results, overflow, infinities and NaN), so the
// kernels call them without a fallback; whether a factor is a power of two is decided once per
// launch (pow2_exponent) and the kernels select their loop by it.

constexpr int kBadPow2 = -100000;  // pow2_exponent of a factor that is not a power of two
constexpr int kScaleExpLimit = 800;  // |log2| bound of defect-correction scales (keeps s e exact)

// Largest power of two <= v, with the exponent clamped to [-kScaleExpLimit, kScaleExpLimit], for
// finite v > 0; 1 otherwise.
__device__ __forceinline__ double pow2_floor(double v) {
  if (!(v > 0.0) || !(v < 1e300)) return 1.0;
  int e = 0;
  frexp(v, &e);  // v = m 2^e, 0.5 <= m < 1
  e -= 1;
  e = e < -kScaleExpLimit ? -kScaleExpLimit : (e > kScaleExpLimit ? kScaleExpLimit : e);
  return ldexp(1.0, e);
}

// p with v = 2^p for a positive normal power of two, else kBadPow2.
__device__ __forceinline__ int pow2_exponent(double v) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(v);
  const int E = (int)((u >> 52) & 0x7ff);
  if ((u & 0x800fffffffffffffULL) != 0ULL || E == 0 || E == 0x7ff) return kBadPow2;
  return E - 1023;
}

// The same test on the host (launchers choose the kernel variant with it).
inline int host_pow2_exponent(double v) {
  unsigned long long u = 0;
  std::memcpy(&u, &v, sizeof(u));
  const int E = (int)((u >> 52) & 0x7ff);
  if ((u & 0x800fffffffffffffULL) != 0ULL || E == 0 || E == 0x7ff) return kBadPow2;
  return E - 1023;
}

// m >> s rounded to nearest, ties to even (1 <= s <= 63).
__device__ __forceinline__ unsigned long long rshift_rne(unsigned long long m, int s) {
  const unsigned long long kept = m >> s;
  const unsigned long long rem = m & ((1ULL << s) - 1ULL);
  const unsigned long long half = 1ULL << (s - 1);
  return kept + ((rem > half || (rem == half && (kept & 1ULL))) ? 1ULL : 0ULL);
}

// Significand (leading one at bit 52) and biased exponent of a finite nonzero double; a
// subnormal is normalised (its exponent then drops below 1).
__device__ __forceinline__ void unpack_f64(unsigned long long u, unsigned long long& M, int& E) {
  E = (int)((u >> 52) & 0x7ff);
  M = u & 0xfffffffffffffULL;
  if (E == 0) {
    const int lz = __clzll((long long)M) - 11;
    M <<= lz;
    E = 1 - lz;
  } else {
    M |= 1ULL << 52;
  }
}

// v * 2^q rounded to nearest even (q = pow2_exponent of the factor): all cases.
static __device__ __noinline__ double ldexp_rne_general(double v, int q) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(v);
  const unsigned long long sign = u & 0x8000000000000000ULL;
  if ((u << 1) == 0ULL || ((u >> 52) & 0x7ff) == 0x7ff) return v;  // zeros, infinities, NaN
  unsigned long long M;
  int E;
  unpack_f64(u, M, E);
  const int En = E + q;
  if (En >= 2047) return __longlong_as_double((long long)(sign | 0x7ff0000000000000ULL));
  if (En >= 1) return __longlong_as_double((long long)(sign | ((unsigned long long)En << 52) | (M & 0xfffffffffffffULL)));
  const int sh = 1 - En;  // subnormal result in units of 2^-1074 (a carry to 2^52 encodes 2^-1022)
  if (sh > 54) return __longlong_as_double((long long)sign);
  return __longlong_as_double((long long)(sign | rshift_rne(M, sh)));
}

// The common cases inline: zeros, and normal in and out (only the exponent field changes).
__device__ __forceinline__ double ldexp_rne(double v, int q) {
  const unsigned hi = (unsigned)__double2hiint(v), lo = (unsigned)__double2loint(v);
  const int E = (int)((hi >> 20) & 0x7ffu);
  const int En = E + q;
  if (E != 0 && E != 0x7ff && En >= 1 && En <= 2046)
    return __hiloint2double((int)((hi & 0x800fffffu) | ((unsigned)En << 20)), (int)lo);
  if (((hi & 0x7fffffffu) | lo) == 0u) return v;
  return ldexp_rne_general(v, q);
}

// float(x * 2^q) rounded to nearest even: all cases.
static __device__ __noinline__ float f32_of_scaled_general(double x, int q) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const unsigned sign = (unsigned)(u >> 32) & 0x80000000u;
  if ((u << 1) == 0ULL) return __uint_as_float(sign);
  if (((u >> 52) & 0x7ff) == 0x7ff)
    return __uint_as_float(sign | 0x7f800000u | ((u & 0xfffffffffffffULL) ? 0x00400000u : 0u));
  unsigned long long M;
  int E;
  unpack_f64(u, M, E);
  const int eL = E - 1023 + q;  // the value lies in [2^eL, 2^(eL+1))
  if (eL > 127) return __uint_as_float(sign | 0x7f800000u);
  if (eL >= -126) {  // normal float: keep 24 of the 53 bits; a carry may reach the exponent (or inf)
    const unsigned r = (unsigned)rshift_rne(M, 29);
    return __uint_as_float(sign | (((unsigned)(eL + 126) << 23) + r));
  }
  const int sh = 29 + (-126 - eL);  // subnormal float in units of 2^-149
  if (sh > 54) return __uint_as_float(sign);
  return __uint_as_float(sign | (unsigned)rshift_rne(M, sh));
}

// The common case inline (normal double to normal float), in 32-bit operations.
__device__ __forceinline__ float f32_of_scaled(double x, int q) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const int E = (int)((hi >> 20) & 0x7ffu);
  const int eL = E - 1023 + q;
  if (E != 0 && E != 0x7ff && eL >= -126 && eL <= 127) {
    const unsigned m23 = ((hi & 0xfffffu) << 3) | (lo >> 29);  // top 23 of the 52 significand bits
    const unsigned rest = lo & 0x1fffffffu;                    // the 29 dropped bits
    const unsigned up = (rest > 0x10000000u || (rest == 0x10000000u && (m23 & 1u))) ? 1u : 0u;
    // a carry out of the significand raises the exponent (to inf past the largest float)
    return __uint_as_float((hi & 0x80000000u) | ((((unsigned)(eL + 127) << 23) | m23) + up));
  }
  if (((hi & 0x7fffffffu) | lo) == 0u) return __uint_as_float(hi & 0x80000000u);
  return f32_of_scaled_general(x, q);
}

// double(e) * 2^p rounded to nearest even (exact unless it leaves the normal range).
__device__ __forceinline__ double f64_of_scaled(float e, int p) {
  const unsigned b = __float_as_uint(e);
  const int Ef = (int)((b >> 23) & 0xffu);
  const int En = Ef - 127 + 1023 + p;
  if (Ef != 0 && Ef != 0xff && En >= 1 && En <= 2046)
    return __hiloint2double((int)((b & 0x80000000u) | ((unsigned)En << 20) | ((b & 0x7fffffu) >> 3)),
                            (int)(b << 29));
  if ((b & 0x7fffffffu) == 0u) return __hiloint2double((int)(b & 0x80000000u), 0);
  return ldexp_rne_general((double)e, p);  // subnormals, infinities, NaN, range ends
}

// 16-byte vector loads and stores (4 floats or 2 doubles).
__device__ __forceinline__ void load_vec(const float* p, float (&o)[4]) {
  const float4 v = __ldg(reinterpret_cast<const float4*>(p));
  o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
}
__device__ __forceinline__ void load_vec(const double* p, double (&o)[2]) {
  const double2 v = __ldg(reinterpret_cast<const double2*>(p));
  o[0] = v.x; o[1] = v.y;
}
__device__ __forceinline__ void store_vec(float* p, const float (&o)[4]) {
  *reinterpret_cast<float4*>(p) = make_float4(o[0], o[1], o[2], o[3]);
}
__device__ __forceinline__ void store_vec(double* p, const double (&o)[2]) {
  *reinterpret_cast<double2*>(p) = make_double2(o[0], o[1]);
}

// Neighbour row Q (0: -y, 1: +y, 2: -z, 3: +z) of packed row (j, k): whether it exists (inside
// the level, or across a periodic axis, where it is the row at the opposite side: Sec. 2.4), and
// its offset within a colour array (the same row serves the cells of either colour). PER = false
// compiles the plain wall tests of a level without periodic axes.
template <int Q, bool PER>
__device__ __forceinline__ bool nb_inside(const Geom& G, int j, int k) {
  return Q == 0 ? j > 0 : (Q == 1 ? j < G.ny - 1 : (Q == 2 ? k > 0 : k < G.nz - 1));
}
template <int Q, bool PER>
__device__ __forceinline__ bool nb_has(const Geom& G, int j, int k) {
  return nb_inside<Q, PER>(G, j, k) || (PER && (G.per & (Q < 2 ? 2 : 4)) != 0);
}
template <int Q, bool PER>
__device__ __forceinline__ long long nb_off(const Geom& G, int j, int k) {
  if (!PER || nb_inside<Q, PER>(G, j, k)) {
    if constexpr (Q < 2) return (Q & 1) ? G.hx : -G.hx;
    else return (Q & 1) ? (long long)G.ny * G.hx : -((long long)G.ny * G.hx);
  }
  if constexpr (Q < 2) return (Q & 1) ? -(long long)(G.ny - 1) * G.hx : (long long)(G.ny - 1) * G.hx;
  else return (Q & 1) ? -(long long)(G.nz - 1) * G.ny * G.hx : (long long)(G.nz - 1) * G.ny * G.hx;
}

// Sum of the six neighbours (in the order -x,+x,-y,+y,-z,+z; absent ones are zero) of the cell at
// index m of row `row` in colour c, where y points at the other colour's array. Across a periodic
// x axis the neighbour of cell 0 (index 0, s = 0) is cell nx-1 (index hx-1 of the other colour)
// and the other way round.
template <typename T, bool PER = true>
__device__ __forceinline__ T nbsum_packed(const T* __restrict__ y, const Geom& G, long long row, int m, int s, int j,
                                          int k) {
  const T* yr = y + row;
  const bool px = PER && (G.per & 1) != 0;
  const T xm = (m == 0 && s == 0) ? (px ? __ldg(yr + G.hx - 1) : T(0)) : __ldg(yr + m + s - 1);
  const T xp = (m == G.hx - 1 && s == 1) ? (px ? __ldg(yr) : T(0)) : __ldg(yr + m + s);
  const T ym = nb_has<0, PER>(G, j, k) ? __ldg(yr + m + nb_off<0, PER>(G, j, k)) : T(0);
  const T yp = nb_has<1, PER>(G, j, k) ? __ldg(yr + m + nb_off<1, PER>(G, j, k)) : T(0);
  const T zm = nb_has<2, PER>(G, j, k) ? __ldg(yr + m + nb_off<2, PER>(G, j, k)) : T(0);
  const T zp = nb_has<3, PER>(G, j, k) ? __ldg(yr + m + nb_off<3, PER>(G, j, k)) : T(0);
  return ((((xm + xp) + ym) + yp) + zm) + zp;
}

// The V-vector of neighbour row Q at m0, or zeros where the row does not exist.
template <int Q, bool PER, typename T, int V>
__device__ __forceinline__ void load_nb_vec(const T* __restrict__ yr, const Geom& G, int m0, int j, int k,
                                            T (&o)[V]) {
  if (nb_has<Q, PER>(G, j, k)) load_vec(yr + m0 + nb_off<Q, PER>(G, j, k), o);
  else
#pragma unroll
    for (int i = 0; i < V; ++i) o[i] = T(0);
}

// ---------------------------------------------------------------------------------------------
// The FP64 scaled residual r~ = g + (x_-x + x_+x + x_-y + x_+y + x_-z + x_+z) - D x_c of one cell
// (D = 6 + d), evaluated in 64-bit fixed point. Each operand is first put in a form that does not
// depend on the cell (FxOp: its 53-bit significand times 2^5 with its sign applied, and its biased
// exponent), so that a value converted once can serve every cell it enters (the packed tile walk
// below goes one step further and aligns each ring row to one exponent; this per-cell form serves
// the natural-order levels). A cell aligns its operands to the largest biased exponent E among them,
// rounding each down to the unit 2^(E-1080) (an arithmetic shift), adds them as integers (the
// magnitudes stay below 2^58 each, so the sum of at most 16 of them fits), and rounds the sum
// once to the nearest double. Each operand loses less than one unit (the centre's loss is scaled
// by D), so the result lies within 16 units, i.e. half an ulp of the largest operand, plus half
// an ulp of itself, of the exact residual: closer than the seven rounded FP64 operations of the
// direct formula. All of it is integer work: on GB300 the FP64 pipe, which the direct formula
// occupies, runs at 1/64 of the FP32 rate. Subnormal operands count as zero (they lie below one
// unit unless every operand is that small); a cell with an infinite or NaN operand takes the
// direct formula.
struct FxOp {
  unsigned lo, hi;  // two's complement of +-significand * 2^5 (0 for zero and subnormal operands)
  unsigned pk;      // biased exponent e in bits 0..15, and (e ? 2047 - e : 0) in bits 16..31
};

__host__ __device__ __forceinline__ unsigned long long fx_bits(double v) {
#ifdef __CUDA_ARCH__
  return (unsigned long long)__double_as_longlong(v);
#else
  unsigned long long u;
  memcpy(&u, &v, sizeof(u));
  return u;
#endif
}

__host__ __device__ __forceinline__ double fx_double(unsigned long long u) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)u);
#else
  double v;
  memcpy(&v, &u, sizeof(v));
  return v;
#endif
}

__host__ __device__ __forceinline__ FxOp fx_op(double v) {
  const unsigned long long u = fx_bits(v);
  const unsigned hi = (unsigned)(u >> 32), lo = (unsigned)u;
  const unsigned e = (hi >> 20) & 0x7ffu;
  const unsigned keep = e ? 0xffffffffu : 0u;
  const unsigned mh = (hi & 0xfffffu) | 0x100000u;
  const unsigned long long mag = ((unsigned long long)(((mh << 5) | (lo >> 27)) & keep) << 32) | ((lo << 5) & keep);
  const unsigned long long neg = (unsigned long long)(long long)((int)hi >> 31);
  const unsigned long long S = (mag ^ neg) - neg;
  FxOp o;
  o.lo = (unsigned)S;
  o.hi = (unsigned)(S >> 32);
  o.pk = e | ((e ? 2047u - e : 0u) << 16);
  return o;
}

// Lane-wise maximum of two pairs of 16-bit fields.
__host__ __device__ __forceinline__ unsigned fx_max2(unsigned a, unsigned b) {
#ifdef __CUDA_ARCH__
  unsigned d;
  asm("max.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
  return d;
#else
  const unsigned l = (a & 0xffffu) > (b & 0xffffu) ? (a & 0xffffu) : (b & 0xffffu);
  const unsigned h = (a >> 16) > (b >> 16) ? (a >> 16) : (b >> 16);
  return l | (h << 16);
#endif
}

// floor(S / 2^(E - e)) for an operand with E - e <= 31 (or S = 0): a funnel shift of the two words.
__host__ __device__ __forceinline__ unsigned long long fx_align31(const FxOp& o, int E) {
  const unsigned d = ((unsigned)E - o.pk) & 31u;  // the upper field of pk drops out of the low 5 bits
#ifdef __CUDA_ARCH__
  const unsigned lo = __funnelshift_r(o.lo, o.hi, d);
  const unsigned hi = (unsigned)((int)o.hi >> d);
  return ((unsigned long long)hi << 32) | lo;
#else
  return (unsigned long long)((long long)(((unsigned long long)o.hi << 32) | o.lo) >> d);
#endif
}

// The same for any exponent gap (shifts of 63 and more leave 0 or -1).
__host__ __device__ __forceinline__ unsigned long long fx_align(const FxOp& o, int E) {
  int d = E - (int)(o.pk & 0xffffu);
  d = d < 63 ? d : 63;
  return (unsigned long long)((long long)(((unsigned long long)o.hi << 32) | o.lo) >> d);
}

// The signed sum S in units 2^(E-1080) as a double: the integer rounded to nearest (ties to even)
// by the conversion instruction, then scaled by the power of two, which is exact unless the result
// leaves the normal range (then it is rounded once more, or overflows to infinity, as ldexp does).
__host__ __device__ __forceinline__ double fx_to_double(unsigned long long S, int E) {
#ifdef __CUDA_ARCH__
  return ldexp_rne(__ll2double_rn((long long)S), E - 1080);
#else
  return ldexp((double)(long long)S, E - 1080);
#endif
}

// The operand back as a double (exact for normal values, infinities and NaN; subnormals give 0).
__host__ __device__ __forceinline__ double fx_value(const FxOp& o) {
  const unsigned long long S = ((unsigned long long)o.hi << 32) | o.lo;
  const unsigned e = o.pk & 0xffffu;
  if (e == 0u) return 0.0;
  const unsigned long long sgn = S & 0x8000000000000000ULL;
  const unsigned long long mag = (sgn ? (0ULL - S) : S) >> 5;
  return fx_double(sgn | ((unsigned long long)e << 52) | (mag & 0xfffffffffffffULL));
}

// The direct FP64 formula, for cells with an infinite or NaN operand.
__host__ __device__ __forceinline__ double fx_direct(const FxOp (&op)[8], int D) {
  const double S = ((((fx_value(op[1]) + fx_value(op[2])) + fx_value(op[3])) + fx_value(op[4])) + fx_value(op[5])) +
                   fx_value(op[6]);
  return fma(-(double)D, fx_value(op[7]), fx_value(op[0]) + S);
}

// r~ of one cell from op[0] = g, op[1..6] = the six neighbours (absent ones as fx_op(0.0)) and
// op[7] = the centre, with D = 6 + d. G0: the right-hand side is zero and op[0] is not read (the
// same exact sum without its zero term, hence the same result).
template <bool G0 = false>
__host__ __device__ __forceinline__ double fx_residual(const FxOp (&op)[8], int D) {
  constexpr int i0 = G0 ? 1 : 0;
  unsigned P = op[7].pk;
#pragma unroll
  for (int i = i0; i < 7; ++i) P = fx_max2(P, op[i].pk);
  const int E = (int)(P & 0xffffu);
  if (E == 0) return 0.0;  // every operand zero or subnormal
  if (E == 2047) {
    if (G0) {
      const FxOp o[8] = {fx_op(0.0), op[1], op[2], op[3], op[4], op[5], op[6], op[7]};
      return fx_direct(o, D);
    }
    return fx_direct(op, D);
  }
  const int emin = 2047 - (int)(P >> 16);  // smallest exponent among the nonzero operands
  unsigned long long acc = 0ULL;
  if (E - emin <= 31) {
#pragma unroll
    for (int i = i0; i < 7; ++i) acc += fx_align31(op[i], E);
    acc -= fx_align31(op[7], E) * (unsigned long long)D;
  } else {
#pragma unroll
    for (int i = i0; i < 7; ++i) acc += fx_align(op[i], E);
    acc -= fx_align(op[7], E) * (unsigned long long)D;
  }
  return fx_to_double(acc, E);
}

// The sum of a cell's six neighbours (absent ones as fx_op(0.0)) in the same fixed point, rounded
// once: within half an ulp of the largest neighbour plus half an ulp of itself of the exact sum
// (closer than five rounded FP64 additions). The FP64 half-sweep takes it so that two of its
// operations stay on the FP64 pipe instead of six.
__host__ __device__ __forceinline__ double fx_sum6(const FxOp (&op)[6]) {
  unsigned P = op[0].pk;
#pragma unroll
  for (int i = 1; i < 6; ++i) P = fx_max2(P, op[i].pk);
  const int E = (int)(P & 0xffffu);
  if (E == 0) return 0.0;  // every operand zero or subnormal
  if (E == 2047)           // an infinite or NaN operand: the direct sum
    return ((((fx_value(op[0]) + fx_value(op[1])) + fx_value(op[2])) + fx_value(op[3])) + fx_value(op[4])) +
           fx_value(op[5]);
  const int emin = 2047 - (int)(P >> 16);
  unsigned long long acc = 0ULL;
  if (E - emin <= 31) {
#pragma unroll
    for (int i = 0; i < 6; ++i) acc += fx_align31(op[i], E);
  } else {
#pragma unroll
    for (int i = 0; i < 6; ++i) acc += fx_align(op[i], E);
  }
  return fx_to_double(acc, E);
}

// The biased exponent of v (0 for zero and subnormal values, 2047 for infinities and NaN).
__device__ __forceinline__ unsigned fx_exp(double v) { return ((unsigned)__double2hiint(v) >> 20) & 0x7ffu; }

// v as a signed integer multiple of 2^(E - 1080), rounded toward -infinity (E >= fx_exp(v);
// subnormal values count as zero): the fixed point of fx_op aligned to the exponent E.
__device__ __forceinline__ long long fx_at(double v, int E) {
  const FxOp o = fx_op(v);
  const int d = E - (int)(o.pk & 0xffffu);
  return (long long)(((unsigned long long)o.hi << 32) | o.lo) >> (d < 63 ? d : 63);
}

// ---------------------------------------------------------------------------------------------
// Red-black Gauss-Seidel half-sweep (Sec. 5.3): every cell of `colour` becomes the solution of
// its own row, phi = (g + sum of neighbours) / (6 + d). ZERO: the level's current iterate is
// zero (first sweep after restriction), so the neighbour sum is exactly zero and is not read.
// Cell (m, j, k) of the colour's array; caller guarantees m < hx, j < ny, k < nz.
template <typename T, bool ZERO, bool PER = true>
__device__ __forceinline__ void smooth_cell(T* __restrict__ x, const T* __restrict__ g, const Geom& G,
                                            const InvDiag<T>& inv, int colour, int m, int j, int k) {
  const int s = (j + k + colour) & 1;
  const long long row = ((long long)k * G.ny + j) * G.hx;
  const long long own = (long long)colour * G.csz + row + m;
  const int d = diag_shift_packed(G, m, s, j, k);
  T S = T(0);
  if (!ZERO) S = nbsum_packed<T, PER>(x + (long long)(1 - colour) * G.csz, G, row, m, s, j, k);
  x[own] = (__ldg(g + own) + S) * inv_of(inv, d);
}

// The same half-sweep for V consecutive cells m0 = V*mv .. m0+V-1 of a colour row (rows whose
// length is a multiple of V). The other colour's row segment m0..m0+V-1 supplies one x-neighbour
// of every cell; the remaining one is the scalar just before (s = 0) or just after (s = 1) the
// segment. Each cell's sum is formed in the same order as in smooth_cell: identical results.
template <typename T, int V, bool ZERO, bool PER = true>
__device__ __forceinline__ void smooth_vec(T* __restrict__ x, const T* __restrict__ g, const Geom& G,
                                           const InvDiag<T>& inv, int colour, int mv, int j, int k) {
  const int m0 = mv * V;
  const int s = (j + k + colour) & 1;
  const long long row = ((long long)k * G.ny + j) * G.hx;
  const long long own = (long long)colour * G.csz + row + m0;
  T gv[V], out[V], invd[V];
  load_vec(g + own, gv);
  inv_diag_vec<T, V>(G, inv, m0, s, j, k, invd);
  if (ZERO) {
#pragma unroll
    for (int i = 0; i < V; ++i) out[i] = (gv[i] + T(0)) * invd[i];
  } else {
    const T* yr = x + (long long)(1 - colour) * G.csz + row;
    T yc[V], ym[V], yp[V], zm[V], zp[V];
    load_vec(yr + m0, yc);
    load_nb_vec<0, PER>(yr, G, m0, j, k, ym);
    load_nb_vec<1, PER>(yr, G, m0, j, k, yp);
    load_nb_vec<2, PER>(yr, G, m0, j, k, zm);
    load_nb_vec<3, PER>(yr, G, m0, j, k, zp);
    // the x-neighbour beyond the segment (the row's other end across a periodic x axis)
    const bool px = PER && (G.per & 1) != 0;
    T extra;
    if (s == 0) extra = (m0 > 0) ? __ldg(yr + m0 - 1) : (px ? __ldg(yr + G.hx - 1) : T(0));
    else extra = (m0 + V < G.hx) ? __ldg(yr + m0 + V) : (px ? __ldg(yr) : T(0));
    if constexpr (sizeof(T) == 8) {
      // FP64: the neighbour sum exactly in fixed point, each loaded value converted once (fx_sum6)
      FxOp fc[V], fym[V], fyp[V], fzm[V], fzp[V];
#pragma unroll
      for (int i = 0; i < V; ++i) {
        fc[i] = fx_op(yc[i]);
        fym[i] = fx_op(ym[i]);
        fyp[i] = fx_op(yp[i]);
        fzm[i] = fx_op(zm[i]);
        fzp[i] = fx_op(zp[i]);
      }
      const FxOp fe = fx_op(extra);
#pragma unroll
      for (int i = 0; i < V; ++i) {
        const FxOp xm = s == 0 ? (i == 0 ? fe : fc[(i + V - 1) % V]) : fc[i];
        const FxOp xp = s == 0 ? fc[i] : (i == V - 1 ? fe : fc[(i + 1) % V]);
        const FxOp op[6] = {xm, xp, fym[i], fyp[i], fzm[i], fzp[i]};
        out[i] = (gv[i] + fx_sum6(op)) * invd[i];
      }
    } else {
#pragma unroll
      for (int i = 0; i < V; ++i) {
        T xm, xp;
        if (s == 0) {
          xm = (i == 0) ? extra : yc[(i + V - 1) % V];
          xp = yc[i];
        } else {
          xm = yc[i];
          xp = (i == V - 1) ? extra : yc[(i + 1) % V];
        }
        const T S = ((((xm + xp) + ym[i]) + yp[i]) + zm[i]) + zp[i];
        out[i] = (gv[i] + S) * invd[i];
      }
    }
  }
  store_vec(x + own, out);
}

// V consecutive coarse values e(I0..I0+V-1, J, K) times omega (I0 a multiple of V), from packed
// colours (two vectors of V/2) or natural order (one vector).
template <typename T, int V>
__device__ __forceinline__ void coarse_row_w(const T* __restrict__ ec, const Geom& Gc, int I0, int J, int K, T omega,
                                             T (&w)[V]) {
  if (Gc.packed) {
    const long long rowc = ((long long)K * Gc.ny + J) * Gc.hx + (I0 >> 1);
    const int C0 = (I0 + J + K) & 1;  // colour of I0 (and I0+2, ...); I0+1, I0+3 have the other
    const T* a = ec + (long long)C0 * Gc.csz + rowc;
    const T* b = ec + (long long)(C0 ^ 1) * Gc.csz + rowc;
    if constexpr (V == 4 && sizeof(T) == 4) {
      // I0 is a multiple of 4 and the coarse rows are an even number of floats long (the fine
      // rows hold whole 4-float vectors), so both pairs are 8-byte aligned
      const float2 pa = __ldg(reinterpret_cast<const float2*>(a));
      const float2 pb = __ldg(reinterpret_cast<const float2*>(b));
      w[0] = mul_rn(omega, pa.x);
      w[1] = mul_rn(omega, pb.x);
      w[2] = mul_rn(omega, pa.y);
      w[3] = mul_rn(omega, pb.y);
    } else {
#pragma unroll
      for (int v = 0; v < V; ++v) w[v] = mul_rn(omega, __ldg(((v & 1) ? b : a) + (v >> 1)));
    }
  } else {
    const long long o = (long long)I0 + (long long)Gc.nx * ((long long)J + (long long)Gc.ny * K);
#pragma unroll
    for (int v = 0; v < V; ++v) w[v] = mul_rn(omega, __ldg(ec + o + v));
  }
}

// Index of coarse cell (I,J,K) in its level's storage (packed colours or natural order).
__device__ __forceinline__ long long coarse_index(const Geom& Gc, int I, int J, int K);

// First post-smoothing half-sweep (black) fused with the constant prolongation of the coarse
// correction e_c (Sec. 3): every red neighbour is read as red + omega * e_parent, the value the
// separate prolongation would have stored. A red cell at packed index m of fine row (j', k') has
// its parent at coarse (m, j'/2, k'/2). The red cells themselves are left uncorrected: the red
// half-sweep that follows overwrites them without reading them. Same arithmetic as prolongation
// followed by smooth_vec, hence identical results.
// PER = false: compiled without periodic support (the kernels choose by the level's walls).
template <typename T, int V, bool PER = true>
__device__ __forceinline__ void smooth_vec_prolong(T* __restrict__ x, const T* __restrict__ g, const Geom& G,
                                                   const InvDiag<T>& inv, const T* __restrict__ ec, const Geom& Gc,
                                                   T omega, int mv, int j, int k) {
  const int per = PER ? G.per : 0;
  const int colour = 1;
  const int m0 = mv * V;
  const int s = (j + k + colour) & 1;
  const long long row = ((long long)k * G.ny + j) * G.hx;
  const long long own = (long long)colour * G.csz + row + m0;
  const T* yr = x + row;  // red array, row (j,k)
  const int J = j >> 1, K = k >> 1;
  T gv[V], out[V], yc[V], ym[V], yp[V], zm[V], zp[V], wc[V], wy[V], wz[V], invd[V];
  inv_diag_vec<T, V>(G, inv, m0, s, j, k, invd);
  load_vec(g + own, gv);
  load_vec(yr + m0, yc);
  // coarse parents: row (J, K) serves the row itself and the y- and z-neighbour rows inside the
  // same coarse cell; the other y (z) neighbour row has its parent in row J -+ 1 (K -+ 1), which
  // across a periodic axis is the coarse row at the opposite side
  coarse_row_w<T, V>(ec, Gc, m0, J, K, omega, wc);
  const bool jy = (j & 1) ? nb_has<1, PER>(G, j, k) : nb_has<0, PER>(G, j, k);
  const bool kz = (k & 1) ? nb_has<3, PER>(G, j, k) : nb_has<2, PER>(G, j, k);
  int Jo = (j & 1) ? J + 1 : J - 1, Ko = (k & 1) ? K + 1 : K - 1;
  if (PER) {
    Jo = Jo == Gc.ny ? 0 : (Jo < 0 ? Gc.ny - 1 : Jo);
    Ko = Ko == Gc.nz ? 0 : (Ko < 0 ? Gc.nz - 1 : Ko);
  }
  if (jy) coarse_row_w<T, V>(ec, Gc, m0, Jo, K, omega, wy);
  if (kz) coarse_row_w<T, V>(ec, Gc, m0, J, Ko, omega, wz);
#pragma unroll
  for (int v = 0; v < V; ++v) yc[v] = add_rn(yc[v], wc[v]);
  // the x-neighbour beyond the segment; across a periodic x axis the red cell at the row's
  // other end, whose parent is coarse cell (hx-1, J, K) or (0, J, K)
  const bool px = (per & 1) != 0;
  T extra = T(0);
  if (s == 0) {
    if (m0 > 0) extra = add_rn(__ldg(yr + m0 - 1), mul_rn(omega, __ldg(ec + coarse_index(Gc, m0 - 1, J, K))));
    else if (px) extra = add_rn(__ldg(yr + G.hx - 1), mul_rn(omega, __ldg(ec + coarse_index(Gc, G.hx - 1, J, K))));
  } else {
    if (m0 + V < G.hx) extra = add_rn(__ldg(yr + m0 + V), mul_rn(omega, __ldg(ec + coarse_index(Gc, m0 + V, J, K))));
    else if (px) extra = add_rn(__ldg(yr), mul_rn(omega, __ldg(ec + coarse_index(Gc, 0, J, K))));
  }
  // (j-1)>>1 is J-1 for even j and J for odd j; (j+1)>>1 is J for even j and J+1 for odd j
  if (nb_has<0, PER>(G, j, k)) {
    load_vec(yr + m0 + nb_off<0, PER>(G, j, k), ym);
#pragma unroll
    for (int v = 0; v < V; ++v) ym[v] = add_rn(ym[v], (j & 1) ? wc[v] : wy[v]);
  } else {
#pragma unroll
    for (int v = 0; v < V; ++v) ym[v] = T(0);
  }
  if (nb_has<1, PER>(G, j, k)) {
    load_vec(yr + m0 + nb_off<1, PER>(G, j, k), yp);
#pragma unroll
    for (int v = 0; v < V; ++v) yp[v] = add_rn(yp[v], (j & 1) ? wy[v] : wc[v]);
  } else {
#pragma unroll
    for (int v = 0; v < V; ++v) yp[v] = T(0);
  }
  if (nb_has<2, PER>(G, j, k)) {
    load_vec(yr + m0 + nb_off<2, PER>(G, j, k), zm);
#pragma unroll
    for (int v = 0; v < V; ++v) zm[v] = add_rn(zm[v], (k & 1) ? wc[v] : wz[v]);
  } else {
#pragma unroll
    for (int v = 0; v < V; ++v) zm[v] = T(0);
  }
  if (nb_has<3, PER>(G, j, k)) {
    load_vec(yr + m0 + nb_off<3, PER>(G, j, k), zp);
#pragma unroll
    for (int v = 0; v < V; ++v) zp[v] = add_rn(zp[v], (k & 1) ? wz[v] : wc[v]);
  } else {
#pragma unroll
    for (int v = 0; v < V; ++v) zp[v] = T(0);
  }
#pragma unroll
  for (int v = 0; v < V; ++v) {
    T xm, xp;
    if (s == 0) {
      xm = (v == 0) ? extra : yc[(v + V - 1) % V];
      xp = yc[v];
    } else {
      xm = yc[v];
      xp = (v == V - 1) ? extra : yc[(v + 1) % V];
    }
    const T S = ((((xm + xp) + ym[v]) + yp[v]) + zm[v]) + zp[v];
    out[v] = (gv[v] + S) * invd[v];
  }
  store_vec(x + own, out);
}

// Index of coarse cell (I,J,K) in its level's storage (packed colours or natural order).
__device__ __forceinline__ long long coarse_index(const Geom& Gc, int I, int J, int K) {
  if (Gc.packed) {
    const int C = (I + J + K) & 1;
    return (long long)C * Gc.csz + ((long long)K * Gc.ny + J) * Gc.hx + (I >> 1);
  }
  return (long long)I + (long long)Gc.nx * ((long long)J + (long long)Gc.ny * K);
}

// Fused residual + averaging restriction (Sec. 3; sweeps "Resid" and "Restr" of Sec. 8.3) for
// coarse cell (I,J,K): the scaled residuals of its 8 children, summed in the order (dk, dj, di),
// times 1/4 give the coarse scaled right-hand side. RED_ONLY: the black cells were just updated
// by a black half-sweep, so their residuals are zero up to rounding and only the 4 red children
// are summed (same order otherwise).
template <typename T, bool RED_ONLY = false, bool PER = true>
__device__ __forceinline__ void resid_restrict_cell(const T* __restrict__ x, const T* __restrict__ g, const Geom& G,
                                                    T* __restrict__ gc, const Geom& Gc, int I, int J, int K) {
  T acc = T(0);
#pragma unroll
  for (int dk = 0; dk < 2; ++dk)
#pragma unroll
    for (int dj = 0; dj < 2; ++dj)
#pragma unroll
      for (int di = 0; di < 2; ++di) {
        const int j = 2 * J + dj, k = 2 * K + dk;
        const int c = (di + dj + dk) & 1;  // colour of child (2I+di, j, k)
        if (RED_ONLY && c == 1) continue;
        const long long row = ((long long)k * G.ny + j) * G.hx;
        const long long own = (long long)c * G.csz + row + I;
        const T S = nbsum_packed<T, PER>(x + (long long)(1 - c) * G.csz, G, row, I, di, j, k);
        const int d = diag_shift_packed(G, I, di, j, k);
        const T r = fmat(neg_diag<T>(d), __ldg(x + own), __ldg(g + own) + S);
        acc = acc + r;
      }
  gc[coarse_index(Gc, I, J, K)] = acc * T(0.25);
}

// resid_restrict_cell for V consecutive coarse cells I0 = V*iv .. I0+V-1 of coarse row (J,K)
// (fine rows whose length hx is a multiple of V). Their children in fine row (j,k) are the V
// consecutive entries I0.. of both colour arrays of that row, so every load is a 16-byte vector
// plus one scalar per colour; each coarse value is summed in the (dk, dj, di) order of
// resid_restrict_cell, so the results are identical.
template <typename T, int V, bool RED_ONLY = false, bool PER = true>
__device__ __forceinline__ void resid_restrict_vec(const T* __restrict__ x, const T* __restrict__ g, const Geom& G,
                                                   T* __restrict__ gc, const Geom& Gc, int iv, int J, int K) {
  const int per = PER ? G.per : 0;
  const int I0 = iv * V;
  T acc[V];
#pragma unroll
  for (int v = 0; v < V; ++v) acc[v] = T(0);
#pragma unroll
  for (int dk = 0; dk < 2; ++dk)
#pragma unroll
    for (int dj = 0; dj < 2; ++dj) {
      const int j = 2 * J + dj, k = 2 * K + dk;
      const long long row = ((long long)k * G.ny + j) * G.hx;
      int dyz = 0;
      if (j == 0) dyz += G.sh[2];
      if (j == G.ny - 1) dyz += G.sh[3];
      if (k == 0) dyz += G.sh[4];
      if (k == G.nz - 1) dyz += G.sh[5];
      // children di = 0 (colour c0) and di = 1 (colour c1) of the V coarse cells
      const int c0 = (dj + dk) & 1, c1 = c0 ^ 1;
      const T* r0 = x + (long long)c0 * G.csz + row;
      const T* r1 = x + (long long)c1 * G.csz + row;
      T x0[V], x1[V], g0[V], g1[V];
      load_vec(r0 + I0, x0);
      load_vec(r1 + I0, x1);
      const bool need0 = !RED_ONLY || c0 == 0, need1 = !RED_ONLY || c1 == 0;  // children computed
      if (need0) load_vec(g + (long long)c0 * G.csz + row + I0, g0);
      if (need1) load_vec(g + (long long)c1 * G.csz + row + I0, g1);
      // x-neighbour of child (I0, di=0) and of child (I0+V-1, di=1) (the row's other end across a
      // periodic x axis)
      const bool px = (per & 1) != 0;
      const T left = !need0 ? T(0) : (I0 > 0 ? __ldg(r1 + I0 - 1) : (px ? __ldg(r1 + G.hx - 1) : T(0)));
      const T right = !need1 ? T(0) : (I0 + V < G.hx ? __ldg(r0 + I0 + V) : (px ? __ldg(r0) : T(0)));
#pragma unroll
      for (int di = 0; di < 2; ++di) {
        if (di == 0 ? !need0 : !need1) continue;
        const T* y = di == 0 ? r1 : r0;  // the other colour's row
        T ym[V], yp[V], zm[V], zp[V];
        load_nb_vec<0, PER>(y, G, I0, j, k, ym);
        load_nb_vec<1, PER>(y, G, I0, j, k, yp);
        load_nb_vec<2, PER>(y, G, I0, j, k, zm);
        load_nb_vec<3, PER>(y, G, I0, j, k, zp);
        if constexpr (sizeof(T) == 8) {
          // FP64: the neighbour sum exactly in fixed point (fx_sum6), as in the FP64 half-sweep
          FxOp fo[V], fym[V], fyp[V], fzm[V], fzp[V];
#pragma unroll
          for (int v = 0; v < V; ++v) {
            fo[v] = fx_op(di == 0 ? x1[v] : x0[v]);  // the other colour's row segment
            fym[v] = fx_op(ym[v]);
            fyp[v] = fx_op(yp[v]);
            fzm[v] = fx_op(zm[v]);
            fzp[v] = fx_op(zp[v]);
          }
          const FxOp fe = fx_op(di == 0 ? left : right);
#pragma unroll
          for (int v = 0; v < V; ++v) {
            const int I = I0 + v;
            const FxOp xm = di == 0 ? (v == 0 ? fe : fo[(v + V - 1) % V]) : fo[v];
            const FxOp xp = di == 0 ? fo[v] : (v == V - 1 ? fe : fo[(v + 1) % V]);
            const FxOp op[6] = {xm, xp, fym[v], fyp[v], fzm[v], fzp[v]};
            const T xv = di == 0 ? x0[v] : x1[v], gv = di == 0 ? g0[v] : g1[v];
            int d = dyz;
            if (I == 0 && di == 0) d += G.sh[0];
            if (I == G.hx - 1 && di == 1) d += G.sh[1];
            acc[v] = acc[v] + fmat(neg_diag<T>(d), xv, gv + fx_sum6(op));
          }
        } else {
#pragma unroll
          for (int v = 0; v < V; ++v) {
            const int I = I0 + v;
            T xm, xp, xv, gv;
            if (di == 0) {  // cell i = 2I: x-neighbours 2I-1 (other colour, index I-1) and 2I+1 (index I)
              xm = (v == 0) ? left : x1[(v + V - 1) % V];
              xp = x1[v];
              xv = x0[v];
              gv = g0[v];
            } else {  // cell i = 2I+1: x-neighbours 2I (index I) and 2I+2 (index I+1)
              xm = x0[v];
              xp = (v == V - 1) ? right : x0[(v + 1) % V];
              xv = x1[v];
              gv = g1[v];
            }
            const T S = ((((xm + xp) + ym[v]) + yp[v]) + zm[v]) + zp[v];
            int d = dyz;
            if (I == 0 && di == 0) d += G.sh[0];
            if (I == G.hx - 1 && di == 1) d += G.sh[1];
            acc[v] = acc[v] + fmat(neg_diag<T>(d), xv, gv + S);
          }
        }
      }
    }
#pragma unroll
  for (int v = 0; v < V; ++v) gc[coarse_index(Gc, I0 + v, J, K)] = acc[v] * T(0.25);
}

// Constant prolongation with the magnified correction (Sec. 3): children += omega * e_parent.
// red_only: the black children are about to be overwritten by a black half-sweep that does not
// read them, so only the red ones are corrected.
template <typename T>
__device__ __forceinline__ void prolong_cell(T* __restrict__ x, const Geom& G, const T* __restrict__ ec,
                                             const Geom& Gc, T omega, int red_only, int I, int J, int K) {
  const T w = mul_rn(omega, __ldg(ec + coarse_index(Gc, I, J, K)));
#pragma unroll
  for (int dk = 0; dk < 2; ++dk)
#pragma unroll
    for (int dj = 0; dj < 2; ++dj)
#pragma unroll
      for (int di = 0; di < 2; ++di) {
        const int c = (di + dj + dk) & 1;
        if (red_only && c) continue;
        const long long idx = (long long)c * G.csz + ((long long)(2 * K + dk) * G.ny + (2 * J + dj)) * G.hx + I;
        x[idx] = add_rn(x[idx], w);
      }
}

// Scaled residual of cell m of packed row (c, j, k); returns r~ = g + sum - (6+d) x (single
// precision: the direct formula; the FP64 levels use the tiled walk below).
template <typename T, bool PER = true>
__device__ __forceinline__ T resid_packed(const T* __restrict__ x, const T* __restrict__ g, const Geom& G, int c,
                                          int m, int j, int k) {
  const int s = (j + k + c) & 1;
  const long long row = ((long long)k * G.ny + j) * G.hx;
  const long long own = (long long)c * G.csz + row + m;
  const int d = diag_shift_packed(G, m, s, j, k);
  const T S = nbsum_packed<T, PER>(x + (long long)(1 - c) * G.csz, G, row, m, s, j, k);
  return fmat(neg_diag<T>(d), __ldg(x + own), __ldg(g + own) + S);
}

// ---------------------------------------------------------------------------------------------
// Block-wide sum in a fixed order (warp shuffles, then warp 0 over the per-warp sums). Works for
// 1D and 2D blocks (threads flattened); result returned to every thread.
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double block_sum(double v, double* red /* >= 33 doubles of shared memory */) {
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int lane = tid & 31, w = tid >> 5;
  const int nw = (blockDim.x * blockDim.y + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    double t = (lane < nw) ? red[lane] : 0.0;
    t = warp_sum(t);
    if (lane == 0) red[32] = t;
  }
  __syncthreads();
  return red[32];
}

// Unpreconditioned CG (Hestenes-Stiefel) on the coarsest grid (Sec. 5.3), one CTA, in double,
// vectors in shared memory `sm` (4 n doubles), natural cell order. Operator: the scaled
// A_L / c_L, i.e. (6 + d_i) p_i - sum of interior neighbours. Stops when ||r|| <= rtol ||b|| or
// after maxit iterations; returns the iteration count.
// The same iteration for coarsest grids of at most 2 x 32 cells, one cell per thread of one warp
// (n <= 32) or two (named barrier 1 over the first 64 threads): each thread keeps its cell's x
// and r in registers, only p (which the neighbours read) lives in shared memory, and the dot
// products are warp_sum reductions, added over the two warps in a fixed order. On GB300 an FP64
// warp instruction takes 64 cycles of its sub-partition's FP64 pipe, so one cell per lane on two
// sub-partitions halves the issue time of the former two-cells-per-lane warp. It computes in the
// level's own precision: double for the FP64 cycle, float for the single-precision inner cycle of
// the mixed solver (stopping at kCoarseRtolF32; in double its FP64 operations took 37 us of
// 64-cycle issue per coarsest solve).
constexpr int kCoarseSmallCells = 64;

template <typename T>
__device__ int coarse_cg_small(T* __restrict__ xo, const T* __restrict__ bi, const Geom& G, double rtol, int maxit,
                               double* __restrict__ sm, double* __restrict__ red_d) {
  T* p = reinterpret_cast<T*>(sm);
  T* red = reinterpret_cast<T*>(red_d);
  const int nx = G.nx, ny = G.ny, nz = G.nz;
  const int n = nx * ny * nz;
  const int W = n > 32 ? 2 : 1;  // warps taking part (uniform)
  const int t = threadIdx.y * blockDim.x + threadIdx.x;
  const int lane = t & 31, w = t >> 5;
  const bool own = t < n;
  auto sync = [&]() {
    if (W == 2) asm volatile("bar.sync 1, 64;" ::: "memory");
    else __syncwarp();
  };
  int slot = 0;
  // sum of one value per thread over the W warps, in a fixed order
  auto psum = [&](T v) -> T {
    v = warp_sum(v);
    if (W == 1) return v;
    if (lane == 0) red[2 * slot + w] = v;
    sync();
    const T sv = red[2 * slot] + red[2 * slot + 1];
    slot ^= 1;  // the next sum writes the other pair; its barrier follows every read of this one
    return sv;
  };
  // the cell's neighbours (bits -x,+x,-y,+y,-z,+z, and their offsets: across a periodic axis the
  // cell at the opposite side) and -(6 + d)
  unsigned nbm = 0u;
  int no[6] = {-1, 1, -nx, nx, -nx * ny, nx * ny};
  T nd = T(0), xi = T(0), ri = T(0);
  if (own) {
    const int ix = t % nx, iy = (t / nx) % ny, iz = t / (nx * ny);
    const int ext[3] = {nx, ny, nz}, pos[3] = {ix, iy, iz}, st[3] = {1, nx, nx * ny};
    int d = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const bool per = (G.per >> a) & 1;
      if (pos[a] > 0) nbm |= 1u << (2 * a);
      else if (per) { nbm |= 1u << (2 * a); no[2 * a] = (ext[a] - 1) * st[a]; }
      else d += G.sh[2 * a];
      if (pos[a] < ext[a] - 1) nbm |= 2u << (2 * a);
      else if (per) { nbm |= 2u << (2 * a); no[2 * a + 1] = -(ext[a] - 1) * st[a]; }
      else d += G.sh[2 * a + 1];
    }
    nd = neg_diag<T>(d);
    ri = bi[t];
    p[t] = ri;
  }
  T rr = psum(ri * ri);  // its barrier also publishes p
  const T bnorm = sqrt(rr);
  const T stop = (T)rtol * bnorm;
  const T stop2 = stop * stop;  // ||r|| <= stop as ||r||^2 <= stop^2: no square root per iteration
  int it = 0;
  if (bnorm > T(0)) {
    while (it < maxit) {
      T a = T(0), pi = T(0);
      if (own) {
        pi = p[t];
        T S = T(0);
#pragma unroll
        for (int q = 0; q < 6; ++q)
          if (nbm & (1u << q)) S += p[t + no[q]];
        a = -nd * pi - S;
      }
      const T pap = psum(pi * a);  // after its barrier nobody reads p of this iteration again
      const T alpha = rr / pap;
      if (own) {
        xi = xi + alpha * pi;
        ri = ri - alpha * a;
      }
      const T rrn = psum(ri * ri);
      ++it;
      if (rrn <= stop2) break;
      const T beta = rrn / rr;
      if (own) p[t] = ri + beta * pi;
      sync();  // p complete before the next product reads its neighbours
      rr = rrn;
    }
  }
  if (own) xo[t] = (T)xi;
  return it;
}

template <typename T>
__device__ int coarse_cg_block(T* __restrict__ xo, const T* __restrict__ bi, const Geom& G, double rtol, int maxit,
                               double* sm, double* red) {
  const int nx = G.nx, ny = G.ny, nz = G.nz;
  const int n = nx * ny * nz;
  if (n <= kCoarseSmallCells) {  // uniform over the block; launches give such grids >= 32 (n <= 32) or 64 threads
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    return tid < (n > 32 ? 64 : 32) ? coarse_cg_small<T>(xo, bi, G, rtol, maxit, sm, red) : 0;
  }
  double* x = sm;
  double* r = x + n;
  double* p = r + n;
  double* ap = p + n;
  double loc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double b = (double)bi[i];
    x[i] = 0.0;
    r[i] = b;
    p[i] = b;
    loc += b * b;
  }
  double rr = block_sum(loc, red);
  const double bnorm = sqrt(rr);
  int it = 0;
  if (bnorm > 0.0) {
    while (it < maxit) {
      loc = 0.0;
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int ix = i % nx, iy = (i / nx) % ny, iz = i / (nx * ny), pl = nx * ny;
        const bool px = (G.per & 1) != 0, py = (G.per & 2) != 0, pz = (G.per & 4) != 0;
        int d = 0;
        double S = 0.0;
        if (ix > 0) S += p[i - 1]; else if (px) S += p[i + nx - 1]; else d += G.sh[0];
        if (ix < nx - 1) S += p[i + 1]; else if (px) S += p[i - (nx - 1)]; else d += G.sh[1];
        if (iy > 0) S += p[i - nx]; else if (py) S += p[i + (ny - 1) * nx]; else d += G.sh[2];
        if (iy < ny - 1) S += p[i + nx]; else if (py) S += p[i - (ny - 1) * nx]; else d += G.sh[3];
        if (iz > 0) S += p[i - pl]; else if (pz) S += p[i + (nz - 1) * pl]; else d += G.sh[4];
        if (iz < nz - 1) S += p[i + pl]; else if (pz) S += p[i - (nz - 1) * pl]; else d += G.sh[5];
        const double a = -neg_diag<double>(d) * p[i] - S;
        ap[i] = a;
        loc += p[i] * a;
      }
      const double pap = block_sum(loc, red);
      const double alpha = rr / pap;
      loc = 0.0;
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        x[i] = x[i] + alpha * p[i];
        const double ri = r[i] - alpha * ap[i];
        r[i] = ri;
        loc += ri * ri;
      }
      const double rrn = block_sum(loc, red);
      ++it;
      if (sqrt(rrn) <= rtol * bnorm) break;
      const double beta = rrn / rr;
      for (int i = threadIdx.x; i < n; i += blockDim.x) p[i] = r[i] + beta * p[i];
      __syncthreads();
      rr = rrn;
    }
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) xo[i] = (T)x[i];
  return it;
}

// ---------------------------------------------------------------------------------------------
// Residual-norm decomposition shared by the single-system and the batched launches: blocks of
// kResBX x kResBY threads, block lb of nb. Packed FP64 levels are cut into tiles of kResTM packed
// columns (one per lane) x kResTJ rows (one per warp) x kResTZ planes, both colours; block lb
// takes tiles lb, lb + nb, ... and each warp marches its row through the tile's planes; the
// operands of a plane pass through shared memory, so every value is read and converted once per
// tile (plus a one-cell halo) and serves the seven cells it enters from there. Packed
// single-precision levels are walked row by row in (k, j, colour) order, kResBY rows at a time,
// threads along the row; a natural-order level (single-level grid) cell by cell. Returns the
// thread's sum of r~^2; by MODE also writes r = r~ c0 in natural order (1) or float(r~ isc) in
// the level's own order (2).
constexpr int kResBX = 64, kResBY = 4;
constexpr int kResTM = 32, kResTJ = 8, kResTZ = 64;
static_assert(kResBX * kResBY == 32 * kResTJ && kResTM == 32, "one warp per tile row");

__host__ __device__ __forceinline__ long long resid_tile_count(const Geom& G, int* nmb = nullptr, int* njb = nullptr) {
  const int a = (G.hx + kResTM - 1) / kResTM, b = (G.ny + kResTJ - 1) / kResTJ, c = (G.nz + kResTZ - 1) / kResTZ;
  if (nmb) *nmb = a;
  if (njb) *njb = b;
  return (long long)a * b * c;
}

// The FP64 walk over the tiles of block lb of nb (packed level). Each tile plane is converted into
// shared memory (a ring of four planes, so one barrier per plane suffices: a plane is rewritten
// only after every warp has passed the barrier of the plane after the one that read it last),
// with a one-cell halo: rows j0-1 and j0+kResTJ loaded by the first and last warp, and the column
// beyond each end of a row loaded by the edge lanes in the colour the row's parity needs there.
//
// The residual r~ = g + (x_-x + x_+x + x_-y + x_+y + x_-z + x_+z) - D x_c (D = 6 + d) is summed in
// 64-bit fixed point with one exponent per ring row. The warp that stores a row (its 32 columns in
// both colours, and the halo column of its edge lanes) takes the largest biased exponent E_R of
// its values (one warp reduction) and stores each value as floor(+-significand 2^5 / 2^(E_R - e)),
// an integer in units of 2^(E_R - 1080) of magnitude below 2^58. A cell reads five rows: its own
// (both x neighbours and the centre, one unit, summed without shifts), the rows j-1 and j+1 of its
// plane and its row in the planes k-1 and k+1. Their exponents are the same for the whole warp;
// with E the largest of them (and of g's, unless the warp's right-hand side is zero) each of the
// five partial sums is shifted down to the unit 2^(E - 1080) and added, g is converted at that
// unit, and the integer is rounded once to a double (fx_to_double). The magnitudes stay below
// 2^62. Each truncation is a floor (two nested floors by powers of two are one), so x_-x, x_+x and
// D x_c lose less than 2 + D units of their row, the shift of their sum, each other neighbour and
// g less than one unit of 2^(E - 1080) each: the result lies within (8 + D) such units, i.e.
// (8 + D)/32 of an ulp of the largest value among the rows the cell reads (and its g), plus half an
// ulp of itself, of the exact residual. (Per-cell alignment, as in fx_residual, is
// bounded by the cell's own largest operand instead; the row exponent moves the alignment shifts
// from every use of a value to its conversion and took the 512^3 walk from 1.33 to 1.11 ms.) A cell
// whose rows hold an infinity or NaN (E = 2047) takes the direct FP64 formula from global memory.
constexpr int kResXR = kResTJ + 2, kResXC = kResTM + 2;

// MODE 3: the residual's restriction instead of its norm (the FP64 cycle's fused residual and
// restriction, Sec. 3): coarse cell (I, J, K) of the next level (gc, geometry Gc) becomes 1/4 of
// the sum of its eight children's scaled residuals. A lane's two cells (packed column m = I, both
// colours) are the children with i = 2I and 2I+1; it adds them over the planes 2K, 2K+1, and the
// warp of row 2J+1 hands its sums through shared memory to the warp of row 2J, which adds them
// after the next barrier and writes the coarse value (tiles start on even rows and planes, and
// levels with a coarser one have even extents, so the pairs never straddle tiles).
template <int MODE, bool PER>
__device__ __forceinline__ double resid_tiles_accum(const double* __restrict__ x, const double* __restrict__ g,
                                                    const Geom& G, long long lb, long long nb, double c0,
                                                    double* __restrict__ outn, float* __restrict__ outp, double isc,
                                                    int p2, double* __restrict__ gc = nullptr,
                                                    const Geom* Gc = nullptr) {
  // ring slot b, row r (0 and kResXR-1 are the halo rows), colour c, column col (0 and kResXC-1 are
  // the halo columns) at b * kSlot + r * kRow + c * kResXC + col
  constexpr int kRow = 2 * kResXC, kSlot = kResXR * kRow;
  __shared__ long long sT[4 * kSlot];  // values in units of their row's 2^(E_row - 1080)
  __shared__ int sE[4 * kResXR];       // E_row of ring slot b, row r at b * kResXR + r
  __shared__ double sR[MODE == 3 ? kResTJ / 2 * kResTM : 1];  // MODE 3: the odd rows' sums
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int w = tid >> 5, lane = tid & 31;
  int nmb, njb;
  const long long ntiles = resid_tile_count(G, &nmb, &njb);
  const int hx = G.hx, ny = G.ny, nz = G.nz;
  const long long plane = (long long)ny * hx;
  auto put = [&](int b, int r, int c, int col, long long v) { sT[b * kSlot + r * kRow + c * kResXC + col] = v; };
  double acc = 0.0;
  for (long long t = lb; t < ntiles; t += nb) {
    const int mb = (int)(t % nmb);
    const long long rest = t / nmb;
    const int jb = (int)(rest % njb);
    const int k0 = (int)(rest / njb) * kResTZ;
    const int k1 = min(k0 + kResTZ, nz);
    const int m = mb * kResTM + lane, j = jb * kResTJ + w;
    const bool live = m < hx && j < ny;
    const int hside = lane == 0 ? -1 : (lane == kResTM - 1 ? 1 : 0);
    const int dj = (j == 0 ? G.sh[2] : 0) + (j == ny - 1 ? G.sh[3] : 0);
    // The values of plane kk this thread contributes to the ring: its own column in both colours,
    // the column beyond the row's end (edge lanes; left end: red cells with s = 0 need black m-1
    // and black cells with s = 0 red m-1; right end likewise with s = 1), and the rows beyond the
    // tile (first and last warp); zero outside the level (the absent neighbours). Fetched one
    // plane ahead of their conversion into slot kk & 3.
    const long long col = (long long)j * hx + m;  // the column's offset within a colour plane
    // Across a periodic axis the values beyond the level's end are those at its other end: the
    // lane just past the last column (or the warp just past the last row) of a ragged tile, and
    // the halo column (row, plane) beyond a wall, load the wrapped column (row, plane) instead.
    const bool px = PER && (G.per & 1) != 0, py = PER && (G.per & 2) != 0, pz = PER && (G.per & 4) != 0;
    const int mw = (m == hx && px) ? 0 : m, jw = (j == ny && py) ? 0 : j;
    const bool lok = mw < hx && jw < ny;  // the thread's own column holds values (live or wrapped)
    const long long lcol = (long long)jw * hx + mw;
    int mh = m + hside;
    if (px) mh = mh < 0 ? hx - 1 : (mh >= hx ? mh - hx : mh);
    const bool hok = hside != 0 && mh >= 0 && mh < hx && j < ny;
    const long long hcoff = (long long)j * hx + mh;
    const bool edge = w == 0 || w == kResTJ - 1;
    int jr = w == 0 ? j - 1 : j + 1;
    if (py) jr = jr < 0 ? ny - 1 : (jr >= ny ? jr - ny : jr);
    const bool rok = edge && jr >= 0 && jr < ny && m < hx;
    const long long rcol = (long long)jr * hx + m;
    struct Raw {
      double own[2], halo, row[2];
    };
    auto hcol = [&](int kk) { return (hside < 0) == (((j + kk) & 1) != 0) ? 0 : 1; };
    auto fetch = [&](int kk, Raw& r) {
      const int kw = pz ? (kk < 0 ? nz - 1 : (kk >= nz ? kk - nz : kk)) : kk;
      const bool zin = kw >= 0 && kw < nz;
      const long long po = (long long)kw * plane;
#pragma unroll
      for (int c = 0; c < 2; ++c) r.own[c] = (lok && zin) ? __ldg(x + c * G.csz + po + lcol) : 0.0;
      r.halo = (hok && zin) ? __ldg(x + hcol(kk) * G.csz + po + hcoff) : 0.0;
      if (edge) {
#pragma unroll
        for (int c = 0; c < 2; ++c) r.row[c] = (rok && zin) ? __ldg(x + c * G.csz + po + rcol) : 0.0;
      }
    };
    auto gload = [&](int c, int kk) { return live ? __ldg(g + c * G.csz + (long long)kk * plane + col) : 0.0; };
    auto store = [&](int kk, const Raw& r) {
      const int b = kk & 3;
      unsigned em = max(fx_exp(r.own[0]), fx_exp(r.own[1]));
      if (hside != 0) em = max(em, fx_exp(r.halo));
      const int er = (int)__reduce_max_sync(0xffffffffu, em);
      if (lane == 0) sE[b * kResXR + w + 1] = er;
#pragma unroll
      for (int c = 0; c < 2; ++c) put(b, w + 1, c, lane + 1, fx_at(r.own[c], er));
      if (hside != 0) put(b, w + 1, hcol(kk), hside < 0 ? 0 : kResXC - 1, fx_at(r.halo, er));
      if (edge) {
        const int rr = w == 0 ? 0 : kResXR - 1;
        const int eh = (int)__reduce_max_sync(0xffffffffu, max(fx_exp(r.row[0]), fx_exp(r.row[1])));
        if (lane == 0) sE[b * kResXR + rr] = eh;
#pragma unroll
        for (int c = 0; c < 2; ++c) put(b, rr, c, lane + 1, fx_at(r.row[c], eh));
      }
    };
    // MODE 3: this lane's sum over its two cells and the plane pair, kept by an even row until the
    // odd row's arrives
    double racc = 0.0, rkeep = 0.0;
    int kpend = -1;
    auto flush = [&]() {
      if (MODE == 3 && kpend >= 0 && (w & 1) == 0 && live)
        gc[coarse_index(*Gc, m, j >> 1, kpend)] = 0.25 * (rkeep + sR[(w >> 1) * kResTM + lane]);
      kpend = -1;
    };
    __syncthreads();  // the previous tile's last reads of the ring are done
    Raw pre;
    fetch(k0 - 1, pre);
    store(k0 - 1, pre);
    fetch(k0, pre);
    store(k0, pre);
    fetch(k0 + 1, pre);
    double gpre[2] = {gload(0, k0), gload(1, k0)};
    for (int k = k0; k < k1; ++k) {
      const Raw cur = pre;
      const double gv[2] = {gpre[0], gpre[1]};
      if (k + 2 <= k1) fetch(k + 2, pre);
      if (k + 1 < k1) {
        gpre[0] = gload(0, k + 1);
        gpre[1] = gload(1, k + 1);
      }
      store(k + 1, cur);
      __syncthreads();
      if (MODE == 3 && (k & 1) == 0) {
        flush();  // the pair of planes before: the odd row's sums were published by this barrier
        racc = 0.0;
      }
      // the two cells of this thread; G0: the right-hand side is zero in every cell of the warp's
      // row (most cells of a charged-particle problem carry no charge), so its term is left out,
      // a uniform branch (7.5 % of the walk's time at 512^3 with 1600 charged spheres)
      auto cells = [&](auto g0) {
        constexpr bool G0 = decltype(g0)::value;
        const int own = (w + 1) * kRow + lane + 1;
        const int B0 = (k & 3) * kSlot + own, BM = ((k - 1) & 3) * kSlot + own, BP = ((k + 1) & 3) * kSlot + own;
        // diagonal shift: the walls of this row and plane, then the x walls per cell
        const int dbase = dj + (k == 0 ? G.sh[4] : 0) + (k == nz - 1 ? G.sh[5] : 0);
        const int e0 = (k & 3) * kResXR + w + 1;
        const int eo = sE[e0], eym = sE[e0 - 1], eyp = sE[e0 + 1];
        const int ezm = sE[((k - 1) & 3) * kResXR + w + 1], ezp = sE[((k + 1) & 3) * kResXR + w + 1];
        const int E5 = max(max(max(eo, eym), max(eyp, ezm)), ezp);
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          const int s = (j + k + c) & 1, o = (1 - c) * kResXC;
          const int d = dbase + (m == 0 && s == 0 ? G.sh[0] : 0) + (m == hx - 1 && s == 1 ? G.sh[1] : 0);
          int E = E5;
          if (!G0) E = max(E, (int)fx_exp(gv[c]));
          auto al = [&](long long v, int ev) {
            const int dd = E - ev;
            return v >> (dd < 63 ? dd : 63);
          };
          // x neighbours: the other colour at m + s - 1 and m + s (columns shifted by the halo)
          const long long A = sT[B0 + o + s - 1] + sT[B0 + o + s] - (long long)(6 + d) * sT[B0 + c * kResXC];
          long long sum = al(A, eo) + al(sT[B0 + o - kRow], eym) + al(sT[B0 + o + kRow], eyp) + al(sT[BM + o], ezm) +
                          al(sT[BP + o], ezp);
          if (!G0) sum += fx_at(gv[c], E);
          const double rd = E == 2047 ? (double)resid_packed<double, PER>(x, g, G, c, m, j, k)
                                      : fx_to_double((unsigned long long)sum, E);
          if (MODE != 3) acc = fma(rd, rd, acc);
          if (MODE == 3) racc += rd;
          if (MODE == 1) outn[(long long)(2 * m + s) + (long long)G.nx * ((long long)j + (long long)ny * k)] = rd * c0;
          if (MODE == 2)
            outp[(long long)c * G.csz + k * plane + col] =
                p2 != kBadPow2 ? f32_of_scaled(rd, p2) : (float)(rd * isc);
        }
      };
      // zero tests on the bits (+-0; an FP64 compare would take the 1/64-rate FP64 pipe); non-live
      // lanes hold 0
      const bool g0 = __all_sync(0xffffffffu, ((fx_bits(gv[0]) | fx_bits(gv[1])) << 1) == 0ULL);
      if (live) {
        if (g0) cells(std::true_type{});
        else cells(std::false_type{});
      }
      if (MODE == 3 && (k & 1) == 1) {
        if (w & 1) sR[(w >> 1) * kResTM + lane] = racc;
        else rkeep = racc;
        kpend = k >> 1;
      }
    }
    if (MODE == 3) {
      __syncthreads();
      flush();
    }
  }
  return acc;
}

template <typename T, int MODE, bool POW2 = false, bool PER = true>
__device__ __forceinline__ double resid_norm_accum_impl(const T* __restrict__ x, const T* __restrict__ g,
                                                        const Geom& G, long long lb, long long nb, double c0,
                                                        double* __restrict__ outn, float* __restrict__ outp,
                                                        double isc, int p2) {
  double acc = 0.0;
  if (G.packed) {
    const long long rows = 2LL * G.nz * G.ny;
    for (long long rw = lb * kResBY + threadIdx.y; rw < rows; rw += nb * kResBY) {
      const int k = (int)(rw / (2LL * G.ny));
      const int rem = (int)(rw - 2LL * G.ny * k);
      const int j = rem >> 1, c = rem & 1;
      const int s = (j + k + c) & 1;
      const long long row = ((long long)k * G.ny + j) * G.hx;
      for (int m = threadIdx.x; m < G.hx; m += kResBX) {
        const double rd = (double)resid_packed<T, PER>(x, g, G, c, m, j, k);
        acc = fma(rd, rd, acc);
        if (MODE == 1) outn[(long long)(2 * m + s) + (long long)G.nx * ((long long)j + (long long)G.ny * k)] = rd * c0;
        if (MODE == 2) outp[(long long)c * G.csz + row + m] = POW2 ? f32_of_scaled(rd, p2) : (float)(rd * isc);
      }
    }
  } else {
    const int nx = G.nx, ny = G.ny, nz = G.nz;
    const long long n = (long long)nx * ny * nz;
    const int tid = threadIdx.y * kResBX + threadIdx.x;
    for (long long i = lb * (kResBX * kResBY) + tid; i < n; i += nb * (kResBX * kResBY)) {
      const int ix = (int)(i % nx), iy = (int)((i / nx) % ny), iz = (int)(i / ((long long)nx * ny));
      int d = 0;
      const long long pl = (long long)nx * ny;
      const bool px = PER && (G.per & 1) != 0, py = PER && (G.per & 2) != 0, pz = PER && (G.per & 4) != 0;
      const T xm = ix > 0 ? x[i - 1] : (px ? x[i + (nx - 1)] : T(0));
      const T xp = ix < nx - 1 ? x[i + 1] : (px ? x[i - (nx - 1)] : T(0));
      const T ym = iy > 0 ? x[i - nx] : (py ? x[i + (long long)(ny - 1) * nx] : T(0));
      const T yp = iy < ny - 1 ? x[i + nx] : (py ? x[i - (long long)(ny - 1) * nx] : T(0));
      const T zm = iz > 0 ? x[i - pl] : (pz ? x[i + (nz - 1) * pl] : T(0));
      const T zp = iz < nz - 1 ? x[i + pl] : (pz ? x[i - (nz - 1) * pl] : T(0));
      if (ix == 0) d += G.sh[0];
      if (ix == nx - 1) d += G.sh[1];
      if (iy == 0) d += G.sh[2];
      if (iy == ny - 1) d += G.sh[3];
      if (iz == 0) d += G.sh[4];
      if (iz == nz - 1) d += G.sh[5];
      double rd;
      if constexpr (sizeof(T) == 8) {
        const FxOp op[8] = {fx_op(g[i]), fx_op(xm), fx_op(xp), fx_op(ym), fx_op(yp), fx_op(zm), fx_op(zp), fx_op(x[i])};
        rd = fx_residual(op, 6 + d);
      } else {
        const T S = ((((xm + xp) + ym) + yp) + zm) + zp;
        rd = (double)fmat(neg_diag<T>(d), x[i], g[i] + S);
      }
      acc = fma(rd, rd, acc);
      if (MODE == 1) outn[i] = rd * c0;
      if (MODE == 2) outp[i] = POW2 ? f32_of_scaled(rd, p2) : (float)(rd * isc);
    }
  }
  return acc;
}

// The residual walk; in MODE 2 the single-precision copy float(r~ isc) is formed by exponent
// arithmetic when isc is a power of two (the branch is uniform over the launch). PER = false:
// the tile walk compiled without periodic halos (levels without a periodic axis).
template <typename T, int MODE, bool PER = true>
__device__ __forceinline__ double resid_norm_accum(const T* __restrict__ x, const T* __restrict__ g, const Geom& G,
                                                   long long lb, long long nb, double c0, double* __restrict__ outn,
                                                   float* __restrict__ outp, double isc) {
  const int p2 = MODE == 2 ? pow2_exponent(isc) : kBadPow2;
  if constexpr (sizeof(T) == 8) {
    if (G.packed) return resid_tiles_accum<MODE, PER>(x, g, G, lb, nb, c0, outn, outp, isc, p2);
  }
  if (p2 != kBadPow2) return resid_norm_accum_impl<T, MODE, true, PER>(x, g, G, lb, nb, c0, outn, outp, isc, p2);
  return resid_norm_accum_impl<T, MODE, false, PER>(x, g, G, lb, nb, c0, outn, outp, isc, kBadPow2);
}

// The single-precision residual copy of a zero iterate (r~ = g exactly) over the same rows of
// The single-precision residual copy of a zero iterate (r~ = g exactly) for block lb of nb of a
// level: float(g isc) over the block's contiguous share of the level's values (both colour arrays
// of a packed level are one contiguous range, a natural-order level is one too), two values per
// thread and step with 16-byte loads where the arrays allow it. Every value is written once, the
// same values as the stencil would give.
__device__ __forceinline__ void resid_zero_rows(const double* __restrict__ g, const Geom& G, long long lb, long long nb,
                                                float* __restrict__ outp, double isc) {
  const int p2 = pow2_exponent(isc);
  auto cv = [&](double v) { return (p2 != kBadPow2) ? f32_of_scaled(v, p2) : (float)(v * isc); };
  const long long n = G.packed ? 2LL * G.csz : (long long)G.nx * G.ny * G.nz;
  const long long per = (((n + nb - 1) / nb) + 1) & ~1LL;  // an even share per block
  const long long a = lb * per, b = a + per < n ? a + per : n;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x, nt = blockDim.x * blockDim.y;
  const bool vec = ((reinterpret_cast<uintptr_t>(g) | reinterpret_cast<uintptr_t>(outp)) & 15) == 0;
  if (vec) {
    for (long long i = a + 2LL * tid; i < b; i += 2LL * nt) {
      if (i + 1 < b) {
        const double2 v = __ldg(reinterpret_cast<const double2*>(g + i));
        *reinterpret_cast<float2*>(outp + i) = make_float2(cv(v.x), cv(v.y));
      } else {
        outp[i] = cv(g[i]);
      }
    }
  } else {
    for (long long i = a + tid; i < b; i += nt) outp[i] = cv(g[i]);
  }
}

// Number of blocks of the residual-norm launch for level G (= the number of partial sums).
__host__ __device__ __forceinline__ int resid_norm_blocks(const Geom& G) {
  if (!G.packed) return 1;
  const long long tiles = resid_tile_count(G);
  return (int)(tiles < kMaxPartials ? tiles : kMaxPartials);
}

// Fixed-order sum of n partials by one block (strided per-thread sums, then block_sum).
__device__ __forceinline__ double sum_partials(const double* __restrict__ partials, int n, double* red) {
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int nt = blockDim.x * blockDim.y;
  double acc = 0.0;
  for (int i = tid; i < n; i += nt) acc += partials[i];
  return block_sum(acc, red);
}

}  // namespace ops
}  // namespace ccmg
