// field_kernels.cu -- E-field, charged-sphere density, Coulomb force and their adjoints (sm_103a).
//
// Sec. 2.4 of the paper: the force on a particle is F = -h^3 sum_b grad(phi)(x_b) rho(x_b)
// (Eq. ElectrostatForce) with an O(h^2) finite-difference gradient; charges are mapped to cells by
// subsampling each cell into sf^3 sub-cells and counting the sub-cell centres inside the sphere.
// Here the gradient is the D3Q7 central difference, with wall ghost values Dirichlet 2g - phi and
// Neumann phi + h g, or (on request) the D3Q19 stencil of the same section where a cell's 18
// neighbours all lie in the domain. The potential is read from the finest level's storage (packed colours, or
// natural order for a single-level grid).
//
// The sub-cell inside test decides an integer count from floating point; it is evaluated with
// explicitly rounded operations (no contraction) in the order (((x-cx)^2 + (y-cy)^2) + (z-cz)^2)
// <= R^2, the sub-cell centre coordinate being (i + (2m+1)/(2 sf)) * h.
#include "ccmg_internal.cuh"
#include "level_ops.cuh"

namespace ccmg {
namespace {

using ops::host_pow2_exponent;
using ops::kBadPow2;
using ops::ldexp_rne;

struct SubOff {
  double o[8];  // (2m+1) / (2 sf), m < sf
};

__device__ __forceinline__ long long nat(const Geom& G, int i, int j, int k) {
  return (long long)i + (long long)G.nx * ((long long)j + (long long)G.ny * k);
}

// v modulo n in [0, n): the cell a coordinate along a periodic axis stands for.
__device__ __forceinline__ int wrap_mod(int v, int n) {
  const int r = v % n;
  return r < 0 ? r + n : r;
}
// The coordinate along axis a (0 x, 1 y, 2 z) wrapped where the axis is periodic (Sec. 2.4: the
// domain extended cyclically), unchanged otherwise.
__device__ __forceinline__ int wrap_axis(const Geom& G, int a, int v) {
  const int n = a == 0 ? G.nx : (a == 1 ? G.ny : G.nz);
  return ((G.per >> a) & 1) ? wrap_mod(v, n) : v;
}

__device__ __forceinline__ double ld_phi(const double* __restrict__ x, const Geom& G, int i, int j, int k) {
  if (G.packed) {
    const int c = (i + j + k) & 1;
    return __ldg(x + (long long)c * G.csz + ((long long)k * G.ny + j) * G.hx + (i >> 1));
  }
  return __ldg(x + nat(G, i, j, k));
}

// phi at the neighbour of (i,j,k) along axis a in direction dir, or the wall ghost value (across
// a periodic axis: the cell at the opposite side).
// FIELD: the faces may carry values per cell (FaceBC::field); the kernels are compiled both ways
// so that the common uniform case keeps its small register footprint.
// PER = false: compiled without periodic support (for kernels launched on levels without one).
template <bool FIELD = true, bool PER = true>
__device__ __forceinline__ double phi_nb(const double* __restrict__ x, const Geom& G, int i, int j, int k, int a,
                                         int dir, double here, double h, const FaceBC& bc) {
  int q[3] = {i, j, k};
  const int n[3] = {G.nx, G.ny, G.nz};
  q[a] += dir;
  if (q[a] < 0 || q[a] >= n[a]) {
    if (PER && ((G.per >> a) & 1)) {  // the cell at the opposite side
      q[a] = q[a] < 0 ? n[a] - 1 : 0;
      return ld_phi(x, G, q[0], q[1], q[2]);
    }
    const int face = 2 * a + (dir > 0 ? 1 : 0);
    const double g = FIELD ? face_value(bc, face, i, j, k, G.nx, G.ny) : bc.value[face];
    if (bc.type[face] == 0) return 2.0 * g - here;
    return here + h * g;
  }
  return ld_phi(x, G, q[0], q[1], q[2]);
}

// E_a = -(phi(+e_a) - phi(-e_a)) / (2h) at cell (i,j,k), a = 0..2. Warps whose cells are all
// interior take a path without any wall code (a warp vote, so the compiler cannot turn the rare
// ghost-value branches into FP64 work done by every cell); (dn - up) * inv2h equals
// -((up - dn) * inv2h) exactly.
// POW2: inv2h = 2^q2 (a power-of-two cell size); the interior products are then exponent shifts
// (ldexp_rne), equal to the FP64 multiply.
template <bool POW2, bool FIELD = true, bool PER = true>
__device__ __forceinline__ void efield_at(const double* __restrict__ x, const Geom& G, int i, int j, int k, double h,
                                          double inv2h, int q2, const FaceBC& bc, double E[3]) {
  const bool interior = i > 0 && i < G.nx - 1 && j > 0 && j < G.ny - 1 && k > 0 && k < G.nz - 1;
  if (__all_sync(__activemask(), interior)) {
    const double d0 = ld_phi(x, G, i - 1, j, k) - ld_phi(x, G, i + 1, j, k);
    const double d1 = ld_phi(x, G, i, j - 1, k) - ld_phi(x, G, i, j + 1, k);
    const double d2 = ld_phi(x, G, i, j, k - 1) - ld_phi(x, G, i, j, k + 1);
    E[0] = POW2 ? ldexp_rne(d0, q2) : d0 * inv2h;
    E[1] = POW2 ? ldexp_rne(d1, q2) : d1 * inv2h;
    E[2] = POW2 ? ldexp_rne(d2, q2) : d2 * inv2h;
  } else {
    const double here = ld_phi(x, G, i, j, k);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const double up = phi_nb<FIELD, PER>(x, G, i, j, k, a, +1, here, h, bc);
      const double dn = phi_nb<FIELD, PER>(x, G, i, j, k, a, -1, here, h, bc);
      E[a] = -((up - dn) * inv2h);
    }
  }
}

// The D3Q19 gradient (Sec. 2.4, "Coulomb force"): grad phi ~ (1/w_1) sum_q w_q phi(x + e_q) e_q / h
// with w_1 = 1/3, 1/18 for the 6 face and 1/36 for the 12 edge directions, taken in the order face
// directions (+x,-x,+y,-y,+z,-z), then (+a+b, -a-b, +a-b, -a+b) for (x,y), (x,z), (y,z); every
// product and sum rounded separately. For cells whose 18 neighbours all lie in the domain.
__constant__ int kD3Q19[18][3] = {{1, 0, 0},  {-1, 0, 0}, {0, 1, 0},  {0, -1, 0}, {0, 0, 1},   {0, 0, -1},
                                  {1, 1, 0},  {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}, {1, 0, 1},   {-1, 0, -1},
                                  {1, 0, -1}, {-1, 0, 1},  {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};

// All 18 neighbours exist: inside the domain, or across a periodic axis.
__device__ __forceinline__ bool d3q19_inside(const Geom& G, int i, int j, int k) {
  return ((G.per & 1) || (i > 0 && i < G.nx - 1)) && ((G.per & 2) || (j > 0 && j < G.ny - 1)) &&
         ((G.per & 4) || (k > 0 && k < G.nz - 1));
}

__device__ __forceinline__ void efield19_at(const double* __restrict__ x, const Geom& G, int i, int j, int k, double h,
                                            double E[3]) {
  double g[3] = {0.0, 0.0, 0.0};
#pragma unroll
  for (int q = 0; q < 18; ++q) {
    const int e0 = kD3Q19[q][0], e1 = kD3Q19[q][1], e2 = kD3Q19[q][2];
    const double w = q < 6 ? 1.0 / 18.0 : 1.0 / 36.0;
    // d3q19_inside holds: a coordinate leaves the domain only along a periodic axis
    const double wv = __dmul_rn(w, ld_phi(x, G, wrap_axis(G, 0, i + e0), wrap_axis(G, 1, j + e1), wrap_axis(G, 2, k + e2)));
    if (e0) g[0] = __dadd_rn(g[0], e0 > 0 ? wv : -wv);
    if (e1) g[1] = __dadd_rn(g[1], e1 > 0 ? wv : -wv);
    if (e2) g[2] = __dadd_rn(g[2], e2 > 0 ? wv : -wv);
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) E[a] = __ddiv_rn(-__dmul_rn(3.0, g[a]), h);  // 1 / w_1 = 3
}

// SFC > 0: the loops run exactly SFC steps (sf == SFC, the common s_f = 2 compiled alone, which
// keeps the kernels small); SFC == 0: any sf <= 8. Same operations in the same order either way.
template <int SFC = 0>
__device__ __forceinline__ int overlap_count(int i, int j, int k, double h, double cx, double cy, double cz, double R2,
                                             int sf, const SubOff& so) {
  constexpr int kMax = SFC > 0 ? SFC : 8;
  int cnt = 0;
#pragma unroll
  for (int mk = 0; mk < kMax; ++mk) {
    if (SFC == 0 && mk >= sf) break;
    const double dz = __dsub_rn(__dmul_rn(__dadd_rn((double)k, so.o[mk]), h), cz);
    const double dz2 = __dmul_rn(dz, dz);
#pragma unroll
    for (int mj = 0; mj < kMax; ++mj) {
      if (SFC == 0 && mj >= sf) break;
      const double dy = __dsub_rn(__dmul_rn(__dadd_rn((double)j, so.o[mj]), h), cy);
      const double dy2 = __dmul_rn(dy, dy);
#pragma unroll
      for (int mi = 0; mi < kMax; ++mi) {
        if (SFC == 0 && mi >= sf) break;
        const double dx = __dsub_rn(__dmul_rn(__dadd_rn((double)i, so.o[mi]), h), cx);
        const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), dy2), dz2);
        cnt += (d2 <= R2) ? 1 : 0;
      }
    }
  }
  return cnt;
}

// Cells [lo, hi] along one axis that can touch the sphere (every other cell has count 0),
// clipped to the domain unless the axis is periodic: there cells beyond an end stand for those at
// the opposite side (the sphere's periodic image), and the kernels keep the unwrapped coordinate
// for the sub-cell positions and wrap it where they touch memory.
__device__ __forceinline__ void cell_range(double c, double R, double h, int n, bool periodic, int& lo, int& hi) {
  int a = (int)floor((c - R) / h) - 1;
  int b = (int)floor((c + R) / h) + 1;
  lo = (a < 0 && !periodic) ? 0 : a;
  hi = (b > n - 1 && !periodic) ? n - 1 : b;
}

struct Box {
  int lo[3], hi[3], nb[3];
  long long ncell;
};

__device__ __forceinline__ Box sphere_box(const Geom& G, double h, const double* c, double R, int dilate) {
  Box B;
  const int n[3] = {G.nx, G.ny, G.nz};
  for (int a = 0; a < 3; ++a) {
    const bool per = (G.per >> a) & 1;
    cell_range(c[a], R, h, n[a], per, B.lo[a], B.hi[a]);
    B.lo[a] = per ? B.lo[a] - dilate : max(B.lo[a] - dilate, 0);
    B.hi[a] = per ? B.hi[a] + dilate : min(B.hi[a] + dilate, n[a] - 1);
    B.nb[a] = B.hi[a] - B.lo[a] + 1;
    if (B.nb[a] < 0) B.nb[a] = 0;
  }
  B.ncell = (long long)B.nb[0] * B.nb[1] * B.nb[2];
  return B;
}

// Natural-order index of the cell an (unwrapped) box coordinate stands for.
__device__ __forceinline__ long long nat_wrapped(const Geom& G, int i, int j, int k) {
  return (long long)wrap_axis(G, 0, i) +
         (long long)G.nx * ((long long)wrap_axis(G, 1, j) + (long long)G.ny * wrap_axis(G, 2, k));
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum of three per-thread values over the block, in a fixed order; result valid in thread 0.
__device__ void block_sum3(double v[3], double (*red)[3]) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  for (int a = 0; a < 3; ++a) v[a] = warp_sum(v[a]);
  if (lane == 0)
    for (int a = 0; a < 3; ++a) red[w][a] = v[a];
  __syncthreads();
  if (w == 0) {
    for (int a = 0; a < 3; ++a) {
      double t = lane < nw ? red[lane][a] : 0.0;
      v[a] = warp_sum(t);
    }
  }
}

// ---------------------------------------------------------------------------------------------

// E with the D3Q19 gradient where all 18 neighbours exist, D3Q7 central differences elsewhere.
__global__ void __launch_bounds__(256) k_efield19(const double* __restrict__ x, Geom G, double h, double inv2h,
                                                  FaceBC bc, double* __restrict__ E) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= G.nx || j >= G.ny) return;
  double e[3];
  if (d3q19_inside(G, i, j, k)) efield19_at(x, G, i, j, k, h, e);
  else efield_at<false>(x, G, i, j, k, h, inv2h, kBadPow2, bc, e);
  const long long N = (long long)G.nx * G.ny * G.nz;
  const long long p = nat(G, i, j, k);
  E[p] = e[0];
  E[N + p] = e[1];
  E[2 * N + p] = e[2];
}

template <bool POW2, bool FIELD>
__global__ void __launch_bounds__(256) k_efield(const double* __restrict__ x, Geom G, double h, double inv2h, int q2,
                                                FaceBC bc,
                                                double* __restrict__ E) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= G.nx || j >= G.ny) return;
  double e[3];
  efield_at<POW2, FIELD>(x, G, i, j, k, h, inv2h, q2, bc, e);
  const long long N = (long long)G.nx * G.ny * G.nz;
  const long long p = nat(G, i, j, k);
  E[p] = e[0];
  E[N + p] = e[1];
  E[2 * N + p] = e[2];
}

// The same on a packed level, two cells per thread: cells 2m and 2m+1 of row (j, k) sit at index m
// of the two colour arrays, so a warp's loads (the pair, its x-neighbours at m-1 and m+1, both
// colours in the four neighbour rows) and its 16-byte stores of each component are contiguous.
// Interior pairs take the differences directly, in efield_at's order; pairs at a wall call
// efield_at per cell.
template <bool POW2, bool FIELD, bool PER>
__global__ void __launch_bounds__(256) k_efield_pair(const double* __restrict__ x, Geom G, double h, double inv2h,
                                                     int q2, FaceBC bc, double* __restrict__ E) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (m >= G.hx || j >= G.ny) return;
  const int i0 = 2 * m;
  const long long N = (long long)G.nx * G.ny * G.nz;
  const long long p = (long long)i0 + (long long)G.nx * ((long long)j + (long long)G.ny * k);
  double e0[3], e1[3];
  const bool interior = m > 0 && m < G.hx - 1 && j > 0 && j < G.ny - 1 && k > 0 && k < G.nz - 1;
  if (__all_sync(__activemask(), interior)) {
    const int c0 = (i0 + j + k) & 1;  // colour of cell 2m; cell 2m+1 has the other
    const long long row = ((long long)k * G.ny + j) * G.hx + m;
    const long long plane = (long long)G.ny * G.hx;
    const double* a0 = x + (long long)c0 * G.csz;        // colour of 2m
    const double* a1 = x + (long long)(c0 ^ 1) * G.csz;  // colour of 2m+1 (and of 2m's y/z neighbours)
    const double p0 = __ldg(a0 + row), p1 = __ldg(a1 + row);
    const double xm = __ldg(a1 + row - 1), xp = __ldg(a0 + row + 1);  // cells 2m-1 and 2m+2
    const double d00 = xm - p1, d10 = p0 - xp;
    const double d01 = __ldg(a1 + row - G.hx) - __ldg(a1 + row + G.hx);
    const double d11 = __ldg(a0 + row - G.hx) - __ldg(a0 + row + G.hx);
    const double d02 = __ldg(a1 + row - plane) - __ldg(a1 + row + plane);
    const double d12 = __ldg(a0 + row - plane) - __ldg(a0 + row + plane);
    e0[0] = POW2 ? ldexp_rne(d00, q2) : d00 * inv2h;
    e0[1] = POW2 ? ldexp_rne(d01, q2) : d01 * inv2h;
    e0[2] = POW2 ? ldexp_rne(d02, q2) : d02 * inv2h;
    e1[0] = POW2 ? ldexp_rne(d10, q2) : d10 * inv2h;
    e1[1] = POW2 ? ldexp_rne(d11, q2) : d11 * inv2h;
    e1[2] = POW2 ? ldexp_rne(d12, q2) : d12 * inv2h;
  } else {
    efield_at<POW2, FIELD, PER>(x, G, i0, j, k, h, inv2h, q2, bc, e0);
    efield_at<POW2, FIELD, PER>(x, G, i0 + 1, j, k, h, inv2h, q2, bc, e1);
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) *reinterpret_cast<double2*>(E + a * N + p) = make_double2(e0[a], e1[a]);
}

// One CTA per sphere: rho(b) += density_s * count / sf^3 over the sphere's cells.
template <int SFC>
__global__ void __launch_bounds__(256) k_sphere_density(Geom G, double h, Spheres sp, int sf, SubOff so,
                                                        double* __restrict__ rho) {
  const int s = blockIdx.x;
  const double c[3] = {sp.c[3 * s], sp.c[3 * s + 1], sp.c[3 * s + 2]};
  const double R = sp.r[s];
  const double R2 = __dmul_rn(R, R);
  const double q = sp.q[s];
  const Box B = sphere_box(G, h, c, R, 0);
  const double sf3 = (double)(sf * sf * sf);
  for (long long t = threadIdx.x; t < B.ncell; t += blockDim.x) {
    const int i = B.lo[0] + (int)(t % B.nb[0]);
    const int j = B.lo[1] + (int)((t / B.nb[0]) % B.nb[1]);
    const int k = B.lo[2] + (int)(t / ((long long)B.nb[0] * B.nb[1]));
    const int cnt = overlap_count<SFC>(i, j, k, h, c[0], c[1], c[2], R2, sf, so);
    if (cnt == 0) continue;
    atomicAdd(rho + nat_wrapped(G, i, j, k), q * ((double)cnt / sf3));
  }
}

// One CTA per sphere: F_s = (h^3 density_s) * sum_b w_{s,b} E(x_b).
template <int SFC, bool FIELD>
__global__ void __launch_bounds__(256) k_force_gather(const double* __restrict__ x, Geom G, double h, double inv2h,
                                                      FaceBC bc, Spheres sp, int sf, SubOff so, int st19,
                                                      double* __restrict__ F) {
  __shared__ double red[32][3];
  const int s = blockIdx.x;
  const double c[3] = {sp.c[3 * s], sp.c[3 * s + 1], sp.c[3 * s + 2]};
  const double R = sp.r[s];
  const double R2 = __dmul_rn(R, R);
  const Box B = sphere_box(G, h, c, R, 0);
  const double sf3 = (double)(sf * sf * sf);
  double acc[3] = {0.0, 0.0, 0.0};
  for (long long t = threadIdx.x; t < B.ncell; t += blockDim.x) {
    const int i = B.lo[0] + (int)(t % B.nb[0]);
    const int j = B.lo[1] + (int)((t / B.nb[0]) % B.nb[1]);
    const int k = B.lo[2] + (int)(t / ((long long)B.nb[0] * B.nb[1]));
    const int cnt = overlap_count<SFC>(i, j, k, h, c[0], c[1], c[2], R2, sf, so);
    if (cnt == 0) continue;
    const double w = (double)cnt / sf3;
    const int iw = wrap_axis(G, 0, i), jw = wrap_axis(G, 1, j), kw = wrap_axis(G, 2, k);
    double e[3];
    if (st19 && d3q19_inside(G, iw, jw, kw)) efield19_at(x, G, iw, jw, kw, h, e);
    else efield_at<false, FIELD>(x, G, iw, jw, kw, h, inv2h, kBadPow2, bc, e);
    for (int a = 0; a < 3; ++a) acc[a] = acc[a] + w * e[a];
  }
  block_sum3(acc, red);
  if (threadIdx.x == 0) {
    const double pre = (h * h * h) * sp.q[s];
    for (int a = 0; a < 3; ++a) F[3 * s + a] = pre * acc[a];
  }
}

// Adjoint of k_force_gather for J = sum wF[s][a] F_s[a], as a gather over the sphere's cell box
// dilated by one: gphi(p) collects, from every cell b whose central difference reads p, the
// derivative of J through that difference; ghost values of wall cells route their part to the
// cell itself and to the wall value (Dirichlet ghost 2g - phi, Neumann phi + h g).
__global__ void __launch_bounds__(256) k_force_adjoint(const double* __restrict__ x, Geom G, double h, double inv2h,
                                                       FaceBC bc, Spheres sp, int sf, SubOff so,
                                                       const double* __restrict__ wF, double* __restrict__ gphi,
                                                       double* __restrict__ gdens, double* __restrict__ gbc) {
  __shared__ double red[32][3];
  const int s = blockIdx.x;
  const double c[3] = {sp.c[3 * s], sp.c[3 * s + 1], sp.c[3 * s + 2]};
  const double R = sp.r[s];
  const double R2 = __dmul_rn(R, R);
  const Box B = sphere_box(G, h, c, R, 1);
  const double sf3 = (double)(sf * sf * sf);
  const double pre = (h * h * h) * sp.q[s];
  const double wa[3] = {wF[3 * s], wF[3 * s + 1], wF[3 * s + 2]};
  const int n[3] = {G.nx, G.ny, G.nz};
  double fsum[3] = {0.0, 0.0, 0.0};
  for (long long t = threadIdx.x; t < B.ncell; t += blockDim.x) {
    const int p[3] = {B.lo[0] + (int)(t % B.nb[0]), B.lo[1] + (int)((t / B.nb[0]) % B.nb[1]),
                      B.lo[2] + (int)(t / ((long long)B.nb[0] * B.nb[1]))};
    double gp = 0.0;
    const int cnt_p = overlap_count(p[0], p[1], p[2], h, c[0], c[1], c[2], R2, sf, so);
    const double w_p = (double)cnt_p / sf3;
    const int pw[3] = {wrap_axis(G, 0, p[0]), wrap_axis(G, 1, p[1]), wrap_axis(G, 2, p[2])};
    if (cnt_p) {
      double e[3];
      efield_at<false>(x, G, pw[0], pw[1], pw[2], h, inv2h, kBadPow2, bc, e);
      for (int a = 0; a < 3; ++a) fsum[a] = fsum[a] + w_p * e[a];
    }
    for (int a = 0; a < 3; ++a) {
      // along a periodic axis every cell has both neighbours (in the box's unwrapped frame) and
      // no ghost
      const bool per = (G.per >> a) & 1;
      // p is the +e_a neighbour of b = p - e_a:  dE_a(b)/dphi(p) = -1/(2h)
      if (per || p[a] - 1 >= 0) {
        int b[3] = {p[0], p[1], p[2]};
        b[a] -= 1;
        const int cb = overlap_count(b[0], b[1], b[2], h, c[0], c[1], c[2], R2, sf, so);
        if (cb) gp = gp - (wa[a] * pre * ((double)cb / sf3)) * inv2h;
      }
      // p is the -e_a neighbour of b = p + e_a:  dE_a(b)/dphi(p) = +1/(2h)
      if (per || p[a] + 1 < n[a]) {
        int b[3] = {p[0], p[1], p[2]};
        b[a] += 1;
        const int cb = overlap_count(b[0], b[1], b[2], h, c[0], c[1], c[2], R2, sf, so);
        if (cb) gp = gp + (wa[a] * pre * ((double)cb / sf3)) * inv2h;
      }
      if (cnt_p && !per) {
        const double gE = wa[a] * pre * w_p;
        if (p[a] == 0) {  // -e_a neighbour is the ghost of face 2a
          const int face = 2 * a;
          const double g = gE * inv2h;
          if (bc.type[face] == 0) {
            atomicAdd(gbc + face, 2.0 * g);
            gp = gp - g;
          } else {
            atomicAdd(gbc + face, h * g);
            gp = gp + g;
          }
        }
        if (p[a] == n[a] - 1) {  // +e_a neighbour is the ghost of face 2a+1
          const int face = 2 * a + 1;
          const double g = -gE * inv2h;
          if (bc.type[face] == 0) {
            atomicAdd(gbc + face, 2.0 * g);
            gp = gp - g;
          } else {
            atomicAdd(gbc + face, h * g);
            gp = gp + g;
          }
        }
      }
    }
    if (gp != 0.0) atomicAdd(gphi + nat_wrapped(G, p[0], p[1], p[2]), gp);
  }
  block_sum3(fsum, red);
  if (threadIdx.x == 0) {
    const double h3 = h * h * h;
    double g = 0.0;
    for (int a = 0; a < 3; ++a) g = g + wa[a] * h3 * fsum[a];
    gdens[s] = g;
  }
}

// One CTA per sphere: gdens[s] = sum_b w_{s,b} gfield[b].
__global__ void __launch_bounds__(256) k_density_adjoint(Geom G, double h, Spheres sp, int sf, SubOff so,
                                                         const double* __restrict__ gf, double* __restrict__ gdens) {
  __shared__ double red[32][3];
  const int s = blockIdx.x;
  const double c[3] = {sp.c[3 * s], sp.c[3 * s + 1], sp.c[3 * s + 2]};
  const double R = sp.r[s];
  const double R2 = __dmul_rn(R, R);
  const Box B = sphere_box(G, h, c, R, 0);
  const double sf3 = (double)(sf * sf * sf);
  double acc[3] = {0.0, 0.0, 0.0};
  for (long long t = threadIdx.x; t < B.ncell; t += blockDim.x) {
    const int i = B.lo[0] + (int)(t % B.nb[0]);
    const int j = B.lo[1] + (int)((t / B.nb[0]) % B.nb[1]);
    const int k = B.lo[2] + (int)(t / ((long long)B.nb[0] * B.nb[1]));
    const int cnt = overlap_count(i, j, k, h, c[0], c[1], c[2], R2, sf, so);
    if (cnt == 0) continue;
    acc[0] = acc[0] + ((double)cnt / sf3) * gf[nat_wrapped(G, i, j, k)];
  }
  block_sum3(acc, red);
  if (threadIdx.x == 0) gdens[s] = acc[0];
}

__global__ void __launch_bounds__(256) k_scale_copy(const double* __restrict__ a, double* __restrict__ b, long long n,
                                                    double s) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    b[i] = a[i] * s;
}

// Six CTAs, one per wall: gbc[q] = sum over the wall's cells of lambda * (2/h^2 or 1/h); a
// periodic face has no value (0).
// With cell permittivities eps (the weighted operator): the sum of lambda * (2 eps/h^2 or eps/h).
__global__ void __launch_bounds__(256) k_face_sums(Geom G, double h, FaceBC bc, const double* __restrict__ lam,
                                                   const double* __restrict__ eps, double* __restrict__ gbc) {
  __shared__ double red[32][3];
  const int q = blockIdx.x;
  const int a = q >> 1;
  const int n[3] = {G.nx, G.ny, G.nz};
  const int fix = (q & 1) ? n[a] - 1 : 0;
  const int u = (a + 1) % 3, v = (a + 2) % 3;
  const long long cnt = (long long)n[u] * n[v];
  double acc[3] = {0.0, 0.0, 0.0};
  for (long long t = threadIdx.x; t < cnt; t += blockDim.x) {
    int p[3];
    p[a] = fix;
    p[u] = (int)(t % n[u]);
    p[v] = (int)(t / n[u]);
    const long long o = nat(G, p[0], p[1], p[2]);
    if (eps) acc[0] = acc[0] + lam[o] * (bc.type[q] == 0 ? 2.0 * eps[o] / (h * h) : eps[o] / h);
    else acc[0] = acc[0] + lam[o];
  }
  block_sum3(acc, red);
  if (threadIdx.x == 0)
    gbc[q] = bc.type[q] == 2 ? 0.0 : (eps ? acc[0] : acc[0] * (bc.type[q] == 0 ? 2.0 / (h * h) : 1.0 / h));
}

SubOff make_suboff(int sf) {
  SubOff so;
  for (int m = 0; m < 8; ++m) so.o[m] = m < sf ? (double)(2 * m + 1) / (double)(2 * sf) : 0.0;
  return so;
}

}  // namespace

cudaError_t launch_efield(const double* x, const Geom& G, double h, const FaceBC& bc, int stencil, double* E,
                          cudaStream_t s) {
  const double inv2h = 1.0 / (2.0 * h);
  const int q2 = host_pow2_exponent(inv2h);
  const bool fld = has_field(bc);
  if (stencil == 19) {
    const int bx = G.nx >= 128 ? 128 : (G.nx >= 64 ? 64 : 32);
    dim3 b(bx, 256 / bx, 1), g((G.nx + bx - 1) / bx, (G.ny + 256 / bx - 1) / (256 / bx), G.nz);
    k_efield19<<<g, b, 0, s>>>(x, G, h, inv2h, bc, E);
    return cudaGetLastError();
  }
  if (G.packed && reinterpret_cast<uintptr_t>(E) % 16 == 0) {
    const int bx = G.hx >= 128 ? 128 : (G.hx >= 64 ? 64 : 32);
    dim3 b(bx, 256 / bx, 1), g((G.hx + bx - 1) / bx, (G.ny + 256 / bx - 1) / (256 / bx), G.nz);
    if (G.per) {  // periodic axes (no per-cell values there; other faces may have them)
      if (q2 != kBadPow2) k_efield_pair<true, true, true><<<g, b, 0, s>>>(x, G, h, inv2h, q2, bc, E);
      else k_efield_pair<false, true, true><<<g, b, 0, s>>>(x, G, h, inv2h, q2, bc, E);
    } else if (fld) {
      if (q2 != kBadPow2) k_efield_pair<true, true, false><<<g, b, 0, s>>>(x, G, h, inv2h, q2, bc, E);
      else k_efield_pair<false, true, false><<<g, b, 0, s>>>(x, G, h, inv2h, q2, bc, E);
    } else {
      if (q2 != kBadPow2) k_efield_pair<true, false, false><<<g, b, 0, s>>>(x, G, h, inv2h, q2, bc, E);
      else k_efield_pair<false, false, false><<<g, b, 0, s>>>(x, G, h, inv2h, q2, bc, E);
    }
    return cudaGetLastError();
  }
  const int bx = G.nx >= 128 ? 128 : (G.nx >= 64 ? 64 : 32);
  dim3 b(bx, 256 / bx, 1), g((G.nx + bx - 1) / bx, (G.ny + 256 / bx - 1) / (256 / bx), G.nz);
  if (fld) {
    if (q2 != kBadPow2) k_efield<true, true><<<g, b, 0, s>>>(x, G, h, inv2h, q2, bc, E);
    else k_efield<false, true><<<g, b, 0, s>>>(x, G, h, inv2h, q2, bc, E);
  } else {
    if (q2 != kBadPow2) k_efield<true, false><<<g, b, 0, s>>>(x, G, h, inv2h, q2, bc, E);
    else k_efield<false, false><<<g, b, 0, s>>>(x, G, h, inv2h, q2, bc, E);
  }
  return cudaGetLastError();
}

cudaError_t launch_sphere_density(const Geom& G, double h, const Spheres& sp, int sf, double* rho, cudaStream_t s) {
  const long long N = (long long)G.nx * G.ny * G.nz;
  cudaError_t e = cudaMemsetAsync(rho, 0, (size_t)N * sizeof(double), s);
  if (e != cudaSuccess || sp.P == 0) return e;
  if (sf == 2) k_sphere_density<2><<<sp.P, 256, 0, s>>>(G, h, sp, sf, make_suboff(sf), rho);
  else if (sf == 1) k_sphere_density<1><<<sp.P, 256, 0, s>>>(G, h, sp, sf, make_suboff(sf), rho);
  else k_sphere_density<0><<<sp.P, 256, 0, s>>>(G, h, sp, sf, make_suboff(sf), rho);
  return cudaGetLastError();
}

cudaError_t launch_force_gather(const double* x, const Geom& G, double h, const FaceBC& bc, int stencil,
                                const Spheres& sp, int sf, double* F, cudaStream_t s) {
  if (sp.P == 0) return cudaSuccess;
  const int st19 = stencil == 19 ? 1 : 0;
  const double inv2h = 1.0 / (2.0 * h);
  const SubOff so = make_suboff(sf);
  if (has_field(bc)) {
    if (sf == 2) k_force_gather<2, true><<<sp.P, 256, 0, s>>>(x, G, h, inv2h, bc, sp, sf, so, st19, F);
    else if (sf == 1) k_force_gather<1, true><<<sp.P, 256, 0, s>>>(x, G, h, inv2h, bc, sp, sf, so, st19, F);
    else k_force_gather<0, true><<<sp.P, 256, 0, s>>>(x, G, h, inv2h, bc, sp, sf, so, st19, F);
  } else {
    if (sf == 2) k_force_gather<2, false><<<sp.P, 256, 0, s>>>(x, G, h, inv2h, bc, sp, sf, so, st19, F);
    else if (sf == 1) k_force_gather<1, false><<<sp.P, 256, 0, s>>>(x, G, h, inv2h, bc, sp, sf, so, st19, F);
    else k_force_gather<0, false><<<sp.P, 256, 0, s>>>(x, G, h, inv2h, bc, sp, sf, so, st19, F);
  }
  return cudaGetLastError();
}

cudaError_t launch_force_adjoint(const double* x, const Geom& G, double h, const FaceBC& bc, const Spheres& sp, int sf,
                                 const double* wF, double* gphi, double* gdens, double* gbc, cudaStream_t s) {
  const long long N = (long long)G.nx * G.ny * G.nz;
  cudaError_t e = cudaMemsetAsync(gphi, 0, (size_t)N * sizeof(double), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(gbc, 0, 6 * sizeof(double), s);
  if (e != cudaSuccess || sp.P == 0) return e;
  k_force_adjoint<<<sp.P, 256, 0, s>>>(x, G, h, 1.0 / (2.0 * h), bc, sp, sf, make_suboff(sf), wF, gphi, gdens, gbc);
  return cudaGetLastError();
}

cudaError_t launch_density_adjoint(const Geom& G, double h, const Spheres& sp, int sf, const double* gfield,
                                   double* gdens, cudaStream_t s) {
  if (sp.P == 0) return cudaSuccess;
  k_density_adjoint<<<sp.P, 256, 0, s>>>(G, h, sp, sf, make_suboff(sf), gfield, gdens);
  return cudaGetLastError();
}

cudaError_t launch_rhs_adjoint(const Geom& G, double h, double inv_eps, const FaceBC& bc, const double* eps,
                               const double* lam, double* grho, double* gbc, cudaStream_t s) {
  const long long N = (long long)G.nx * G.ny * G.nz;
  long long blocks = (N + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  k_scale_copy<<<(int)blocks, 256, 0, s>>>(lam, grho, N, eps ? 1.0 : inv_eps);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_face_sums<<<6, 256, 0, s>>>(G, h, bc, lam, eps, gbc);
  return cudaGetLastError();
}

}  // namespace ccmg
