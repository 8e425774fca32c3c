// level_kernels.cu -- per-level multigrid kernels for sm_103a (Sec. 3 and Sec. 4.3 of the paper).
//
// All kernels work on the checkerboard-separated level layout described in ccmg_internal.cuh
// (two colour arrays per field, unit-stride rows) with the scaled right-hand side g = f / c_l.
// Templated on the storage/arithmetic type T (double for the FP64 solver, float for the inner
// cycle of the mixed-precision defect correction). The coarsest-grid CG always computes in
// double.
#include "ccmg_internal.cuh"

namespace ccmg {
namespace {

__device__ __forceinline__ double fmat(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float fmat(float a, float b, float c) { return __fmaf_rn(a, b, c); }

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

// Sum of the six neighbours (in the order -x,+x,-y,+y,-z,+z; absent ones are zero) of the cell at
// index m of row `row` in colour c, where y points at the other colour's array.
template <typename T>
__device__ __forceinline__ T nbsum_packed(const T* __restrict__ y, const Geom& G, long long row, int m, int s, int j,
                                          int k) {
  const long long plane = (long long)G.ny * G.hx;
  const T* yr = y + row;
  const T xm = (m == 0 && s == 0) ? T(0) : __ldg(yr + m + s - 1);
  const T xp = (m == G.hx - 1 && s == 1) ? T(0) : __ldg(yr + m + s);
  const T ym = (j > 0) ? __ldg(yr + m - G.hx) : T(0);
  const T yp = (j < G.ny - 1) ? __ldg(yr + m + G.hx) : T(0);
  const T zm = (k > 0) ? __ldg(yr + m - plane) : T(0);
  const T zp = (k < G.nz - 1) ? __ldg(yr + m + plane) : T(0);
  return ((((xm + xp) + ym) + yp) + zm) + zp;
}

// ---------------------------------------------------------------------------------------------
// Red-black Gauss-Seidel half-sweep (Sec. 4.3): every cell of `colour` becomes the solution of
// its own row, phi = (g + sum of neighbours) / (6 + d). ZERO: the level's current iterate is
// zero (first sweep after restriction), so the neighbour sum is exactly zero and is not read.
template <typename T, bool ZERO>
__global__ void __launch_bounds__(256) k_smooth(T* __restrict__ x, const T* __restrict__ g, Geom G, InvDiag<T> inv,
                                                int colour) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (m >= G.hx || j >= G.ny) return;
  const int s = (j + k + colour) & 1;
  const long long row = ((long long)k * G.ny + j) * G.hx;
  const long long own = (long long)colour * G.csz + row + m;
  const int d = diag_shift_packed(G, m, s, j, k);
  T S = T(0);
  if (!ZERO) S = nbsum_packed(x + (long long)(1 - colour) * G.csz, G, row, m, s, j, k);
  x[own] = (__ldg(g + own) + S) * inv_of(inv, d);
}

// ---------------------------------------------------------------------------------------------
// Fused residual + averaging restriction (Sec. 3; sweeps "Resid" and "Restr" of Sec. 6.3). One
// thread per coarse cell (I,J,K): the scaled residuals of its 8 children, summed in the order
// (dk, dj, di), times 1/4 give the coarse scaled right-hand side.
template <typename T>
__global__ void __launch_bounds__(256) k_resid_restrict(const T* __restrict__ x, const T* __restrict__ g, Geom G,
                                                        T* __restrict__ gc, Geom Gc) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  const int J = blockIdx.y * blockDim.y + threadIdx.y;
  const int K = blockIdx.z;
  if (I >= Gc.nx || J >= Gc.ny) return;
  T acc = T(0);
#pragma unroll
  for (int dk = 0; dk < 2; ++dk)
#pragma unroll
    for (int dj = 0; dj < 2; ++dj)
#pragma unroll
      for (int di = 0; di < 2; ++di) {
        const int j = 2 * J + dj, k = 2 * K + dk;
        const int c = (di + dj + dk) & 1;  // colour of child (2I+di, j, k)
        const long long row = ((long long)k * G.ny + j) * G.hx;
        const long long own = (long long)c * G.csz + row + I;
        const T S = nbsum_packed(x + (long long)(1 - c) * G.csz, G, row, I, di, j, k);
        const int d = diag_shift_packed(G, I, di, j, k);
        const T r = fmat(-T(6 + d), __ldg(x + own), __ldg(g + own) + S);
        acc = acc + r;
      }
  const T val = acc * T(0.25);
  long long o;
  if (Gc.packed) {
    const int C = (I + J + K) & 1;
    o = (long long)C * Gc.csz + ((long long)K * Gc.ny + J) * Gc.hx + (I >> 1);
  } else {
    o = (long long)I + (long long)Gc.nx * ((long long)J + (long long)Gc.ny * K);
  }
  gc[o] = val;
}

// ---------------------------------------------------------------------------------------------
// Constant prolongation with the magnified correction (Sec. 3): children += omega * e_parent.
// red_only: the black children are about to be overwritten by a black half-sweep that does not
// read them, so only the red ones are corrected.
template <typename T>
__global__ void __launch_bounds__(256) k_prolong(T* __restrict__ x, Geom G, const T* __restrict__ ec, Geom Gc,
                                                 T omega, int red_only) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  const int J = blockIdx.y * blockDim.y + threadIdx.y;
  const int K = blockIdx.z;
  if (I >= Gc.nx || J >= Gc.ny) return;
  long long o;
  if (Gc.packed) {
    const int C = (I + J + K) & 1;
    o = (long long)C * Gc.csz + ((long long)K * Gc.ny + J) * Gc.hx + (I >> 1);
  } else {
    o = (long long)I + (long long)Gc.nx * ((long long)J + (long long)Gc.ny * K);
  }
  const T w = omega * __ldg(ec + o);
#pragma unroll
  for (int dk = 0; dk < 2; ++dk)
#pragma unroll
    for (int dj = 0; dj < 2; ++dj)
#pragma unroll
      for (int di = 0; di < 2; ++di) {
        const int c = (di + dj + dk) & 1;
        if (red_only && c) continue;
        const long long idx = (long long)c * G.csz + ((long long)(2 * K + dk) * G.ny + (2 * J + dj)) * G.hx + I;
        x[idx] = x[idx] + w;
      }
}

// ---------------------------------------------------------------------------------------------
// Block-wide sum in a fixed order (warp shuffles, then warp 0 over the per-warp sums).
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ double block_sum(double v, double* red /* >= 33 doubles of shared memory */) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
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

// Unpreconditioned CG (Hestenes-Stiefel) on the coarsest grid (Sec. 4.3), one CTA, in double,
// vectors in shared memory, natural cell order. Operator: the scaled A_L / c_L, i.e.
// (6 + d_i) p_i - sum of interior neighbours. Stops when ||r|| <= rtol ||b|| or after maxit.
template <typename T>
__global__ void __launch_bounds__(1024) k_coarse_cg(T* __restrict__ xo, const T* __restrict__ bi, Geom G, double rtol,
                                                    int maxit, int* iters) {
  extern __shared__ double sm[];
  __shared__ double red[33];
  const int nx = G.nx, ny = G.ny, nz = G.nz;
  const int n = nx * ny * nz;
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
        const int ix = i % nx, iy = (i / nx) % ny, iz = i / (nx * ny);
        int d = 0;
        double S = 0.0;
        if (ix > 0) S += p[i - 1]; else d += G.sh[0];
        if (ix < nx - 1) S += p[i + 1]; else d += G.sh[1];
        if (iy > 0) S += p[i - nx]; else d += G.sh[2];
        if (iy < ny - 1) S += p[i + nx]; else d += G.sh[3];
        if (iz > 0) S += p[i - nx * ny]; else d += G.sh[4];
        if (iz < nz - 1) S += p[i + nx * ny]; else d += G.sh[5];
        const double a = (double)(6 + d) * p[i] - S;
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
  if (threadIdx.x == 0 && iters) *iters = it;
}

// ---------------------------------------------------------------------------------------------
// Scaled residual over a packed level with per-block partial sums of r~^2 (the termination test
// of Algorithm 1). Grid-stride over rows (colour, k, j) so the partial count is the grid size.
template <typename T, int MODE>
__global__ void __launch_bounds__(256) k_resid_norm(const T* __restrict__ x, const T* __restrict__ g, Geom G,
                                                    double* __restrict__ partials, double c0,
                                                    double* __restrict__ outn, float* __restrict__ outp,
                                                    const double* __restrict__ inv_scale) {
  __shared__ double red[33];
  const int bx = blockDim.x, by = blockDim.y;
  const long long rows = 2LL * G.nz * G.ny;
  double isc = 0.0;
  if (MODE == 2) isc = inv_scale[0];
  double acc = 0.0;
  for (long long rw = (long long)blockIdx.x * by + threadIdx.y; rw < rows; rw += (long long)gridDim.x * by) {
    const int c = (int)(rw / ((long long)G.nz * G.ny));
    const int rem = (int)(rw - (long long)c * G.nz * G.ny);
    const int k = rem / G.ny, j = rem - k * G.ny;
    const int s = (j + k + c) & 1;
    const long long row = ((long long)k * G.ny + j) * G.hx;
    const T* y = x + (long long)(1 - c) * G.csz;
    for (int m = threadIdx.x; m < G.hx; m += bx) {
      const long long own = (long long)c * G.csz + row + m;
      const T S = nbsum_packed(y, G, row, m, s, j, k);
      const int d = diag_shift_packed(G, m, s, j, k);
      const T r = fmat(-T(6 + d), __ldg(x + own), __ldg(g + own) + S);
      const double rd = (double)r;
      acc = fma(rd, rd, acc);
      if (MODE == 1) outn[(long long)(2 * m + s) + (long long)G.nx * ((long long)j + (long long)G.ny * k)] = rd * c0;
      if (MODE == 2) outp[own] = (float)(rd * isc);
    }
  }
  // flatten the 2D block for the reduction
  const int tid = threadIdx.y * bx + threadIdx.x;
  const int lane = tid & 31, w = tid >> 5, nw = (bx * by + 31) >> 5;
  acc = warp_sum(acc);
  if (lane == 0) red[w] = acc;
  __syncthreads();
  if (w == 0) {
    double t = (lane < nw) ? red[lane] : 0.0;
    t = warp_sum(t);
    if (lane == 0) partials[blockIdx.x] = t;
  }
}

// Residual of a natural-order (single-level) grid: used when the finest level is also the
// coarsest. One block.
template <typename T, int MODE>
__global__ void __launch_bounds__(256) k_resid_norm_natural(const T* __restrict__ x, const T* __restrict__ g, Geom G,
                                                            double* __restrict__ partials, double c0,
                                                            double* __restrict__ outn, float* __restrict__ outp,
                                                            const double* __restrict__ inv_scale) {
  __shared__ double red[33];
  const int nx = G.nx, ny = G.ny, nz = G.nz;
  const long long n = (long long)nx * ny * nz;
  double isc = 0.0;
  if (MODE == 2) isc = inv_scale[0];
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int ix = (int)(i % nx), iy = (int)((i / nx) % ny), iz = (int)(i / ((long long)nx * ny));
    int d = 0;
    T S = T(0);
    S = S + (ix > 0 ? x[i - 1] : T(0));
    S = S + (ix < nx - 1 ? x[i + 1] : T(0));
    S = S + (iy > 0 ? x[i - nx] : T(0));
    S = S + (iy < ny - 1 ? x[i + nx] : T(0));
    S = S + (iz > 0 ? x[i - (long long)nx * ny] : T(0));
    S = S + (iz < nz - 1 ? x[i + (long long)nx * ny] : T(0));
    if (ix == 0) d += G.sh[0];
    if (ix == nx - 1) d += G.sh[1];
    if (iy == 0) d += G.sh[2];
    if (iy == ny - 1) d += G.sh[3];
    if (iz == 0) d += G.sh[4];
    if (iz == nz - 1) d += G.sh[5];
    const T r = fmat(-T(6 + d), x[i], g[i] + S);
    const double rd = (double)r;
    acc = fma(rd, rd, acc);
    if (MODE == 1) outn[i] = rd * c0;
    if (MODE == 2) outp[i] = (float)(rd * isc);
  }
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) partials[blockIdx.x] = acc;
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
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc += partials[i];
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) {
    scal[slot] = acc;
    if (slot_rel >= 0) {
      const double ref = scal[slot_ref];
      scal[slot_rel] = ref > 0.0 ? sqrt(acc) / sqrt(ref) : sqrt(acc);
    }
  }
}

__global__ void k_set_scale(double* scal, int src, int dst, double n) {
  const double v = sqrt(scal[src] / n);
  const double s = (v > 0.0 && v == v && v < 1e300) ? v : 1.0;
  scal[dst] = s;
  scal[dst + 1] = 1.0 / s;
}

// ---------------------------------------------------------------------------------------------
// Right-hand side (Sec. 2.4 and Sec. 4.3, "the RHS is adapted to the BCs ... only on the finest
// grid"): f = rho/eps + wall terms (term[q] precomputed per face), stored scaled, g = f * h^2.
struct WallTerms {
  double t[6];
};
template <typename T>
__global__ void __launch_bounds__(256) k_set_rhs(T* __restrict__ gout, Geom G, const double* __restrict__ rho,
                                                 double inv_eps, double hsq, WallTerms wt, int raw) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= G.nx || j >= G.ny) return;
  const long long p = (long long)i + (long long)G.nx * ((long long)j + (long long)G.ny * k);
  double v = rho[p];
  if (!raw) {
    v = v * inv_eps;
    if (i == 0) v = v + wt.t[0];
    if (i == G.nx - 1) v = v + wt.t[1];
    if (j == 0) v = v + wt.t[2];
    if (j == G.ny - 1) v = v + wt.t[3];
    if (k == 0) v = v + wt.t[4];
    if (k == G.nz - 1) v = v + wt.t[5];
  }
  long long o = p;
  if (G.packed) o = (long long)((i + j + k) & 1) * G.csz + ((long long)k * G.ny + j) * G.hx + (i >> 1);
  gout[o] = (T)(v * hsq);
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

__global__ void __launch_bounds__(256) k_update_mixed(double* __restrict__ x, const float* __restrict__ e, long long n,
                                                      const double* __restrict__ scal, int slot) {
  const double sc = scal[slot];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    x[i] = fma(sc, (double)e[i], x[i]);
}

// Launch shape for a (w x h x depth) thread grid with 256-thread blocks.
void shape(int w, int h, int depth, dim3& b, dim3& g) {
  const int bx = w >= 128 ? 128 : (w >= 64 ? 64 : 32);
  const int by = 256 / bx;
  b = dim3(bx, by, 1);
  g = dim3((w + bx - 1) / bx, (h + by - 1) / by, depth);
}

int resid_grid(const Geom& G) {
  const long long rows = 2LL * G.nz * G.ny;
  long long blocks = (rows + 1) / 2;
  const long long cap = 152 * 8;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  return (int)blocks;
}

}  // namespace

// ================================ launchers ================================================

template <typename T>
cudaError_t launch_smooth(T* x, const T* g, const Geom& G, const InvDiag<T>& inv, int colour, bool zero_start,
                          cudaStream_t s) {
  dim3 b, gr;
  shape(G.hx, G.ny, G.nz, b, gr);
  if (zero_start)
    k_smooth<T, true><<<gr, b, 0, s>>>(x, g, G, inv, colour);
  else
    k_smooth<T, false><<<gr, b, 0, s>>>(x, g, G, inv, colour);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_resid_restrict(const T* x, const T* g, const Geom& G, T* gc, const Geom& Gc, cudaStream_t s) {
  dim3 b, gr;
  shape(Gc.nx, Gc.ny, Gc.nz, b, gr);
  k_resid_restrict<T><<<gr, b, 0, s>>>(x, g, G, gc, Gc);
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
  if (G.packed) {
    const int grid = resid_grid(G);
    const int bx = G.hx >= 128 ? 128 : (G.hx >= 64 ? 64 : 32);
    dim3 b(bx, 256 / bx, 1);
    if (mode == 0) k_resid_norm<T, 0><<<grid, b, 0, s>>>(x, g, G, partials, c0, out_natural, out_packed, inv_scale);
    if (mode == 1) k_resid_norm<T, 1><<<grid, b, 0, s>>>(x, g, G, partials, c0, out_natural, out_packed, inv_scale);
    if (mode == 2) k_resid_norm<T, 2><<<grid, b, 0, s>>>(x, g, G, partials, c0, out_natural, out_packed, inv_scale);
    *nparts = grid;
  } else {
    if (mode == 0) k_resid_norm_natural<T, 0><<<1, 256, 0, s>>>(x, g, G, partials, c0, out_natural, out_packed, inv_scale);
    if (mode == 1) k_resid_norm_natural<T, 1><<<1, 256, 0, s>>>(x, g, G, partials, c0, out_natural, out_packed, inv_scale);
    if (mode == 2) k_resid_norm_natural<T, 2><<<1, 256, 0, s>>>(x, g, G, partials, c0, out_natural, out_packed, inv_scale);
    *nparts = 1;
  }
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

template <typename T>
cudaError_t launch_set_rhs(T* g, const Geom& G, const double* rho, double inv_eps, double h, const FaceBC& bc, int raw,
                           cudaStream_t s) {
  WallTerms wt;
  for (int q = 0; q < 6; ++q)
    wt.t[q] = bc.type[q] == 0 ? 2.0 * bc.value[q] / (h * h) : bc.value[q] / h;
  dim3 b, gr;
  shape(G.nx, G.ny, G.nz, b, gr);
  k_set_rhs<T><<<gr, b, 0, s>>>(g, G, rho, inv_eps, h * h, wt, raw);
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

cudaError_t launch_update_mixed(double* x, const float* e, long long n, const double* scal, int slot, cudaStream_t s) {
  long long blocks = (n + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (blocks < 1) blocks = 1;
  k_update_mixed<<<(int)blocks, 256, 0, s>>>(x, e, n, scal, slot);
  return cudaGetLastError();
}

#define CCMG_INSTANTIATE(T)                                                                                         \
  template cudaError_t launch_smooth<T>(T*, const T*, const Geom&, const InvDiag<T>&, int, bool, cudaStream_t);     \
  template cudaError_t launch_resid_restrict<T>(const T*, const T*, const Geom&, T*, const Geom&, cudaStream_t);    \
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
