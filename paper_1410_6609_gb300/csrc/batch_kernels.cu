// batch_kernels.cu -- multigrid operations over many independent systems in one launch.
//
// Each launch walks a table of entries (one system at one level, see BEntry), each entry split
// into virtual blocks (start[] holds their offsets). The launch is persistent: a CTA takes
// virtual blocks blockIdx.x, blockIdx.x + gridDim.x, ..., finds the first one's entry by binary
// search and then advances the entry index as it goes (the offsets ascend), skips a virtual block
// whose system is inactive (converged or out of cycles), and runs the same per-thread body as
// the single-system kernel (level_ops.cuh) at the decoded coordinates. The residual norm reproduces
// the single-system block decomposition and reduction order per system, so every system's
// iterates are bit-identical to a solve of that system alone.
#include "level_ops.cuh"

namespace ccmg {
namespace {

using namespace ops;

__device__ __forceinline__ int find_entry(const int* __restrict__ start, int count, int b) {
  int lo = 0, hi = count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(start + mid) <= b) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Vector entries map a block to a chunk of one plane's (row, vector) pairs, taken row-major:
// the rows of a plane are contiguous in a colour array, so every lane has work and a warp's
// accesses are contiguous whatever the row length (entry.gx = chunks per plane, gy = 1). Other
// entries keep a 2D tile of (packed index, row).
__device__ __forceinline__ bool flat_coords(int lb, int gx, int per_row, int rows, int& a, int& row, int& plane) {
  const int nt = blockDim.x * blockDim.y;
  plane = lb / gx;
  const int idx = (lb - plane * gx) * nt + threadIdx.y * blockDim.x + threadIdx.x;
  row = idx / per_row;
  a = idx - row * per_row;
  return row < rows;
}

// Iteration over a launch's virtual blocks (see the file comment); `body` gets the entry and the
// block's index within it. Every thread of a CTA sees the same sequence, so bodies may use
// __syncthreads.
template <typename F>
__device__ __forceinline__ void for_vblocks(const BEntry* __restrict__ E, const int* __restrict__ start, int count,
                                            int total, const int* __restrict__ active, F body) {
  if ((int)blockIdx.x >= total) return;
  int e = find_entry(start, count, blockIdx.x);
  for (int b = blockIdx.x; b < total; b += gridDim.x) {
    while (__ldg(start + e + 1) <= b) ++e;
    if (!active[E[e].sys]) continue;
    body(E[e], e, b - __ldg(start + e));
  }
}

template <typename T, bool ZERO, bool PER>
__global__ void __launch_bounds__(256) kb_smooth(const BEntry* __restrict__ E, const int* __restrict__ start, int count,
                                                 int total, const int* __restrict__ active, InvDiag<T> inv,
                                                 int colour) {
  constexpr int V = 16 / sizeof(T);
  for_vblocks(E, start, count, total, active, [&](const BEntry& en, int, int lb) {
    const Geom G = en.G;
    T* x = (T*)en.x;
    const T* g = (const T*)en.g;
    if (en.vec) {
      int mv, j, k;
      if (flat_coords(lb, en.gx, G.hx / V, G.ny, mv, j, k)) smooth_vec<T, V, ZERO, PER>(x, g, G, inv, colour, mv, j, k);
    } else {
      const int bxi = lb % en.gx, rest = lb / en.gx;
      const int byi = rest % en.gy, k = rest / en.gy;
      const int j = byi * blockDim.y + threadIdx.y;
      const int m = bxi * blockDim.x + threadIdx.x;
      if (m < G.hx && j < G.ny) smooth_cell<T, ZERO, PER>(x, g, G, inv, colour, m, j, k);
    }
  });
}

// PER: compiled with periodic-axis support (launched when some system of the launch has one).
template <bool PER>
__global__ void __launch_bounds__(256) kb_smooth_prolong(const BEntry* __restrict__ E, const int* __restrict__ start,
                                                         int count, int total, const int* __restrict__ active,
                                                         InvDiag<float> inv, float omega) {
  for_vblocks(E, start, count, total, active, [&](const BEntry& en, int, int lb) {
    const Geom G = en.G;
    float* x = (float*)en.x;
    const float* g = (const float*)en.g;
    if (en.vec) {
      int mv, j, k;
      if (flat_coords(lb, en.gx, G.hx / 4, G.ny, mv, j, k))
        smooth_vec_prolong<float, 4, PER>(x, g, G, inv, (const float*)en.xc, en.Gc, omega, mv, j, k);
    } else {
      const int bxi = lb % en.gx, rest = lb / en.gx;
      const int byi = rest % en.gy, k = rest / en.gy;
      const int j = byi * blockDim.y + threadIdx.y;
      const int m = bxi * blockDim.x + threadIdx.x;
      if (m < G.hx && j < G.ny) smooth_cell<float, false, PER>(x, g, G, inv, 1, m, j, k);
    }
  });
}

template <typename T, bool RED_ONLY, bool PER>
__global__ void __launch_bounds__(256) kb_resid_restrict(const BEntry* __restrict__ E, const int* __restrict__ start,
                                                         int count, int total, const int* __restrict__ active) {
  for_vblocks(E, start, count, total, active, [&](const BEntry& en, int, int lb) {
    const Geom G = en.G, Gc = en.Gc;
    if (en.vec) {
      constexpr int V = 16 / sizeof(T);
      int iv, J, K;
      if (flat_coords(lb, en.gx, Gc.nx / V, Gc.ny, iv, J, K))
        resid_restrict_vec<T, V, RED_ONLY, PER>((const T*)en.x, (const T*)en.g, G, (T*)en.gc, Gc, iv, J, K);
    } else {
      const int bxi = lb % en.gx, rest = lb / en.gx;
      const int byi = rest % en.gy, K = rest / en.gy;
      const int I = bxi * blockDim.x + threadIdx.x;
      const int J = byi * blockDim.y + threadIdx.y;
      if (I < Gc.nx && J < Gc.ny)
        resid_restrict_cell<T, RED_ONLY, PER>((const T*)en.x, (const T*)en.g, G, (T*)en.gc, Gc, I, J, K);
    }
  });
}

template <typename T>
__global__ void __launch_bounds__(256) kb_prolong(const BEntry* __restrict__ E, const int* __restrict__ start, int count,
                                                  int total, const int* __restrict__ active, T omega, int red_only) {
  for_vblocks(E, start, count, total, active, [&](const BEntry& en, int, int lb) {
    const Geom G = en.G, Gc = en.Gc;
    int I, J, K;
    if (flat_coords(lb, en.gx, Gc.nx, Gc.ny, I, J, K))
      prolong_cell<T>((T*)en.x, G, (const T*)en.xc, Gc, omega, red_only, I, J, K);
  });
}

// One CTA per system: CG on the system's coarsest grid.
template <typename T>
__global__ void __launch_bounds__(1024) kb_coarse_cg(const BEntry* __restrict__ E, const int* __restrict__ active,
                                                     double rtol) {
  extern __shared__ double sm[];
  __shared__ double red[33];
  const BEntry& en = E[blockIdx.x];
  if (!active[en.sys]) return;
  const Geom G = en.G;
  const int n = G.nx * G.ny * G.nz;
  coarse_cg_block<T>((T*)en.x, (const T*)en.g, G, rtol, 2 * n, sm, red);
}

template <int MODE, bool PER>
__global__ void __launch_bounds__(256, 3) kb_resid_norm(const BEntry* __restrict__ E, const int* __restrict__ start,
                                                     int count, int total, const int* __restrict__ active,
                                                     const int* __restrict__ zero, const double* __restrict__ scal,
                                                     double* __restrict__ partials) {
  __shared__ double red[33];
  for_vblocks(E, start, count, total, active, [&](const BEntry& en, int e, int lb) {
    const int nb = __ldg(start + e + 1) - __ldg(start + e);
    const double isc = (MODE == 2) ? scal[kScalStride * en.sys + kSlotInvScale] : 0.0;
    if (zero[en.sys]) {  // a zero iterate: r = f, no stencil (kb_finalize takes the norm of f)
      if (MODE == 2) resid_zero_rows((const double*)en.g, en.G, lb, nb, (float*)en.aux, isc);
      if (threadIdx.x == 0 && threadIdx.y == 0) partials[__ldg(start + e) + lb] = 0.0;
      return;
    }
    double acc = resid_norm_accum<double, MODE, PER>((const double*)en.x, (const double*)en.g, en.G, lb, nb, 0.0, nullptr,
                                                (float*)en.aux, isc);
    acc = block_sum(acc, red);
    if (threadIdx.x == 0 && threadIdx.y == 0) partials[__ldg(start + e) + lb] = acc;
  });
}

__global__ void __launch_bounds__(256) kb_finalize(const BEntry* __restrict__ E, const int* __restrict__ start,
                                                   const int* __restrict__ active, const int* __restrict__ zero,
                                                   const double* __restrict__ partials, double* __restrict__ scal) {
  __shared__ double red[33];
  const int e = blockIdx.x;
  const int sys = E[e].sys;
  if (!active[sys]) return;
  double acc = sum_partials(partials + start[e], start[e + 1] - start[e], red);
  // a zero iterate has r = f exactly; its norm is the one taken when f was set (as a single
  // context reports it without evaluating the stencil)
  if (zero[sys]) acc = scal[kScalStride * sys + kSlotGsum];
  if (threadIdx.x == 0) {
    double* sc = scal + kScalStride * sys;
    sc[kSlotRsum] = acc;
    const double ref = sc[kSlotGsum];
    sc[kSlotRel] = ref > 0.0 ? sqrt(acc) / sqrt(ref) : sqrt(acc);
  }
}

// phi += s e; for a system whose iterate is zero (possibly never written) phi = fma(s, e, +0),
// without reading phi (as k_set_mixed). Systems stepping by recurrence (rec[sys]) are left to
// kb_defect_rec.
__global__ void __launch_bounds__(256) kb_update(const BEntry* __restrict__ E, const int* __restrict__ start, int count,
                                                 int total, const int* __restrict__ active, const int* __restrict__ rec,
                                                 const int* __restrict__ zero, const double* __restrict__ scal) {
  for_vblocks(E, start, count, total, active, [&](const BEntry& en, int e, int lb) {
    if (rec && rec[en.sys]) return;
    const long long nb = __ldg(start + e + 1) - __ldg(start + e);
    const Geom G = en.G;
    const long long n = G.packed ? 2 * G.csz : G.csz;
    double* x = (double*)en.x;
    const float* ev = (const float*)en.aux;
    const double sc = scal[kScalStride * en.sys + kSlotScale];
    const int p = pow2_exponent(sc);
    const long long i0 = (long long)lb * blockDim.x + threadIdx.x, st = nb * blockDim.x;
    const bool pow2 = p != kBadPow2 && p >= -kScaleExpLimit && p <= kScaleExpLimit;
    if (zero[en.sys]) {
      if (pow2)
        for (long long i = i0; i < n; i += st) {
          const double v = f64_of_scaled(ev[i], p);
          x[i] = (__double_as_longlong(v) == (long long)0x8000000000000000ULL) ? 0.0 : v;
        }
      else
        for (long long i = i0; i < n; i += st) x[i] = fma(sc, (double)ev[i], 0.0);
    } else if (pow2) {
      for (long long i = i0; i < n; i += st) x[i] = x[i] + f64_of_scaled(ev[i], p);
    } else {
      for (long long i = i0; i < n; i += st) x[i] = fma(sc, (double)ev[i], x[i]);
    }
  });
}

__global__ void kb_set_scale(const BEntry* __restrict__ E, int count, const int* __restrict__ active,
                             const int* __restrict__ rec, double* __restrict__ scal) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= count) return;
  const int sys = E[e].sys;
  if (!active[sys] || (rec && rec[sys])) return;
  const Geom G = E[e].G;
  const double n = (double)(G.packed ? 2 * G.csz : G.csz);
  double* sc = scal + kScalStride * sys;
  const double s = pow2_floor(sqrt(sc[kSlotRsum] / n));
  sc[kSlotScale] = s;
  sc[kSlotInvScale] = 1.0 / s;
}

// Persistent grid: per_sm CTAs per SM (of kSMs), at most the launch's virtual blocks.
constexpr int kSMs = 152;
int persist(const BLaunch& L, int per_sm = 8) {
  const long long g = (long long)kSMs * per_sm;
  return (int)(L.blocks < g ? L.blocks : g);
}

}  // namespace

template <typename T>
cudaError_t launch_b_smooth(const BLaunch& L, const int* active, const InvDiag<T>& inv, int colour, bool zero,
                            cudaStream_t s) {
  if (L.count == 0 || L.blocks == 0) return cudaSuccess;
  if (zero)  // no neighbour is read
    kb_smooth<T, true, false><<<persist(L), L.block, 0, s>>>(L.entries, L.start, L.count, L.blocks, active, inv, colour);
  else if (L.per)
    kb_smooth<T, false, true><<<persist(L), L.block, 0, s>>>(L.entries, L.start, L.count, L.blocks, active, inv, colour);
  else
    kb_smooth<T, false, false><<<persist(L), L.block, 0, s>>>(L.entries, L.start, L.count, L.blocks, active, inv, colour);
  return cudaGetLastError();
}

cudaError_t launch_b_smooth_prolong(const BLaunch& L, const int* active, const InvDiag<float>& inv, float omega,
                                    cudaStream_t s) {
  if (L.count == 0 || L.blocks == 0) return cudaSuccess;
  if (L.per)
    kb_smooth_prolong<true><<<persist(L), L.block, 0, s>>>(L.entries, L.start, L.count, L.blocks, active, inv, omega);
  else
    kb_smooth_prolong<false><<<persist(L), L.block, 0, s>>>(L.entries, L.start, L.count, L.blocks, active, inv, omega);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_b_resid_restrict(const BLaunch& L, const int* active, bool red_only, cudaStream_t s) {
  if (L.count == 0 || L.blocks == 0) return cudaSuccess;
  if (L.per) {
    if (red_only)
      kb_resid_restrict<T, true, true><<<persist(L), L.block, 0, s>>>(L.entries, L.start, L.count, L.blocks, active);
    else
      kb_resid_restrict<T, false, true><<<persist(L), L.block, 0, s>>>(L.entries, L.start, L.count, L.blocks, active);
  } else {
    if (red_only)
      kb_resid_restrict<T, true, false><<<persist(L), L.block, 0, s>>>(L.entries, L.start, L.count, L.blocks, active);
    else
      kb_resid_restrict<T, false, false><<<persist(L), L.block, 0, s>>>(L.entries, L.start, L.count, L.blocks, active);
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_b_prolong(const BLaunch& L, const int* active, T omega, bool red_only, cudaStream_t s) {
  if (L.count == 0 || L.blocks == 0) return cudaSuccess;
  kb_prolong<T><<<persist(L), L.block, 0, s>>>(L.entries, L.start, L.count, L.blocks, active, omega,
                                                red_only ? 1 : 0);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_b_coarse_cg(const BLaunch& L, const int* active, size_t smem, double rtol, cudaStream_t s) {
  if (L.count == 0) return cudaSuccess;
  kb_coarse_cg<T><<<L.count, L.block, smem, s>>>(L.entries, active, rtol);
  return cudaGetLastError();
}

cudaError_t prepare_b_coarse_cg() {
  const int bytes = (int)(4 * kMaxCoarseCells * sizeof(double));
  cudaError_t e = cudaFuncSetAttribute(kb_coarse_cg<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(kb_coarse_cg<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

cudaError_t launch_b_resid_norm(const BLaunch& L, const int* active, const int* zero, int mode, double* scal,
                                double* partials, cudaStream_t s) {
  if (L.count == 0 || L.blocks == 0) return cudaSuccess;
  const dim3 b(kResBX, kResBY, 1);
  const dim3 g = persist(L, 12);
  if (mode == 2 && L.per)
    kb_resid_norm<2, true><<<g, b, 0, s>>>(L.entries, L.start, L.count, L.blocks, active, zero, scal, partials);
  else if (mode == 2)
    kb_resid_norm<2, false><<<g, b, 0, s>>>(L.entries, L.start, L.count, L.blocks, active, zero, scal, partials);
  else if (L.per)
    kb_resid_norm<0, true><<<g, b, 0, s>>>(L.entries, L.start, L.count, L.blocks, active, zero, scal, partials);
  else
    kb_resid_norm<0, false><<<g, b, 0, s>>>(L.entries, L.start, L.count, L.blocks, active, zero, scal, partials);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  kb_finalize<<<L.count, 256, 0, s>>>(L.entries, L.start, active, zero, partials, scal);
  return cudaGetLastError();
}

cudaError_t launch_b_update(const BLaunch& L, const int* active, const int* rec, const int* zero, const double* scal,
                            cudaStream_t s) {
  if (L.count == 0 || L.blocks == 0) return cudaSuccess;
  kb_update<<<persist(L), 256, 0, s>>>(L.entries, L.start, L.count, L.blocks, active, rec, zero, scal);
  return cudaGetLastError();
}

cudaError_t launch_b_set_scale(const BLaunch& L, const int* active, const int* rec, double* scal, cudaStream_t s) {
  if (L.count == 0) return cudaSuccess;
  kb_set_scale<<<(L.count + 63) / 64, 64, 0, s>>>(L.entries, L.count, active, rec, scal);
  return cudaGetLastError();
}

#define CCMG_B_INSTANTIATE(T)                                                                                  \
  template cudaError_t launch_b_smooth<T>(const BLaunch&, const int*, const InvDiag<T>&, int, bool, cudaStream_t); \
  template cudaError_t launch_b_resid_restrict<T>(const BLaunch&, const int*, bool, cudaStream_t);              \
  template cudaError_t launch_b_prolong<T>(const BLaunch&, const int*, T, bool, cudaStream_t);                  \
  template cudaError_t launch_b_coarse_cg<T>(const BLaunch&, const int*, size_t, double, cudaStream_t);

CCMG_B_INSTANTIATE(double)
CCMG_B_INSTANTIATE(float)

}  // namespace ccmg
