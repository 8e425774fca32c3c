// static_scratch.cu -- residual norm of a caller's fields without any device allocation.
//
// Some callers cannot let a library call cudaMalloc or cudaFree: their device memory is owned
// and budgeted by another allocator (a framework's caching allocator or a fixed memory pool
// that has already claimed the device), or they run latency-critical loops in which an
// allocation call, which may synchronise the whole device, is not acceptable. For them this
// file offers a variant of the residual-norm reduction whose per-plane partial sums live in a
// file-scope static device array instead of a context's buffer. The paper has no counterpart:
// it is a deployment convenience.
//
// The array below is part of the module: every GPU that loads libccmg holds it (64 KiB) until
// the process exits, whether or not this entry point is called. Host code cannot use the
// array's name as a device address, so the first call on each device looks the address up with
// cudaGetSymbolAddress (with that device current) and caches it together with the CUDA context
// it belongs to: the address is a property of the context, so a call made under another context
// of the same device (after cudaDeviceReset, or under a context the caller created with the
// driver API) looks it up again instead of using a stale address.
#include <mutex>

#include <cuda.h>

#include "../../include/ccmg.h"

namespace {

constexpr int kStaticMaxPlanes = 4096;  // largest nz accepted
constexpr int kMaxDevices = 64;

// Two partial sums per z-plane: sum of r^2 and sum of f^2. Every call overwrites the entries of
// its own planes before reading them, so nothing has to start at zero.
__device__ __align__(256) double g_plane_partials[2 * kStaticMaxPlanes];

std::mutex g_mu;
struct ScratchAddr {
  CUcontext ctx;   // context the address was looked up in
  double* ptr;     // device address of g_plane_partials there
};
ScratchAddr g_scratch[kMaxDevices] = {};

// One block per z-plane: r = f - A_0 phi in natural order (Sec. 2.4 stencil with the walls
// folded in, periodic axes wrapping around), partial sums of r^2 and f^2 for the plane, fixed reduction order.
__global__ void __launch_bounds__(256) k_plane_residual(const double* __restrict__ phi, const double* __restrict__ f,
                                                        int nx, int ny, int nz, double c0, int4 sh_lo, int4 sh_hi,
                                                        double* __restrict__ partials) {
  __shared__ double red[2][32];
  const int k = blockIdx.x;
  const long long plane = (long long)nx * ny;
  const int sh[6] = {sh_lo.x, sh_lo.y, sh_lo.z, sh_lo.w, sh_hi.x, sh_hi.y};
  const int per = sh_hi.z;  // periodic axes (bit a: axis a wraps around)
  double rr = 0.0, ff = 0.0;
  for (long long t = threadIdx.x; t < plane; t += blockDim.x) {
    const int i = (int)(t % nx), j = (int)(t / nx);
    const long long p = t + plane * k;
    double S = 0.0;
    int d = 0;
    if (i > 0) S += phi[p - 1]; else if (per & 1) S += phi[p + (nx - 1)]; else d += sh[0];
    if (i < nx - 1) S += phi[p + 1]; else if (per & 1) S += phi[p - (nx - 1)]; else d += sh[1];
    if (j > 0) S += phi[p - nx]; else if (per & 2) S += phi[p + (long long)(ny - 1) * nx]; else d += sh[2];
    if (j < ny - 1) S += phi[p + nx]; else if (per & 2) S += phi[p - (long long)(ny - 1) * nx]; else d += sh[3];
    if (k > 0) S += phi[p - plane]; else if (per & 4) S += phi[p + (nz - 1) * plane]; else d += sh[4];
    if (k < nz - 1) S += phi[p + plane]; else if (per & 4) S += phi[p - (nz - 1) * plane]; else d += sh[5];
    const double fv = f[p];
    const double r = fv - c0 * ((double)(6 + d) * phi[p] - S);
    rr = fma(r, r, rr);
    ff = fma(fv, fv, ff);
  }
  for (int o = 16; o > 0; o >>= 1) {
    rr += __shfl_xor_sync(0xffffffffu, rr, o);
    ff += __shfl_xor_sync(0xffffffffu, ff, o);
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (lane == 0) {
    red[0][w] = rr;
    red[1][w] = ff;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int q = 0; q < nw; ++q) {
      a += red[0][q];
      b += red[1][q];
    }
    partials[2 * k] = a;
    partials[2 * k + 1] = b;
  }
}

// Sum the per-plane partials in plane order: out[0] = ||r|| / ||f|| (||r|| if f = 0), out[1] = ||r||.
__global__ void k_plane_finalize(const double* __restrict__ partials, int nz, double* __restrict__ out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double rr = 0.0, ff = 0.0;
  for (int k = 0; k < nz; ++k) {
    rr += partials[2 * k];
    ff += partials[2 * k + 1];
  }
  const double rn = sqrt(rr);
  out[0] = ff > 0.0 ? rn / sqrt(ff) : rn;
  out[1] = rn;
}

// The current CUDA context (cuCtxGetCurrent, fetched from the driver at run time so that the
// library does not link against libcuda).
using CtxGetCurrentFn = CUresult (*)(CUcontext*);
mg_status current_context(CUcontext* out) {
  static CtxGetCurrentFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !p)
      return MG_ERR_CUDA;
    fn = reinterpret_cast<CtxGetCurrentFn>(p);
  }
  *out = nullptr;
  return fn(out) == CUDA_SUCCESS && *out ? MG_OK : MG_ERR_CUDA;  // null: no context current
}

// Device address of g_plane_partials on the current device, looked up once per device and
// context (set-up on the first call, with that device current).
mg_status scratch_for_current_device(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return MG_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return MG_ERR_INVALID;
  CUcontext ctx = nullptr;
  mg_status st = current_context(&ctx);
  std::lock_guard<std::mutex> lock(g_mu);
  if (st == MG_OK && g_scratch[dev].ptr && g_scratch[dev].ctx == ctx) {
    *out = g_scratch[dev].ptr;
    return MG_OK;
  }
  // first call under this context (or no context current yet: the lookup initialises the
  // runtime's primary context of the device, which is then the current one)
  void* ptr = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&ptr, g_plane_partials);
  if (e != cudaSuccess || !ptr) return MG_ERR_CUDA;
  if ((st = current_context(&ctx)) != MG_OK) return st;
  g_scratch[dev] = ScratchAddr{ctx, (double*)ptr};
  *out = (double*)ptr;
  return MG_OK;
}

}  // namespace

extern "C" {

mg_status mg_residual_norm_static(int nx, int ny, int nz, double h, const int* h_bc_type6, const double* d_phi,
                                  const double* d_f, double* d_out2, void* stream) {
  // sizes first: nothing is touched for a request beyond the static scratch
  if (nz > kStaticMaxPlanes) return MG_ERR_INVALID;
  if (nx < 1 || ny < 1 || nz < 1 || !(h > 0.0)) return MG_ERR_INVALID;
  if (!h_bc_type6 || !d_phi || !d_f || !d_out2) return MG_ERR_INVALID;
  int sh[6], per = 0;
  for (int q = 0; q < 6; ++q) {
    const int t = h_bc_type6[q];
    if (t != MG_BC_DIRICHLET && t != MG_BC_NEUMANN && t != MG_BC_PERIODIC) return MG_ERR_INVALID;
    sh[q] = t == MG_BC_DIRICHLET ? 1 : (t == MG_BC_NEUMANN ? -1 : 0);
  }
  for (int a = 0; a < 3; ++a) {
    if ((h_bc_type6[2 * a] == MG_BC_PERIODIC) != (h_bc_type6[2 * a + 1] == MG_BC_PERIODIC)) return MG_ERR_INVALID;
    if (h_bc_type6[2 * a] == MG_BC_PERIODIC) per |= 1 << a;
  }
  double* scratch = nullptr;
  const mg_status st = scratch_for_current_device(&scratch);
  if (st != MG_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  k_plane_residual<<<nz, 256, 0, s>>>(d_phi, d_f, nx, ny, nz, 1.0 / (h * h), make_int4(sh[0], sh[1], sh[2], sh[3]),
                                       make_int4(sh[4], sh[5], per, 0), scratch);
  k_plane_finalize<<<1, 32, 0, s>>>(scratch, nz, d_out2);
  return cudaGetLastError() == cudaSuccess ? MG_OK : MG_ERR_CUDA;
}

}  // extern "C"
