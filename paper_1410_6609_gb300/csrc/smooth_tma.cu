// smooth_tma.cu -- single-precision red-black Gauss-Seidel half-sweep with TMA z-slab staging
// (sm_103a).
//
// The half-sweep of Sec. 4.3 (phi_i = (g_i + sum of neighbours) / (6 + d_i) on every cell of one
// colour) reads the other colour's array around each cell: the same row for the x-neighbours,
// rows j+-1 and planes k+-1 for the rest. Here a CTA owns a tile of 32 x 4-cell vectors by 8
// rows and marches it through a slab of z-planes. The other colour's planes come into shared
// memory by TMA (cp.async.bulk.tensor, completion on an mbarrier per ring slot) as boxes of
// 136 x 10 floats (the tile plus a one-row and a 4-float x halo), together with the 128 x 8 box of
// the right-hand side one plane behind, in a ring of kSlots slots: planes k-1, k, k+1 are read
// while the next kSlots-3 are in flight. Out-of-range box elements (walls) arrive as zeros,
// which is exactly the absent-neighbour term of the folded boundary stencil. Each other-colour
// value is fetched from L2 once per CTA instead of five times per cell; results are stored
// straight from registers. The arithmetic is that of ops::smooth_vec (same operands, same
// order), so the results are bit-identical.
//
// Every wait on an mbarrier is bounded (clock64 budget); a CTA that runs out sets the context's
// error flag, waits (bounded) for the copies it has in flight and returns.
#include "ccmg_internal.cuh"
#include "level_ops.cuh"

namespace ccmg {
namespace {

using ops::inv_of;

constexpr int kTX = 32;                    // 4-float vectors per tile row
constexpr int kTY = 8;                     // rows per tile
constexpr int kHaloX = 4;                  // floats on each side of the tile row (16-byte aligned box start)
constexpr int kBoxX = 4 * kTX + 2 * kHaloX;  // 136
constexpr int kBoxY = kTY + 2;             // 10
constexpr int kSlots = 6;
constexpr int kBoxBytes = kBoxX * kBoxY * 4;                 // 5440: other-colour box
constexpr int kGBoxBytes = 4 * kTX * kTY * 4;                // 4096: right-hand-side box
constexpr int kGOff = ((kBoxBytes + 127) / 128) * 128;       // 5504: the rhs box within a slot
constexpr int kSlotBytes = ((kGOff + kGBoxBytes + 127) / 128) * 128;  // 9600
constexpr int kSmemBytes = kSlots * kSlotBytes + 64;         // + the mbarriers
// tensor-copy destinations in shared memory must be 128-byte aligned
static_assert(kGOff % 128 == 0 && kSlotBytes % 128 == 0, "TMA destinations need 128-byte alignment");
constexpr long long kWaitCycles = 4000000000LL;           // wait budget, about 2 s at 2 GHz

__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_test(unsigned bar, unsigned parity) {
  unsigned done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(bar), "r"(parity)
      : "memory");
  return done != 0;
}
// Bounded wait for the phase of the given parity; false when `budget` clock cycles ran out.
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity, long long budget) {
  if (mbar_test(bar, parity)) return true;
  const long long t0 = clock64();
  for (;;) {
    if (mbar_test(bar, parity)) return true;
    if (clock64() - t0 > budget) return false;
  }
}
__device__ __forceinline__ void tma_load_box(unsigned dst, const CUtensorMap* map, int x, int y, int z,
                                             unsigned bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
          dst),
      "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}

struct Work {
  int x0, y0, k0, k1;  // tile origin (colour-array index, row) and planes [k0, k1)
};
__device__ __forceinline__ Work work_item(const Geom& G, int kz, long long w) {
  const int tiles_x = (G.hx + 4 * kTX - 1) / (4 * kTX);
  const int tiles_y = (G.ny + kTY - 1) / kTY;
  const long long per_slab = (long long)tiles_x * tiles_y;
  const int slab = (int)(w / per_slab);
  const int rem = (int)(w - per_slab * slab);
  Work t;
  t.x0 = (rem % tiles_x) * 4 * kTX;
  t.y0 = (rem / tiles_x) * kTY;
  t.k0 = slab * kz;
  t.k1 = min(t.k0 + kz, G.nz);
  return t;
}

// One persistent CTA of 32 x 8 threads; thread (tx, ty) owns the vector m0 = x0 + 4 tx of row
// y0 + ty in every plane of the item. Loads are numbered per CTA in issue order (seq); load n
// uses slot n % kSlots and completes phase n / kSlots of that slot's mbarrier. Load i of an item
// brings other-colour plane k0-1+i and, for i >= 2, right-hand-side plane k0-2+i. withhold >= 0
// (the failure-path self-test only) leaves that load of each CTA's first item unissued, so the
// waits for it run out of their `budget`.
__global__ void __launch_bounds__(kTX* kTY) k_smooth_tma(float* __restrict__ x, Geom G, InvDiag<float> inv,
                                                        int colour, int kz, long long nwork,
                                                        const __grid_constant__ CUtensorMap other,
                                                        const __grid_constant__ CUtensorMap rhs, int* err,
                                                        long long budget, int withhold) {
  extern __shared__ __align__(128) unsigned char smem[];
  float* ring = reinterpret_cast<float*>(smem);
  unsigned long long* bars = reinterpret_cast<unsigned long long*>(smem + kSlots * kSlotBytes);
  const int tx = threadIdx.x, ty = threadIdx.y;
  const bool leader = tx == 0 && ty == 0;
  if (leader) {
    for (int q = 0; q < kSlots; ++q) mbar_init(smem_addr(bars + q), 1);
    mbar_fence_init();
  }
  __syncthreads();

  const unsigned ring0 = smem_addr(ring);
  const unsigned bar0 = smem_addr(bars);
  float* const xo = x + (long long)colour * G.csz;
  int seq = 0;     // loads issued by this CTA before the current item
  int issued = 0;  // loads issued so far (leader)
  bool failed = false;

  for (long long w = blockIdx.x; w < nwork && !failed; w += gridDim.x) {
    const Work t = work_item(G, kz, w);
    const int np = (t.k1 - t.k0) + 2;  // other-colour planes k0-1 .. k1
    // load i of the item into slot (seq+i) % kSlots
    auto issue = [&](int i) {
      if (seq == 0 && i == withhold) return;
      const int n = seq + i;
      const int q = n % kSlots;
      const unsigned bar = bar0 + 8u * q;
      const unsigned dst = ring0 + (unsigned)(q * kSlotBytes);
      const bool with_rhs = i >= 2;
      mbar_expect_tx(bar, kBoxBytes + (with_rhs ? kGBoxBytes : 0));
      tma_load_box(dst, &other, t.x0 - kHaloX, t.y0 - 1, t.k0 - 1 + i, bar);
      if (with_rhs) tma_load_box(dst + kGOff, &rhs, t.x0, t.y0, t.k0 - 2 + i, bar);
      issued = n + 1;
    };
    __syncthreads();  // every thread is done with the previous item's slots
    if (leader)
      for (int i = 0; i < np && i < kSlots - 1; ++i) issue(i);

    const int m0 = t.x0 + 4 * tx;
    const int j = t.y0 + ty;
    const bool mine = m0 < G.hx && j < G.ny;
    for (int k = t.k0; k < t.k1; ++k) {
      const int i = k - t.k0 + 1;  // load index of plane k (k-1 is i-1; k+1 and g(k) are i+1)
      const long long row = ((long long)k * G.ny + j) * G.hx;
      bool ok = true;
      for (int d = (k == t.k0 ? -1 : 1); d <= 1; ++d) {
        const int n = seq + i + d;
        ok = ok && mbar_wait(bar0 + 8u * (unsigned)(n % kSlots), (unsigned)((n / kSlots) & 1), budget);
      }
      // the barrier also retires iteration k-1, freeing the slot of load i-2 for load i+kSlots-2
      if (__syncthreads_or(!ok)) {
        failed = true;
        break;
      }
      if (leader && i + kSlots - 2 < np) issue(i + kSlots - 2);
      if (mine) {
        const int s = (j + k + colour) & 1;
        const float* pk = ring + (size_t)((seq + i) % kSlots) * (kSlotBytes / 4);
        const float* pm = ring + (size_t)((seq + i - 1) % kSlots) * (kSlotBytes / 4);
        const float* pp = ring + (size_t)((seq + i + 1) % kSlots) * (kSlotBytes / 4);
        const int c0 = (ty + 1) * kBoxX + kHaloX + 4 * tx;
        const float4 yc = *reinterpret_cast<const float4*>(pk + c0);
        const float4 ym = *reinterpret_cast<const float4*>(pk + c0 - kBoxX);
        const float4 yp = *reinterpret_cast<const float4*>(pk + c0 + kBoxX);
        const float4 zm = *reinterpret_cast<const float4*>(pm + c0);
        const float4 zp = *reinterpret_cast<const float4*>(pp + c0);
        const float extra = s == 0 ? pk[c0 - 1] : pk[c0 + 4];
        const float4 gv = *reinterpret_cast<const float4*>(pp + kGOff / 4 + ty * (4 * kTX) + 4 * tx);
        const float ycv[4] = {yc.x, yc.y, yc.z, yc.w}, ymv[4] = {ym.x, ym.y, ym.z, ym.w};
        const float ypv[4] = {yp.x, yp.y, yp.z, yp.w}, zmv[4] = {zm.x, zm.y, zm.z, zm.w};
        const float zpv[4] = {zp.x, zp.y, zp.z, zp.w}, gvv[4] = {gv.x, gv.y, gv.z, gv.w};
        int dbase = 0;
        if (j == 0) dbase += G.sh[2];
        if (j == G.ny - 1) dbase += G.sh[3];
        if (k == 0) dbase += G.sh[4];
        if (k == G.nz - 1) dbase += G.sh[5];
        float out[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          float xm, xp;
          if (s == 0) {
            xm = (e == 0) ? extra : ycv[e - 1 < 0 ? 0 : e - 1];
            xp = ycv[e];
          } else {
            xm = ycv[e];
            xp = (e == 3) ? extra : ycv[e + 1 > 3 ? 3 : e + 1];
          }
          const float S = ((((xm + xp) + ymv[e]) + ypv[e]) + zmv[e]) + zpv[e];
          int d = dbase;
          if (m0 + e == 0 && s == 0) d += G.sh[0];
          if (m0 + e == G.hx - 1 && s == 1) d += G.sh[1];
          out[e] = (gvv[e] + S) * inv_of(inv, d);
        }
        *reinterpret_cast<float4*>(xo + row + m0) = make_float4(out[0], out[1], out[2], out[3]);
      }
    }
    seq += np;
  }

  if (failed && leader) {
    atomicExch(err, 1);
    // let the copies already issued land before the CTA's shared memory is released (bounded)
    for (int n = issued > kSlots ? issued - kSlots : 0; n < issued; ++n)
      if (!(seq == 0 && n == withhold)) mbar_wait(bar0 + 8u * (unsigned)(n % kSlots), (unsigned)((n / kSlots) & 1), budget);
  }
}

}  // namespace

bool tma_sweep_applies(const Geom& G) {
  // rows of whole 4-float vectors and enough planes to march
  return G.packed && (G.hx % 4) == 0 && G.nz >= 8 && (long long)G.hx * G.ny * G.nz >= (1LL << 16);
}

bool tma_sweep_pays(const Geom& G) {
  // measured on GB300: ahead of the direct-load kernel at 512^3 (2^25 cells per colour), even at
  // 256^3, behind below that (too few tiles to keep every SM's copies in flight)
  return tma_sweep_applies(G) && (long long)G.hx * G.ny * G.nz >= (1LL << 24);
}

cudaError_t prepare_tma_sweep(TmaSweep& t, float* x, const float* g, const Geom& G, int device) {
  t.ok = 0;
  if (!tma_sweep_applies(G)) return cudaSuccess;
  using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  static EncodeFn encode = nullptr;
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess) return e;
    if (q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
    encode = reinterpret_cast<EncodeFn>(fn);
  }
  const cuuint64_t dims[3] = {(cuuint64_t)G.hx, (cuuint64_t)G.ny, (cuuint64_t)G.nz};
  const cuuint64_t strides[2] = {(cuuint64_t)G.hx * 4, (cuuint64_t)G.hx * G.ny * 4};
  const cuuint32_t box[3] = {(cuuint32_t)kBoxX, (cuuint32_t)kBoxY, 1};
  const cuuint32_t gbox[3] = {(cuuint32_t)(4 * kTX), (cuuint32_t)kTY, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  for (int c = 0; c < 2; ++c) {
    float* base = x + (long long)(1 - c) * G.csz;          // a colour-c sweep reads colour 1-c
    float* gbase = const_cast<float*>(g) + (long long)c * G.csz;  // and its own right-hand side
    if (reinterpret_cast<uintptr_t>(base) % 16 != 0 || reinterpret_cast<uintptr_t>(gbase) % 16 != 0)
      return cudaSuccess;
    CUresult r = encode(&t.other[c], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    r = encode(&t.rhs[c], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, gbase, dims, strides, gbox, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  }
  cudaError_t e = cudaFuncSetAttribute(k_smooth_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
  if (e != cudaSuccess) return e;
  int per_sm = 0, sms = 0;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_smooth_tma, kTX * kTY, kSmemBytes)) != cudaSuccess)
    return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device)) != cudaSuccess) return e;
  if (per_sm < 1) return cudaSuccess;
  const long long tiles = (long long)((G.hx + 4 * kTX - 1) / (4 * kTX)) * ((G.ny + kTY - 1) / kTY);
  const long long slots = (long long)per_sm * sms;
  // planes per item: at least four items per resident CTA, at most 32 planes
  int kz = 32;
  while (kz > 8 && tiles * ((G.nz + kz - 1) / kz) < 4 * slots) kz /= 2;
  t.kz = kz;
  t.nwork = tiles * ((G.nz + kz - 1) / kz);
  t.grid = (int)(t.nwork < slots ? t.nwork : slots);
  t.ok = 1;
  return cudaSuccess;
}

cudaError_t launch_smooth_tma(float* x, const Geom& G, const InvDiag<float>& inv, int colour, const TmaSweep& t,
                              int* err, cudaStream_t s) {
  if (!t.ok) return cudaErrorInvalidValue;
  k_smooth_tma<<<t.grid, dim3(kTX, kTY, 1), kSmemBytes, s>>>(x, G, inv, colour, t.kz, t.nwork, t.other[colour],
                                                              t.rhs[colour], err, kWaitCycles, -1);
  return cudaGetLastError();
}

cudaError_t launch_smooth_tma_withheld(float* x, const Geom& G, const InvDiag<float>& inv, const TmaSweep& t, int* err,
                                       long long budget_cycles, cudaStream_t s) {
  if (!t.ok) return cudaErrorInvalidValue;
  k_smooth_tma<<<t.grid, dim3(kTX, kTY, 1), kSmemBytes, s>>>(x, G, inv, 0, t.kz, t.nwork, t.other[0], t.rhs[0], err,
                                                              budget_cycles, 2);
  return cudaGetLastError();
}

}  // namespace ccmg
