// smooth_tma.cu -- single-precision red-black Gauss-Seidel half-sweep with TMA z-slab staging
// (sm_103a).
//
// The half-sweep of Sec. 5.3 (phi_i = (g_i + sum of neighbours) / (6 + d_i) on every cell of one
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
#include <cstring>

#include "ccmg_internal.cuh"
#include "level_ops.cuh"

namespace ccmg {
namespace {

using ops::FxOp;
using ops::fx_op;
using ops::fx_sum6;
using ops::fx_exp;
using ops::fx_at;
using ops::fx_to_double;
using ops::inv_of;

constexpr int kHaloX = 4;  // floats on each side of the tile row (16-byte aligned box start)
constexpr long long kWaitCycles = 4000000000LL;  // wait budget, about 2 s at 2 GHz

constexpr int kCHalo = 4;  // coarse floats on each side of a tile's parents (16-byte aligned box start)

__host__ __device__ constexpr int round128(int b) { return ((b + 127) / 128) * 128; }

// Tile of TX 4-float vectors (one per thread column) by TY rows (one per thread row), ring of
// SLOTS plane slots. PRO: the black sweep fused with the prolongation; each slot then also holds
// the coarse-correction rows (both coarse colour arrays) under the other-colour box.
template <int TX, int TY, int SLOTS, bool PRO = false, bool PER = false>
struct Cfg {
  static constexpr int kTX = TX;
  static constexpr int kBoxX = 4 * TX + 2 * kHaloX;    // other-colour box width (floats)
  static constexpr int kCBoxX = 2 * TX + 2 * kCHalo;   // parents of the other-colour box, per coarse colour
  static constexpr int kTY = TY;
  static constexpr int kSlots = SLOTS;
  static constexpr bool kPro = PRO;
  static constexpr bool kPer = PER;  // levels with periodic axes: wrapped halos (the walls-only build keeps its registers)
  static constexpr int kBoxY = TY + 2;
  static constexpr int kBoxBytes = kBoxX * kBoxY * 4;                  // other-colour box
  static constexpr int kGBoxBytes = 4 * TX * TY * 4;                   // right-hand-side box
  static constexpr int kCBoxY = TY / 2 + 2;                            // coarse rows of the parents
  static constexpr int kCBoxBytes = kCBoxX * kCBoxY * 4;               // one coarse colour's box
  static constexpr int kGOff = round128(kBoxBytes);                    // rhs box within a slot
  static constexpr int kC0Off = round128(kGOff + kGBoxBytes);          // coarse colour-0 box
  static constexpr int kC1Off = round128(kC0Off + kCBoxBytes);         // coarse colour-1 box
  static constexpr int kSlotBytes = PRO ? round128(kC1Off + kCBoxBytes) : round128(kGOff + kGBoxBytes);
  static constexpr int kSmemBytes = SLOTS * kSlotBytes + 8 * SLOTS;    // + the mbarriers
  // tensor-copy destinations in shared memory must be 128-byte aligned
  static_assert(kGOff % 128 == 0 && kC0Off % 128 == 0 && kC1Off % 128 == 0 && kSlotBytes % 128 == 0,
                "TMA destinations need 128-byte alignment");
  static_assert(SLOTS >= 4, "planes k-1, k, k+1 and at least one copy in flight");
  static_assert(TY % 2 == 0, "tiles cover whole coarse rows");
};
using Product = Cfg<32, 8, 6>;           // 9600-byte slots, 57.6 KB per CTA, 3 CTAs per SM
using ProductPer = Cfg<32, 8, 6, false, true>;  // the same on levels with a periodic axis
using ProductPro = Cfg<32, 8, 5, true>;  // 13184-byte slots, 65.9 KB per CTA, 3 CTAs per SM (6 slots: 2 per SM, slower)
// Batched systems (rows of 32 to 96 packed values): tiles of 32 packed columns by 32 rows, the
// same slot sizes (a 40 x 34-float box is 1360 floats, as 136 x 10).
using BatchCfg = Cfg<8, 32, 6>;
using BatchPro = Cfg<8, 32, 5, true>;
// the fused sweep reads the other colour through the plain sweep's tensor maps, whose boxes are
// Product::kBoxY rows high: the expected transaction bytes must match them
static_assert(ProductPro::kTY == Product::kTY, "the fused sweep shares the plain sweep's other-colour boxes");

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
// Orders this thread's earlier generic-proxy writes to shared memory before later accesses by the
// async proxy (the tensor copies that refill the same ring slots). Without it a late plain store
// of a slot could land after the copy that reuses the slot.
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
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
template <class C>
__device__ __forceinline__ Work work_item(const Geom& G, int kz, long long w) {
  constexpr int kTX = C::kTX, kTY = C::kTY;
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
// With C::kPro the sweep is the first black post-smoothing sweep fused with the prolongation of
// the coarse correction e_c (Sec. 3): every red value read is red + omega e_c(parent), the parent
// of the red cell at packed index m of fine row (j', k') being coarse cell (m, j'/2, k'/2), both
// operations rounded separately as in ops::smooth_vec_prolong; the coarse rows arrive with each
// red plane (coarse plane floor(p/2) for red plane p), out-of-range parents as zeros, and each
// landed red plane is corrected once in shared memory before the cells read it.
// BATCH: the work items of many systems' finest levels (table `bsys` of nbsys systems, items
// numbered consecutively system by system); each item takes its system's geometry, iterate and
// tensor maps from the table, and the items of systems whose active flag is 0 are skipped. The
// arguments x, G, kz and the four maps are then unused.
template <class C, bool BATCH = false>
__global__ void __launch_bounds__(C::kTX* C::kTY) k_smooth_tma(float* __restrict__ x0, Geom G0, InvDiag<float> inv,
                                                              int colour, int kz0, long long nwork,
                                                              const __grid_constant__ CUtensorMap other,
                                                              const __grid_constant__ CUtensorMap rhs,
                                                              const __grid_constant__ CUtensorMap coarse0,
                                                              const __grid_constant__ CUtensorMap coarse1, float omega,
                                                              int* err, long long budget, int withhold,
                                                              const BTmaSys* __restrict__ bsys, int nbsys,
                                                              const int* __restrict__ active) {
  constexpr int kTX = C::kTX, kBoxX = C::kBoxX, kCBoxX = C::kCBoxX;
  constexpr int kTY = C::kTY, kSlots = C::kSlots, kBoxBytes = C::kBoxBytes, kGBoxBytes = C::kGBoxBytes;
  constexpr int kGOff = C::kGOff, kSlotBytes = C::kSlotBytes, kCBoxBytes = C::kCBoxBytes;
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
  int seq = 0;     // loads issued by this CTA before the current item
  int issued = 0;  // loads issued so far (leader)
  bool failed = false;
  int sb = 0;      // BATCH: the table entry of the current item (items ascend per CTA)

  for (long long w = blockIdx.x; w < nwork && !failed; w += gridDim.x) {
    // the item's level: the launch's one, or (BATCH) its system's from the table
    Geom G = G0;
    float* x = x0;
    int kz = kz0;
    long long wl = w;
    const CUtensorMap *mo = &other, *mr = &rhs, *mc0 = &coarse0, *mc1 = &coarse1;
    if constexpr (BATCH) {
      while (sb + 1 < nbsys && bsys[sb + 1].w0 <= w) ++sb;
      if (!__ldg(active + bsys[sb].sys)) continue;  // uniform over the CTA
      G = bsys[sb].G;
      x = bsys[sb].x;
      kz = bsys[sb].kz;
      wl = w - bsys[sb].w0;
      mo = &bsys[sb].other[colour];
      mr = &bsys[sb].rhs[colour];
      mc0 = &bsys[sb].coarse[0];
      mc1 = &bsys[sb].coarse[1];
    }
    float* const xo = x + (long long)colour * G.csz;
    const Work t = work_item<C>(G, kz, wl);
    const int np = (t.k1 - t.k0) + 2;  // other-colour planes k0-1 .. k1
    // load i of the item into slot (seq+i) % kSlots
    auto issue = [&](int i) {
      if (seq == 0 && i == withhold) return;
      const int n = seq + i;
      const int q = n % kSlots;
      const unsigned bar = bar0 + 8u * q;
      const unsigned dst = ring0 + (unsigned)(q * kSlotBytes);
      const bool with_rhs = i >= 2;
      mbar_expect_tx(bar, kBoxBytes + (with_rhs ? kGBoxBytes : 0) + (C::kPro ? 2 * kCBoxBytes : 0));
      int kp = t.k0 - 1 + i;  // other-colour plane; across a periodic z axis the opposite one
      if (C::kPer && (G.per & 4)) kp = kp < 0 ? G.nz - 1 : (kp >= G.nz ? kp - G.nz : kp);
      tma_load_box(dst, mo, t.x0 - kHaloX, t.y0 - 1, kp, bar);
      if (with_rhs) tma_load_box(dst + kGOff, mr, t.x0, t.y0, t.k0 - 2 + i, bar);
      if (C::kPro) {
        const int kc = (t.k0 - 1 + i + 2) / 2 - 1;  // floor(p / 2) for red plane p >= -1
        tma_load_box(dst + C::kC0Off, mc0, t.x0 / 2 - kCHalo, t.y0 / 2 - 1, kc, bar);
        tma_load_box(dst + C::kC1Off, mc1, t.x0 / 2 - kCHalo, t.y0 / 2 - 1, kc, bar);
      }
      issued = n + 1;
    };
    __syncthreads();  // every thread is done with the previous item's slots
    if (leader)
      for (int i = 0; i < np && i < kSlots - 1; ++i) issue(i);

    const int m0 = t.x0 + 4 * tx;
    const int j = t.y0 + ty;
    const bool mine = m0 < G.hx && j < G.ny;
    // ring positions of loads i-1, i, i+1 (planes k-1, k, k+1) and the phase parity of load
    // i+1, advanced by one slot per plane instead of being recomputed
    int qm = seq % kSlots, qk = (seq + 1) % kSlots, qp = (seq + 2) % kSlots;
    unsigned php = (unsigned)(((seq + 2) / kSlots) & 1);
    float* xrow = xo + ((long long)t.k0 * G.ny + j) * G.hx + m0;  // own row of plane k
    const long long plane_stride = (long long)G.ny * G.hx;
    // walls touched by this thread's cells in every plane but the first and last (x and y);
    // without any, every cell's diagonal is 6
    const bool xy_wall = j == 0 || j == G.ny - 1 || (m0 == 0) || (m0 + 4 >= G.hx);
    const int hxe_col = (G.hx - t.x0 + kHaloX < kBoxX) ? G.hx - t.x0 + kHaloX : -1;
    // PRO: red plane p in slot q becomes red + omega e_c(parent) in place. The parent of the red
    // cell at packed index m of fine row (j', p) is coarse cell (m, j'/2, p/2), of colour
    // (m + j'/2 + p/2) & 1 at packed index m >> 1; its coarse row sits in box row
    // j'/2 - (y0/2 - 1), column (m >> 1) - (x0/2 - kCHalo). Out-of-range red values and parents
    // arrived as zeros, so walls stay zero.
    // The box positions a thread corrects (vectors f = tid and tid + 256 of the box) are fixed for
    // the tile: the red vector's offset in a slot, its parents' row offset in a coarse box, and the
    // parity of m + J; only the coarse plane's parity changes from plane to plane.
    constexpr int kVecs = kBoxX / 4 * C::kBoxY;
    constexpr int kNT = kTX * C::kTY;
    constexpr int kPerThr = (kVecs + kNT - 1) / kNT;
    int cvo[kPerThr], cco[kPerThr], cpar[kPerThr];
    if constexpr (C::kPro) {
#pragma unroll
      for (int u = 0; u < kPerThr; ++u) {
        const int f = ty * kTX + tx + u * kNT;
        const int by = f / (kBoxX / 4), bx = 4 * (f - by * (kBoxX / 4));
        const int m = t.x0 - kHaloX + bx, J = (t.y0 - 1 + by) >> 1;
        cvo[u] = f < kVecs ? by * kBoxX + bx : -1;
        cco[u] = (J - (t.y0 / 2 - 1)) * kCBoxX + (bx >> 1) + (kCHalo - kHaloX / 2);
        cpar[u] = (m + J) & 1;
      }
    }
    auto correct = [&](int q, int p) {
      float* slot = ring + q * (kSlotBytes / 4);
      const int K = (p + 2) / 2 - 1;  // floor(p / 2) for p >= -1
#pragma unroll
      for (int u = 0; u < kPerThr; ++u) {
        if (cvo[u] < 0) continue;
        const bool even0 = ((cpar[u] + K) & 1) == 0;  // parent I = m has colour 0
        const float* ca = slot + (even0 ? C::kC0Off : C::kC1Off) / 4 + cco[u];
        const float* cb = slot + (even0 ? C::kC1Off : C::kC0Off) / 4 + cco[u];
        const float2 pa = *reinterpret_cast<const float2*>(ca);
        const float2 pb = *reinterpret_cast<const float2*>(cb);
        float4* v = reinterpret_cast<float4*>(slot + cvo[u]);
        float4 r = *v;
        r.x = __fadd_rn(r.x, __fmul_rn(omega, pa.x));
        r.y = __fadd_rn(r.y, __fmul_rn(omega, pb.x));
        r.z = __fadd_rn(r.z, __fmul_rn(omega, pa.y));
        r.w = __fadd_rn(r.w, __fmul_rn(omega, pb.y));
        *v = r;
      }
    };
    // Periodic x / y axes: the copy engine fills the box beyond the level with zeros; the halo
    // values the sweep reads there (the column beyond each end of the tile's rows, and the rows
    // beyond the level's first and last row) are the other colour's values at the opposite side.
    // Each thread owns at most three of them (two of the wrapped rows, one of the columns): their
    // box positions (hidx) and offsets within a plane (hoff, -1: zero) are fixed for the tile, the
    // values of plane k+2 are loaded while plane k is computed and written into its slot after it
    // lands, before the barrier that publishes it.
    int hidx[3] = {-1, -1, -1};
    int hoff[3] = {-1, -1, -1};  // within a plane: ny * hx entries
    float hval[3] = {0.0f, 0.0f, 0.0f};
    if constexpr (C::kPer) {
      // every wrapped halo row value has a slot (two per thread) and every column value a thread
      static_assert(kBoxX <= kTX * C::kTY, "two wrapped halo rows need kBoxX <= threads per CTA");
      static_assert(2 * C::kBoxY <= kTX * C::kTY, "the wrapped halo columns need 2 kBoxY <= threads per CTA");
      const int nt = kTX * kTY, tid = ty * kTX + tx;
      const bool px = (G.per & 1) != 0, py = (G.per & 2) != 0;
      if (py) {  // box row 0 holds row -1 for the first tile, box row ny-y0+1 holds row ny
        const int rlo = t.y0 == 0 ? 0 : -1, rhi = G.ny - t.y0 + 1 < C::kBoxY ? G.ny - t.y0 + 1 : -1;
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int f = tid + u * nt;
          if (f >= 2 * kBoxX) continue;
          const int r = f < kBoxX ? rlo : rhi;
          if (r < 0) continue;
          const int col = f < kBoxX ? f : f - kBoxX;
          const int sy = f < kBoxX ? G.ny - 1 : 0;
          int gx = t.x0 - kHaloX + col;
          if (px) gx = gx < 0 ? gx + G.hx : (gx >= G.hx ? gx - G.hx : gx);
          hidx[u] = r * kBoxX + col;
          hoff[u] = (gx >= 0 && gx < G.hx) ? sy * G.hx + gx : -1;
        }
      }
      if (px && tid < 2 * C::kBoxY) {  // box columns kHaloX-1 (x0 = 0) and hx-x0+kHaloX (in the box)
        const int r = tid % C::kBoxY;
        const bool left = tid < C::kBoxY;
        const int gy = t.y0 - 1 + r;
        if (gy >= 0 && gy < G.ny) {
          if (left && t.x0 == 0) {
            hidx[2] = r * kBoxX + kHaloX - 1;
            hoff[2] = gy * G.hx + G.hx - 1;
          } else if (!left && hxe_col >= 0) {
            hidx[2] = r * kBoxX + hxe_col;
            hoff[2] = gy * G.hx;
          }
        }
      }
    }
    const float* const oth_base = x + (long long)(1 - colour) * G.csz;
    auto gather = [&](int p) {  // the halo values of plane p (zeros for a wall plane)
      int pw = p;
      if (G.per & 4) pw = pw < 0 ? G.nz - 1 : (pw >= G.nz ? pw - G.nz : pw);
      const bool in = pw >= 0 && pw < G.nz;
      const float* src = oth_base + (long long)(in ? pw : 0) * G.ny * G.hx;
#pragma unroll
      for (int u = 0; u < 3; ++u) hval[u] = (hidx[u] >= 0 && hoff[u] >= 0 && in) ? __ldg(src + hoff[u]) : 0.0f;
    };
    auto scatter = [&](int q) {
      float* slot = ring + q * (kSlotBytes / 4);
#pragma unroll
      for (int u = 0; u < 3; ++u)
        if (hidx[u] >= 0) slot[hidx[u]] = hval[u];
    };
    for (int k = t.k0; k < t.k1; ++k) {
      const int i = k - t.k0 + 1;  // load index of plane k (k-1 is i-1; k+1 and g(k) are i+1)
      bool ok = true;
      if (k == t.k0) {
        ok = mbar_wait(bar0 + 8u * (unsigned)qm, (unsigned)((seq / kSlots) & 1), budget);
        ok = ok && mbar_wait(bar0 + 8u * (unsigned)qk, (unsigned)(((seq + 1) / kSlots) & 1), budget);
      }
      ok = ok && mbar_wait(bar0 + 8u * (unsigned)qp, php, budget);
      if constexpr (C::kPer) {  // the fused sweep (PRO) is not run on periodic levels
        if (ok && (G.per & 3)) {
          if (k == t.k0) {  // the item's first three planes: loaded here
            gather(k - 1);
            scatter(qm);
            gather(k);
            scatter(qk);
            gather(k + 1);
          }
          scatter(qp);                     // plane k+1 (loaded during the previous plane)
          if (k + 1 < t.k1) gather(k + 2);  // in flight while plane k is computed
        }
      }
      if constexpr (C::kPro) {
        // red planes k-1 and k arrived with the item's first plane, k+1 just now: add the
        // prolongated correction to them in place, once, before any cell reads them
        if (ok) {
          if (k == t.k0) {
            correct(qm, k - 1);
            correct(qk, k);
          }
          correct(qp, k + 1);
        }
      }
      // plain stores into ring slots (wrapped halos, corrected planes) are ordered before the
      // tensor copies that will refill those slots
      if constexpr (C::kPro) fence_proxy_async_smem();
      else if constexpr (C::kPer)
        if (G.per & 3) fence_proxy_async_smem();
      // the barrier also retires iteration k-1 (and publishes the corrected planes), freeing the
      // slot of load i-2 for load i+kSlots-2
      if (__syncthreads_or(!ok)) {
        failed = true;
        break;
      }
      if (leader && i + kSlots - 2 < np) issue(i + kSlots - 2);
      if (mine) {
        const int s = (j + k + colour) & 1;
        const float* pk = ring + qk * (kSlotBytes / 4);
        const float* pm = ring + qm * (kSlotBytes / 4);
        const float* pp = ring + qp * (kSlotBytes / 4);
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
        const float zpv[4] = {zp.x, zp.y, zp.z, zp.w};
        const float gvv[4] = {gv.x, gv.y, gv.z, gv.w};
        float invd[4];
        if (xy_wall || k == 0 || k == G.nz - 1) {
          int dbase = 0;
          if (j == 0) dbase += G.sh[2];
          if (j == G.ny - 1) dbase += G.sh[3];
          if (k == 0) dbase += G.sh[4];
          if (k == G.nz - 1) dbase += G.sh[5];
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            int d = dbase;
            if (m0 + e == 0 && s == 0) d += G.sh[0];
            if (m0 + e == G.hx - 1 && s == 1) d += G.sh[1];
            invd[e] = inv_of(inv, d);
          }
        } else {
#pragma unroll
          for (int e = 0; e < 4; ++e) invd[e] = inv.v[3];  // 1/6
        }
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
          out[e] = (gvv[e] + S) * invd[e];
        }
        *reinterpret_cast<float4*>(xrow) = make_float4(out[0], out[1], out[2], out[3]);
      }
      xrow += plane_stride;
      qm = qk;
      qk = qp;
      if (++qp == kSlots) {
        qp = 0;
        php ^= 1u;
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

// ---------------------------------------------------------------------------------------------
// FP64 half-sweep with TMA z-slab staging (FP64 mode, levels without a periodic axis):
// phi = (g + S) / (6 + d) with the six-neighbour sum S formed exactly in 64-bit fixed point. A CTA
// of 32 x 8 threads owns a tile of 64 x 8 cells of the colour (two per thread, a 16-byte vector)
// and marches it through a slab of planes; the other colour's planes arrive as 68 x 10-double
// boxes (tile plus a one-row and a 2-double x halo, 16-byte aligned start) in four raw slots.
// Every landed plane gets one exponent, the largest biased exponent E_p among its box values
// (each warp reduces its share, the CTA takes the maximum of the eight), and every value is
// converted once, as floor(+-significand 2^5 / 2^(E_p - e)), an integer in units of 2^(E_p - 1080)
// of magnitude below 2^58, into a ring of four converted planes. A cell's four in-plane neighbours
// share one unit and are added without shifts; with E the largest of the three planes' exponents
// the in-plane sum and the two z neighbours are shifted to the unit 2^(E - 1080) (shifts the same
// for the whole CTA), added and rounded once to a double. Each floor loses less than one unit, so
// S lies within 7 units of 2^(E - 1080), 7/32 of an ulp of the largest value in the three boxes,
// plus half an ulp of itself, of the exact sum; then + g and x 1/(6 + d) as in the direct-load
// sweep, whose per-cell alignment (fx_sum6) is bounded by the cell's own largest neighbour instead.
// A tile plane next to an infinity or NaN takes the direct FP64 sum from global memory.
// The right-hand side, read once, comes by a plain vector load issued before the plane's wait.
// Load i (other-colour plane k0-1+i) goes to raw slot and converted plane (seq + i) % 4. The
// exponent of a plane must be known before its values are converted, so the pipeline runs one
// plane deeper than the copies: at plane k (load index i) the threads take the exponents of load
// i+2, convert load i+1 with the exponent published at the previous barrier, and one barrier
// publishes both; then the raw slot of load i+1 takes load i+5 and the cells read loads i-1, i,
// i+1. A converted plane is rewritten two barriers after its last read.
constexpr int k64TX = 32, k64TY = 8;
constexpr int k64Halo = 2;                              // doubles on each side of a tile row
constexpr int k64BoxX = 2 * k64TX + 2 * k64Halo;        // 68
constexpr int k64BoxY = k64TY + 2;                      // 10
constexpr int k64BoxN = k64BoxX * k64BoxY;              // values per converted plane
constexpr int k64BoxBytes = k64BoxN * 8;                // 5440
constexpr int k64SlotBytes = round128(k64BoxBytes);    // 5504
constexpr int k64Slots = 4;
constexpr int k64Fx = 4;  // converted planes
constexpr int k64Warps = k64TX * k64TY / 32;
constexpr int k64SmemBytes = k64Slots * k64SlotBytes + k64Fx * k64BoxN * 8 + k64Slots * k64Warps * 4 + 8 * k64Slots;
static_assert(k64SlotBytes % 128 == 0, "TMA destinations need 128-byte alignment");
static_assert((k64Slots * k64SlotBytes) % 8 == 0 && (k64Fx * k64BoxN * 8) % 8 == 0 && (k64Slots * k64Warps * 4) % 8 == 0,
              "ring alignment");
static_assert(k64BoxN <= 3 * k64TX * k64TY, "three box values per thread at most");

__global__ void __launch_bounds__(k64TX* k64TY, 4)
    k_smooth_tma64(double* __restrict__ x, const double* __restrict__ g, Geom G, InvDiag<double> inv, int colour, int kz,
                   long long nwork, const __grid_constant__ CUtensorMap other, int* err, long long budget,
                   int withhold) {
  extern __shared__ __align__(128) unsigned char smem[];
  unsigned char* raw = smem;
  long long* fT = reinterpret_cast<long long*>(smem + k64Slots * k64SlotBytes);  // converted planes
  int* pexp = reinterpret_cast<int*>(fT + k64Fx * k64BoxN);  // per raw slot, each warp's largest exponent
  unsigned long long* bars = reinterpret_cast<unsigned long long*>(pexp + k64Slots * k64Warps);
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * k64TX + tx, wid = tid >> 5;
  const bool leader = tid == 0;
  if (leader) {
    for (int q = 0; q < k64Slots; ++q) mbar_init(smem_addr(bars + q), 1);
    mbar_fence_init();
  }
  __syncthreads();
  const unsigned raw0 = smem_addr(raw), bar0 = smem_addr(bars);
  double* const xo = x + (long long)colour * G.csz;
  const double* const xoth = x + (long long)(1 - colour) * G.csz;
  int seq = 0, issued = 0;
  bool failed = false;
  for (long long w = blockIdx.x; w < nwork && !failed; w += gridDim.x) {
    const int tiles_x = (G.hx + 2 * k64TX - 1) / (2 * k64TX), tiles_y = (G.ny + k64TY - 1) / k64TY;
    const long long per_slab = (long long)tiles_x * tiles_y;
    const int slab = (int)(w / per_slab), rem = (int)(w - per_slab * slab);
    const int x0 = (rem % tiles_x) * 2 * k64TX, y0 = (rem / tiles_x) * k64TY;
    const int k0 = slab * kz, k1 = min(k0 + kz, G.nz);
    const int np = (k1 - k0) + 2;
    auto issue = [&](int i) {
      if (seq == 0 && i == withhold) return;  // the failure-path self-test only
      const int n = seq + i, q = n % k64Slots;
      const unsigned bar = bar0 + 8u * q, dst = raw0 + (unsigned)(q * k64SlotBytes);
      mbar_expect_tx(bar, k64BoxBytes);
      tma_load_box(dst, &other, x0 - k64Halo, y0 - 1, k0 - 1 + i, bar);
      issued = n + 1;
    };
    auto wait = [&](int i) {
      const int n = seq + i;
      return mbar_wait(bar0 + 8u * (unsigned)(n % k64Slots), (unsigned)((n / k64Slots) & 1), budget);
    };
    auto rawp = [&](int i) { return reinterpret_cast<const double*>(raw + ((seq + i) % k64Slots) * k64SlotBytes); };
    // the largest exponent among this warp's share of load i's box, for the plane's exponent
    auto scan = [&](int i) {
      const double* src = rawp(i);
      unsigned e = 0u;
#pragma unroll
      for (int u = 0; u < 3; ++u) {
        const int f = tid + u * k64TX * k64TY;
        if (f < k64BoxN) e = max(e, fx_exp(src[f]));
      }
      e = __reduce_max_sync(0xffffffffu, e);
      if ((tid & 31) == 0) pexp[((seq + i) % k64Slots) * k64Warps + wid] = (int)e;
    };
    auto plane_exp = [&](int i) {
      const int* pe = pexp + ((seq + i) % k64Slots) * k64Warps;
      int e = pe[0];
#pragma unroll
      for (int q = 1; q < k64Warps; ++q) e = max(e, pe[q]);
      return e;
    };
    // load i's box into converted plane (seq + i) % k64Fx at the plane's exponent E
    auto convert = [&](int i, int E) {
      const double* src = rawp(i);
      long long* dT = fT + ((seq + i) % k64Fx) * k64BoxN;
#pragma unroll
      for (int u = 0; u < 3; ++u) {
        const int f = tid + u * k64TX * k64TY;
        if (f < k64BoxN) dT[f] = fx_at(src[f], E);
      }
    };
    __syncthreads();  // every thread is done with the previous item's slots
    if (leader)
      for (int i = 0; i < np && i < k64Slots; ++i) issue(i);
    bool ok = wait(0) && wait(1) && wait(2);
    if (ok) {
      scan(0);
      scan(1);
      scan(2);
    }
    if (__syncthreads_or(!ok)) {
      failed = true;
      break;
    }
    int Em = plane_exp(0), Ek = plane_exp(1);  // exponents of loads i-1 and i at plane k
    convert(0, Em);
    convert(1, Ek);
    const int m0 = x0 + 2 * tx, j = y0 + ty;
    const bool mine = m0 < G.hx && j < G.ny;
    const bool xy_wall = j == 0 || j == G.ny - 1 || m0 == 0 || m0 + 2 >= G.hx;
    const int c0 = (ty + 1) * k64BoxX + k64Halo + 2 * tx;  // box position of m0 in row j
    double* xrow = xo + ((long long)k0 * G.ny + j) * G.hx + m0;
    const double* grow = g + (xrow - x);
    const long long plane_stride = (long long)G.ny * G.hx;
    for (int k = k0; k < k1; ++k) {
      const int i = k - k0 + 1;  // load index of plane k
      // the cell pair's right-hand side, read while the copies land and are converted
      const double2 gv = mine ? __ldg(reinterpret_cast<const double2*>(grow)) : make_double2(0.0, 0.0);
      const int Ep = plane_exp(i + 1);  // published by the previous barrier
      if (i + 2 < np) {
        ok = ok && wait(i + 2);
        if (ok) scan(i + 2);
      }
      convert(i + 1, Ep);
      if (__syncthreads_or(!ok)) {
        failed = true;
        break;
      }
      if (leader) {  // raw slots whose planes are converted: loads 0..2 at the first plane, then i+1
        if (i == 1)
          for (int n = k64Slots; n < k64Slots + 2 && n < np; ++n) issue(n);
        if (i + k64Slots + 1 < np) issue(i + k64Slots + 1);
      }
      if (mine) {
        const int s = (j + k + colour) & 1;
        double invd[2];
        if (xy_wall || k == 0 || k == G.nz - 1) {
          int dbase = 0;
          if (j == 0) dbase += G.sh[2];
          if (j == G.ny - 1) dbase += G.sh[3];
          if (k == 0) dbase += G.sh[4];
          if (k == G.nz - 1) dbase += G.sh[5];
#pragma unroll
          for (int e = 0; e < 2; ++e) {
            int d = dbase;
            if (m0 + e == 0 && s == 0) d += G.sh[0];
            if (m0 + e == G.hx - 1 && s == 1) d += G.sh[1];
            invd[e] = inv_of(inv, d);
          }
        } else {
          invd[0] = invd[1] = inv.v[3];
        }
        const int E = max(max(Em, Ek), Ep);
        double S[2];
        if (E != 2047) {
          const long long* pm = fT + ((seq + i - 1) % k64Fx) * k64BoxN;
          const long long* pk = fT + ((seq + i) % k64Fx) * k64BoxN;
          const long long* pp = fT + ((seq + i + 1) % k64Fx) * k64BoxN;
          const int dk = min(E - Ek, 63), dm = min(E - Em, 63), dp = min(E - Ep, 63);
          // x-neighbours: other colour at m + s - 1 and m + s for cells m0 and m0 + 1
          const long long xa = pk[c0 + s - 1], xb = pk[c0 + s], xc = pk[c0 + s + 1];
          const long long in0 = xa + xb + pk[c0 - k64BoxX] + pk[c0 + k64BoxX];
          const long long in1 = xb + xc + pk[c0 - k64BoxX + 1] + pk[c0 + k64BoxX + 1];
          S[0] = fx_to_double((unsigned long long)((in0 >> dk) + (pm[c0] >> dm) + (pp[c0] >> dp)), E);
          S[1] = fx_to_double((unsigned long long)((in1 >> dk) + (pm[c0 + 1] >> dm) + (pp[c0 + 1] >> dp)), E);
        } else {  // an infinity or NaN in the three planes: the direct sum of the values
          auto nb = [&](int mm, int jj, int kk) {
            return (mm >= 0 && mm < G.hx && jj >= 0 && jj < G.ny && kk >= 0 && kk < G.nz)
                       ? __ldg(xoth + ((long long)kk * G.ny + jj) * G.hx + mm)
                       : 0.0;
          };
#pragma unroll
          for (int e = 0; e < 2; ++e) {
            const int mm = m0 + e;
            S[e] = ((((nb(mm + s - 1, j, k) + nb(mm + s, j, k)) + nb(mm, j - 1, k)) + nb(mm, j + 1, k)) +
                    nb(mm, j, k - 1)) +
                   nb(mm, j, k + 1);
          }
        }
        *reinterpret_cast<double2*>(xrow) = make_double2((gv.x + S[0]) * invd[0], (gv.y + S[1]) * invd[1]);
      }
      Em = Ek;
      Ek = Ep;
      xrow += plane_stride;
      grow += plane_stride;
    }
    seq += np;
  }
  if (failed && leader) {
    atomicExch(err, 1);
    for (int n = issued > k64Slots ? issued - k64Slots : 0; n < issued; ++n)
      if (!(seq == 0 && n == withhold))
        mbar_wait(bar0 + 8u * (unsigned)(n % k64Slots), (unsigned)((n / k64Slots) & 1), budget);
  }
}

}  // namespace

bool tma_sweep_applies(const Geom& G) {
  // rows of whole 4-float vectors and enough planes to march (periodic axes: the kernel loads the
  // wrapped halos itself)
  return G.packed && (G.hx % 4) == 0 && G.nz >= 8 && (long long)G.hx * G.ny * G.nz >= (1LL << 16);
}

bool tma_sweep_pays(const Geom& G) {
  // measured on GB300: ahead of the direct-load kernel at 512^3 (2^25 cells per colour), even at
  // 256^3, behind below that (too few tiles to keep every SM's copies in flight). Not on periodic
  // levels: with their wrapped halo values (loaded a plane ahead) the kernel holds 88 registers
  // and two CTAs per SM, and the periodic 512^3 time step took 14.9 ms with it against 13.7 ms
  // with the direct-load sweep
  return tma_sweep_applies(G) && G.per == 0 && (long long)G.hx * G.ny * G.nz >= (1LL << 24);
}

namespace {

using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

cudaError_t encoder(EncodeFn* out) {
  static EncodeFn encode = nullptr;
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess) return e;
    if (q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
    encode = reinterpret_cast<EncodeFn>(fn);
  }
  *out = encode;
  return cudaSuccess;
}

// 3D float map of one colour array of level G (x = packed index, y = row, z = plane).
cudaError_t colour_map(EncodeFn encode, CUtensorMap* map, const float* base, const Geom& G, int box_x, int box_y) {
  const cuuint64_t dims[3] = {(cuuint64_t)G.hx, (cuuint64_t)G.ny, (cuuint64_t)G.nz};
  const cuuint64_t strides[2] = {(cuuint64_t)G.hx * 4, (cuuint64_t)G.hx * G.ny * 4};
  const cuuint32_t box[3] = {(cuuint32_t)box_x, (cuuint32_t)box_y, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  const CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(base), dims, strides, box,
                            estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// Persistent grid and slab length for configuration C on level G.
template <class C>
cudaError_t size_launch(const Geom& G, int device, int& kz, long long& nwork, int& grid) {
  cudaError_t e = cudaFuncSetAttribute(k_smooth_tma<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::kSmemBytes);
  if (e != cudaSuccess) return e;
  int per_sm = 0, sms = 0;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_smooth_tma<C>, C::kTX * C::kTY, C::kSmemBytes)) !=
      cudaSuccess)
    return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device)) != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const long long tiles = (long long)((G.hx + 4 * C::kTX - 1) / (4 * C::kTX)) * ((G.ny + C::kTY - 1) / C::kTY);
  const long long slots = (long long)per_sm * sms;
  // planes per item: long slabs (each starts by loading two extra planes), but at least two
  // items per resident CTA; 64 planes measured best at 512^3
  kz = 64;
  while (kz > 8 && tiles * ((G.nz + kz - 1) / kz) < 2 * slots) kz /= 2;
  nwork = tiles * ((G.nz + kz - 1) / kz);
  grid = (int)(nwork < slots ? nwork : slots);
  return cudaSuccess;
}

template <class C>
cudaError_t prepare_tma_sweep_cfg(TmaSweep& t, float* x, const float* g, const Geom& G, int device) {
  t.ok = 0;
  if (!tma_sweep_applies(G)) return cudaSuccess;
  EncodeFn encode = nullptr;
  cudaError_t e = encoder(&encode);
  if (e != cudaSuccess) return e;
  for (int c = 0; c < 2; ++c) {
    const float* base = x + (long long)(1 - c) * G.csz;  // a colour-c sweep reads colour 1-c
    const float* gbase = g + (long long)c * G.csz;       // and its own right-hand side
    if (reinterpret_cast<uintptr_t>(base) % 16 != 0 || reinterpret_cast<uintptr_t>(gbase) % 16 != 0)
      return cudaSuccess;
    if ((e = colour_map(encode, &t.other[c], base, G, C::kBoxX, C::kBoxY)) != cudaSuccess) return e;
    if ((e = colour_map(encode, &t.rhs[c], gbase, G, 4 * C::kTX, C::kTY)) != cudaSuccess) return e;
  }
  if ((e = size_launch<C>(G, device, t.kz, t.nwork, t.grid)) != cudaSuccess) return e;
  t.ok = 1;
  return cudaSuccess;
}

// The prolongation-fused black sweep of level G with coarse correction ec on level Gc (packed).
template <class C>
cudaError_t prepare_tma_prolong_cfg(TmaSweep& t, const float* ec, const Geom& Gc, const Geom& G, int device) {
  t.ok_pro = 0;
  // the fused prolongation sweep takes the plain sweep's zero halos; periodic levels keep the
  // separate direct-load fused sweep
  if (!t.ok || G.per != 0 || !Gc.packed || (Gc.hx % 4) != 0 || Gc.hx * 2 != G.hx || Gc.ny * 2 != G.ny ||
      Gc.nz * 2 != G.nz)
    return cudaSuccess;
  EncodeFn encode = nullptr;
  cudaError_t e = encoder(&encode);
  if (e != cudaSuccess) return e;
  for (int c = 0; c < 2; ++c) {
    const float* base = ec + (long long)c * Gc.csz;
    if (reinterpret_cast<uintptr_t>(base) % 16 != 0) return cudaSuccess;
    if ((e = colour_map(encode, &t.coarse[c], base, Gc, C::kCBoxX, C::kCBoxY)) != cudaSuccess) return e;
  }
  if ((e = size_launch<C>(G, device, t.kz_pro, t.nwork_pro, t.grid_pro)) != cudaSuccess) return e;
  t.ok_pro = 1;
  return cudaSuccess;
}

template <class C>
cudaError_t launch_smooth_tma_cfg(float* x, const Geom& G, const InvDiag<float>& inv, int colour, const TmaSweep& t,
                                  int* err, long long budget, int withhold, cudaStream_t s) {
  if (!t.ok) return cudaErrorInvalidValue;
  k_smooth_tma<C><<<t.grid, dim3(C::kTX, C::kTY, 1), C::kSmemBytes, s>>>(
      x, G, inv, colour, t.kz, t.nwork, t.other[colour], t.rhs[colour], t.other[colour], t.other[colour], 0.0f, err,
      budget, withhold, nullptr, 0, nullptr);
  return cudaGetLastError();
}

// The FP64 sweep: 3D double map of one colour array of level G.
cudaError_t colour_map64(EncodeFn encode, CUtensorMap* map, const double* base, const Geom& G, int box_x, int box_y) {
  const cuuint64_t dims[3] = {(cuuint64_t)G.hx, (cuuint64_t)G.ny, (cuuint64_t)G.nz};
  const cuuint64_t strides[2] = {(cuuint64_t)G.hx * 8, (cuuint64_t)G.hx * G.ny * 8};
  const cuuint32_t box[3] = {(cuuint32_t)box_x, (cuuint32_t)box_y, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  const CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3, const_cast<double*>(base), dims, strides, box,
                            estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

}  // namespace

bool tma_sweep64_applies(const Geom& G) {
  // rows of whole 16-byte vectors, enough planes to march, walls only (no periodic axis)
  return G.packed && (G.hx % 2) == 0 && G.nz >= 8 && G.per == 0 && (long long)G.hx * G.ny * G.nz >= (1LL << 16);
}

bool tma_sweep64_pays(const Geom& G) { return tma_sweep64_applies(G) && (long long)G.hx * G.ny * G.nz >= (1LL << 22); }

cudaError_t prepare_tma_sweep64(TmaSweep& t, double* x, const double* g, const Geom& G, int device) {
  t.ok = 0;
  if (!tma_sweep64_applies(G)) return cudaSuccess;
  EncodeFn encode = nullptr;
  cudaError_t e = encoder(&encode);
  if (e != cudaSuccess) return e;
  for (int c = 0; c < 2; ++c) {
    const double* base = x + (long long)(1 - c) * G.csz;
    const double* gbase = g + (long long)c * G.csz;
    if (reinterpret_cast<uintptr_t>(base) % 16 != 0 || reinterpret_cast<uintptr_t>(gbase) % 16 != 0)
      return cudaSuccess;
    if ((e = colour_map64(encode, &t.other[c], base, G, k64BoxX, k64BoxY)) != cudaSuccess) return e;
  }
  if ((e = cudaFuncSetAttribute(k_smooth_tma64, cudaFuncAttributeMaxDynamicSharedMemorySize, k64SmemBytes)) !=
      cudaSuccess)
    return e;
  int per_sm = 0, sms = 0;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_smooth_tma64, k64TX * k64TY, k64SmemBytes)) !=
      cudaSuccess)
    return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device)) != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const long long tiles = (long long)((G.hx + 2 * k64TX - 1) / (2 * k64TX)) * ((G.ny + k64TY - 1) / k64TY);
  const long long slots = (long long)per_sm * sms;
  int kz = 64;
  while (kz > 8 && tiles * ((G.nz + kz - 1) / kz) < 2 * slots) kz /= 2;
  t.kz = kz;
  t.nwork = tiles * ((G.nz + kz - 1) / kz);
  t.grid = (int)(t.nwork < slots ? t.nwork : slots);
  t.ok = 1;
  return cudaSuccess;
}

cudaError_t launch_smooth_tma64(double* x, const double* g, const Geom& G, const InvDiag<double>& inv, int colour,
                                const TmaSweep& t, int* err, cudaStream_t s) {
  if (!t.ok) return cudaErrorInvalidValue;
  k_smooth_tma64<<<t.grid, dim3(k64TX, k64TY, 1), k64SmemBytes, s>>>(x, g, G, inv, colour, t.kz, t.nwork,
                                                                    t.other[colour], err, kWaitCycles, -1);
  return cudaGetLastError();
}

cudaError_t launch_smooth_tma64_withheld(double* x, const double* g, const Geom& G, const InvDiag<double>& inv,
                                         const TmaSweep& t, int* err, long long budget_cycles, cudaStream_t s) {
  if (!t.ok) return cudaErrorInvalidValue;
  k_smooth_tma64<<<t.grid, dim3(k64TX, k64TY, 1), k64SmemBytes, s>>>(x, g, G, inv, 0, t.kz, t.nwork, t.other[0],
                                                                    err, budget_cycles, 2);
  return cudaGetLastError();
}

cudaError_t prepare_tma_sweep(TmaSweep& t, float* x, const float* g, const Geom& G, int device) {
  return G.per ? prepare_tma_sweep_cfg<ProductPer>(t, x, g, G, device)
               : prepare_tma_sweep_cfg<Product>(t, x, g, G, device);
}

cudaError_t prepare_tma_prolong(TmaSweep& t, const float* ec, const Geom& Gc, const Geom& G, int device) {
  return prepare_tma_prolong_cfg<ProductPro>(t, ec, Gc, G, device);
}

cudaError_t launch_smooth_tma(float* x, const Geom& G, const InvDiag<float>& inv, int colour, const TmaSweep& t,
                              int* err, cudaStream_t s) {
  return G.per ? launch_smooth_tma_cfg<ProductPer>(x, G, inv, colour, t, err, kWaitCycles, -1, s)
               : launch_smooth_tma_cfg<Product>(x, G, inv, colour, t, err, kWaitCycles, -1, s);
}

cudaError_t launch_smooth_prolong_tma(float* x, const Geom& G, const InvDiag<float>& inv, const TmaSweep& t,
                                      float omega, int* err, cudaStream_t s) {
  if (!t.ok_pro) return cudaErrorInvalidValue;
  k_smooth_tma<ProductPro><<<t.grid_pro, dim3(ProductPro::kTX, ProductPro::kTY, 1), ProductPro::kSmemBytes, s>>>(
      x, G, inv, 1, t.kz_pro, t.nwork_pro, t.other[1], t.rhs[1], t.coarse[0], t.coarse[1], omega, err, kWaitCycles,
      -1, nullptr, 0, nullptr);
  return cudaGetLastError();
}

cudaError_t prepare_tma_batch(BTmaSys* sys, int n, float* const* x, const float* const* g, const Geom* G,
                              const float* const* xc, const Geom* Gc, const int* sys_index, long long* total,
                              int* grid, int* ok, int device) {
  *ok = 0;
  for (int i = 0; i < n; ++i) {
    const Geom &F = G[i], &C = Gc[i];
    const bool halves = C.nx * 2 == F.nx && C.ny * 2 == F.ny && C.nz * 2 == F.nz;
    if (!F.packed || F.per || F.hx % 4 != 0 || F.nz < 8 || !C.packed || C.hx % 4 != 0 || !halves) return cudaSuccess;
    for (int c = 0; c < 2; ++c)
      if (reinterpret_cast<uintptr_t>(x[i] + c * F.csz) % 16 || reinterpret_cast<uintptr_t>(g[i] + c * F.csz) % 16 ||
          reinterpret_cast<uintptr_t>(xc[i] + c * C.csz) % 16)
        return cudaSuccess;
  }
  EncodeFn encode = nullptr;
  cudaError_t e = encoder(&encode);
  if (e != cudaSuccess) return e;
  static_assert(BatchPro::kBoxX == BatchCfg::kBoxX && BatchPro::kBoxY == BatchCfg::kBoxY,
                "the fused batched sweep reads the other colour through the plain sweep's maps");
  long long w = 0;
  for (int i = 0; i < n; ++i) {
    BTmaSys& d = sys[i];
    std::memset(&d, 0, sizeof(d));
    const Geom &F = G[i], &C = Gc[i];
    for (int c = 0; c < 2; ++c) {
      if ((e = colour_map(encode, &d.other[c], x[i] + (long long)(1 - c) * F.csz, F, BatchCfg::kBoxX,
                          BatchCfg::kBoxY)) != cudaSuccess)
        return e;
      if ((e = colour_map(encode, &d.rhs[c], g[i] + (long long)c * F.csz, F, 4 * BatchCfg::kTX, BatchCfg::kTY)) !=
          cudaSuccess)
        return e;
      if ((e = colour_map(encode, &d.coarse[c], xc[i] + (long long)c * C.csz, C, BatchPro::kCBoxX,
                          BatchPro::kCBoxY)) != cudaSuccess)
        return e;
    }
    d.G = F;
    d.x = x[i];
    d.sys = sys_index[i];
    d.kz = F.nz < 64 ? F.nz : 64;  // slabs of up to 64 planes
    const long long tiles =
        (long long)((F.hx + 4 * BatchCfg::kTX - 1) / (4 * BatchCfg::kTX)) * ((F.ny + BatchCfg::kTY - 1) / BatchCfg::kTY);
    d.nwork = tiles * ((F.nz + d.kz - 1) / d.kz);
    d.w0 = w;
    w += d.nwork;
  }
  // persistent grid: the smaller of the two kernels' resident CTAs
  int per_a = 0, per_b = 0, sms = 0;
  if ((e = cudaFuncSetAttribute(k_smooth_tma<BatchCfg, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                BatchCfg::kSmemBytes)) != cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(k_smooth_tma<BatchPro, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                BatchPro::kSmemBytes)) != cudaSuccess)
    return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_a, k_smooth_tma<BatchCfg, true>,
                                                         BatchCfg::kTX * BatchCfg::kTY, BatchCfg::kSmemBytes)) !=
      cudaSuccess)
    return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_b, k_smooth_tma<BatchPro, true>,
                                                         BatchPro::kTX * BatchPro::kTY, BatchPro::kSmemBytes)) !=
      cudaSuccess)
    return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device)) != cudaSuccess) return e;
  const long long slots = (long long)(per_a < per_b ? per_a : per_b) * sms;
  if (slots < 1) return cudaErrorInvalidConfiguration;
  *total = w;
  *grid = (int)(w < slots ? w : slots);
  *ok = 1;
  return cudaSuccess;
}

cudaError_t launch_b_smooth_tma(const BTmaSys* d_sys, int n, long long total, int grid, const int* active,
                                const InvDiag<float>& inv, int colour, int* err, cudaStream_t s) {
  CUtensorMap none{};
  k_smooth_tma<BatchCfg, true><<<grid, dim3(BatchCfg::kTX, BatchCfg::kTY, 1), BatchCfg::kSmemBytes, s>>>(
      nullptr, Geom{}, inv, colour, 0, total, none, none, none, none, 0.0f, err, kWaitCycles, -1, d_sys, n, active);
  return cudaGetLastError();
}

cudaError_t launch_b_smooth_prolong_tma(const BTmaSys* d_sys, int n, long long total, int grid, const int* active,
                                        const InvDiag<float>& inv, float omega, int* err, cudaStream_t s) {
  CUtensorMap none{};
  k_smooth_tma<BatchPro, true><<<grid, dim3(BatchPro::kTX, BatchPro::kTY, 1), BatchPro::kSmemBytes, s>>>(
      nullptr, Geom{}, inv, 1, 0, total, none, none, none, none, omega, err, kWaitCycles, -1, d_sys, n, active);
  return cudaGetLastError();
}

cudaError_t launch_smooth_tma_withheld(float* x, const Geom& G, const InvDiag<float>& inv, const TmaSweep& t, int* err,
                                       long long budget_cycles, cudaStream_t s) {
  return launch_smooth_tma_cfg<Product>(x, G, inv, 0, t, err, budget_cycles, 2, s);
}

}  // namespace ccmg
