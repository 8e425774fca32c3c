// ccmg_internal.cuh -- internal types and kernel launchers of libccmg (not part of the ABI).
//
// Storage of a multigrid level. Every level except the coarsest stores its cells in the
// checkerboard-separated order that red-black Gauss-Seidel works in (Sec. 5.3: the unknowns are
// rearranged in a checker-board manner so that each colour updates in parallel): two arrays per
// field, one per colour, each of (nx/2) x ny x nz entries, x fastest. Cell (i,j,k) has colour
// c = (i+j+k) & 1 and sits at index m = i/2 of row (j,k) of its colour's array; within the row,
// i = 2m + s with s = (j+k+c) & 1. Then
//   - its two x-neighbours are at m+s-1 and m+s of the other colour's row (j,k),
//   - its four y/z-neighbours are at the same m in the other colour's rows (j+-1,k), (j,k+-1),
// so a half-sweep reads one colour and writes the other with unit-stride, fully used lines.
// The coarsest level (solved by CG, possibly with odd dimensions) is stored in natural order.
//
// Every level stores the scaled right-hand side g_l = f_l / c_l (c_l = 1/(2^l h^2) is the
// coefficient of the Galerkin operator on level l), so the smoother is
//   phi_i = (g_i + sum of neighbours) / (6 + d_i),
// the scaled residual is r_i / c_l = g_i + sum - (6 + d_i) phi_i, and the averaging restriction
// into the next level's scaled right-hand side is (1/4) * (sum of the 8 children's scaled
// residuals): all level-to-level factors are powers of two.
#pragma once
#include <cuda.h>  // CUtensorMap (types only; the encoder is fetched from the driver at run time)
#include <cuda_runtime.h>
#include <stdint.h>

namespace ccmg {

constexpr int kMaxLevels = 24;
constexpr int kMaxCoarseCells = 4096;
// Relative residuals at which the coarsest CG stops: FP64 levels 1e-14; the single-precision
// levels of the mixed solver's inner cycles 1e-5 (float cannot reach 1e-14, and the inner
// cycles' correction needs no more on the coarsest grid).
constexpr double kCoarseRtol = 1e-14, kCoarseRtolF32 = 1e-5;
template <typename T>
constexpr double coarse_rtol() { return sizeof(T) == sizeof(float) ? kCoarseRtolF32 : kCoarseRtol; }

struct Geom {
  int nx, ny, nz;  // cells per axis
  int hx;          // nx / 2 on packed levels
  long long csz;   // entries per colour array (packed) or nx*ny*nz (natural)
  int packed;      // 1: red/black arrays; 0: natural order
  int sh[6];       // diagonal shift of each face (+1 Dirichlet, -1 Neumann, 0 periodic)
  int per;         // bit a set: axis a (0 x, 1 y, 2 z) is periodic (its neighbour wraps around)
};

// Diagonal shift of a face of type t (0 Dirichlet, 1 Neumann, 2 periodic; Sec. 2.4).
inline int face_shift(int t) { return t == 0 ? 1 : (t == 1 ? -1 : 0); }
// nullptr if six face types form a valid, non-singular set: each Dirichlet, Neumann or periodic,
// periodic faces in opposite pairs, and at least one Dirichlet face (Neumann and periodic walls
// alone leave the constant in the null space); else the reason.
inline const char* check_bc_types(const int* type6) {
  bool dirichlet = false;
  for (int q = 0; q < 6; ++q) {
    if (type6[q] < 0 || type6[q] > 2) return "bc_type must be MG_BC_DIRICHLET, MG_BC_NEUMANN or MG_BC_PERIODIC";
    if (type6[q] == 0) dirichlet = true;
  }
  for (int a = 0; a < 3; ++a)
    if ((type6[2 * a] == 2) != (type6[2 * a + 1] == 2)) return "periodic faces come in opposite pairs";
  if (!dirichlet) return "walls without a Dirichlet face give a singular problem";
  return nullptr;
}

// Periodic-axis bits of six face types (both faces of an axis periodic).
inline int periodic_bits(const int* type6) {
  int b = 0;
  for (int a = 0; a < 3; ++a)
    if (type6[2 * a] == 2 && type6[2 * a + 1] == 2) b |= 1 << a;
  return b;
}

template <typename T>
struct InvDiag {
  T v[7];  // 1 / (6 + d) for d = -3 .. 3
};

// Wall conditions of the six faces (0:-x 1:+x 2:-y 3:+y 4:-z 5:+z): type 0 Dirichlet, 1 Neumann,
// 2 periodic (both faces of an axis; no value), with one value per face, or, where field[q] is set, one value per face cell (faces 0,1: index
// j + ny k; 2,3: i + nx k; 4,5: i + nx j), device memory the context owns.
struct FaceBC {
  int type[6];
  double value[6];
  const double* field[6];
};

// Index of boundary cell (i, j, k) in face q's per-cell array, and the number of face cells.
__host__ __device__ __forceinline__ long long face_index(int q, int i, int j, int k, int nx, int ny) {
  return q < 2 ? (long long)j + (long long)ny * k
               : (q < 4 ? (long long)i + (long long)nx * k : (long long)i + (long long)nx * j);
}
__host__ __device__ __forceinline__ long long face_cells(int q, int nx, int ny, int nz) {
  return q < 2 ? (long long)ny * nz : (q < 4 ? (long long)nx * nz : (long long)nx * ny);
}

inline bool has_field(const FaceBC& bc) {
  for (int q = 0; q < 6; ++q)
    if (bc.field[q]) return true;
  return false;
}

// The value of face q's condition at its boundary cell (i, j, k).
__device__ __forceinline__ double face_value(const FaceBC& bc, int q, int i, int j, int k, int nx, int ny) {
  const double* f = bc.field[q];
  return f ? __ldg(f + face_index(q, i, j, k, nx, ny)) : bc.value[q];
}

// Variable permittivity and reaction term (var_kernels.cu): var_arrays() coefficient arrays per
// level (D, wx, wy, wz, 1/D, Dw, M, each of the level's cell count, in its storage order) at vc[l].
long long var_cells(const Geom& G);
int var_arrays();
cudaError_t launch_var_setup(const double* eps, const double* react, double h, double omega, const Geom* geo, int L,
                             const FaceBC& bc, double* const* vc, cudaStream_t s);
cudaError_t launch_var_coarsen_all(const Geom* geo, int L, double* const* vc, double omega, cudaStream_t s);
cudaError_t launch_pb_update(const double* x, const double* g0, double* vc, const Geom& G, const double* k2, double h,
                             double* f, double* partials, int* nparts, cudaStream_t s);
cudaError_t launch_axpy(double* y, const double* x, long long n, cudaStream_t s);
cudaError_t launch_fill(double* y, double v, long long n, cudaStream_t s);
template <typename T>
cudaError_t launch_var_smooth(T* x, const T* g, const T* vc, const Geom& G, int colour, bool zero, cudaStream_t s);
template <typename T>
cudaError_t launch_var_resid_restrict(const T* x, const T* g, const T* vc, const Geom& G, T* gc, const Geom& Gc,
                                      cudaStream_t s);
// mode 0: partial sums; 1: also the natural-order residual; 2: also the float copy float(r~ isc)
cudaError_t launch_var_resid_norm(const double* x, const double* g, const double* vc, const Geom& G, double c0,
                                  double* partials, int* nparts, int mode, double* out_natural, float* out_packed,
                                  const double* inv_scale, cudaStream_t s);
template <typename T>
cudaError_t launch_var_coarse_cg(T* x, const T* b, const T* vc, const Geom& Gc, double rtol, int maxit, int* d_iters,
                                 cudaStream_t s);
// single-precision copies of the cycle's coefficients (var_arrays32() arrays per level)
int var_arrays32();
cudaError_t launch_var_to_f32(const double* const* vc, float* const* v32, const Geom* geo, int L, cudaStream_t s);
cudaError_t prepare_var_coarse_cg();
cudaError_t launch_var_set_rhs(double* g, const Geom& G, const double* rho, const double* eps, double h,
                               const FaceBC& bc, cudaStream_t s);

// Kernel launchers (all enqueue on `s`; return cudaGetLastError()).
template <typename T>
cudaError_t launch_smooth(T* x, const T* g, const Geom& G, const InvDiag<T>& inv, int colour, bool zero_start,
                          cudaStream_t s);
// Black half-sweep of single-precision level (x, g, G) fused with the prolongation of the
// coarse correction ec (level Gc) into its red neighbours; rows must be a multiple of 4 long.
cudaError_t launch_smooth_prolong(float* x, const float* g, const Geom& G, const InvDiag<float>& inv, const float* ec,
                                  const Geom& Gc, float omega, cudaStream_t s);
// TMA-staged single-precision half-sweep (smooth_tma.cu): persistent CTAs march tiles of a level
// through z-slabs, the other colour's planes staged in shared memory by tensor-map copies.
struct TmaSweep {
  CUtensorMap other[2];   // other[c]: the colour-(1-c) array, read by a colour-c half-sweep
  CUtensorMap rhs[2];     // rhs[c]: the colour-c right-hand side
  CUtensorMap coarse[2];  // the next level's correction (both colours), for the fused prolongation
  long long nwork, nwork_pro;  // tiles x slabs
  int kz, kz_pro;              // planes per slab
  int grid, grid_pro;          // persistent CTAs
  int ok;                      // 1 when the level uses this path
  int ok_pro;                  // 1 when its first black post-sweep runs fused with the prolongation
};
// The finest level of one system of a batch, for the batched TMA-staged half-sweep: its tensor
// maps (other[c], rhs[c] as in TmaSweep; coarse[] the next level's correction, for the fused
// prolongation), geometry, iterate, slab length and its first work item in the launch.
struct BTmaSys {  // aligned as its CUtensorMap members
  CUtensorMap other[2];
  CUtensorMap rhs[2];
  CUtensorMap coarse[2];
  Geom G;
  float* x;
  int sys;
  int kz;
  long long w0;     // first work item (items of one system are consecutive)
  long long nwork;  // tiles x slabs
};
// The FP64 half-sweep staged the same way (levels without a periodic axis): same results as
// launch_smooth<double> (the neighbour sum in exact fixed point, each value converted once).
bool tma_sweep64_applies(const Geom& G);
bool tma_sweep64_pays(const Geom& G);
cudaError_t prepare_tma_sweep64(TmaSweep& t, double* x, const double* g, const Geom& G, int device);
cudaError_t launch_smooth_tma64(double* x, const double* g, const Geom& G, const InvDiag<double>& inv, int colour, const TmaSweep& t,
                                int* err, cudaStream_t s);
cudaError_t launch_smooth_tma64_withheld(double* x, const double* g, const Geom& G, const InvDiag<double>& inv, const TmaSweep& t,
                                         int* err, long long budget_cycles, cudaStream_t s);
bool tma_sweep_applies(const Geom& G);  // the kernel can run on this level
bool tma_sweep_pays(const Geom& G);     // ... and is the faster of the two here
// Encode the tensor maps of level arrays x and g (both colours) and size the launch; t.ok = 0
// when the level does not qualify.
cudaError_t prepare_tma_sweep(TmaSweep& t, float* x, const float* g, const Geom& G, int device);
// Same result as launch_smooth<float>(x, g, ..., zero_start = false), bit for bit (g is the one
// the maps were made for). On a wait that runs out of its budget a CTA sets *err = 1 and returns.
cudaError_t launch_smooth_tma(float* x, const Geom& G, const InvDiag<float>& inv, int colour, const TmaSweep& t,
                              int* err, cudaStream_t s);
// The fused prolongation + black sweep in the same scheme (t prepared with a packed coarse level
// ec, Gc of half the size in every direction); same result as launch_smooth_prolong.
cudaError_t prepare_tma_prolong(TmaSweep& t, const float* ec, const Geom& Gc, const Geom& G, int device);
cudaError_t launch_smooth_prolong_tma(float* x, const Geom& G, const InvDiag<float>& inv, const TmaSweep& t,
                                      float omega, int* err, cudaStream_t s);
// Batched systems: fills sys (one entry per system: finest level x, g of geometry G, next level xc,
// Gc packed with whole 4-float rows) with tensor maps, slab lengths and work offsets; returns in
// *total the number of work items and in *grid the persistent grid of the launches below; *ok = 0
// when some system does not qualify (then nothing else is written).
cudaError_t prepare_tma_batch(BTmaSys* sys, int n, float* const* x, const float* const* g, const Geom* G,
                              const float* const* xc, const Geom* Gc, const int* sys_index, long long* total,
                              int* grid, int* ok, int device);
// The batched half-sweep of colour `colour` over the finest levels in the device table d_sys (n
// entries, total work items), systems with active[sys] == 0 skipped; same results as the
// single-system sweep of each. The fused prolongation variant: first black post-sweep.
cudaError_t launch_b_smooth_tma(const BTmaSys* d_sys, int n, long long total, int grid, const int* active,
                                const InvDiag<float>& inv, int colour, int* err, cudaStream_t s);
cudaError_t launch_b_smooth_prolong_tma(const BTmaSys* d_sys, int n, long long total, int grid, const int* active,
                                        const InvDiag<float>& inv, float omega, int* err, cudaStream_t s);
// Failure-path self-test: the same red half-sweep with one plane copy of every CTA's first item
// never issued, and a wait budget of budget_cycles; every CTA then sets *err and returns.
cudaError_t launch_smooth_tma_withheld(float* x, const Geom& G, const InvDiag<float>& inv, const TmaSweep& t, int* err,
                                       long long budget_cycles, cudaStream_t s);

template <typename T>
// red_only: restrict only the red children's residuals (right after a black half-sweep the black
// residuals are zero up to rounding).
cudaError_t launch_resid_restrict(const T* x, const T* g, const Geom& G, T* gc, const Geom& Gc, bool red_only,
                                  cudaStream_t s);
// FP64 residual + restriction by the fixed-point residual walk (packed levels of at least one
// tile width); the direct-load kernel above serves the other levels and single precision.
bool resid_restrict_walk_applies(const Geom& G);
cudaError_t launch_resid_restrict_walk(const double* x, const double* g, const Geom& G, double* gc, const Geom& Gc,
                                       cudaStream_t s);
template <typename T>
cudaError_t launch_prolong(T* x, const Geom& G, const T* ec, const Geom& Gc, T omega, bool red_only,
                           cudaStream_t s);
template <typename T>
cudaError_t launch_coarse_cg(T* x, const T* b, const Geom& Gc, double rtol, int maxit, int* d_iters,
                             cudaStream_t s);
cudaError_t prepare_coarse_cg();

// Scaled residual r~ = g + sum - (6+d) x over the finest level. Writes per-block partial sums
// of r~^2 to `partials` (at most kMaxPartials) and, by mode:
//   0: nothing else;
//   1: r = r~ * c0 in natural order, double (d_out_natural);
//   2: float(r~ * inv_scale[0]) into a packed float array of the same geometry (d_out_packed).
constexpr int kMaxPartials = 4096;
template <typename T>
cudaError_t launch_resid_norm(const T* x, const T* g, const Geom& G, double* partials, int* nparts, int mode,
                              double c0, double* out_natural, float* out_packed, const double* inv_scale,
                              cudaStream_t s);
// Sum of squares of a packed or natural field (||g||^2), same partial-sum protocol.
template <typename T>
cudaError_t launch_sumsq(const T* a, long long n, double* partials, int* nparts, cudaStream_t s);
// Fixed-order sum of partials into scal[slot]; if slot_rel >= 0 also writes
// scal[slot_rel] = sqrt(scal[slot]) / sqrt(scal[slot_ref]) (or sqrt(scal[slot]) if ref is 0).
cudaError_t launch_finalize(const double* partials, int nparts, double* scal, int slot, int slot_rel, int slot_ref,
                            cudaStream_t s);
// scal[dst] = sqrt(scal[src] / n) if positive else 1; scal[dst+1] = 1 / scal[dst].
cudaError_t launch_set_scale(double* scal, int src, int dst, double n, cudaStream_t s);

// g = (rho/eps + wall terms) * h^2 written into a packed (or natural) level-0 array.
template <typename T>
cudaError_t launch_set_rhs(T* g, const Geom& G, const double* rho, double inv_eps, double h, const FaceBC& bc,
                           int raw, cudaStream_t s);
// Natural-order double <-> level layout and precision.
template <typename T>
cudaError_t launch_pack(T* dst, const Geom& G, const double* src, double scale, cudaStream_t s);
template <typename T>
cudaError_t launch_unpack(double* dst, const T* src, const Geom& G, double scale, cudaStream_t s);
// Termination residual of a zero iterate (r = f exactly): scal[rsum] = scal[gsum], scal[rel] = 1
// (0 if f = 0); with outp also float(g * scal[inv_scale]) over n entries (mixed precision).
cudaError_t launch_resid_zero(const double* g, long long n, float* outp, double* scal, int slot_rsum, int slot_rel,
                              int slot_gsum, int slot_inv_scale, cudaStream_t s);
// x64 += scal[slot] * double(e32) elementwise over n entries.
cudaError_t launch_scale_convert(const double* x, const float* e, const double* y, long long n, double sc, float* xf,
                                 double* yo, double* xs, cudaStream_t s);
// x = s e for an iterate that is zero (x is not read).
cudaError_t launch_set_mixed(double* x, const float* e, long long n, const double* scal, int slot, cudaStream_t s);
cudaError_t launch_update_mixed(double* x, const float* e, long long n, const double* scal, int slot, cudaStream_t s);
// The outer step with the residual carried by recurrence (defect_kernels.cu): x += s e (x = s e
// for a zero, unwritten iterate: `zero`, the pair then formed from g / s), the residual pair
// (qh, ql) in units of s = scal[slot] becomes (pair - A e) in units of scal[slot_next], and the
// per-block sums of squares of the new qh go to partials (*nparts of them). Packed levels with
// rows of whole 4-float vectors (defect_rec_applies).
bool defect_rec_applies(const Geom& G);
cudaError_t launch_defect_rec(double* x, const float* e, float* qh, float* ql, const double* g, const Geom& G,
                              double* scal, int slot, int slot_next, bool zero, double* partials, int* nparts,
                              cudaStream_t s);
// scal[rsum] = sum(partials) scal[next]^2, scal[rel] = sqrt(rsum / scal[gsum]), then the next
// scale and its inverse move into scal[scale], scal[scale + 1].
cudaError_t launch_defect_finalize(const double* partials, int nparts, double* scal, int slot_rsum, int slot_rel,
                                   int slot_gsum, int slot_scale, int slot_next, cudaStream_t s);
// Natural-order double field times 2^q -> the packed float pair (qh, ql) (verification).
cudaError_t launch_pack_pair(float* qh, float* ql, const Geom& G, const double* src, int q, cudaStream_t s);

// Fields and forces (finest level, FP64 packed potential).
struct Spheres {
  int P;
  const double* c;  // P*3
  const double* r;  // P
  const double* q;  // P (density), may be null where unused
};
// E = -grad phi, [3][N] natural order; stencil 7 (D3Q7 central differences) or 19 (D3Q19 where
// all 18 neighbours exist, D3Q7 elsewhere).
cudaError_t launch_efield(const double* x, const Geom& G, double h, const FaceBC& bc, int stencil, double* E,
                          cudaStream_t s);
cudaError_t launch_sphere_density(const Geom& G, double h, const Spheres& sp, int sf, double* rho, cudaStream_t s);
cudaError_t launch_force_gather(const double* x, const Geom& G, double h, const FaceBC& bc, int stencil,
                                const Spheres& sp, int sf, double* F, cudaStream_t s);
cudaError_t launch_force_adjoint(const double* x, const Geom& G, double h, const FaceBC& bc, const Spheres& sp, int sf,
                                 const double* wF, double* gphi, double* gdens, double* gbc, cudaStream_t s);
cudaError_t launch_density_adjoint(const Geom& G, double h, const Spheres& sp, int sf, const double* gfield,
                                   double* gdens, cudaStream_t s);
cudaError_t launch_rhs_adjoint(const Geom& G, double h, double inv_eps, const FaceBC& bc, const double* eps,
                               const double* lam, double* grho, double* gbc, cudaStream_t s);

// ------------------------------------------------------------------------------------------------
// Batched launches over many independent systems of different sizes. One entry describes one
// system at one level; an entry owns the block range [start[e], start[e+1]) of the launch, laid
// out as gx * gy * gz blocks (gz = planes). A block whose system is inactive returns at once.
struct BEntry {
  Geom G;        // the entry's level
  Geom Gc;       // next-coarser level (restriction / prolongation entries)
  void* x;       // level iterate (T)
  void* g;       // level scaled right-hand side (T)
  void* xc;      // next-coarser iterate
  void* gc;      // next-coarser right-hand side
  void* aux;     // residual entries: float residual output (mixed); update entries: float correction
  int sys;       // system index
  int gx, gy, gz;
  int vec;       // smoother: 16-byte vector path
  int pad;
};

struct BLaunch {
  const BEntry* entries;  // device
  const int* start;       // device, count + 1 block offsets
  int count;
  int blocks;             // start[count]
  dim3 block;
  int per;                // some system of the launch has a periodic axis
};

template <typename T>
cudaError_t launch_b_smooth(const BLaunch& L, const int* active, const InvDiag<T>& inv, int colour, bool zero,
                            cudaStream_t s);
template <typename T>
cudaError_t launch_b_resid_restrict(const BLaunch& L, const int* active, bool red_only, cudaStream_t s);
template <typename T>
cudaError_t launch_b_prolong(const BLaunch& L, const int* active, T omega, bool red_only, cudaStream_t s);
// First black post-sweep (single precision): fused with the prolongation for vector entries (as
// launch_smooth_prolong), a plain black sweep for the others (prolonged before).
cudaError_t launch_b_smooth_prolong(const BLaunch& L, const int* active, const InvDiag<float>& inv, float omega,
                                    cudaStream_t s);
template <typename T>
cudaError_t launch_b_coarse_cg(const BLaunch& L, const int* active, size_t smem, double rtol, cudaStream_t s);
cudaError_t prepare_b_coarse_cg();
// The wall terms of a right-hand side (Sec. 2.4): t[q] = 2 value / h^2 (Dirichlet), value / h
// (Neumann), 0 (periodic) for a face with one value; field[q] for a face with values per cell.
struct WallTerms {
  double t[6];
  const double* field[6];
  int type[6];
  double h;
};
WallTerms make_wall_terms(const FaceBC& bc, double h);

// One system of a batched right-hand-side setting (mg_batch_set_rhs_all): its finest level, the
// factors and wall terms of its set_rhs, its scalars, and the block layout of its sum of squares
// (the one launch_sumsq takes, so that the norms equal a single context's).
struct RhsJob {
  Geom G;
  double* g;          // finest scaled right-hand side
  const double* rho;  // this call's charge density, natural order
  double inv_eps, hsq;
  int qe, qh, pow2, fld;
  WallTerms wt;
  int pair;      // packed level and 16-byte aligned rho: two cells per thread
  long long b0;  // first block of this system in the right-hand-side launch
  int sb0, sbn;  // its sum-of-squares blocks: first, count
  double* scal;  // its scalars
  double n;      // its cells
};
// The parts of a job that do not change from call to call (all but rho, pair and b0).
void rhs_job_static(RhsJob& j, const Geom& G, double* g, double inv_eps, double h, const FaceBC& bc, double* scal);
// Right-hand sides, their sums of squares (partials: one per sum-of-squares block of all jobs),
// norms into slot_gsum and the first defect-correction scale into slot_scale (and its
// reciprocal) of every job's scalars: three launches for the whole batch.
cudaError_t launch_set_rhs_all(const RhsJob* d_jobs, int B, long long nblocks, int nsblocks, double* partials,
                               int slot_gsum, int slot_scale, cudaStream_t s);

// Per-system scalars of a batch: kScalStride doubles per system, same slots as a single context.
constexpr int kScalStride = 8;
constexpr int kSlotGsum = 0, kSlotRsum = 1, kSlotRel = 2, kSlotScale = 3, kSlotInvScale = 4;
constexpr int kSlotNext = 5;  // the next scale (and its inverse at 6) while a recurrence step runs
// FP64 residual of every system's finest level (mode 0 or 2, as launch_resid_norm), per-block
// partials, then one finalize block per system: rsum, rel = sqrt(rsum / gsum) in its slots.
// zero[s] != 0: system s's iterate is exactly zero, its norm is taken from the gsum slot.
cudaError_t launch_b_resid_norm(const BLaunch& L, const int* active, const int* zero, int mode, double* scal,
                                double* partials, cudaStream_t s);
// x64 += scale * double(e32) on every active system's finest level (update entries), except the
// systems that step by recurrence (rec[sys]; rec may be null).
cudaError_t launch_b_update(const BLaunch& L, const int* active, const int* rec, const int* zero, const double* scal,
                            cudaStream_t s);
// scale = sqrt(rsum / n) (1 if not positive and finite), inv_scale = 1 / scale, per system (not
// those with rec[sys]; rec may be null).
cudaError_t launch_b_set_scale(const BLaunch& L, const int* active, const int* rec, double* scal, cudaStream_t s);
// The recurrence step over the active systems with rec[sys] (defect_kernels.cu): per system the
// next scale, the step (bit-identical to its single-system launch, entries of defect_rec_blocks
// virtual blocks: x phi, g g, xc e, gc the pair's hi, aux its lo), the norm and scale update.
int defect_rec_blocks(const Geom& G);
cudaError_t launch_b_defect_step(const BLaunch& L, const int* active, const int* rec, const int* zero, double* scal,
                                 double* partials, cudaStream_t s);

}  // namespace ccmg
