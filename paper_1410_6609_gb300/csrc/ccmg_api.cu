// ccmg_api.cu -- host side of libccmg: the C ABI declared in include/ccmg.h.
//
// A context owns the level hierarchy on one device (Sec. 5.3: the multigrid solver allocates all
// coarse-grid data itself), the wall conditions and a few device scalars. The V-cycle of Sec. 3 /
// Sec. 5.3 is enqueued as a fixed kernel sequence, captured once into a CUDA graph on a private
// stream and replayed on the caller's stream; the termination test of Algorithm 1 is a second,
// small graph (residual norm + fixed-order reduction) followed by one 8-byte read-back.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <type_traits>

#include "../../include/ccmg.h"
#include "ccmg_internal.cuh"

using namespace ccmg;

namespace {

enum Slot {
  S_GSUM = 0, S_RSUM = 1, S_REL = 2, S_SCALE = 3, S_INV_SCALE = 4, S_PB_REF = 5, S_PB_REL = 6,
  S_NEXT = 8,  // the next outer step's scale and its inverse (9) while a recurrence step runs
  S_COUNT = 10
};

thread_local std::string g_create_error;

}  // namespace

struct mg_ctx {
  mg_params p{};
  cudaStream_t stream = nullptr;  // caller's stream
  cudaStream_t cap = nullptr;     // private stream used only for graph capture
  int L = 0;
  Geom geo[kMaxLevels]{};
  double* x64[kMaxLevels]{};
  double* g64[kMaxLevels]{};
  float* x32[kMaxLevels]{};
  float* g32[kMaxLevels]{};
  double* partials = nullptr;
  double* scal = nullptr;
  double* h_pin = nullptr;
  int* d_iters = nullptr;
  InvDiag<double> inv64{};
  InvDiag<float> inv32{};
  FaceBC bc{};
  cudaGraphExec_t g_cycle = nullptr;
  cudaGraphExec_t g_cycle0 = nullptr;  // mixed: the first cycle from a zero iterate (phi = s e)
  cudaGraphExec_t g_resid = nullptr;
  cudaGraphExec_t g_resid0 = nullptr;  // the termination residual of a zero iterate (r = f)
  cudaGraphExec_t g_check = nullptr;   // mixed: the termination residual without the float copy
  cudaGraphExec_t g_rec = nullptr;   // mixed: a cycle whose update carries the residual by recurrence
  cudaGraphExec_t g_rec0 = nullptr;  // the same from a zero iterate
  long long n_cycle = 0, n_cycle0 = 0, n_resid = 0, n_resid0 = 0, n_rec = 0, n_rec0 = 0,
            n_check = 0;  // kernel nodes per graph
  float* q_lo = nullptr;     // mixed: low part of the residual pair whose high part is g32[0] (recurrence)
  bool rec_on = false;       // mixed solves carry the residual by recurrence between direct checks
  long long cnt_cycles = 0, cnt_rec = 0, cnt_direct = 0;  // outer cycles, those by recurrence, direct residuals
  bool phi_zero = true;                // the finest iterate is known to be exactly zero
  bool x_lazy = false;                 // mixed: x64[0] holds no data, its value is zero
  long long launches = 0;
  double* d_rho = nullptr;  // step_host scratch: density field
  double* d_sph = nullptr;  // step_host scratch: 8*P doubles (centres, radius, density, forces)
  int sph_cap = 0;
  TmaSweep tma[kMaxLevels]{};  // TMA-staged single-precision half-sweeps, per level
  TmaSweep tma64[kMaxLevels]{};  // TMA-staged FP64 half-sweeps (FP64 mode), per level
  unsigned char rr_walk[kMaxLevels]{};  // FP64 residual + restriction by the fixed-point walk, per level
  int* d_err = nullptr;        // set by a kernel whose bounded wait ran out
  int grad_stencil = 7;        // gradient of mg_efield / mg_force_gather: 7 (D3Q7) or 19 (D3Q19)
  double* d_bcf[6] = {};       // per-cell wall values of each face (allocated on first use)
  double* d_eps = nullptr;     // weighted operator: cell permittivities (null: the constant operator)
  bool eps_set = false;        // d_eps came from mg_set_permittivity (else the constant eps)
  double* d_k2 = nullptr;      // reaction coefficients (screened / Poisson-Boltzmann), or null
  double* vc[kMaxLevels]{};    // weighted coefficients per level (D, wx, wy, wz, 1/D, Dw, M)
  float* vc32[kMaxLevels]{};   // MG_MIXED: their single-precision copies (D, wx, wy, wz, 1/D)
  double* d_pb = nullptr;      // Newton state: base right-hand side and potential (2 finest fields)
  std::string err;
};

namespace {

mg_status fail(mg_ctx* c, mg_status st, const std::string& msg) {
  if (c) c->err = msg;
  else g_create_error = msg;
  return st;
}

mg_status cuda_fail(mg_ctx* c, cudaError_t e, const char* where) {
  return fail(c, MG_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(call, where)                                  \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return cuda_fail(c, e_, where); \
  } while (0)

bool mixed(const mg_ctx* c) { return c->p.prec == MG_MIXED; }
long long cells(const Geom& G) { return G.packed ? 2 * G.csz : G.csz; }
double level_coeff(const mg_ctx* c, int l) { return 1.0 / (std::ldexp(1.0, l) * c->p.h * c->p.h); }

void free_all(mg_ctx* c) {
  if (c->g_cycle) cudaGraphExecDestroy(c->g_cycle);
  if (c->g_cycle0) cudaGraphExecDestroy(c->g_cycle0);
  if (c->g_resid) cudaGraphExecDestroy(c->g_resid);
  if (c->g_resid0) cudaGraphExecDestroy(c->g_resid0);
  if (c->g_check) cudaGraphExecDestroy(c->g_check);
  if (c->g_rec) cudaGraphExecDestroy(c->g_rec);
  if (c->g_rec0) cudaGraphExecDestroy(c->g_rec0);
  cudaFree(c->q_lo);
  for (int l = 0; l < kMaxLevels; ++l) {
    cudaFree(c->x64[l]);
    cudaFree(c->g64[l]);
    cudaFree(c->x32[l]);
    cudaFree(c->g32[l]);
  }
  for (int q = 0; q < 6; ++q) cudaFree(c->d_bcf[q]);
  cudaFree(c->d_eps);
  cudaFree(c->d_k2);
  cudaFree(c->d_pb);
  for (int l = 0; l < kMaxLevels; ++l) {
    cudaFree(c->vc[l]);
    cudaFree(c->vc32[l]);
  }
  cudaFree(c->partials);
  cudaFree(c->scal);
  cudaFree(c->d_iters);
  cudaFree(c->d_rho);
  cudaFree(c->d_sph);
  cudaFree(c->d_err);
  if (c->h_pin) cudaFreeHost(c->h_pin);
  if (c->cap) cudaStreamDestroy(c->cap);
}

// ------------------------------------------------------------------------------------------
// Enqueue helpers (usable inside stream capture)

// One half-sweep of level l: the TMA-staged kernel where the level has one (single precision,
// not from a zero iterate), else the vectorised one; identical results.
template <typename T>
cudaError_t sweep(mg_ctx* c, T* x, const T* g, const InvDiag<T>& inv, int l, int colour, bool zero, cudaStream_t s) {
  if constexpr (std::is_same<T, float>::value) {
    if (!zero && c->tma[l].ok && x == c->x32[l] && g == c->g32[l])
      return launch_smooth_tma(x, c->geo[l], inv, colour, c->tma[l], c->d_err, s);
  } else {
    if (!zero && c->tma64[l].ok && x == c->x64[l] && g == c->g64[l])
      return launch_smooth_tma64(x, g, c->geo[l], inv, colour, c->tma64[l], c->d_err, s);
  }
  return launch_smooth<T>(x, g, c->geo[l], inv, colour, zero, s);
}

// The V-cycle with the weighted operators (the same steps, weighted kernels), in double on the
// FP64 hierarchy or in single precision on the inner-cycle hierarchy of MG_MIXED.
template <typename T>
cudaError_t enqueue_vcycle_var(mg_ctx* c, T* const* xs, T* const* gs, const T* const* vcs, int l, bool zero,
                               cudaStream_t s, long long* nk) {
  const Geom& G = c->geo[l];
  T* x = xs[l];
  const T* g = gs[l];
  cudaError_t e;
  if (l == c->L - 1) {
    ++*nk;
    return launch_var_coarse_cg<T>(x, g, vcs[l], G, 1e-14, 2 * G.nx * G.ny * G.nz, c->d_iters, s);
  }
  if (zero && c->p.nu1 == 0) {
    e = cudaMemsetAsync(x, 0, sizeof(T) * (size_t)cells(G), s);
    if (e != cudaSuccess) return e;
  }
  for (int it = 0; it < c->p.nu1; ++it) {
    if ((e = launch_var_smooth<T>(x, g, vcs[l], G, 0, zero && it == 0, s)) != cudaSuccess) return e;
    if ((e = launch_var_smooth<T>(x, g, vcs[l], G, 1, false, s)) != cudaSuccess) return e;
    *nk += 2;
  }
  if ((e = launch_var_resid_restrict<T>(x, g, vcs[l], G, gs[l + 1], c->geo[l + 1], s)) != cudaSuccess) return e;
  ++*nk;
  if ((e = enqueue_vcycle_var<T>(c, xs, gs, vcs, l + 1, true, s, nk)) != cudaSuccess) return e;
  // the correction factor is in the coarse operators (var_kernels.cu): weight 1 here
  if ((e = launch_prolong<T>(x, G, xs[l + 1], c->geo[l + 1], T(1), c->p.nu2 >= 1, s)) != cudaSuccess) return e;
  ++*nk;
  for (int it = 0; it < c->p.nu2; ++it) {
    if ((e = launch_var_smooth<T>(x, g, vcs[l], G, 1, false, s)) != cudaSuccess) return e;
    if ((e = launch_var_smooth<T>(x, g, vcs[l], G, 0, false, s)) != cudaSuccess) return e;
    *nk += 2;
  }
  return cudaSuccess;
}

template <typename T>
cudaError_t enqueue_vcycle(mg_ctx* c, T* const* x, T* const* g, const InvDiag<T>& inv, int l, bool zero,
                           cudaStream_t s, long long* nk) {
  const Geom& G = c->geo[l];
  cudaError_t e;
  if (l == c->L - 1) {
    const int n = G.nx * G.ny * G.nz;
    ++*nk;
    return launch_coarse_cg<T>(x[l], g[l], G, coarse_rtol<T>(), 2 * n, c->d_iters, s);
  }
  if (zero && c->p.nu1 == 0) {
    e = cudaMemsetAsync(x[l], 0, sizeof(T) * (size_t)cells(G), s);
    if (e != cudaSuccess) return e;
  }
  for (int it = 0; it < c->p.nu1; ++it) {
    if ((e = sweep<T>(c, x[l], g[l], inv, l, 0, zero && it == 0, s)) != cudaSuccess) return e;
    if ((e = sweep<T>(c, x[l], g[l], inv, l, 1, false, s)) != cudaSuccess) return e;
    *nk += 2;
  }
  // single precision: after a black half-sweep the black residuals are at float rounding level,
  // below what the inner cycle resolves, so only the red residuals are restricted. Double
  // precision keeps them: near FP64 convergence those rounding residuals are the residual.
  const bool red_only = std::is_same<T, float>::value && c->p.nu1 >= 1;
  if constexpr (std::is_same<T, double>::value) {
    if (c->rr_walk[l] && x == c->x64 && !red_only)
      e = launch_resid_restrict_walk(x[l], g[l], G, g[l + 1], c->geo[l + 1], s);
    else
      e = launch_resid_restrict<T>(x[l], g[l], G, g[l + 1], c->geo[l + 1], red_only, s);
  } else {
    e = launch_resid_restrict<T>(x[l], g[l], G, g[l + 1], c->geo[l + 1], red_only, s);
  }
  if (e != cudaSuccess) return e;
  ++*nk;
  if ((e = enqueue_vcycle<T>(c, x, g, inv, l + 1, true, s, nk)) != cudaSuccess) return e;
  // single precision, vector rows: the prolongation is fused into the first black half-sweep
  const bool fuse = std::is_same<T, float>::value && (G.hx % 4 == 0) && c->p.nu2 >= 1;
  if (!fuse) {
    if ((e = launch_prolong<T>(x[l], G, x[l + 1], c->geo[l + 1], (T)c->p.cgc_weight, c->p.nu2 >= 1, s)) !=
        cudaSuccess)
      return e;
    ++*nk;
  }
  for (int it = 0; it < c->p.nu2; ++it) {
    if (fuse && it == 0 && c->tma[l].ok_pro)
      e = launch_smooth_prolong_tma((float*)x[l], G, c->inv32, c->tma[l], (float)c->p.cgc_weight, c->d_err, s);
    else if (fuse && it == 0)
      e = launch_smooth_prolong((float*)x[l], (const float*)g[l], G, c->inv32, (const float*)x[l + 1],
                                c->geo[l + 1], (float)c->p.cgc_weight, s);
    else
      e = sweep<T>(c, x[l], g[l], inv, l, 1, false, s);
    if (e != cudaSuccess) return e;
    if ((e = sweep<T>(c, x[l], g[l], inv, l, 0, false, s)) != cudaSuccess) return e;
    *nk += 2;
  }
  return cudaSuccess;
}

// One cycle: FP64 V-cycle, or (mixed) mixed_inner single-precision V-cycles on the scaled
// residual that the residual graph left in g32[0] (the first from e = 0), followed by
// phi += scale * e (phi = scale * e for a zero iterate, `first`) and the next scale.
cudaError_t enqueue_cycle(mg_ctx* c, cudaStream_t s, long long* nk, bool first) {
  if (c->d_eps && !mixed(c)) return enqueue_vcycle_var<double>(c, c->x64, c->g64, c->vc, 0, false, s, nk);
  if (!mixed(c)) return enqueue_vcycle<double>(c, c->x64, c->g64, c->inv64, 0, false, s, nk);
  cudaError_t e = cudaSuccess;
  for (int it = 0; it < c->p.mixed_inner; ++it) {
    e = c->d_eps ? enqueue_vcycle_var<float>(c, c->x32, c->g32, c->vc32, 0, it == 0, s, nk)
                 : enqueue_vcycle<float>(c, c->x32, c->g32, c->inv32, 0, it == 0, s, nk);
    if (e != cudaSuccess) return e;
  }
  e = first ? launch_set_mixed(c->x64[0], c->x32[0], cells(c->geo[0]), c->scal, S_SCALE, s)
            : launch_update_mixed(c->x64[0], c->x32[0], cells(c->geo[0]), c->scal, S_SCALE, s);
  if (e != cudaSuccess) return e;
  if ((e = launch_set_scale(c->scal, S_RSUM, S_SCALE, (double)cells(c->geo[0]), s)) != cudaSuccess) return e;
  *nk += 2;
  return cudaSuccess;
}

// A mixed cycle whose update also carries the residual by recurrence: mixed_inner single-
// precision V-cycles on the scaled residual's high part g32[0] (the first from e = 0), the next
// scale from the residual's norm into scal[S_NEXT], then phi += s e (phi = s e from a zero
// iterate, `first`) with the residual pair (g32[0], q_lo) updated to (r - s A e) / s_next, its
// norm and relative norm (scal[S_RSUM], scal[S_REL]), and s_next made current. From a zero
// iterate the pair is formed from g64[0] (r = f); otherwise it must hold the current residual
// (rec_avail).
cudaError_t enqueue_cycle_rec(mg_ctx* c, cudaStream_t s, long long* nk, bool first) {
  cudaError_t e = cudaSuccess;
  for (int it = 0; it < c->p.mixed_inner; ++it)
    if ((e = enqueue_vcycle<float>(c, c->x32, c->g32, c->inv32, 0, it == 0, s, nk)) != cudaSuccess) return e;
  if ((e = launch_set_scale(c->scal, S_RSUM, S_NEXT, (double)cells(c->geo[0]), s)) != cudaSuccess) return e;
  int np = 0;
  e = launch_defect_rec(c->x64[0], c->x32[0], c->g32[0], c->q_lo, c->g64[0], c->geo[0], c->scal, S_SCALE, S_NEXT,
                        first, c->partials, &np, s);
  if (e != cudaSuccess) return e;
  if ((e = launch_defect_finalize(c->partials, np, c->scal, S_RSUM, S_REL, S_GSUM, S_SCALE, S_NEXT, s)) != cudaSuccess)
    return e;
  *nk += 3;
  return cudaSuccess;
}

// Termination quantity ||r|| / ||f|| into scal[S_REL]; in mixed mode also the scaled
// single-precision residual for the next inner cycle.
cudaError_t enqueue_resid(mg_ctx* c, int mode, double* out_natural, cudaStream_t s, long long* nk) {
  int np = 0;
  if (c->d_eps) {
    cudaError_t e = launch_var_resid_norm(c->x64[0], c->g64[0], c->vc[0], c->geo[0], level_coeff(c, 0), c->partials,
                                          &np, mode, out_natural, mode == 2 ? c->g32[0] : nullptr,
                                          c->scal + S_INV_SCALE, s);
    if (e != cudaSuccess) return e;
    *nk += 2;
    return launch_finalize(c->partials, np, c->scal, S_RSUM, S_REL, S_GSUM, s);
  }
  cudaError_t e = launch_resid_norm<double>(c->x64[0], c->g64[0], c->geo[0], c->partials, &np, mode,
                                            level_coeff(c, 0), out_natural, mode == 2 ? c->g32[0] : nullptr,
                                            c->scal + S_INV_SCALE, s);
  if (e != cudaSuccess) return e;
  *nk += 2;
  return launch_finalize(c->partials, np, c->scal, S_RSUM, S_REL, S_GSUM, s);
}

template <typename F>
mg_status capture(mg_ctx* c, cudaGraphExec_t* out, long long* nodes, F body, const char* what) {
  if (*out) return MG_OK;
  cudaError_t e = cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return cuda_fail(c, e, what);
  long long nk = 0;
  cudaError_t eb = body(c->cap, &nk);
  cudaGraph_t g = nullptr;
  cudaError_t ee = cudaStreamEndCapture(c->cap, &g);
  if (eb != cudaSuccess || ee != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return cuda_fail(c, eb != cudaSuccess ? eb : ee, what);
  }
  e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    *out = nullptr;
    return cuda_fail(c, e, what);
  }
  *nodes = nk;
  return MG_OK;
}

mg_status ensure_graphs(mg_ctx* c) {
  mg_status st = capture(c, &c->g_cycle, &c->n_cycle,
                         [c](cudaStream_t s, long long* nk) { return enqueue_cycle(c, s, nk, false); },
                         "capture cycle");
  if (st != MG_OK) return st;
  if (mixed(c)) {
    st = capture(c, &c->g_cycle0, &c->n_cycle0,
                 [c](cudaStream_t s, long long* nk) { return enqueue_cycle(c, s, nk, true); }, "capture cycle");
    if (st != MG_OK) return st;
  }
  if (c->rec_on && !c->d_eps) {
    st = capture(c, &c->g_rec, &c->n_rec,
                 [c](cudaStream_t s, long long* nk) { return enqueue_cycle_rec(c, s, nk, false); }, "capture cycle");
    if (st != MG_OK) return st;
    st = capture(c, &c->g_rec0, &c->n_rec0,
                 [c](cudaStream_t s, long long* nk) { return enqueue_cycle_rec(c, s, nk, true); }, "capture cycle");
    if (st != MG_OK) return st;
  }
  const int mode = mixed(c) ? 2 : 0;
  st = capture(c, &c->g_resid, &c->n_resid,
               [c, mode](cudaStream_t s, long long* nk) { return enqueue_resid(c, mode, nullptr, s, nk); },
               "capture residual");
  if (st != MG_OK) return st;
  if (mixed(c)) {
    st = capture(c, &c->g_check, &c->n_check,
                 [c](cudaStream_t s, long long* nk) { return enqueue_resid(c, 0, nullptr, s, nk); },
                 "capture residual");
    if (st != MG_OK) return st;
  }
  return capture(c, &c->g_resid0, &c->n_resid0,
                 [c](cudaStream_t s, long long* nk) {
                   ++*nk;
                   return launch_resid_zero(c->g64[0], cells(c->geo[0]), mixed(c) ? c->g32[0] : nullptr, c->scal,
                                            S_RSUM, S_REL, S_GSUM, S_INV_SCALE, s);
                 },
                 "capture zero residual");
}

mg_status run_graph(mg_ctx* c, cudaGraphExec_t g, long long nodes, const char* what) {
  CK(cudaGraphLaunch(g, c->stream), what);
  c->launches += nodes;
  return MG_OK;
}

// One cycle of the solve; the first one from a zero iterate that was never written (mixed
// mode) stores phi = s e instead of adding to it.
mg_status run_cycle(mg_ctx* c) {
  mg_status st = c->x_lazy ? run_graph(c, c->g_cycle0, c->n_cycle0, "cycle")
                           : run_graph(c, c->g_cycle, c->n_cycle, "cycle");
  if (st != MG_OK) return st;
  c->x_lazy = false;
  c->phi_zero = false;
  ++c->cnt_cycles;
  return MG_OK;
}

mg_status check_err_flag(mg_ctx* c);

// A cycle that carries the residual by recurrence, then its relative residual (scal[S_REL]) read
// back: an estimate that only a direct evaluation (read_rel) confirms.
mg_status run_cycle_rec(mg_ctx* c, double* rel) {
  mg_status st = c->x_lazy ? run_graph(c, c->g_rec0, c->n_rec0, "cycle")
                           : run_graph(c, c->g_rec, c->n_rec, "cycle");
  if (st != MG_OK) return st;
  c->x_lazy = false;
  c->phi_zero = false;
  ++c->cnt_cycles;
  ++c->cnt_rec;
  CK(cudaMemcpyAsync(c->h_pin, c->scal + S_REL, sizeof(double), cudaMemcpyDeviceToHost, c->stream), "read residual");
  CK(cudaMemcpyAsync(c->h_pin + 1, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "read error flag");
  CK(cudaStreamSynchronize(c->stream), "residual sync");
  *rel = c->h_pin[0];
  return check_err_flag(c);
}

// Write the zeros of a finest iterate that mg_set_solution(NULL) left unwritten, before a call
// that reads it.
mg_status materialize(mg_ctx* c) {
  if (!c->x_lazy) return MG_OK;
  CK(cudaMemsetAsync(c->x64[0], 0, sizeof(double) * (size_t)cells(c->geo[0]), c->stream), "zero iterate");
  c->x_lazy = false;
  return MG_OK;
}

// The device error flag as read into h_pin[1]: a kernel whose bounded wait ran out (the result
// of that launch is incomplete). The flag is cleared for the calls that follow.
mg_status check_err_flag(mg_ctx* c) {
  int flag = 0;
  std::memcpy(&flag, c->h_pin + 1, sizeof(int));
  if (flag == 0) return MG_OK;
  cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream);
  return fail(c, MG_ERR_TIMEOUT, "a kernel's bounded wait for its staged copies ran out; the result is incomplete");
}

// Relative residual of the current state: run the residual graph, read scal[S_REL]. check: in
// mixed mode, without the single-precision copy of the residual (for a value that is expected to
// end the solve; a cycle after it needs read_rel without check first).
mg_status read_rel(mg_ctx* c, double* rel, bool check = false) {
  // a zero iterate has r = f: its residual needs no stencil evaluation
  mg_status st = c->phi_zero ? run_graph(c, c->g_resid0, c->n_resid0, "residual")
                 : (check && c->g_check) ? run_graph(c, c->g_check, c->n_check, "residual")
                                         : run_graph(c, c->g_resid, c->n_resid, "residual");
  if (st != MG_OK) return st;
  if (!c->phi_zero) ++c->cnt_direct;
  CK(cudaMemcpyAsync(c->h_pin, c->scal + S_REL, sizeof(double), cudaMemcpyDeviceToHost, c->stream), "read residual");
  CK(cudaMemcpyAsync(c->h_pin + 1, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "read error flag");
  CK(cudaStreamSynchronize(c->stream), "residual sync");
  *rel = c->h_pin[0];
  return check_err_flag(c);
}

mg_status check_sph(mg_ctx* c, int P, const double* ctr, const double* rad, int sf) {
  if (P < 0 || (P > 0 && (!ctr || !rad))) return fail(c, MG_ERR_INVALID, "invalid sphere arrays");
  if (sf < 1 || sf > 8) return fail(c, MG_ERR_INVALID, "subsampling factor must be in 1..8");
  return MG_OK;
}

}  // namespace

// ============================================================================================

extern "C" {

void mg_default_params(mg_params* p, int nx, int ny, int nz, double h) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->nx = nx;
  p->ny = ny;
  p->nz = nz;
  p->h = h;
  for (int q = 0; q < 6; ++q) {
    p->bc_type[q] = MG_BC_DIRICHLET;
    p->bc_value[q] = 0.0;
  }
  p->nu1 = 2;
  p->nu2 = 2;
  p->cgc_weight = 2.0;
  p->prec = MG_FP64;
  p->eps = 1.0;
  p->mixed_inner = 4;
}

const char* mg_last_error(const mg_ctx* c) { return c ? c->err.c_str() : g_create_error.c_str(); }

mg_status mg_create(const mg_params* p, void* stream, mg_ctx** out) {
  mg_ctx* c = nullptr;
  if (!p || !out) return fail(c, MG_ERR_INVALID, "null argument");
  *out = nullptr;
  const int d[3] = {p->nx, p->ny, p->nz};
  for (int a = 0; a < 3; ++a)
    if (d[a] < 4 || (d[a] % 2) != 0) return fail(c, MG_ERR_INVALID, "grid dimensions must be even and >= 4");
  if (!(p->h > 0.0) || !std::isfinite(p->h)) return fail(c, MG_ERR_INVALID, "h must be positive");
  if (!(p->eps > 0.0) || !std::isfinite(p->eps)) return fail(c, MG_ERR_INVALID, "eps must be positive");
  if (const char* why = check_bc_types(p->bc_type)) return fail(c, MG_ERR_INVALID, why);
  for (int q = 0; q < 6; ++q)
    if (!std::isfinite(p->bc_value[q])) return fail(c, MG_ERR_INVALID, "bc_value must be finite");
  if (p->nu1 < 0 || p->nu1 > 16 || p->nu2 < 1 || p->nu2 > 16)
    return fail(c, MG_ERR_INVALID, "need 0 <= nu1 <= 16 and 1 <= nu2 <= 16");
  if (!std::isfinite(p->cgc_weight)) return fail(c, MG_ERR_INVALID, "cgc_weight must be finite");
  if (p->prec != MG_FP64 && p->prec != MG_MIXED) return fail(c, MG_ERR_INVALID, "prec must be MG_FP64 or MG_MIXED");
  if (p->prec == MG_MIXED && (p->mixed_inner < 1 || p->mixed_inner > 16))
    return fail(c, MG_ERR_INVALID, "mixed_inner must be in 1..16");

  c = new mg_ctx();
  c->p = *p;
  c->stream = (cudaStream_t)stream;
  for (int q = 0; q < 6; ++q) {
    c->bc.type[q] = p->bc_type[q];
    c->bc.value[q] = p->bc_value[q];
  }
  // level hierarchy: halve while every dimension is even and its half is >= 3 (Sec. 3)
  int dims[3] = {p->nx, p->ny, p->nz};
  for (;;) {
    if (c->L >= kMaxLevels) break;
    Geom& G = c->geo[c->L];
    G.nx = dims[0];
    G.ny = dims[1];
    G.nz = dims[2];
    for (int q = 0; q < 6; ++q) G.sh[q] = face_shift(p->bc_type[q]);
    G.per = periodic_bits(p->bc_type);
    ++c->L;
    bool ok = true;
    for (int a = 0; a < 3; ++a)
      if ((dims[a] % 2) != 0 || dims[a] / 2 < 3) ok = false;
    if (!ok) break;
    for (int a = 0; a < 3; ++a) dims[a] /= 2;
  }
  for (int l = 0; l < c->L; ++l) {
    Geom& G = c->geo[l];
    G.packed = (l < c->L - 1) ? 1 : 0;
    G.hx = G.nx / 2;
    G.csz = G.packed ? (long long)G.hx * G.ny * G.nz : (long long)G.nx * G.ny * G.nz;
  }
  const Geom& Gc = c->geo[c->L - 1];
  if ((long long)Gc.nx * Gc.ny * Gc.nz > kMaxCoarseCells) {
    delete c;
    return fail(nullptr, MG_ERR_INVALID,
                "coarsest grid has more than 4096 cells: choose dimensions with more factors of two");
  }
  for (int d6 = -3; d6 <= 3; ++d6) {
    c->inv64.v[d6 + 3] = 1.0 / (double)(6 + d6);
    c->inv32.v[d6 + 3] = 1.0f / (float)(6 + d6);
  }

  cudaError_t e = cudaSuccess;
  auto alloc = [&](void** ptr, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(ptr, bytes);
  };
  for (int l = 0; l < c->L; ++l) {
    const size_t n = (size_t)cells(c->geo[l]);
    if (!mixed(c) || l == 0) {
      alloc((void**)&c->x64[l], n * sizeof(double));
      alloc((void**)&c->g64[l], n * sizeof(double));
    }
    if (mixed(c)) {
      alloc((void**)&c->x32[l], n * sizeof(float));
      alloc((void**)&c->g32[l], n * sizeof(float));
    }
  }
  // MG_MIXED: the outer steps carry the residual by recurrence (defect_kernels.cu) on finest levels
  // of whole 4-float rows; CCMG_DEFECT=walk evaluates it directly after every step instead
  const char* defect_env = std::getenv("CCMG_DEFECT");
  c->rec_on = mixed(c) && defect_rec_applies(c->geo[0]) && !(defect_env && std::strcmp(defect_env, "walk") == 0);
  if (c->rec_on) alloc((void**)&c->q_lo, (size_t)cells(c->geo[0]) * sizeof(float));
  alloc((void**)&c->partials, kMaxPartials * sizeof(double));
  alloc((void**)&c->scal, S_COUNT * sizeof(double));
  alloc((void**)&c->d_iters, sizeof(int));
  alloc((void**)&c->d_err, sizeof(int));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&c->h_pin, 8 * sizeof(double));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = prepare_coarse_cg();
  if (e == cudaSuccess) e = prepare_var_coarse_cg();
  // TMA-staged half-sweeps on the single-precision levels where they are the faster kernel;
  // CCMG_SWEEP=vec keeps the direct-load kernel everywhere, CCMG_SWEEP=tma takes the TMA one on
  // every level it can run on (both for comparing and testing the two)
  const char* sweep_env = std::getenv("CCMG_SWEEP");
  const bool no_tma = sweep_env && std::strcmp(sweep_env, "vec") == 0;
  const bool all_tma = sweep_env && std::strcmp(sweep_env, "tma") == 0;
  if (mixed(c) && !no_tma) {
    int dev = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    for (int l = 0; l + 1 < c->L && e == cudaSuccess; ++l)
      if (all_tma ? tma_sweep_applies(c->geo[l]) : tma_sweep_pays(c->geo[l])) {
        e = prepare_tma_sweep(c->tma[l], c->x32[l], c->g32[l], c->geo[l], dev);
        if (e == cudaSuccess) e = prepare_tma_prolong(c->tma[l], c->x32[l + 1], c->geo[l + 1], c->geo[l], dev);
      }
  }
  if (!mixed(c) && !no_tma) {  // FP64 mode: the FP64 half-sweeps of the large levels staged the same way
    int dev = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    for (int l = 0; l + 1 < c->L && e == cudaSuccess; ++l)
      if (all_tma ? tma_sweep64_applies(c->geo[l]) : tma_sweep64_pays(c->geo[l]))
        e = prepare_tma_sweep64(c->tma64[l], c->x64[l], c->g64[l], c->geo[l], dev);
  }
  // FP64 mode: the residual + restriction of the large levels by the fixed-point residual walk;
  // CCMG_RESTRICT=vec keeps the direct-load kernel everywhere, =walk takes the walk on every
  // packed level it can run on
  if (!mixed(c)) {
    const char* rr_env = std::getenv("CCMG_RESTRICT");
    const bool rr_vec = rr_env && std::strcmp(rr_env, "vec") == 0;
    const bool rr_all = rr_env && std::strcmp(rr_env, "walk") == 0;
    for (int l = 0; l + 1 < c->L; ++l)
      c->rr_walk[l] = !rr_vec && resid_restrict_walk_applies(c->geo[l]) &&
                      (rr_all || cells(c->geo[l]) >= (1LL << 25));  // measured: 1.22 vs 1.50 ms at 512^3;
                                                                      // 0.20 vs 0.19 at 256^3, slower below
  }
  if (e != cudaSuccess) {
    const bool oom = (e == cudaErrorMemoryAllocation);
    std::string msg = std::string("mg_create: ") + cudaGetErrorString(e);
    cudaGetLastError();
    free_all(c);
    delete c;
    return fail(nullptr, oom ? MG_ERR_OOM : MG_ERR_CUDA, msg);
  }
  // zero state: phi = 0, f = 0, scalars 0 (scale 1)
  for (int l = 0; l < c->L; ++l) {
    const size_t n = (size_t)cells(c->geo[l]);
    if (c->x64[l]) e = cudaMemsetAsync(c->x64[l], 0, n * sizeof(double), c->stream);
    if (e == cudaSuccess && c->g64[l]) e = cudaMemsetAsync(c->g64[l], 0, n * sizeof(double), c->stream);
    if (e == cudaSuccess && c->x32[l]) e = cudaMemsetAsync(c->x32[l], 0, n * sizeof(float), c->stream);
    if (e == cudaSuccess && c->g32[l]) e = cudaMemsetAsync(c->g32[l], 0, n * sizeof(float), c->stream);
    if (e != cudaSuccess) break;
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(c->scal, 0, S_COUNT * sizeof(double), c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    std::string msg = std::string("mg_create: ") + cudaGetErrorString(e);
    free_all(c);
    delete c;
    return fail(nullptr, MG_ERR_CUDA, msg);
  }
  *out = c;
  return MG_OK;
}

mg_status mg_destroy(mg_ctx* c) {
  if (!c) return MG_ERR_INVALID;
  cudaStreamSynchronize(c->stream);
  free_all(c);
  delete c;
  return MG_OK;
}

int mg_num_levels(const mg_ctx* c) { return c ? c->L : 0; }

mg_status mg_level_dims(const mg_ctx* c, int level, int* dims) {
  if (!c || !dims || level < 0 || level >= c->L) return MG_ERR_INVALID;
  dims[0] = c->geo[level].nx;
  dims[1] = c->geo[level].ny;
  dims[2] = c->geo[level].nz;
  return MG_OK;
}

long long mg_kernel_launches(const mg_ctx* c) { return c ? c->launches : 0; }

mg_status mg_selftest_wait_timeout(mg_ctx* c, int level) {
  if (!c) return MG_ERR_INVALID;
  if (level < 0 || level >= c->L - 1 || !(c->tma[level].ok || c->tma64[level].ok))
    return fail(c, MG_ERR_INVALID, "the level has no TMA-staged half-sweep");
  if (c->tma[level].ok)
    CK(launch_smooth_tma_withheld(c->x32[level], c->geo[level], c->inv32, c->tma[level], c->d_err, 20000000LL,
                                  c->stream),
       "wait-timeout self-test");
  else
    CK(launch_smooth_tma64_withheld(c->x64[level], c->g64[level], c->geo[level], c->inv64, c->tma64[level], c->d_err, 20000000LL,
                                    c->stream),
       "wait-timeout self-test");
  c->launches += 1;
  CK(cudaMemcpyAsync(c->h_pin + 1, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "self-test flag");
  CK(cudaStreamSynchronize(c->stream), "self-test sync");
  return check_err_flag(c);
}

int mg_level_sweep_kind(const mg_ctx* c, int level) {
  if (!c || level < 0 || level >= c->L - 1) return -1;
  return (c->tma[level].ok || c->tma64[level].ok) ? 1 : 0;
}

mg_status mg_set_bc_values(mg_ctx* c, const double* v) {
  if (!c) return MG_ERR_INVALID;
  if (!v) return fail(c, MG_ERR_INVALID, "null bc values");
  for (int q = 0; q < 6; ++q) {
    if (!std::isfinite(v[q])) return fail(c, MG_ERR_INVALID, "bc values must be finite");
  }
  for (int q = 0; q < 6; ++q) {
    c->bc.value[q] = v[q];
    c->p.bc_value[q] = v[q];
  }
  return MG_OK;
}

mg_status mg_set_bc_field(mg_ctx* c, int face, const double* d_values) {
  if (!c) return MG_ERR_INVALID;
  if (face < 0 || face > 5) return fail(c, MG_ERR_INVALID, "face must be 0..5");
  if (!d_values) {
    c->bc.field[face] = nullptr;
    return MG_OK;
  }
  if (c->bc.type[face] == MG_BC_PERIODIC) return fail(c, MG_ERR_INVALID, "a periodic face has no wall values");
  const Geom& G = c->geo[0];
  const size_t bytes = (size_t)face_cells(face, G.nx, G.ny, G.nz) * sizeof(double);
  if (!c->d_bcf[face]) {
    const cudaError_t e = cudaMalloc((void**)&c->d_bcf[face], bytes);
    if (e != cudaSuccess) {
      c->d_bcf[face] = nullptr;
      cudaGetLastError();
      return fail(c, e == cudaErrorMemoryAllocation ? MG_ERR_OOM : MG_ERR_CUDA, "bc field allocation");
    }
  }
  CK(cudaMemcpyAsync(c->d_bcf[face], d_values, bytes, cudaMemcpyDeviceToDevice, c->stream), "set_bc_field");
  CK(cudaStreamSynchronize(c->stream), "set_bc_field");  // the caller's array is free on return
  c->bc.field[face] = c->d_bcf[face];
  return MG_OK;
}

static mg_status set_rhs_impl(mg_ctx* c, const double* d_rho, int raw) {
  if (!c) return MG_ERR_INVALID;
  if (!d_rho) return fail(c, MG_ERR_INVALID, "null right-hand side");
  const Geom& G = c->geo[0];
  if (c->d_eps && !raw)
    CK(launch_var_set_rhs(c->g64[0], G, d_rho, c->d_eps, c->p.h, c->bc, c->stream), "set_rhs");
  else
    CK(launch_set_rhs<double>(c->g64[0], G, d_rho, 1.0 / c->p.eps, c->p.h, c->bc, raw, c->stream), "set_rhs");
  int np = 0;
  CK(launch_sumsq<double>(c->g64[0], cells(G), c->partials, &np, c->stream), "set_rhs norm");
  CK(launch_finalize(c->partials, np, c->scal, S_GSUM, -1, 0, c->stream), "set_rhs norm");
  CK(launch_set_scale(c->scal, S_GSUM, S_SCALE, (double)cells(G), c->stream), "set_rhs scale");
  c->launches += 4;
  return MG_OK;
}

}  // extern "C"

namespace {

// The cycle and residual graphs hold the operator's kernels: drop them to be captured again.
void drop_graphs(mg_ctx* c) {
  for (cudaGraphExec_t* gx : {&c->g_cycle, &c->g_cycle0, &c->g_resid, &c->g_resid0, &c->g_rec, &c->g_rec0, &c->g_check})
    if (*gx) {
      cudaGraphExecDestroy(*gx);
      *gx = nullptr;
    }
}

// Buffers of the weighted operator (permittivities and coefficients of every level); a new
// permittivity array is filled with the constant eps of the parameters when `fill`.
mg_status var_alloc(mg_ctx* c, bool fill) {
  if (c->d_eps) return MG_OK;
  const Geom& G = c->geo[0];
  const size_t n = (size_t)G.nx * G.ny * G.nz;
  bool ok = cudaMalloc((void**)&c->d_eps, n * sizeof(double)) == cudaSuccess;
  for (int l = 0; l < c->L && ok; ++l) {
    ok = cudaMalloc((void**)&c->vc[l], (size_t)var_arrays() * cells(c->geo[l]) * sizeof(double)) == cudaSuccess;
    if (ok && mixed(c))
      ok = cudaMalloc((void**)&c->vc32[l], (size_t)var_arrays32() * cells(c->geo[l]) * sizeof(float)) == cudaSuccess;
  }
  if (!ok) {
    cudaGetLastError();
    cudaFree(c->d_eps);
    c->d_eps = nullptr;
    for (int l = 0; l < c->L; ++l) {
      cudaFree(c->vc[l]);
      cudaFree(c->vc32[l]);
      c->vc[l] = nullptr;
      c->vc32[l] = nullptr;
    }
    return fail(c, MG_ERR_OOM, "weighted operator");
  }
  if (fill) CK(launch_fill(c->d_eps, c->p.eps, (long long)n, c->stream), "permittivity");
  return MG_OK;
}

void var_release(mg_ctx* c) {
  cudaStreamSynchronize(c->stream);
  cudaFree(c->d_eps);
  c->d_eps = nullptr;
  for (int l = 0; l < c->L; ++l) {
    cudaFree(c->vc[l]);
    cudaFree(c->vc32[l]);
    c->vc[l] = nullptr;
    c->vc32[l] = nullptr;
  }
}

// The coefficients of every level from the permittivities and the reaction coefficients (and
// their single-precision copies for the inner cycle of MG_MIXED).
mg_status var_rebuild(mg_ctx* c) {
  CK(launch_var_setup(c->d_eps, c->d_k2, c->p.h, c->p.cgc_weight, c->geo, c->L, c->bc, c->vc, c->stream),
     "weighted coefficients");
  c->launches += c->L;
  if (mixed(c)) {
    CK(launch_var_to_f32(c->vc, c->vc32, c->geo, c->L, c->stream), "weighted coefficients");
    c->launches += c->L;
  }
  CK(cudaStreamSynchronize(c->stream), "weighted coefficients");
  return MG_OK;
}

}  // namespace

extern "C" {

mg_status mg_set_permittivity(mg_ctx* c, const double* d_eps) {
  if (!c) return MG_ERR_INVALID;
  drop_graphs(c);
  mg_status st;
  c->eps_set = d_eps != nullptr;
  if (!d_eps) {
    if (!c->d_k2) {
      var_release(c);
      return MG_OK;
    }
    // the reaction term stays: the weighted operator with the constant permittivity
    CK(launch_fill(c->d_eps, c->p.eps, (long long)c->geo[0].nx * c->geo[0].ny * c->geo[0].nz, c->stream),
       "permittivity");
    return var_rebuild(c);
  }
  if ((st = var_alloc(c, false)) != MG_OK) return st;
  const Geom& G = c->geo[0];
  const size_t n = (size_t)G.nx * G.ny * G.nz;
  CK(cudaMemcpyAsync(c->d_eps, d_eps, n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream), "permittivity");
  return var_rebuild(c);
}

mg_status mg_set_reaction(mg_ctx* c, const double* d_k2) {
  if (!c) return MG_ERR_INVALID;
  drop_graphs(c);
  const Geom& G = c->geo[0];
  const size_t n = (size_t)G.nx * G.ny * G.nz;
  if (!d_k2) {
    CK(cudaStreamSynchronize(c->stream), "reaction");
    cudaFree(c->d_k2);
    c->d_k2 = nullptr;
    if (c->d_eps && !c->eps_set) var_release(c);  // the constant operator again
    return c->d_eps ? var_rebuild(c) : MG_OK;
  }
  mg_status st = var_alloc(c, true);
  if (st != MG_OK) return st;
  if (!c->d_k2 && cudaMalloc((void**)&c->d_k2, n * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    c->d_k2 = nullptr;
    return fail(c, MG_ERR_OOM, "reaction");
  }
  CK(cudaMemcpyAsync(c->d_k2, d_k2, n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream), "reaction");
  return var_rebuild(c);
}

mg_status mg_solve_pb(mg_ctx* c, double tol, int max_newton, double inner_tol, int max_cycles, int* h_newton,
                      double* h_rel) {
  if (!c) return MG_ERR_INVALID;
  if (!c->d_k2) return fail(c, MG_ERR_INVALID, "no reaction coefficients (mg_set_reaction)");
  if (!(tol >= 0.0) || !(inner_tol >= 0.0) || max_newton < 0 || max_cycles < 0)
    return fail(c, MG_ERR_INVALID, "need tolerances >= 0 and counts >= 0");
  mg_status st = ensure_graphs(c);
  if (st != MG_OK) return st;
  const Geom& G = c->geo[0];
  const long long n = cells(G);
  if (!c->d_pb && cudaMalloc((void**)&c->d_pb, 2 * (size_t)n * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    c->d_pb = nullptr;
    return fail(c, MG_ERR_OOM, "Newton state");
  }
  double* g0 = c->d_pb;
  double* phi = c->d_pb + n;
  if ((st = materialize(c)) != MG_OK) return st;
  CK(cudaMemcpyAsync(g0, c->g64[0], n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream), "Newton");
  CK(cudaMemcpyAsync(phi, c->x64[0], n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream), "Newton");
  int np = 0;
  CK(launch_sumsq<double>(g0, n, c->partials, &np, c->stream), "Newton");
  CK(launch_finalize(c->partials, np, c->scal, S_PB_REF, -1, 0, c->stream), "Newton");
  int it = 0;
  double rel = 0.0;
  for (;;) {
    // F = f - A_eps phi - k2 sinh(phi) into the right-hand side, and the linearised diagonal
    CK(launch_pb_update(phi, g0, c->vc[0], G, c->d_k2, c->p.h, c->g64[0], c->partials, &np, c->stream), "Newton");
    CK(launch_finalize(c->partials, np, c->scal, S_GSUM, S_PB_REL, S_PB_REF, c->stream), "Newton");
    c->launches += 2;
    CK(cudaMemcpyAsync(c->h_pin, c->scal + S_PB_REL, sizeof(double), cudaMemcpyDeviceToHost, c->stream), "Newton");
    CK(cudaStreamSynchronize(c->stream), "Newton");
    rel = c->h_pin[0];
    if (!(rel >= tol) || it >= max_newton) break;
    // (A_eps + k2 cosh(phi)) delta = F with homogeneous walls, from delta = 0
    CK(launch_var_coarsen_all(c->geo, c->L, c->vc, c->p.cgc_weight, c->stream), "Newton");
    c->launches += c->L - 1;
    if (mixed(c)) {  // the inner cycle's coefficients and the scale of its first defect-correction step
      CK(launch_var_to_f32(c->vc, c->vc32, c->geo, c->L, c->stream), "Newton");
      CK(launch_set_scale(c->scal, S_GSUM, S_SCALE, (double)n, c->stream), "Newton");
      c->launches += c->L + 1;
    }
    CK(cudaMemsetAsync(c->x64[0], 0, n * sizeof(double), c->stream), "Newton");
    c->phi_zero = true;
    st = mg_solve(c, inner_tol, max_cycles, nullptr, nullptr);
    if (st != MG_OK && st != MG_ERR_NOT_CONVERGED) return st;  // an inexact step is still a step
    CK(launch_axpy(phi, c->x64[0], n, c->stream), "Newton");
    c->launches += 1;
    ++it;
  }
  // the potential into the iterate; the right-hand side back to f
  CK(cudaMemcpyAsync(c->x64[0], phi, n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream), "Newton");
  CK(cudaMemcpyAsync(c->g64[0], g0, n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream), "Newton");
  CK(cudaStreamSynchronize(c->stream), "Newton");
  c->phi_zero = false;
  if (h_newton) *h_newton = it;
  if (h_rel) *h_rel = rel;
  if (!std::isfinite(rel)) return fail(c, MG_ERR_NOT_CONVERGED, "Newton residual is not finite");
  if (rel >= tol) return fail(c, MG_ERR_NOT_CONVERGED, "Newton did not reach the tolerance");
  return MG_OK;
}

int mg_has_permittivity(const mg_ctx* c) { return c && c->d_eps ? 1 : 0; }
int mg_has_reaction(const mg_ctx* c) { return c && c->d_k2 ? 1 : 0; }

mg_status mg_set_rhs(mg_ctx* c, const double* d_rho) { return set_rhs_impl(c, d_rho, 0); }
mg_status mg_set_rhs_f(mg_ctx* c, const double* d_f) { return set_rhs_impl(c, d_f, 1); }

mg_status mg_set_solution(mg_ctx* c, const double* d_phi) {
  if (!c) return MG_ERR_INVALID;
  c->phi_zero = (d_phi == nullptr);
  if (mixed(c) && !d_phi) {  // nothing is written: the first cycle stores phi = s e
    c->x_lazy = true;
    return MG_OK;
  }
  CK(launch_pack<double>(c->x64[0], c->geo[0], d_phi, 1.0, c->stream), "set_solution");
  c->launches += 1;
  c->x_lazy = false;
  return MG_OK;
}

mg_status mg_get_solution(mg_ctx* c, double* d_phi) {
  if (!c) return MG_ERR_INVALID;
  if (!d_phi) return fail(c, MG_ERR_INVALID, "null output");
  mg_status st = materialize(c);
  if (st != MG_OK) return st;
  CK(launch_unpack<double>(d_phi, c->x64[0], c->geo[0], 1.0, c->stream), "get_solution");
  c->launches += 1;
  return MG_OK;
}

mg_status mg_vcycle(mg_ctx* c, int ncycles) {
  if (!c) return MG_ERR_INVALID;
  if (ncycles < 0) return fail(c, MG_ERR_INVALID, "ncycles must be >= 0");
  mg_status st = ensure_graphs(c);
  if (st != MG_OK) return st;
  for (int k = 0; k < ncycles; ++k) {
    if (mixed(c)) {
      if (c->phi_zero) st = run_graph(c, c->g_resid0, c->n_resid0, "residual");
      else st = run_graph(c, c->g_resid, c->n_resid, "residual");
      if (st != MG_OK) return st;
    }
    if ((st = run_cycle(c)) != MG_OK) return st;
  }
  return MG_OK;
}

mg_status mg_solve(mg_ctx* c, double tol, int max_cycles, int* h_cycles, double* h_rel) {
  if (!c) return MG_ERR_INVALID;
  if (!(tol >= 0.0) || max_cycles < 0) return fail(c, MG_ERR_INVALID, "need tol >= 0 and max_cycles >= 0");
  mg_status st = ensure_graphs(c);
  if (st != MG_OK) return st;
  int k = 0;
  double rel = 0.0, rel0 = -1.0, rel_prev = -1.0;
  mg_status out = MG_OK;
  // MG_MIXED with the constant operator: a cycle may carry the residual by recurrence (from a zero
  // iterate, or after another such cycle), which leaves an estimate of the relative residual in
  // place of its direct evaluation. The direct evaluation follows whenever the estimate would end
  // the solve (below the tolerance, non-finite, diverged, or at max_cycles), so every result the
  // solve returns is evaluated directly. The recurrence is skipped for a cycle that the last
  // contraction predicts to reach the tolerance: that cycle is followed by the direct evaluation.
  const bool use_rec = c->rec_on && !c->d_eps && !c->d_k2;
  bool estimate = false;  // rel is the recurrence's estimate
  bool final = false;     // the last cycle was predicted to reach the tolerance, or was the last allowed
  // the solve stops on this value (and needs no single-precision copy of the residual)
  auto ends = [&](double v) {
    return !(v >= tol) || !std::isfinite(v) || (rel0 >= 0.0 && v > 1e3 * rel0) || k >= max_cycles;
  };
  for (;;) {
    if (!estimate || ends(rel)) {
      // a cycle predicted to reach the tolerance is checked without the single-precision copy
      // (0.13 ms of the walk at 512^3); if the solve goes on after all, the copy is made then
      if ((st = read_rel(c, &rel, final)) != MG_OK) return st;
      if (final && !ends(rel) && (st = read_rel(c, &rel)) != MG_OK) return st;
      estimate = false;
    }
    if (!std::isfinite(rel)) {
      out = fail(c, MG_ERR_NOT_CONVERGED, "residual is not finite");
      break;
    }
    if (rel0 < 0.0) rel0 = rel;
    if (rel > 1e3 * rel0 && rel > tol) {
      out = fail(c, MG_ERR_DIVERGED, "residual grew by more than 1e3");
      break;
    }
    if (!(rel >= tol)) break;
    if (k >= max_cycles) {
      out = fail(c, MG_ERR_NOT_CONVERGED, "max_cycles reached before the tolerance");
      break;
    }
    // the recurrence continues from a zero iterate or from its own last step
    final = mixed(c) && ((rel_prev > 0.0 && rel * (rel / rel_prev) < tol) || k + 1 >= max_cycles);
    const bool rec_next = use_rec && (c->x_lazy || estimate) && !final;
    rel_prev = rel;
    if (rec_next) {
      if ((st = run_cycle_rec(c, &rel)) != MG_OK) return st;
      estimate = true;
    } else {
      if ((st = run_cycle(c)) != MG_OK) return st;
      estimate = false;
    }
    ++k;
  }
  if (h_cycles) *h_cycles = k;
  if (h_rel) *h_rel = rel;
  return out;
}

mg_status mg_residual(mg_ctx* c, double* h_rel, double* d_r) {
  if (!c) return MG_ERR_INVALID;
  mg_status st = materialize(c);
  if (st != MG_OK) return st;
  long long nk = 0;
  CK(enqueue_resid(c, d_r ? 1 : 0, d_r, c->stream, &nk), "residual");
  c->launches += nk;
  ++c->cnt_direct;
  CK(cudaMemcpyAsync(c->h_pin, c->scal + S_REL, sizeof(double), cudaMemcpyDeviceToHost, c->stream), "residual");
  CK(cudaMemcpyAsync(c->h_pin + 1, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "residual");
  CK(cudaStreamSynchronize(c->stream), "residual sync");
  if (h_rel) *h_rel = c->h_pin[0];
  return check_err_flag(c);
}

mg_status mg_efield(mg_ctx* c, double* d_E) {
  if (!c) return MG_ERR_INVALID;
  if (!d_E) return fail(c, MG_ERR_INVALID, "null output");
  mg_status st = materialize(c);
  if (st != MG_OK) return st;
  CK(launch_efield(c->x64[0], c->geo[0], c->p.h, c->bc, c->grad_stencil, d_E, c->stream), "efield");
  c->launches += 1;
  return MG_OK;
}

mg_status mg_sphere_density(mg_ctx* c, int P, const double* ctr, const double* rad, const double* dens, int sf,
                            double* d_rho) {
  if (!c) return MG_ERR_INVALID;
  mg_status st = check_sph(c, P, ctr, rad, sf);
  if (st != MG_OK) return st;
  if (!d_rho || (P > 0 && !dens)) return fail(c, MG_ERR_INVALID, "null argument");
  Spheres sp{P, ctr, rad, dens};
  CK(launch_sphere_density(c->geo[0], c->p.h, sp, sf, d_rho, c->stream), "sphere_density");
  c->launches += P > 0 ? 1 : 0;
  return MG_OK;
}

mg_status mg_force_gather(mg_ctx* c, int P, const double* ctr, const double* rad, const double* dens, int sf,
                          double* d_F) {
  if (!c) return MG_ERR_INVALID;
  mg_status st = check_sph(c, P, ctr, rad, sf);
  if (st != MG_OK) return st;
  if ((P > 0 && (!dens || !d_F))) return fail(c, MG_ERR_INVALID, "null argument");
  Spheres sp{P, ctr, rad, dens};
  if ((st = materialize(c)) != MG_OK) return st;
  CK(launch_force_gather(c->x64[0], c->geo[0], c->p.h, c->bc, c->grad_stencil, sp, sf, d_F, c->stream), "force_gather");
  c->launches += P > 0 ? 1 : 0;
  return MG_OK;
}

mg_status mg_force_gather_adjoint(mg_ctx* c, int P, const double* ctr, const double* rad, const double* dens, int sf,
                                  const double* d_wF, double* d_gphi, double* d_gdens, double* d_gbc) {
  if (!c) return MG_ERR_INVALID;
  mg_status st = check_sph(c, P, ctr, rad, sf);
  if (st != MG_OK) return st;
  if (!d_gphi || !d_gbc || (P > 0 && (!dens || !d_wF || !d_gdens))) return fail(c, MG_ERR_INVALID, "null argument");
  if (c->grad_stencil != 7) return fail(c, MG_ERR_INVALID, "the force adjoint is implemented for the D3Q7 gradient");
  Spheres sp{P, ctr, rad, dens};
  if ((st = materialize(c)) != MG_OK) return st;
  CK(launch_force_adjoint(c->x64[0], c->geo[0], c->p.h, c->bc, sp, sf, d_wF, d_gphi, d_gdens, d_gbc, c->stream),
     "force_gather_adjoint");
  c->launches += P > 0 ? 1 : 0;
  return MG_OK;
}

mg_status mg_set_gradient_stencil(mg_ctx* c, int stencil) {
  if (!c) return MG_ERR_INVALID;
  if (stencil != 7 && stencil != 19) return fail(c, MG_ERR_INVALID, "the gradient stencil must be 7 or 19");
  c->grad_stencil = stencil;
  return MG_OK;
}

int mg_gradient_stencil(const mg_ctx* c) { return c ? c->grad_stencil : -1; }

mg_status mg_sphere_density_adjoint(mg_ctx* c, int P, const double* ctr, const double* rad, int sf,
                                    const double* d_gfield, double* d_gdens) {
  if (!c) return MG_ERR_INVALID;
  mg_status st = check_sph(c, P, ctr, rad, sf);
  if (st != MG_OK) return st;
  if (P > 0 && (!d_gfield || !d_gdens)) return fail(c, MG_ERR_INVALID, "null argument");
  Spheres sp{P, ctr, rad, nullptr};
  CK(launch_density_adjoint(c->geo[0], c->p.h, sp, sf, d_gfield, d_gdens, c->stream), "sphere_density_adjoint");
  c->launches += P > 0 ? 1 : 0;
  return MG_OK;
}

mg_status mg_rhs_adjoint(mg_ctx* c, const double* d_lam, double* d_grho, double* d_gbc) {
  if (!c) return MG_ERR_INVALID;
  if (!d_lam || !d_grho || !d_gbc) return fail(c, MG_ERR_INVALID, "null argument");
  CK(launch_rhs_adjoint(c->geo[0], c->p.h, 1.0 / c->p.eps, c->bc, c->d_eps, d_lam, d_grho, d_gbc, c->stream),
     "rhs_adjoint");
  c->launches += 2;
  return MG_OK;
}

mg_status mg_adjoint_solve(mg_ctx* c, const double* d_g, double* d_lambda, double tol, int max_cycles, int* h_cycles,
                           double* h_rel) {
  if (!c) return MG_ERR_INVALID;
  if (!d_g || !d_lambda) return fail(c, MG_ERR_INVALID, "null argument");
  if (!(tol >= 0.0) || max_cycles < 0) return fail(c, MG_ERR_INVALID, "need tol >= 0 and max_cycles >= 0");
  // the adjoint system has homogeneous walls: g is the right-hand side as it is (the wall values
  // of the forward problem are neither read nor changed)
  mg_status st = mg_set_rhs_f(c, d_g);
  if (st != MG_OK) return st;
  if ((st = mg_set_solution(c, nullptr)) != MG_OK) return st;
  const mg_status solve_st = mg_solve(c, tol, max_cycles, h_cycles, h_rel);
  if (solve_st != MG_OK && solve_st != MG_ERR_NOT_CONVERGED) return solve_st;
  if ((st = mg_get_solution(c, d_lambda)) != MG_OK) return st;
  return solve_st;
}

mg_status mg_step_host(mg_ctx* c, int P, const double* h_ctr, const double* h_rad, const double* h_dens, int sf,
                       double tol, int max_cycles, double* h_F, int* h_cycles, double* h_rel) {
  if (!c) return MG_ERR_INVALID;
  mg_status st = check_sph(c, P, h_ctr, h_rad, sf);
  if (st != MG_OK) return st;
  if (P > 0 && (!h_dens || !h_F)) return fail(c, MG_ERR_INVALID, "null argument");
  if (max_cycles < 0 || !(tol == tol)) return fail(c, MG_ERR_INVALID, "need max_cycles >= 0 and a tolerance");
  const Geom& G = c->geo[0];
  if (!c->d_rho) CK(cudaMalloc((void**)&c->d_rho, sizeof(double) * (size_t)G.nx * G.ny * G.nz), "step scratch");
  if (P > c->sph_cap) {
    cudaFree(c->d_sph);
    c->d_sph = nullptr;
    c->sph_cap = 0;
    CK(cudaMalloc((void**)&c->d_sph, sizeof(double) * 8 * (size_t)P), "step scratch");
    c->sph_cap = P;
  }
  double* dc = c->d_sph;
  double* dr = dc + 3 * (size_t)c->sph_cap;
  double* dq = dr + c->sph_cap;
  double* dF = dq + c->sph_cap;
  if (P > 0) {
    CK(cudaMemcpyAsync(dc, h_ctr, sizeof(double) * 3 * P, cudaMemcpyHostToDevice, c->stream), "step copy");
    CK(cudaMemcpyAsync(dr, h_rad, sizeof(double) * P, cudaMemcpyHostToDevice, c->stream), "step copy");
    CK(cudaMemcpyAsync(dq, h_dens, sizeof(double) * P, cudaMemcpyHostToDevice, c->stream), "step copy");
  }
  if ((st = mg_sphere_density(c, P, dc, dr, dq, sf, c->d_rho)) != MG_OK) return st;
  if ((st = mg_set_rhs(c, c->d_rho)) != MG_OK) return st;
  mg_status solve_st = MG_OK;
  if (tol < 0.0) {  // fixed number of cycles from the current solution (the time loop of Sec. 8.1)
    if ((st = mg_vcycle(c, max_cycles)) != MG_OK) return st;
    if (h_cycles) *h_cycles = max_cycles;
    if (h_rel && (st = mg_residual(c, h_rel, nullptr)) != MG_OK) return st;
  } else {
    solve_st = mg_solve(c, tol, max_cycles, h_cycles, h_rel);
    if (solve_st != MG_OK && solve_st != MG_ERR_NOT_CONVERGED) return solve_st;
  }
  if (P > 0) {
    if ((st = mg_force_gather(c, P, dc, dr, dq, sf, dF)) != MG_OK) return st;
    CK(cudaMemcpyAsync(h_F, dF, sizeof(double) * 3 * P, cudaMemcpyDeviceToHost, c->stream), "step copy");
  }
  CK(cudaStreamSynchronize(c->stream), "step sync");
  return solve_st;
}

// ---------------------------------------------------------------------------------------------
// Level-wise operations

mg_status mg_level_set(mg_ctx* c, int level, int which, const double* d_in) {
  if (!c) return MG_ERR_INVALID;
  if (level < 0 || level >= c->L || (which != 0 && which != 1) || !d_in)
    return fail(c, MG_ERR_INVALID, "bad level, field or pointer");
  const double scale = which == 0 ? 1.0 : 1.0 / level_coeff(c, level);
  if (mixed(c))
    CK(launch_pack<float>(which == 0 ? c->x32[level] : c->g32[level], c->geo[level], d_in, scale, c->stream),
       "level_set");
  else
    CK(launch_pack<double>(which == 0 ? c->x64[level] : c->g64[level], c->geo[level], d_in, scale, c->stream),
       "level_set");
  if (!mixed(c) && level == 0 && which == 0) c->phi_zero = false;
  c->launches += 1;
  return MG_OK;
}

mg_status mg_level_get(mg_ctx* c, int level, int which, double* d_out) {
  if (!c) return MG_ERR_INVALID;
  if (level >= 0 && level < c->L && which >= 2 && which <= 5 && d_out) {  // permittivity coefficients
    if (!c->d_eps) return fail(c, MG_ERR_INVALID, "no variable permittivity is set");
    CK(launch_unpack<double>(d_out, c->vc[level] + (which - 2) * cells(c->geo[level]), c->geo[level], 1.0,
                             c->stream),
       "level_get");
    c->launches += 1;
    return MG_OK;
  }
  if (level < 0 || level >= c->L || (which != 0 && which != 1) || !d_out)
    return fail(c, MG_ERR_INVALID, "bad level, field or pointer");
  const double scale = which == 0 ? 1.0 : level_coeff(c, level);
  if (mixed(c))
    CK(launch_unpack<float>(d_out, which == 0 ? c->x32[level] : c->g32[level], c->geo[level], scale, c->stream),
       "level_get");
  else
    CK(launch_unpack<double>(d_out, which == 0 ? c->x64[level] : c->g64[level], c->geo[level], scale, c->stream),
       "level_get");
  c->launches += 1;
  return MG_OK;
}

mg_status mg_op_smooth(mg_ctx* c, int level, int colour) {
  if (c && !mixed(c) && level == 0) c->phi_zero = false;
  if (!c) return MG_ERR_INVALID;
  if (level < 0 || level >= c->L - 1 || (colour != 0 && colour != 1))
    return fail(c, MG_ERR_INVALID, "smoothing needs a non-coarsest level and colour 0 or 1");
  if (c->d_eps && mixed(c))
    CK(launch_var_smooth<float>(c->x32[level], c->g32[level], c->vc32[level], c->geo[level], colour, false,
                                c->stream),
       "smooth");
  else if (c->d_eps)
    CK(launch_var_smooth<double>(c->x64[level], c->g64[level], c->vc[level], c->geo[level], colour, false, c->stream),
       "smooth");
  else if (mixed(c))
    CK(sweep<float>(c, c->x32[level], c->g32[level], c->inv32, level, colour, false, c->stream), "smooth");
  else
    CK(sweep<double>(c, c->x64[level], c->g64[level], c->inv64, level, colour, false, c->stream), "smooth");
  c->launches += 1;
  return MG_OK;
}

static mg_status residual_restrict_op(mg_ctx* c, int level, bool red_only) {
  if (!c) return MG_ERR_INVALID;
  if (level < 0 || level >= c->L - 1) return fail(c, MG_ERR_INVALID, "restriction needs a non-coarsest level");
  if (c->d_eps && red_only) return fail(c, MG_ERR_INVALID, "the red-only restriction is single precision");
  if (c->d_eps && mixed(c))
    CK(launch_var_resid_restrict<float>(c->x32[level], c->g32[level], c->vc32[level], c->geo[level],
                                        c->g32[level + 1], c->geo[level + 1], c->stream),
       "residual_restrict");
  else if (c->d_eps)
    CK(launch_var_resid_restrict<double>(c->x64[level], c->g64[level], c->vc[level], c->geo[level],
                                         c->g64[level + 1], c->geo[level + 1], c->stream),
       "residual_restrict");
  else if (mixed(c))
    CK(launch_resid_restrict<float>(c->x32[level], c->g32[level], c->geo[level], c->g32[level + 1],
                                    c->geo[level + 1], red_only, c->stream),
       "residual_restrict");
  else if (c->rr_walk[level] && !red_only)
    CK(launch_resid_restrict_walk(c->x64[level], c->g64[level], c->geo[level], c->g64[level + 1],
                                  c->geo[level + 1], c->stream),
       "residual_restrict");
  else
    CK(launch_resid_restrict<double>(c->x64[level], c->g64[level], c->geo[level], c->g64[level + 1],
                                     c->geo[level + 1], red_only, c->stream),
       "residual_restrict");
  c->launches += 1;
  return MG_OK;
}

mg_status mg_op_residual_restrict(mg_ctx* c, int level) { return residual_restrict_op(c, level, false); }
mg_status mg_op_residual_restrict_red(mg_ctx* c, int level) { return residual_restrict_op(c, level, true); }

mg_status mg_op_prolong_smooth(mg_ctx* c, int level) {
  if (!c) return MG_ERR_INVALID;
  if (level < 0 || level >= c->L - 1) return fail(c, MG_ERR_INVALID, "prolongation needs a non-coarsest level");
  const Geom& G = c->geo[level];
  if (!mixed(c) || c->d_eps || !G.packed || G.hx % 4 != 0)
    return fail(c, MG_ERR_INVALID,
                "the fused prolongation sweep runs on single-precision levels of the constant operator with rows of "
                "whole 4-float vectors");
  if (c->tma[level].ok_pro)
    CK(launch_smooth_prolong_tma(c->x32[level], G, c->inv32, c->tma[level], (float)c->p.cgc_weight, c->d_err,
                                 c->stream),
       "prolong_smooth");
  else
    CK(launch_smooth_prolong(c->x32[level], c->g32[level], G, c->inv32, c->x32[level + 1], c->geo[level + 1],
                             (float)c->p.cgc_weight, c->stream),
       "prolong_smooth");
  c->launches += 1;
  return MG_OK;
}

int mg_level_prolong_sweep_kind(const mg_ctx* c, int level) {
  if (!c || level < 0 || level >= c->L - 1) return -1;
  const Geom& G = c->geo[level];
  if (!mixed(c) || c->d_eps || !G.packed || G.hx % 4 != 0) return -1;
  return c->tma[level].ok_pro ? 1 : 0;
}

mg_status mg_op_prolong_correct(mg_ctx* c, int level) {
  if (c && !mixed(c) && level == 0) c->phi_zero = false;
  if (!c) return MG_ERR_INVALID;
  if (level < 0 || level >= c->L - 1) return fail(c, MG_ERR_INVALID, "prolongation needs a non-coarsest level");
  if (mixed(c))
    CK(launch_prolong<float>(c->x32[level], c->geo[level], c->x32[level + 1], c->geo[level + 1],
                             (float)c->p.cgc_weight, false, c->stream),
       "prolong");
  else
    CK(launch_prolong<double>(c->x64[level], c->geo[level], c->x64[level + 1], c->geo[level + 1], c->p.cgc_weight,
                              false, c->stream),
       "prolong");
  c->launches += 1;
  return MG_OK;
}

mg_status mg_op_coarse_solve(mg_ctx* c, int* h_iters) {
  if (!c) return MG_ERR_INVALID;
  const int l = c->L - 1;
  const Geom& G = c->geo[l];
  const int n = G.nx * G.ny * G.nz;
  if (!mixed(c) && l == 0) c->phi_zero = false;  // single-level grid: the CG writes the finest iterate
  if (c->d_eps && mixed(c))
    CK(launch_var_coarse_cg<float>(c->x32[l], c->g32[l], c->vc32[l], G, 1e-14, 2 * n, c->d_iters, c->stream),
       "coarse_solve");
  else if (c->d_eps)
    CK(launch_var_coarse_cg<double>(c->x64[l], c->g64[l], c->vc[l], G, 1e-14, 2 * n, c->d_iters, c->stream),
       "coarse_solve");
  else if (mixed(c))
    CK(launch_coarse_cg<float>(c->x32[l], c->g32[l], G, kCoarseRtolF32, 2 * n, c->d_iters, c->stream), "coarse_solve");
  else
    CK(launch_coarse_cg<double>(c->x64[l], c->g64[l], G, 1e-14, 2 * n, c->d_iters, c->stream), "coarse_solve");
  c->launches += 1;
  int it = 0;
  CK(cudaMemcpyAsync(c->h_pin, c->d_iters, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "coarse_solve");
  CK(cudaStreamSynchronize(c->stream), "coarse_solve");
  std::memcpy(&it, c->h_pin, sizeof(int));
  if (h_iters) *h_iters = it;
  return MG_OK;
}

mg_status mg_op_residual_norm(mg_ctx* c) {
  if (!c) return MG_ERR_INVALID;
  mg_status st = materialize(c);
  if (st != MG_OK) return st;
  long long nk = 0;
  CK(enqueue_resid(c, mixed(c) ? 2 : 0, nullptr, c->stream, &nk), "residual_norm");
  c->launches += nk;
  ++c->cnt_direct;
  return MG_OK;
}

mg_status mg_op_defect_update(mg_ctx* c, int zero_start, double sc, double sc_next, const double* d_phi,
                              const double* d_e, const double* d_r, double* d_phi_out, double* d_hi_out,
                              double* d_lo_out, double* h_sumsq) {
  if (!c) return MG_ERR_INVALID;
  if (!c->rec_on) return fail(c, MG_ERR_INVALID, "the recurrence step needs MG_MIXED and finest rows of whole 4-float vectors");
  // both scales powers of two in [2^-800, 2^800], as the solver's are
  int p = 0, pn = 0;
  const bool ok = sc > 0.0 && sc_next > 0.0 && std::isfinite(sc) && std::isfinite(sc_next) &&
                  std::frexp(sc, &p) == 0.5 && std::frexp(sc_next, &pn) == 0.5 && std::abs(p - 1) <= 800 &&
                  std::abs(pn - 1) <= 800;
  if (!ok) return fail(c, MG_ERR_INVALID, "scales must be powers of two in [2^-800, 2^800]");
  p -= 1;
  if (!d_e || !d_r || (!zero_start && !d_phi) || !d_phi_out || !d_hi_out || !d_lo_out || !h_sumsq)
    return fail(c, MG_ERR_INVALID, "null argument");
  const Geom& G = c->geo[0];
  CK(launch_pack<float>(c->x32[0], G, d_e, 1.0, c->stream), "defect_update");
  if (zero_start) {
    CK(launch_pack<double>(c->g64[0], G, d_r, 1.0, c->stream), "defect_update");
  } else {
    CK(launch_pack<double>(c->x64[0], G, d_phi, 1.0, c->stream), "defect_update");
    CK(launch_pack_pair(c->g32[0], c->q_lo, G, d_r, -p, c->stream), "defect_update");
  }
  const double sv[2] = {sc, 1.0 / sc}, nv[2] = {sc_next, 1.0 / sc_next};
  CK(cudaMemcpyAsync(c->scal + S_SCALE, sv, sizeof(sv), cudaMemcpyHostToDevice, c->stream), "defect_update");
  CK(cudaMemcpyAsync(c->scal + S_NEXT, nv, sizeof(nv), cudaMemcpyHostToDevice, c->stream), "defect_update");
  int np = 0;
  CK(launch_defect_rec(c->x64[0], c->x32[0], c->g32[0], c->q_lo, c->g64[0], G, c->scal, S_SCALE, S_NEXT,
                       zero_start != 0, c->partials, &np, c->stream),
     "defect_update");
  CK(launch_defect_finalize(c->partials, np, c->scal, S_RSUM, S_REL, S_GSUM, S_SCALE, S_NEXT, c->stream),
     "defect_update");
  CK(launch_unpack<double>(d_phi_out, c->x64[0], G, 1.0, c->stream), "defect_update");
  CK(launch_unpack<float>(d_hi_out, c->g32[0], G, 1.0, c->stream), "defect_update");
  CK(launch_unpack<float>(d_lo_out, c->q_lo, G, 1.0, c->stream), "defect_update");
  CK(cudaMemcpyAsync(c->h_pin, c->scal + S_RSUM, sizeof(double), cudaMemcpyDeviceToHost, c->stream), "defect_update");
  CK(cudaStreamSynchronize(c->stream), "defect_update");
  *h_sumsq = c->h_pin[0];
  c->x_lazy = false;
  c->phi_zero = false;
  c->launches += zero_start ? 8 : 9;
  return MG_OK;
}

mg_status mg_outer_counts(const mg_ctx* c, long long* h_counts3) {
  if (!c || !h_counts3) return MG_ERR_INVALID;
  h_counts3[0] = c->cnt_cycles;
  h_counts3[1] = c->cnt_rec;
  h_counts3[2] = c->cnt_direct;
  return MG_OK;
}

mg_status mg_op_defect_step(mg_ctx* c) {
  if (!c) return MG_ERR_INVALID;
  if (!c->rec_on) return fail(c, MG_ERR_INVALID, "the recurrence step needs MG_MIXED and finest rows of whole 4-float vectors");
  mg_status st = materialize(c);
  if (st != MG_OK) return st;
  const Geom& G = c->geo[0];
  int np = 0;
  CK(launch_set_scale(c->scal, S_RSUM, S_NEXT, (double)cells(G), c->stream), "defect_step");
  CK(launch_defect_rec(c->x64[0], c->x32[0], c->g32[0], c->q_lo, c->g64[0], G, c->scal, S_SCALE, S_NEXT, false,
                       c->partials, &np, c->stream),
     "defect_step");
  CK(launch_defect_finalize(c->partials, np, c->scal, S_RSUM, S_REL, S_GSUM, S_SCALE, S_NEXT, c->stream),
     "defect_step");
  c->phi_zero = false;
  c->launches += 3;
  return MG_OK;
}

mg_status mg_op_scale_convert(const double* d_x, const float* d_e, const double* d_y, long long n, double sc,
                              float* d_xf, double* d_yo, double* d_xs, void* stream) {
  if (n < 0 || !(sc > 0.0) || !std::isfinite(sc) || !std::isfinite(1.0 / sc)) return MG_ERR_INVALID;
  if (n == 0) return MG_OK;
  if (!d_x || !d_e || !d_y || !d_xf || !d_yo || !d_xs) return MG_ERR_INVALID;
  if (launch_scale_convert(d_x, d_e, d_y, n, sc, d_xf, d_yo, d_xs, (cudaStream_t)stream) != cudaSuccess)
    return MG_ERR_CUDA;
  return MG_OK;
}

}  // extern "C"
