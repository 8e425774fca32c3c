// batch_api.cu -- many independent Poisson systems of different sizes solved together.
//
// Each system is the single-system problem of ccmg_api.cu (own dimensions, cell size, walls,
// right-hand side). Every multigrid operation is ONE launch over all systems that take part in it
// (batch_kernels.cu). Systems with different level counts are scheduled by depth below the finest
// level: descend (smoothing + residual/restriction at depth d for every system with more than d+1
// levels), one coarse-CG launch for all systems, ascend. Per-system activity flags in device memory
// let converged systems drop out of the same captured graphs. The smoother and transfer tile
// shapes are chosen by mg_batch_autotune, which times the whole batched cycle per candidate.
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>
#include <algorithm>

#include "../../include/ccmg.h"
#include "level_ops.cuh"

using namespace ccmg;

namespace {

struct BSys {
  mg_params p{};
  int L = 0;
  Geom geo[kMaxLevels]{};
  double* x64[kMaxLevels]{};
  double* g64[kMaxLevels]{};
  float* x32[kMaxLevels]{};
  float* g32[kMaxLevels]{};
  float* q_lo = nullptr;  // mixed: low part of the residual pair whose high part is g32[0] (recurrence)
  FaceBC bc{};
};

struct Plan {
  int e0 = 0, s0 = 0, count = 0, blocks = 0;
  dim3 block{1, 1, 1};
  int per = 0;  // some entry's level has a periodic axis
};

thread_local std::string g_batch_error;

long long cells(const Geom& G) { return G.packed ? 2 * G.csz : G.csz; }

const int kCandidates[][4] = {{32, 8, 64, 4}, {64, 4, 64, 4}, {128, 2, 64, 4}, {16, 16, 32, 8},
                              {32, 8, 32, 8}, {64, 4, 128, 2}, {8, 32, 32, 8}, {128, 2, 128, 2}};
constexpr int kNumCandidates = sizeof(kCandidates) / sizeof(kCandidates[0]);

}  // namespace

struct mg_batch {
  int B = 0;
  int prec = MG_FP64;
  int nu1 = 2, nu2 = 2, inner = 4;
  double omega = 2.0;
  cudaStream_t stream = nullptr;
  cudaStream_t cap = nullptr;
  std::vector<BSys> sys;
  int maxL = 0;
  char* arena = nullptr;
  InvDiag<double> inv64{};
  InvDiag<float> inv32{};
  int tile[4] = {64, 4, 64, 4};  // smoother (bx, by), transfers (bx, by)
  std::vector<BEntry> h_entries;
  std::vector<int> h_starts;
  BEntry* d_entries = nullptr;
  int* d_starts = nullptr;
  size_t cap_entries = 0, cap_starts = 0;
  Plan smooth[kMaxLevels], xfer[kMaxLevels], restr[kMaxLevels], cg, resid, update;
  Plan defect;  // finest levels of the systems that can step by recurrence (q_lo set)
  bool rec_on = false;  // mixed solves carry residuals by recurrence (CCMG_DEFECT=walk: never)
  int* d_rec = nullptr;  // per system: this cycle steps by recurrence (all zero outside mg_batch_solve)
  int* h_rec = nullptr;
  Plan xfer_nv[kMaxLevels];  // prolongation entries of the systems whose rows are not whole vectors
  size_t cg_smem = 0;
  int* d_active = nullptr;
  int* h_active = nullptr;
  int* d_zero = nullptr;  // per system: iterate known to be exactly zero
  int* h_zero = nullptr;
  std::vector<char> lazy;  // per system (mixed): finest iterate zero but never written
  // pinned staging slots for flag uploads: a slot is rewritten only after the copy that read it
  // last has run (its event), so a later host-side change never leaks into an earlier upload
  static constexpr int kFlagSlots = 16;
  int* h_flag_ring = nullptr;
  // mg_batch_set_rhs_all: the job table on the device, its staging ring on the host (two slots,
  // each reused once its copy has run), the sum-of-squares partials of all systems
  RhsJob* d_rhs = nullptr;
  RhsJob* h_rhs = nullptr;
  cudaEvent_t rhs_ev[2]{};
  int rhs_slot = 0;
  int rhs_nsb = 0;
  double* d_rhs_partials = nullptr;
  cudaEvent_t flag_ev[kFlagSlots]{};
  int flag_slot = 0;
  double* d_scal = nullptr;
  double* h_scal = nullptr;
  double* d_partials = nullptr;
  size_t cap_partials = 0;
  cudaGraphExec_t g_cycle = nullptr, g_resid = nullptr;
  long long n_cycle = 0, n_resid = 0;
  long long launches = 0;
  // single precision: the finest levels' half-sweeps TMA-staged (one table entry per system), when
  // every system's finest level qualifies
  BTmaSys* d_tma = nullptr;
  long long tma_total = 0;
  int tma_grid = 0;
  bool tma_ok = false;
  int* d_err = nullptr;  // set by a kernel whose bounded wait ran out
  int* h_err = nullptr;
  std::string err;
};

namespace {

mg_status bfail(mg_batch* b, mg_status st, const std::string& msg) {
  if (b) b->err = msg;
  else g_batch_error = msg;
  return st;
}

#define BCK(call, where)                                                                             \
  do {                                                                                               \
    cudaError_t e_ = (call);                                                                         \
    if (e_ != cudaSuccess) return bfail(b, MG_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e_)); \
  } while (0)

bool bmixed(const mg_batch* b) { return b->prec == MG_MIXED; }

BLaunch bl(const mg_batch* b, const Plan& p) {
  BLaunch L;
  L.entries = b->d_entries + p.e0;
  L.start = b->d_starts + p.s0;
  L.count = p.count;
  L.blocks = p.blocks;
  L.block = p.block;
  L.per = p.per;
  return L;
}

void add_plan(mg_batch* b, Plan& p, const std::vector<BEntry>& ents, dim3 block) {
  p.e0 = (int)b->h_entries.size();
  p.s0 = (int)b->h_starts.size();
  p.count = (int)ents.size();
  p.block = block;
  int acc = 0;
  p.per = 0;
  for (const BEntry& e : ents) {
    b->h_starts.push_back(acc);
    acc += e.gx * e.gy * e.gz;
    b->h_entries.push_back(e);
    if (e.G.per) p.per = 1;
  }
  b->h_starts.push_back(acc);
  p.blocks = acc;
}

void destroy_graphs(mg_batch* b) {
  if (b->g_cycle) cudaGraphExecDestroy(b->g_cycle);
  if (b->g_resid) cudaGraphExecDestroy(b->g_resid);
  b->g_cycle = b->g_resid = nullptr;
}

int ceil_div(long long a, long long c) { return (int)((a + c - 1) / c); }

// Build every launch's entry table for the current tiles and upload it.
mg_status plan(mg_batch* b) {
  destroy_graphs(b);
  b->h_entries.clear();
  b->h_starts.clear();
  const bool mx = bmixed(b);
  const int V = mx ? 4 : 2;
  const int sbx = b->tile[0], sby = b->tile[1], tbx = b->tile[2], tby = b->tile[3];
  for (int d = 0; d < kMaxLevels; ++d) {
    b->smooth[d] = Plan();
    b->xfer[d] = Plan();
    b->xfer_nv[d] = Plan();
    b->restr[d] = Plan();
  }
  for (int d = 0; d + 1 < b->maxL; ++d) {
    std::vector<BEntry> es, et, er, etn;
    for (int s = 0; s < b->B; ++s) {
      BSys& S = b->sys[s];
      if (d >= S.L - 1) continue;
      BEntry e{};
      e.G = S.geo[d];
      e.Gc = S.geo[d + 1];
      e.x = mx ? (void*)S.x32[d] : (void*)S.x64[d];
      e.g = mx ? (void*)S.g32[d] : (void*)S.g64[d];
      e.xc = mx ? (void*)S.x32[d + 1] : (void*)S.x64[d + 1];
      e.gc = mx ? (void*)S.g32[d + 1] : (void*)S.g64[d + 1];
      e.sys = s;
      // vector entries and the prolongation take chunks of a plane's (row, element) pairs with
      // sbx * sby (tbx * tby) threads per block; the rest a 2D (element, row) tile
      BEntry es1 = e;
      es1.vec = (e.G.hx % V == 0) ? 1 : 0;
      if (es1.vec) {
        es1.gx = ceil_div((long long)(e.G.hx / V) * e.G.ny, sbx * sby);
        es1.gy = 1;
      } else {
        es1.gx = ceil_div(e.G.hx, sbx);
        es1.gy = ceil_div(e.G.ny, sby);
      }
      es1.gz = e.G.nz;
      es.push_back(es1);
      BEntry et1 = e;  // prolongation: one thread per coarse cell
      et1.gx = ceil_div((long long)e.Gc.nx * e.Gc.ny, tbx * tby);
      et1.gy = 1;
      et1.gz = e.Gc.nz;
      et.push_back(et1);
      if (e.G.hx % V != 0) etn.push_back(et1);
      BEntry er1 = e;  // residual + restriction: V coarse cells per thread where rows allow
      er1.vec = (e.G.hx % V == 0) ? 1 : 0;
      if (er1.vec) {
        er1.gx = ceil_div((long long)(e.Gc.nx / V) * e.Gc.ny, tbx * tby);
        er1.gy = 1;
      } else {
        er1.gx = ceil_div(e.Gc.nx, tbx);
        er1.gy = ceil_div(e.Gc.ny, tby);
      }
      er1.gz = e.Gc.nz;
      er.push_back(er1);
    }
    add_plan(b, b->smooth[d], es, dim3(sbx, sby, 1));
    add_plan(b, b->xfer[d], et, dim3(tbx, tby, 1));
    add_plan(b, b->xfer_nv[d], etn, dim3(tbx, tby, 1));
    add_plan(b, b->restr[d], er, dim3(tbx, tby, 1));
  }
  {  // coarsest grids: one CTA each, as many threads as the largest single-system launch would use
    std::vector<BEntry> ec;
    int threads = 32, nmax = 1;
    for (int s = 0; s < b->B; ++s) {
      BSys& S = b->sys[s];
      BEntry e{};
      e.G = S.geo[S.L - 1];
      e.x = mx ? (void*)S.x32[S.L - 1] : (void*)S.x64[S.L - 1];
      e.g = mx ? (void*)S.g32[S.L - 1] : (void*)S.g64[S.L - 1];
      e.sys = s;
      e.gx = e.gy = e.gz = 1;
      ec.push_back(e);
      const int n = e.G.nx * e.G.ny * e.G.nz;
      int t = ((n + 31) / 32) * 32;
      if (t > 256) t = 256;
      if (t > threads) threads = t;
      if (n > nmax) nmax = n;
    }
    add_plan(b, b->cg, ec, dim3(threads, 1, 1));
    b->cg_smem = (size_t)4 * nmax * sizeof(double);
  }
  {  // finest-level FP64 residual (the termination test) and the mixed-precision update
    std::vector<BEntry> er, eu;
    for (int s = 0; s < b->B; ++s) {
      BSys& S = b->sys[s];
      BEntry e{};
      e.G = S.geo[0];
      e.x = S.x64[0];
      e.g = S.g64[0];
      e.aux = mx ? (void*)S.g32[0] : nullptr;
      e.sys = s;
      e.gx = ops::resid_norm_blocks(S.geo[0]);
      e.gy = e.gz = 1;
      er.push_back(e);
      BEntry u = e;
      u.aux = mx ? (void*)S.x32[0] : nullptr;
      u.gx = std::max(1, std::min(ceil_div(cells(S.geo[0]), 256), 152 * 16));
      eu.push_back(u);
    }
    add_plan(b, b->resid, er, dim3(ops::kResBX, ops::kResBY, 1));
    add_plan(b, b->update, eu, dim3(256, 1, 1));
  }
  {  // the recurrence step: each system as many virtual blocks as its single-system launch has CTAs
    std::vector<BEntry> ed;
    for (int s = 0; s < b->B; ++s) {
      BSys& S = b->sys[s];
      if (!S.q_lo) continue;
      BEntry e{};
      e.G = S.geo[0];
      e.x = S.x64[0];
      e.g = S.g64[0];
      e.xc = S.x32[0];
      e.gc = S.g32[0];
      e.aux = S.q_lo;
      e.sys = s;
      e.gx = defect_rec_blocks(S.geo[0]);
      e.gy = e.gz = 1;
      if (e.gx < 1) return bfail(b, MG_ERR_CUDA, "batch plan: no occupancy for the recurrence step");
      ed.push_back(e);
    }
    add_plan(b, b->defect, ed, dim3(256, 1, 1));
  }
  if (b->h_entries.size() > b->cap_entries) {
    cudaFree(b->d_entries);
    b->d_entries = nullptr;
    b->cap_entries = 0;
    BCK(cudaMalloc((void**)&b->d_entries, b->h_entries.size() * sizeof(BEntry)), "batch plan");
    b->cap_entries = b->h_entries.size();
  }
  if (b->h_starts.size() > b->cap_starts) {
    cudaFree(b->d_starts);
    b->d_starts = nullptr;
    b->cap_starts = 0;
    BCK(cudaMalloc((void**)&b->d_starts, b->h_starts.size() * sizeof(int)), "batch plan");
    b->cap_starts = b->h_starts.size();
  }
  const size_t np = std::max({(size_t)b->resid.blocks, (size_t)b->defect.blocks, (size_t)kMaxPartials});
  if (np > b->cap_partials) {
    cudaFree(b->d_partials);
    b->d_partials = nullptr;
    b->cap_partials = 0;
    BCK(cudaMalloc((void**)&b->d_partials, np * sizeof(double)), "batch plan");
    b->cap_partials = np;
  }
  BCK(cudaMemcpyAsync(b->d_entries, b->h_entries.data(), b->h_entries.size() * sizeof(BEntry), cudaMemcpyHostToDevice,
                      b->stream),
      "batch plan");
  BCK(cudaMemcpyAsync(b->d_starts, b->h_starts.data(), b->h_starts.size() * sizeof(int), cudaMemcpyHostToDevice,
                      b->stream),
      "batch plan");
  BCK(cudaStreamSynchronize(b->stream), "batch plan");
  return MG_OK;
}

template <typename T>
cudaError_t enqueue_bvcycle(mg_batch* b, const InvDiag<T>& inv, bool zero0, cudaStream_t s, long long* nk) {
  cudaError_t e;
  const int* act = b->d_active;
  for (int d = 0; d + 1 < b->maxL; ++d) {
    const BLaunch Ls = bl(b, b->smooth[d]);
    if (Ls.count == 0) continue;
    const bool zero = (d > 0) || zero0;
    // the finest levels' sweeps TMA-staged (single precision; not from a zero iterate)
    auto sweep = [&](int colour, bool z) -> cudaError_t {
      if constexpr (sizeof(T) == sizeof(float))
        if (d == 0 && !z && b->tma_ok)
          return launch_b_smooth_tma(b->d_tma, b->B, b->tma_total, b->tma_grid, act, inv, colour, b->d_err, s);
      return launch_b_smooth<T>(Ls, act, inv, colour, z, s);
    };
    for (int it = 0; it < b->nu1; ++it) {
      if ((e = sweep(0, zero && it == 0)) != cudaSuccess) return e;
      if ((e = sweep(1, false)) != cudaSuccess) return e;
      *nk += 2;
    }
    // as the single-system cycle: red-only restriction in single precision only
    const bool red_only = sizeof(T) == sizeof(float) && b->nu1 >= 1;
    if ((e = launch_b_resid_restrict<T>(bl(b, b->restr[d]), act, red_only, s)) != cudaSuccess) return e;
    ++*nk;
  }
  if ((e = launch_b_coarse_cg<T>(bl(b, b->cg), act, b->cg_smem, coarse_rtol<T>(), s)) != cudaSuccess) return e;
  ++*nk;
  // single precision, as the single-system cycle: the prolongation is fused into the first black
  // sweep of the systems whose rows are whole vectors; the others prolong first
  const bool fuse = sizeof(T) == sizeof(float) && b->nu2 >= 1;
  for (int d = b->maxL - 2; d >= 0; --d) {
    const BLaunch Ls = bl(b, b->smooth[d]);
    if (Ls.count == 0) continue;
    const BLaunch Lp = bl(b, fuse ? b->xfer_nv[d] : b->xfer[d]);
    if ((e = launch_b_prolong<T>(Lp, act, (T)b->omega, b->nu2 >= 1, s)) != cudaSuccess) return e;
    *nk += Lp.count > 0 ? 1 : 0;
    const bool tma = sizeof(T) == sizeof(float) && d == 0 && b->tma_ok;
    for (int it = 0; it < b->nu2; ++it) {
      if (fuse && it == 0 && tma)
        e = launch_b_smooth_prolong_tma(b->d_tma, b->B, b->tma_total, b->tma_grid, act, b->inv32, (float)b->omega,
                                        b->d_err, s);
      else if (fuse && it == 0)
        e = launch_b_smooth_prolong(Ls, act, b->inv32, (float)b->omega, s);
      else if (tma)
        e = launch_b_smooth_tma(b->d_tma, b->B, b->tma_total, b->tma_grid, act, b->inv32, 1, b->d_err, s);
      else
        e = launch_b_smooth<T>(Ls, act, inv, 1, false, s);
      if (e != cudaSuccess) return e;
      if (tma)
        e = launch_b_smooth_tma(b->d_tma, b->B, b->tma_total, b->tma_grid, act, b->inv32, 0, b->d_err, s);
      else
        e = launch_b_smooth<T>(Ls, act, inv, 0, false, s);
      if (e != cudaSuccess) return e;
      *nk += 2;
    }
  }
  return cudaSuccess;
}

cudaError_t enqueue_bcycle(mg_batch* b, cudaStream_t s, long long* nk) {
  if (!bmixed(b)) return enqueue_bvcycle<double>(b, b->inv64, false, s, nk);
  cudaError_t e;
  for (int it = 0; it < b->inner; ++it)
    if ((e = enqueue_bvcycle<float>(b, b->inv32, it == 0, s, nk)) != cudaSuccess) return e;
  // phi += s e and the next scale for the systems that evaluate their residual directly; the
  // recurrence step (with its own next scale and norm) for those with rec[sys]
  if ((e = launch_b_update(bl(b, b->update), b->d_active, b->d_rec, b->d_zero, b->d_scal, s)) != cudaSuccess) return e;
  if (b->defect.count > 0) {
    if ((e = launch_b_defect_step(bl(b, b->defect), b->d_active, b->d_rec, b->d_zero, b->d_scal, b->d_partials, s)) !=
        cudaSuccess)
      return e;
    *nk += 4;
  }
  if ((e = launch_b_set_scale(bl(b, b->resid), b->d_active, b->d_rec, b->d_scal, s)) != cudaSuccess) return e;
  *nk += 2;
  return cudaSuccess;
}

cudaError_t enqueue_bresid(mg_batch* b, cudaStream_t s, long long* nk) {
  *nk += 2;
  return launch_b_resid_norm(bl(b, b->resid), b->d_active, b->d_zero, bmixed(b) ? 2 : 0, b->d_scal, b->d_partials,
                             s);
}

template <typename F>
mg_status bcapture(mg_batch* b, cudaGraphExec_t* out, long long* nodes, F body, const char* what) {
  if (*out) return MG_OK;
  cudaError_t e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return bfail(b, MG_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
  long long nk = 0;
  cudaError_t eb = body(b->cap, &nk);
  cudaGraph_t g = nullptr;
  cudaError_t ee = cudaStreamEndCapture(b->cap, &g);
  if (eb != cudaSuccess || ee != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return bfail(b, MG_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(eb != cudaSuccess ? eb : ee));
  }
  e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    *out = nullptr;
    return bfail(b, MG_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
  }
  *nodes = nk;
  return MG_OK;
}

mg_status bgraphs(mg_batch* b) {
  mg_status st = bcapture(b, &b->g_cycle, &b->n_cycle,
                          [b](cudaStream_t s, long long* nk) { return enqueue_bcycle(b, s, nk); }, "batch cycle");
  if (st != MG_OK) return st;
  return bcapture(b, &b->g_resid, &b->n_resid,
                  [b](cudaStream_t s, long long* nk) { return enqueue_bresid(b, s, nk); }, "batch residual");
}

mg_status brun(mg_batch* b, cudaGraphExec_t g, long long nodes, const char* what) {
  BCK(cudaGraphLaunch(g, b->stream), what);
  b->launches += nodes;
  return MG_OK;
}

mg_status upload_flags(mg_batch* b, int* d_dst, const int* h_src) {
  const int k = b->flag_slot;
  b->flag_slot = (k + 1) % mg_batch::kFlagSlots;
  int* slot = b->h_flag_ring + (size_t)k * b->B;
  BCK(cudaEventSynchronize(b->flag_ev[k]), "flag upload");
  std::memcpy(slot, h_src, (size_t)b->B * sizeof(int));
  BCK(cudaMemcpyAsync(d_dst, slot, (size_t)b->B * sizeof(int), cudaMemcpyHostToDevice, b->stream), "flag upload");
  BCK(cudaEventRecord(b->flag_ev[k], b->stream), "flag upload");
  return MG_OK;
}

mg_status set_all_active(mg_batch* b, int v) {
  for (int s = 0; s < b->B; ++s) b->h_active[s] = v;
  if (mg_status st = upload_flags(b, b->d_active, b->h_active); st != MG_OK) return st;
  return MG_OK;
}

mg_status upload_zero(mg_batch* b) { return upload_flags(b, b->d_zero, b->h_zero); }

// After a cycle graph ran: the iterates of the systems that took part are no longer zero (and a
// never-written one has been stored by the update).
mg_status clear_zero_of_active(mg_batch* b) {
  bool changed = false;
  for (int s = 0; s < b->B; ++s)
    if (b->h_active[s] && b->h_zero[s]) {
      b->h_zero[s] = 0;
      b->lazy[s] = 0;
      changed = true;
    }
  return changed ? upload_zero(b) : MG_OK;
}

// Write the zeros of a finest iterate that set_solution(NULL) left unwritten.
mg_status materialize(mg_batch* b, int s) {
  if (!b->lazy[s]) return MG_OK;
  BCK(cudaMemsetAsync(b->sys[s].x64[0], 0, sizeof(double) * (size_t)cells(b->sys[s].geo[0]), b->stream),
      "zero iterate");
  b->lazy[s] = 0;
  return MG_OK;
}

void free_batch(mg_batch* b) {
  destroy_graphs(b);
  cudaFree(b->d_tma);
  cudaFree(b->d_err);
  if (b->h_err) cudaFreeHost(b->h_err);
  cudaFree(b->arena);
  cudaFree(b->d_entries);
  cudaFree(b->d_starts);
  cudaFree(b->d_active);
  cudaFree(b->d_zero);
  cudaFree(b->d_rec);
  if (b->h_rec) cudaFreeHost(b->h_rec);
  cudaFree(b->d_scal);
  cudaFree(b->d_partials);
  if (b->h_active) cudaFreeHost(b->h_active);
  if (b->h_zero) cudaFreeHost(b->h_zero);
  if (b->h_flag_ring) cudaFreeHost(b->h_flag_ring);
  for (int k = 0; k < mg_batch::kFlagSlots; ++k)
    if (b->flag_ev[k]) cudaEventDestroy(b->flag_ev[k]);
  if (b->h_scal) cudaFreeHost(b->h_scal);
  cudaFree(b->d_rhs);
  cudaFree(b->d_rhs_partials);
  if (b->h_rhs) cudaFreeHost(b->h_rhs);
  for (int k = 0; k < 2; ++k)
    if (b->rhs_ev[k]) cudaEventDestroy(b->rhs_ev[k]);
  if (b->cap) cudaStreamDestroy(b->cap);
}

// The TMA-staged half-sweeps of the systems' finest single-precision levels (as a single context
// stages its largest levels): one table entry per system, made when every system qualifies
// (packed finest level with whole 4-float rows and at least 8 planes, no periodic axis, a packed
// next level of half the size). CCMG_SWEEP=vec keeps the direct-load sweeps (as for a context).
mg_status prepare_batch_tma(mg_batch* b) {
  b->tma_ok = false;
  if (!bmixed(b)) return MG_OK;
  const char* env = std::getenv("CCMG_SWEEP");
  if (env && std::strcmp(env, "vec") == 0) return MG_OK;
  std::vector<float*> x(b->B);
  std::vector<const float*> g(b->B), xc(b->B);
  std::vector<Geom> G(b->B), Gc(b->B);
  std::vector<int> idx(b->B);
  for (int s = 0; s < b->B; ++s) {
    const BSys& S = b->sys[s];
    if (S.L < 2) return MG_OK;
    x[s] = S.x32[0];
    g[s] = S.g32[0];
    xc[s] = S.x32[1];
    G[s] = S.geo[0];
    Gc[s] = S.geo[1];
    idx[s] = s;
  }
  std::vector<BTmaSys> tab(b->B);
  int ok = 0, dev = 0;
  BCK(cudaGetDevice(&dev), "batch TMA maps");
  BCK(prepare_tma_batch(tab.data(), b->B, x.data(), g.data(), G.data(), xc.data(), Gc.data(), idx.data(),
                        &b->tma_total, &b->tma_grid, &ok, dev),
      "batch TMA maps");
  if (!ok) return MG_OK;
  BCK(cudaMalloc((void**)&b->d_tma, tab.size() * sizeof(BTmaSys)), "batch TMA maps");
  BCK(cudaMemcpy(b->d_tma, tab.data(), tab.size() * sizeof(BTmaSys), cudaMemcpyHostToDevice), "batch TMA maps");
  b->tma_ok = true;
  return MG_OK;
}

mg_status check_sys(mg_batch* b, int s) {
  if (!b) return MG_ERR_INVALID;
  if (s < 0 || s >= b->B) return bfail(b, MG_ERR_INVALID, "system index out of range");
  return MG_OK;
}

}  // namespace

extern "C" {

const char* mg_batch_last_error(const mg_batch* b) { return b ? b->err.c_str() : g_batch_error.c_str(); }

mg_status mg_batch_create(int B, const mg_params* params, void* stream, mg_batch** out) {
  mg_batch* b = nullptr;
  if (!params || !out || B < 1) return bfail(b, MG_ERR_INVALID, "need B >= 1 and non-null params and out");
  *out = nullptr;
  const mg_params& p0 = params[0];
  for (int s = 0; s < B; ++s) {
    // validate each system with the single-system rules
    const mg_params& p = params[s];
    const int d[3] = {p.nx, p.ny, p.nz};
    for (int a = 0; a < 3; ++a)
      if (d[a] < 4 || (d[a] % 2) != 0) return bfail(b, MG_ERR_INVALID, "grid dimensions must be even and >= 4");
    if (!(p.h > 0.0) || !std::isfinite(p.h) || !(p.eps > 0.0) || !std::isfinite(p.eps))
      return bfail(b, MG_ERR_INVALID, "h and eps must be positive");
    if (const char* why = check_bc_types(p.bc_type)) return bfail(b, MG_ERR_INVALID, why);
    for (int q = 0; q < 6; ++q)
      if (!std::isfinite(p.bc_value[q])) return bfail(b, MG_ERR_INVALID, "bc_value must be finite");
    if (p.prec != p0.prec || p.nu1 != p0.nu1 || p.nu2 != p0.nu2 || p.cgc_weight != p0.cgc_weight ||
        (p0.prec == MG_MIXED && p.mixed_inner != p0.mixed_inner))
      return bfail(b, MG_ERR_INVALID, "all systems of a batch share prec, nu1, nu2, cgc_weight and mixed_inner");
  }
  if (p0.nu1 < 1 || p0.nu1 > 16 || p0.nu2 < 1 || p0.nu2 > 16)
    return bfail(b, MG_ERR_INVALID, "a batch needs 1 <= nu1, nu2 <= 16");
  if (p0.prec != MG_FP64 && p0.prec != MG_MIXED) return bfail(b, MG_ERR_INVALID, "prec must be MG_FP64 or MG_MIXED");
  if (p0.prec == MG_MIXED && (p0.mixed_inner < 1 || p0.mixed_inner > 16))
    return bfail(b, MG_ERR_INVALID, "mixed_inner must be in 1..16");
  if (!std::isfinite(p0.cgc_weight)) return bfail(b, MG_ERR_INVALID, "cgc_weight must be finite");

  b = new mg_batch();
  b->B = B;
  b->prec = p0.prec;
  b->nu1 = p0.nu1;
  b->nu2 = p0.nu2;
  b->inner = p0.mixed_inner;
  b->omega = p0.cgc_weight;
  // mixed solves carry each system's residual by recurrence between direct checks where its
  // finest level has rows of whole 4-float vectors, as single contexts do; CCMG_DEFECT=walk
  // evaluates it directly after every step
  const char* defect_env = std::getenv("CCMG_DEFECT");
  b->rec_on = bmixed(b) && !(defect_env && std::strcmp(defect_env, "walk") == 0);
  b->stream = (cudaStream_t)stream;
  b->sys.resize(B);
  for (int d6 = -3; d6 <= 3; ++d6) {
    b->inv64.v[d6 + 3] = 1.0 / (double)(6 + d6);
    b->inv32.v[d6 + 3] = 1.0f / (float)(6 + d6);
  }
  // hierarchies (Sec. 3 coarsening rule) and the arena size
  size_t bytes = 0;
  auto reserve = [&bytes](size_t n) {
    const size_t off = bytes;
    bytes += (n + 255) / 256 * 256;
    return off;
  };
  std::vector<std::vector<size_t>> offs(B);
  for (int s = 0; s < B; ++s) {
    BSys& S = b->sys[s];
    S.p = params[s];
    for (int q = 0; q < 6; ++q) {
      S.bc.type[q] = S.p.bc_type[q];
      S.bc.value[q] = S.p.bc_value[q];
    }
    int dims[3] = {S.p.nx, S.p.ny, S.p.nz};
    for (;;) {
      if (S.L >= kMaxLevels) break;
      Geom& G = S.geo[S.L];
      G.nx = dims[0];
      G.ny = dims[1];
      G.nz = dims[2];
      for (int q = 0; q < 6; ++q) G.sh[q] = face_shift(S.p.bc_type[q]);
      G.per = periodic_bits(S.p.bc_type);
      ++S.L;
      bool ok = true;
      for (int a = 0; a < 3; ++a)
        if ((dims[a] % 2) != 0 || dims[a] / 2 < 3) ok = false;
      if (!ok) break;
      for (int a = 0; a < 3; ++a) dims[a] /= 2;
    }
    for (int l = 0; l < S.L; ++l) {
      Geom& G = S.geo[l];
      G.packed = (l < S.L - 1) ? 1 : 0;
      G.hx = G.nx / 2;
      G.csz = G.packed ? (long long)G.hx * G.ny * G.nz : (long long)G.nx * G.ny * G.nz;
    }
    const Geom& Gc = S.geo[S.L - 1];
    if ((long long)Gc.nx * Gc.ny * Gc.nz > kMaxCoarseCells) {
      delete b;
      return bfail(nullptr, MG_ERR_INVALID, "a coarsest grid has more than 4096 cells");
    }
    if (S.L > b->maxL) b->maxL = S.L;
    for (int l = 0; l < S.L; ++l) {
      const size_t n = (size_t)cells(S.geo[l]);
      if (!bmixed(b) || l == 0) {
        offs[s].push_back(reserve(n * sizeof(double)));
        offs[s].push_back(reserve(n * sizeof(double)));
      }
      if (bmixed(b)) {
        offs[s].push_back(reserve(n * sizeof(float)));
        offs[s].push_back(reserve(n * sizeof(float)));
      }
    }
    if (b->rec_on && defect_rec_applies(S.geo[0]))
      offs[s].push_back(reserve((size_t)cells(S.geo[0]) * sizeof(float)));  // q_lo
  }
  cudaError_t e = cudaMalloc((void**)&b->arena, bytes);
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_active, B * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_rec, B * sizeof(int));
  if (e == cudaSuccess) e = cudaMemsetAsync(b->d_rec, 0, B * sizeof(int), b->stream);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&b->h_rec, B * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_zero, B * sizeof(int));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&b->h_zero, B * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_scal, (size_t)B * kScalStride * sizeof(double));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&b->h_active, B * sizeof(int));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&b->h_flag_ring, (size_t)mg_batch::kFlagSlots * B * sizeof(int));
  for (int k = 0; k < mg_batch::kFlagSlots && e == cudaSuccess; ++k)
    e = cudaEventCreateWithFlags(&b->flag_ev[k], cudaEventDisableTiming);
  b->lazy.assign(B, 0);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&b->h_scal, (size_t)B * kScalStride * sizeof(double));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = prepare_b_coarse_cg();
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_err, sizeof(int));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&b->h_err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemsetAsync(b->d_err, 0, sizeof(int), b->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->arena, 0, bytes, b->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->d_scal, 0, (size_t)B * kScalStride * sizeof(double), b->stream);
  if (e == cudaSuccess) {  // mg_batch_set_rhs_all: one sum-of-squares partial per block of each system
    long long nsb = 0;
    for (int s = 0; s < B; ++s) {
      RhsJob j;
      rhs_job_static(j, b->sys[s].geo[0], nullptr, 1.0, 1.0, b->sys[s].bc, nullptr);
      nsb += j.sbn;
    }
    b->rhs_nsb = (int)nsb;
    e = cudaMalloc((void**)&b->d_rhs_partials, (size_t)nsb * sizeof(double));
  }
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_rhs, (size_t)B * sizeof(RhsJob));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&b->h_rhs, (size_t)2 * B * sizeof(RhsJob));
  for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = cudaEventCreateWithFlags(&b->rhs_ev[k], cudaEventDisableTiming);
  if (e != cudaSuccess) {
    const bool oom = (e == cudaErrorMemoryAllocation);
    std::string msg = std::string("mg_batch_create: ") + cudaGetErrorString(e);
    cudaGetLastError();
    free_batch(b);
    delete b;
    return bfail(nullptr, oom ? MG_ERR_OOM : MG_ERR_CUDA, msg);
  }
  for (int s = 0; s < B; ++s) {
    BSys& S = b->sys[s];
    size_t k = 0;
    for (int l = 0; l < S.L; ++l) {
      if (!bmixed(b) || l == 0) {
        S.x64[l] = (double*)(b->arena + offs[s][k++]);
        S.g64[l] = (double*)(b->arena + offs[s][k++]);
      }
      if (bmixed(b)) {
        S.x32[l] = (float*)(b->arena + offs[s][k++]);
        S.g32[l] = (float*)(b->arena + offs[s][k++]);
      }
    }
    if (b->rec_on && defect_rec_applies(S.geo[0])) S.q_lo = (float*)(b->arena + offs[s][k++]);
  }
  for (int s = 0; s < B; ++s) b->h_zero[s] = 1;  // the arena starts zeroed
  mg_status st = prepare_batch_tma(b);
  if (st == MG_OK) st = plan(b);
  if (st == MG_OK) st = set_all_active(b, 1);
  if (st == MG_OK) st = upload_zero(b);
  if (st != MG_OK) {
    std::string msg = b->err;
    free_batch(b);
    delete b;
    return bfail(nullptr, st, msg);
  }
  *out = b;
  return MG_OK;
}

mg_status mg_batch_destroy(mg_batch* b) {
  if (!b) return MG_ERR_INVALID;
  cudaStreamSynchronize(b->stream);
  free_batch(b);
  delete b;
  return MG_OK;
}

int mg_batch_size(const mg_batch* b) { return b ? b->B : 0; }

mg_status mg_batch_set_rhs(mg_batch* b, int s, const double* d_rho) {
  mg_status st = check_sys(b, s);
  if (st != MG_OK) return st;
  if (!d_rho) return bfail(b, MG_ERR_INVALID, "null right-hand side");
  BSys& S = b->sys[s];
  const Geom& G = S.geo[0];
  double* sc = b->d_scal + (size_t)kScalStride * s;
  int np = 0;
  BCK(launch_set_rhs<double>(S.g64[0], G, d_rho, 1.0 / S.p.eps, S.p.h, S.bc, 0, b->stream), "batch set_rhs");
  BCK(launch_sumsq<double>(S.g64[0], cells(G), b->d_partials, &np, b->stream), "batch set_rhs");
  BCK(launch_finalize(b->d_partials, np, sc, kSlotGsum, -1, 0, b->stream), "batch set_rhs");
  BCK(launch_set_scale(sc, kSlotGsum, kSlotScale, (double)cells(G), b->stream), "batch set_rhs");
  b->launches += 4;
  return MG_OK;
}

mg_status mg_batch_set_rhs_all(mg_batch* b, const double* const* h_rho) {
  if (!b) return MG_ERR_INVALID;
  if (!h_rho) return bfail(b, MG_ERR_INVALID, "null array of right-hand sides");
  for (int s = 0; s < b->B; ++s)
    if (!h_rho[s]) return bfail(b, MG_ERR_INVALID, "null right-hand side in the array");
  const int k = b->rhs_slot;
  b->rhs_slot ^= 1;
  BCK(cudaEventSynchronize(b->rhs_ev[k]), "batch set_rhs_all");  // the slot's previous copy has run
  RhsJob* J = b->h_rhs + (size_t)k * b->B;
  long long nb = 0;
  int sb = 0;
  for (int s = 0; s < b->B; ++s) {
    BSys& S = b->sys[s];
    const Geom& G = S.geo[0];
    rhs_job_static(J[s], G, S.g64[0], 1.0 / S.p.eps, S.p.h, S.bc, b->d_scal + (size_t)kScalStride * s);
    J[s].rho = h_rho[s];
    J[s].pair = G.packed && reinterpret_cast<uintptr_t>(h_rho[s]) % 16 == 0;
    J[s].b0 = nb;
    J[s].sb0 = sb;
    const long long items = J[s].pair ? (long long)G.hx * G.ny * G.nz : (long long)G.nx * G.ny * G.nz;
    nb += (items + 255) / 256;
    sb += J[s].sbn;
  }
  BCK(cudaMemcpyAsync(b->d_rhs, J, (size_t)b->B * sizeof(RhsJob), cudaMemcpyHostToDevice, b->stream),
      "batch set_rhs_all");
  BCK(cudaEventRecord(b->rhs_ev[k], b->stream), "batch set_rhs_all");
  BCK(launch_set_rhs_all(b->d_rhs, b->B, nb, sb, b->d_rhs_partials, kSlotGsum, kSlotScale, b->stream),
      "batch set_rhs_all");
  b->launches += 3;
  return MG_OK;
}

mg_status mg_batch_set_solution(mg_batch* b, int s, const double* d_phi) {
  mg_status st = check_sys(b, s);
  if (st != MG_OK) return st;
  b->h_zero[s] = (d_phi == nullptr) ? 1 : 0;
  if (bmixed(b) && !d_phi) {  // nothing is written: the first cycle's update stores phi = s e
    b->lazy[s] = 1;
    return upload_zero(b);
  }
  BCK(launch_pack<double>(b->sys[s].x64[0], b->sys[s].geo[0], d_phi, 1.0, b->stream), "batch set_solution");
  b->launches += 1;
  b->lazy[s] = 0;
  return upload_zero(b);
}

mg_status mg_batch_get_solution(mg_batch* b, int s, double* d_phi) {
  mg_status st = check_sys(b, s);
  if (st != MG_OK) return st;
  if (!d_phi) return bfail(b, MG_ERR_INVALID, "null output");
  if ((st = materialize(b, s)) != MG_OK) return st;
  BCK(launch_unpack<double>(d_phi, b->sys[s].x64[0], b->sys[s].geo[0], 1.0, b->stream), "batch get_solution");
  b->launches += 1;
  return MG_OK;
}

mg_status mg_batch_vcycle(mg_batch* b, int ncycles) {
  if (!b) return MG_ERR_INVALID;
  if (ncycles < 0) return bfail(b, MG_ERR_INVALID, "ncycles must be >= 0");
  mg_status st = bgraphs(b);
  if (st == MG_OK) st = set_all_active(b, 1);
  for (int k = 0; k < ncycles && st == MG_OK; ++k) {
    if (bmixed(b)) st = brun(b, b->g_resid, b->n_resid, "batch residual");
    if (st == MG_OK) st = brun(b, b->g_cycle, b->n_cycle, "batch cycle");
    if (st == MG_OK) st = clear_zero_of_active(b);
  }
  return st;
}

mg_status mg_batch_solve(mg_batch* b, double tol, int max_cycles, int* h_cycles, double* h_rel) {
  if (!b) return MG_ERR_INVALID;
  if (!(tol >= 0.0) || max_cycles < 0) return bfail(b, MG_ERR_INVALID, "need tol >= 0 and max_cycles >= 0");
  mg_status st = bgraphs(b);
  if (st != MG_OK) return st;
  const int B = b->B;
  // per system, as mg_solve: a cycle from a never-written zero iterate, or after another such
  // cycle, carries the residual by recurrence unless the last contraction predicts that it reaches
  // the tolerance; its estimate is replaced by the direct residual before it ends the solve
  std::vector<int> cyc(B, 0), conv(B, 0), run(B, 1), est(B, 0);
  std::vector<double> rel(B, 0.0), relp(B, -1.0);
  auto finish = [&](mg_status out) {
    for (int s = 0; s < B; ++s) b->h_rec[s] = 0;  // the recurrence flags stay zero outside a solve
    mg_status u = upload_flags(b, b->d_rec, b->h_rec);
    if (u == MG_OK) u = set_all_active(b, 1);
    return out != MG_OK ? out : u;
  };
  auto read_scal = [&](const char* what) -> mg_status {
    BCK(cudaMemcpyAsync(b->h_scal, b->d_scal, (size_t)B * kScalStride * sizeof(double), cudaMemcpyDeviceToHost,
                        b->stream),
        what);
    BCK(cudaMemcpyAsync(b->h_err, b->d_err, sizeof(int), cudaMemcpyDeviceToHost, b->stream), what);
    BCK(cudaStreamSynchronize(b->stream), what);
    if (*b->h_err) {  // a staged sweep's bounded wait ran out: the iterates are incomplete
      cudaMemsetAsync(b->d_err, 0, sizeof(int), b->stream);
      return bfail(b, MG_ERR_TIMEOUT, "a kernel's bounded wait for its staged copies ran out; the result is incomplete");
    }
    return MG_OK;
  };
  for (;;) {
    // direct residuals of the running systems whose value is not an estimate, or whose estimate
    // would end their solve
    bool anyd = false;
    for (int s = 0; s < B; ++s) {
      b->h_active[s] = run[s] && (!est[s] || !(rel[s] >= tol) || !std::isfinite(rel[s]) || cyc[s] >= max_cycles);
      anyd = anyd || b->h_active[s];
    }
    if (anyd) {
      if ((st = upload_flags(b, b->d_active, b->h_active)) != MG_OK) return finish(st);
      if ((st = brun(b, b->g_resid, b->n_resid, "batch residual")) != MG_OK) return finish(st);
      if ((st = read_scal("batch residual")) != MG_OK) return finish(st);
      for (int s = 0; s < B; ++s)
        if (b->h_active[s]) {
          rel[s] = b->h_scal[(size_t)kScalStride * s + kSlotRel];
          est[s] = 0;
        }
    }
    bool any = false;
    for (int s = 0; s < B; ++s) {
      if (!run[s]) continue;
      if (!std::isfinite(rel[s])) {
        run[s] = 0;
      } else if (!(rel[s] >= tol)) {
        run[s] = 0;
        conv[s] = 1;
      } else if (cyc[s] >= max_cycles) {
        run[s] = 0;
      } else {
        any = true;
      }
    }
    if (!any) break;
    bool anyrec = false;
    for (int s = 0; s < B; ++s) {
      b->h_active[s] = run[s];
      b->h_rec[s] = run[s] && b->sys[s].q_lo && (b->lazy[s] || est[s]) &&
                    !(relp[s] > 0.0 && rel[s] * (rel[s] / relp[s]) < tol);
      if (run[s]) relp[s] = rel[s];
      anyrec = anyrec || b->h_rec[s];
    }
    if ((st = upload_flags(b, b->d_active, b->h_active)) != MG_OK) return finish(st);
    if ((st = upload_flags(b, b->d_rec, b->h_rec)) != MG_OK) return finish(st);
    if ((st = brun(b, b->g_cycle, b->n_cycle, "batch cycle")) != MG_OK) return finish(st);
    if ((st = clear_zero_of_active(b)) != MG_OK) return finish(st);
    for (int s = 0; s < B; ++s) {
      cyc[s] += b->h_active[s];
      if (b->h_active[s] && !b->h_rec[s]) est[s] = 0;
    }
    if (anyrec) {  // the estimates of the systems that stepped by recurrence
      if ((st = read_scal("batch cycle")) != MG_OK) return finish(st);
      for (int s = 0; s < B; ++s)
        if (b->h_rec[s]) {
          rel[s] = b->h_scal[(size_t)kScalStride * s + kSlotRel];
          est[s] = 1;
        }
    }
  }
  bool all = true;
  for (int s = 0; s < B; ++s) {
    if (h_cycles) h_cycles[s] = cyc[s];
    if (h_rel) h_rel[s] = rel[s];
    if (!conv[s]) all = false;
  }
  if ((st = finish(MG_OK)) != MG_OK) return st;
  if (!all) return bfail(b, MG_ERR_NOT_CONVERGED, "some systems did not reach the tolerance");
  return MG_OK;
}

mg_status mg_batch_set_tiles(mg_batch* b, const int* h_tiles4) {
  if (!b) return MG_ERR_INVALID;
  if (!h_tiles4) return bfail(b, MG_ERR_INVALID, "null tiles");
  for (int q = 0; q < 2; ++q) {
    const int bx = h_tiles4[2 * q], by = h_tiles4[2 * q + 1];
    if (bx < 1 || by < 1 || bx * by > 256 || (bx * by) % 32 != 0)
      return bfail(b, MG_ERR_INVALID, "tile bx*by must be a multiple of 32 and at most 256");
  }
  for (int q = 0; q < 4; ++q) b->tile[q] = h_tiles4[q];
  return plan(b);
}

mg_status mg_batch_get_tiles(const mg_batch* b, int* h_tiles4) {
  if (!b || !h_tiles4) return MG_ERR_INVALID;
  for (int q = 0; q < 4; ++q) h_tiles4[q] = b->tile[q];
  return MG_OK;
}

mg_status mg_batch_autotune(mg_batch* b, int reps, int* h_best4, double* h_ms, int* h_ncand) {
  if (!b) return MG_ERR_INVALID;
  if (reps < 1) reps = 1;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  BCK(cudaEventCreate(&e0), "autotune");
  BCK(cudaEventCreate(&e1), "autotune");
  double best = 1e300;
  int bi = 0;
  mg_status st = MG_OK;
  for (int c = 0; c < kNumCandidates && st == MG_OK; ++c) {
    st = mg_batch_set_tiles(b, kCandidates[c]);
    if (st == MG_OK) st = bgraphs(b);
    if (st == MG_OK) st = set_all_active(b, 1);
    if (st == MG_OK) st = brun(b, b->g_cycle, b->n_cycle, "autotune");
    if (st != MG_OK) break;
    cudaEventRecord(e0, b->stream);
    for (int r = 0; r < reps && st == MG_OK; ++r) st = brun(b, b->g_cycle, b->n_cycle, "autotune");
    cudaEventRecord(e1, b->stream);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    const double per = ms / reps;
    if (h_ms) h_ms[c] = per;
    if (per < best) {
      best = per;
      bi = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != MG_OK) return st;
  if (h_ncand) *h_ncand = kNumCandidates;
  if (h_best4)
    for (int q = 0; q < 4; ++q) h_best4[q] = kCandidates[bi][q];
  // the timed cycles may have changed the iterates: no longer known to be zero
  for (int s = 0; s < b->B; ++s) {
    b->h_zero[s] = 0;
    b->lazy[s] = 0;
  }
  if ((st = upload_zero(b)) != MG_OK) return st;
  return mg_batch_set_tiles(b, kCandidates[bi]);
}

long long mg_batch_kernel_launches(const mg_batch* b) { return b ? b->launches : 0; }

}  // extern "C"
