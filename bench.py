"""Benchmark of the electrostatics step (charged spheres -> multigrid Poisson solve -> E-field ->
Coulomb forces) on one or more GB300s; prints ONE JSON line on rank 0.

A step is one pass of the hot path over the workload: subsampled sphere charge density, RHS with
wall terms, solve from zero to the relative-residual tolerance (FP32 V(2,2)-cycles inside FP64
defect correction for the default 512^3 workload), the E-field, and the force on every sphere.
value = fine-grid cells solved per second (MLUP/s, the paper's metric, Sec. 8.1), whole job.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload spheres512|spheres256|...]
  python bench.py --impl reference ...   # the CPU oracle on the same workload (bounded sample)

Several GPUs run independent replicas of the workload (one process per GPU, no collective on
the data path); the timing is the maximum over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1410_6609_gb300 import synth  # noqa: E402

METRIC = "V-cycle MLUP/s & time-to-1e-9 residual vs FP64 GPU; % HBM roofline"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="spheres512", choices=sorted(synth.WORKLOADS))
    ap.add_argument("--precision", choices=["fp64", "mixed"], default=None,
                    help="override the workload's precision (profiling runs)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the FP64 comparison and kernel timings")
    return ap.parse_args()


def workload_config(w, rank_seed_offset=0):
    if w.sphere_count:
        source = (f"{w.sphere_count} spheres R={w.sphere_radius:g} (N(0,1) charge, zero sum, subsampling "
                  f"{w.subsample}), phi=0/1 on z walls, Neumann 0 on x/y")
    else:
        source = "f = 3 pi^2 sin(pi x) sin(pi y) sin(pi z) on the unit cube, homogeneous Dirichlet walls"
    return {
        "workload": f"{w.name}: {w.dims[0]}x{w.dims[1]}x{w.dims[2]} cells, {source}, "
                    f"{'FP32 V(2,2) inside FP64 defect correction' if w.precision == 'mixed' else 'FP64 V(2,2)'} "
                    f"to {w.tol:g} relative residual from zero, then E-field{' and forces' if w.sphere_count else ''}",
        "grid": list(w.dims),
        "spheres": w.sphere_count,
        "tol": w.tol,
        "precision": w.precision,
        "cycle": "V(2,2), x2 coarse-grid correction, CG coarsest",
        "l2": "inputs larger than L2 (each fine-grid field >= 134 MB for 256^3 and up)",
        "seed": w.seed + rank_seed_offset,
    }


# ------------------------------------------------------------------------------------------
# Clock sampling during the timed region

CLOCK_FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
CLOCK_REASONS = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")


class ClockSampler:
    """nvidia-smi sampling every 50 ms, started before the warm-up; summary() keeps the samples
    whose timestamps fall inside the marked timed region (the nearest ones if it was shorter than
    the sampling period)."""

    def __init__(self, gpu_index: int):
        self.proc = None
        self.gpu_index = gpu_index
        self.window = None
        # the raw samples (CCMG_CLOCKS_DIR, else the temporary directory); the JSON line carries the summary
        d = os.environ.get("CCMG_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(d, f"clocks_bench_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu_index), f"--query-gpu={CLOCK_FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
            return self
        t_end = time.time() + 5.0  # the first sample, so that the timed region is covered
        while time.time() < t_end and self.proc.poll() is None:
            self.f.flush()
            if os.path.getsize(self.path) > 0:
                break
            time.sleep(0.02)
        return self

    def mark(self, t0: float, t1: float):
        self.window = (t0, t1)

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def _rows(self):
        import datetime
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 10:
                    continue
                try:
                    ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                    rows.append((ts, float(parts[2]), float(parts[3]), parts[6:10]))
                except ValueError:
                    continue
        return rows

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = self._rows()
        if self.window is not None and rows:
            t0, t1 = self.window
            inside = [r for r in rows if t0 <= r[0] <= t1]
            if not inside:  # region shorter than the period: the samples nearest to it
                mid = 0.5 * (t0 + t1)
                inside = sorted(rows, key=lambda r: abs(r[0] - mid))[:2]
            rows = inside
        reasons = {nm for r in rows for nm, v in zip(CLOCK_REASONS, r[3]) if v.lower().startswith("active")}
        out = {"sm_mhz": statistics.median(r[1] for r in rows) if rows else None,
               "sm_max_mhz": max(r[2] for r in rows) if rows else None,
               "reasons": sorted(reasons), "samples": len(rows), "period_ms": 50}
        if self.window is not None:
            out["window_ms"] = round(1e3 * (self.window[1] - self.window[0]), 1)
        return out


# ------------------------------------------------------------------------------------------
# CPU oracle timings (whole steps on the host cores)

def host_threads() -> int:
    return os.cpu_count() or 1


def oracle_step(w, sp, threads: int):
    """One whole step of the oracle on workload w, the same work as one GPU step: subsampled
    sphere density, right-hand side with the wall terms, solve from zero to the workload's
    tolerance in its precision (FP32 V(2,2)-cycles inside FP64 defect correction for 'mixed'),
    E-field and forces. Returns (seconds, details, phi, f)."""
    import oracle
    used = oracle.set_threads(threads)
    nx, ny, nz = w.dims
    t0 = time.perf_counter()
    if w.sphere_count:
        rho = oracle.sphere_density((nz, ny, nx), w.h, sp.centers, sp.radius, sp.density, w.subsample, w.bc_type)
        f = oracle.rhs(rho, w.h, w.bc_type, w.bc_value)
    else:  # the manufactured solution: the analytic right-hand side, homogeneous walls
        f = synth.manufactured_rhs(nx)[0]
    t1 = time.perf_counter()
    solve = oracle.solve_mixed if w.precision == "mixed" else oracle.solve
    phi, k, rel = solve(f, w.h, w.bc_type, tol=w.tol, max_cycles=100)
    t2 = time.perf_counter()
    oracle.efield(phi, w.h, w.bc_type, w.bc_value)
    if w.sphere_count:
        oracle.force_gather(phi, w.h, w.bc_type, w.bc_value, sp.centers, sp.radius, sp.density, w.subsample)
    t3 = time.perf_counter()
    info = {"threads": used, "density_rhs_s": round(t1 - t0, 3), "solve_s": round(t2 - t1, 3),
            "efield_forces_s": round(t3 - t2, 3), "cycles": k, "rel_residual": rel}
    return t3 - t0, info, phi, f


def oracle_adjoint_step(w, sp, threads: int):
    """The adjoint workload on the oracle: J = sum of z-forces and its gradient with respect to
    the sphere densities and the wall values (forward solve, force adjoint, one adjoint solve)."""
    import oracle
    used = oracle.set_threads(threads)
    nx, ny, nz = w.dims
    wF = np.zeros((sp.count, 3))
    wF[:, 2] = 1.0
    t0 = time.perf_counter()
    J, gq, gv, info = oracle.force_objective_and_grad((nz, ny, nx), w.h, w.bc_type, w.bc_value, sp.centers,
                                                      sp.radius, sp.density, wF, w.subsample, tol=w.tol)
    return time.perf_counter() - t0, {"threads": used, "cycles": list(info["cycles"]), "dJ_dV_top": float(gv[5])}


def oracle_baseline(w, sp, steps: int = 2):
    """cpu_baseline of the GPU arm: whole oracle steps of the bench workload on all host cores
    (a bounded sample of `steps` steps), the last step's potential and right-hand side kept for
    comparing the GPU solution with."""
    threads = host_threads()
    times, info, phi, f = [], None, None, None
    for _ in range(steps):
        t, info, phi, f = oracle_step(w, sp, threads)
        times.append(t)
    t_step = statistics.mean(times)
    N = int(np.prod(w.dims))
    nx, ny, nz = w.dims
    cb = {"value": N / t_step / 1e6, "unit": "MLUP/s", "cores": info["threads"], "kind": "oracle",
          "sample": (f"{steps} whole oracle steps (plain C, OpenMP over z-planes, {info['threads']} threads) on the "
                     f"full {nx}x{ny}x{nz} workload: density+RHS, {w.precision} solve from zero to {w.tol:g} "
                     f"({info['cycles']} {'outer steps' if w.precision == 'mixed' else 'cycles'}), E-field, forces; "
                     f"{t_step:.2f} s per step"),
          "ms_per_step": t_step * 1e3, "last_step": info}
    return cb, phi, f


# ------------------------------------------------------------------------------------------
# ------------------------------------------------------------------------------------------

def max_over_ranks(x: float, world: int, device: str = "cpu") -> float:
    """Maximum of a per-rank scalar over all ranks (the step time every replica waits for)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_mlups(cells_per_rank: int, world: int, ms: float) -> float:
    """MLUP/s of the whole job: every replica solves cells_per_rank cells in ms milliseconds."""
    return world * cells_per_rank / (ms / 1e3) / 1e6


def parallelism(world: int) -> str:
    return "single" if world <= 1 else f"replicas{world}"


def run_reference(args):
    """The oracle on the host cores: the same workload, metric and config as the GPU arm, each
    step one whole oracle step (density, RHS, solve to the tolerance, E-field, forces) on all host
    threads; warm-up steps run the same work untimed. Rank 0 only."""
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if rank != 0:
        return
    w = workload(args)
    sp = w.spheres()
    threads = host_threads()
    for _ in range(args.warmup):
        oracle_step(w, sp, threads)
    times = []
    t_all = time.perf_counter()
    for _ in range(args.steps):
        t, info, _, _ = oracle_step(w, sp, threads)
        times.append(t)
    wall = time.perf_counter() - t_all
    t_step = statistics.mean(times)
    N = int(np.prod(w.dims))
    value = N / t_step / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "MLUP/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_step * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if w.precision == "fp64" else "f64+f32",
        "data": "synthetic", "config": {**workload_config(w), "parallelism": parallelism(world)},
        "cycles_per_step": info["cycles"], "final_rel_residual": info["rel_residual"],
        "cpu_baseline": {"value": value, "unit": "MLUP/s", "cores": info["threads"], "kind": "oracle",
                         "sample": (f"{args.steps} whole oracle steps (after {args.warmup} untimed) on all "
                                    f"{info['threads']} host threads in {wall:.1f} s; last step {info}")},
        "e2e": {"value": value, "unit": "MLUP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    if not args.no_extras:
        line["oracle_extras"] = reference_extras(w, sp, threads)
    print(json.dumps(line), flush=True)


def reference_extras(w, sp, threads):
    """The oracle on the other configurations of the method (manufactured 32^3, 256^3 FP64, the
    adjoint at 256^3) at all host threads, and the headline workload and the 256^3 one at one
    thread: one whole step each."""
    out = {"host_threads": threads}
    for name in ("manufactured32", "spheres256"):
        wx = synth.WORKLOADS[name]
        spx = wx.spheres() if wx.sphere_count else None
        t, info, phi, _ = oracle_step(wx, spx, threads)
        d = {"ms_per_step": t * 1e3, "mlups": int(np.prod(wx.dims)) / t / 1e6, **info}
        if name == "manufactured32":
            ex = synth.manufactured_exact(wx.dims[0])
            d["rel_error_vs_exact"] = float(np.linalg.norm(phi - ex) / np.linalg.norm(ex))
        out[name] = d
        t1, info1, _, _ = oracle_step(wx, spx, 1)
        out[name]["one_thread"] = {"ms_per_step": t1 * 1e3, "mlups": int(np.prod(wx.dims)) / t1 / 1e6}
    wa = synth.WORKLOADS["adjoint256"]
    t, info = oracle_adjoint_step(wa, wa.spheres(), threads)
    out["adjoint256"] = {"ms_forward_and_gradient": t * 1e3, **info}
    t1, info1, _, _ = oracle_step(w, sp, 1)
    out[w.name + "_one_thread"] = {"ms_per_step": t1 * 1e3, "mlups": int(np.prod(w.dims)) / t1 / 1e6, **info1}
    return out


def workload(args):
    w = synth.WORKLOADS[args.workload]
    if args.precision and args.precision != w.precision:
        import dataclasses
        w = dataclasses.replace(w, precision=args.precision, name=f"{w.name}-{args.precision}")
    return w


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_1410_6609_gb300.solver import Poisson

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    w = workload(args)
    nx, ny, nz = w.dims
    N = nx * ny * nz
    sp = synth.random_spheres(w.dims, w.sphere_count, w.sphere_radius, w.seed + 100 * rank, w.h)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    c, r, q = dev(sp.centers), dev(sp.radius), dev(sp.density)
    P = Poisson(w.dims, h=w.h, bc_type=w.bc_type, bc_value=w.bc_value, precision=w.precision)
    rho = P.new_field()
    E = P.new_field(3)
    F = torch.empty(sp.count, 3, dtype=torch.float64, device="cuda")
    stream = P.stream
    cycles_seen = []

    def step():
        P.sphere_density(c, r, q, w.subsample, out=rho)
        P.set_rhs(rho)
        P.set_solution(None)
        k, rel = P.solve(w.tol, 100)
        P.efield(out=E)
        P.force_gather(c, r, q, w.subsample, out=F)
        cycles_seen.append((k, rel))

    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        cycles_seen.clear()
        launches0 = P.kernel_launches
        counts0 = P.outer_counts()
        barrier()
        torch.cuda.synchronize()
        t_wall0 = time.time()
        ev0.record(stream)
        for _ in range(args.steps):
            step()
        ev1.record(stream)
        torch.cuda.synchronize()
        clk.mark(t_wall0, time.time())
        barrier()
    ms = ev0.elapsed_time(ev1) / args.steps
    launches = (P.kernel_launches - launches0) // args.steps
    counts = [(b - a) / args.steps for a, b in zip(counts0, P.outer_counts())]
    outer = {"cycles": counts[0], "by_recurrence": counts[1], "direct_residuals": counts[2]}
    ms_all = max_over_ranks(ms, world, "cuda")
    value = whole_job_mlups(N, world, ms_all)
    k_step = cycles_seen[-1][0]
    rel_final = max(v for _, v in cycles_seen)
    want_cpu = rank == 0 and world == 1 and not args.no_cpu_baseline
    phi_gpu = P.solution().cpu().numpy() if want_cpu else None  # the last timed step's potential

    extras = {}
    if not args.no_extras:
        extras = measure_extras(P, w, sp, c, r, q, rho, stream, k_step, outer)

    # e2e: the public host-buffer call (spheres in, forces out) plus the E-field, timed by wall clock
    P.set_solution(None)
    P.step_host(sp.centers, sp.radius, sp.density, w.subsample, w.tol, 100)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        P.set_solution(None)
        Fh, k_e2e, _ = P.step_host(sp.centers, sp.radius, sp.density, w.subsample, w.tol, 100)
        P.efield(out=E)
        torch.cuda.synchronize()
    t_e2e = (time.perf_counter() - t0) / args.steps
    e2e = {"value": world * N / t_e2e / 1e6, "unit": "MLUP/s", "ms_per_step": t_e2e * 1e3,
           "h2d_bytes_per_step": int(sp.centers.nbytes + sp.radius.nbytes + sp.density.nbytes),
           "d2h_bytes_per_step": int(Fh.nbytes)}

    cpu = vs_oracle = None
    if want_cpu:
        import oracle
        cpu, phi_or, f_or = oracle_baseline(w, sp)
        # the GPU step's potential against the oracle: the oracle's own FP64 residual of it, and
        # its distance from the oracle's solution of the same step
        vs_oracle = {"oracle_rel_residual_of_gpu_solution": oracle.rel_residual(phi_gpu, f_or, w.h, w.bc_type),
                     "rel_error_vs_oracle_solution": float(np.linalg.norm(phi_gpu - phi_or) / np.linalg.norm(phi_or)),
                     "oracle_precision": w.precision, "tol": w.tol}
        del phi_or, f_or, phi_gpu

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "MLUP/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_all, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if w.precision == "fp64" else "f64+f32", "data": "synthetic",
            "config": {**workload_config(w), "parallelism": parallelism(world)},
            "cycles_per_step": k_step, "final_rel_residual": rel_final, "outer_steps_per_step": outer,
            "gpu_launches": int(launches),
            "e2e": e2e,
            "clocks": clk.summary(),
            **extras,
        }
        if cpu is not None:
            line["cpu_baseline"] = cpu
            line["vs_oracle"] = vs_oracle
        print(json.dumps(line), flush=True)
    P.close()
    if world > 1:
        dist.destroy_process_group()


def _time(fn, stream, reps):
    import torch
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    fn()
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(reps):
        fn()
    ev1.record(stream)
    torch.cuda.synchronize()
    return ev0.elapsed_time(ev1) / reps


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0}, "fallback"


# FP64 issue peak: 1.25 TFLOP/s nominal FP64 with an FMA counted as two FLOPs, i.e. 625 G FP64
# instruction lanes per second at 2070 MHz (152 SMs x ~2 lanes/clk); every DADD/DMUL/DFMA lane is one op.
FP64_OPS_PEAK = 0.625  # Tops/s

# DRAM bytes (read + write) per launch of a kernel, from one ncu capture of that kernel on the
# same workload (profiles/); None where no capture of the current kernel exists.
MEASURED_TRAFFIC = {
    # ncu dram__bytes_read.sum + dram__bytes_write.sum of one finest-level FP32 half-sweep of the
    # 512^3 mixed step (one-pass capture of that kernel alone, TMA kernel as of commit d5485bd):
    # 545.2 MB read + 234.7 MB written, mean of two launches; the algorithmic figure is 805.3 MB
    # (the rest of the writes are still in L2 when the launch ends)
    ("spheres512", "k_smooth_tma"): 779_890_000,
}


def measure_extras(P, w, sp, c, r, q, rho, stream, k_step, outer):
    """Kernel-level timings for the roofline, the FP64 GPU solve at the same tolerance, and the
    error of the mixed solution against it."""
    import torch

    from paper_1410_6609_gb300.solver import Poisson

    peaks, src = load_peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    nx, ny, nz = w.dims
    N = nx * ny * nz
    out = {}
    kern = {}
    phi_m = P.solution().clone()  # the step's solution, before the kernel timings below reuse the state
    # outer FP64 residual (+ single-precision scaled residual in mixed mode)
    t_res = _time(P.op_residual_norm, stream, 10)
    mixed = w.precision == "mixed"
    bytes_res = N * (8 + 8 + (4 if mixed else 0))
    kern["residual_fp64"] = {"ms": t_res, "GB/s": bytes_res / t_res / 1e6,
                             "launches_per_step": outer["direct_residuals"], "bytes_per_launch": int(bytes_res),
                             "bound": "integer ALU (64-bit fixed-point sum per cell)",
                             "note": "plus one stencil-free residual of the zero start per step"}
    if outer["by_recurrence"] > 0:
        # the outer step that carries the residual by recurrence (phi += s e, residual pair - A e)
        t_def = _time(P.op_defect_step, stream, 10)
        bytes_def = N * 36
        kern["defect_update"] = {"ms": t_def, "GB/s": bytes_def / t_def / 1e6,
                                 "launches_per_step": outer["by_recurrence"], "bytes_per_launch": bytes_def,
                                 "device_kernel": "k_defect_rec",
                                 "note": "reads e (4 B), phi (8), the residual pair (8), writes phi and the pair; "
                                         "the first step from zero reads g (8 B) and no phi: 28 B per cell"}
    # smoother half-sweep and fused residual+restriction on the finest level
    esz = 4 if mixed else 8
    inner = P.mixed_inner if mixed else 1  # finest-level V-cycles per outer step
    t_sm = _time(lambda: P.op_smooth(0, 0), stream, 20)
    sweep_kernel = ("k_smooth_tma" if P.level_sweep_kind(0) == "tma" else
                    ("k_smooth_vec<float,4,0>" if mixed else "k_smooth_vec<double,2,0>"))
    kern["smooth_half_sweep"] = {"ms": t_sm, "GB/s": 1.5 * N * esz / t_sm / 1e6, "Tops/s": 0.5 * N * 7 / t_sm / 1e9,
                                 "launches_per_step": 8 * k_step * inner, "precision": "f32" if mixed else "f64",
                                 "bytes_per_launch": int(1.5 * N * esz), "device_kernel": sweep_kernel,
                                 "note": "the first post-smoothing black sweep runs fused with the prolongation"
                                 if mixed else ""}
    # the restriction the cycle runs: red children only in single precision (after a black sweep)
    t_rr = _time(lambda: P.op_residual_restrict(0, red_only=mixed), stream, 20)
    rr_bytes = (1.5 * N * esz + N * esz / 8) if mixed else (2 * N * esz + N * esz / 8)
    kern["resid_restrict"] = {"ms": t_rr, "GB/s": rr_bytes / t_rr / 1e6,
                              "Tops/s": N * (4 if mixed else 8) / t_rr / 1e9, "launches_per_step": k_step * inner,
                              "precision": "f32" if mixed else "f64", "red_only": mixed,
                              "bytes_per_launch": int(rr_bytes)}
    # the state changed: restore a consistent solve state for later use
    for name, d in kern.items():
        d["share_ms_per_step"] = d["ms"] * d["launches_per_step"]
    dom = max(kern, key=lambda n: kern[n]["share_ms_per_step"])
    d = kern[dom]
    alu = not mixed and "Tops/s" in d  # the FP64 smoother and restriction are bound by the FP64 pipe
    traffic = MEASURED_TRAFFIC.get((w.name, d.get("device_kernel", dom)))
    if alu:
        out["roofline"] = {"bound": "alu", "kernel": dom, "achieved": d["Tops/s"], "peak": FP64_OPS_PEAK,
                           "unit": "Tops/s (FP64 lane-ops)", "frac": d["Tops/s"] / FP64_OPS_PEAK,
                           "traffic": traffic, "peak_source": "nominal FP64 1.25 TFLOP/s (FMA=2) at 2070 MHz",
                           "hbm_frac": d["GB/s"] / hbm}
    else:
        out["roofline"] = {"bound": "hbm", "kernel": dom, "achieved": d["GB/s"], "peak": hbm, "unit": "GB/s",
                           "frac": d["GB/s"] / hbm, "traffic": traffic, "peak_source": src,
                           "algorithmic_bytes": d["bytes_per_launch"]}
    out["kernels"] = kern

    # FP64 GPU solve of the same problem to the same tolerance, and the error between them
    P64 = Poisson(w.dims, h=w.h, bc_type=w.bc_type, bc_value=w.bc_value, precision="fp64")
    P64.set_rhs(rho)

    def solve64():
        P64.set_solution(None)
        return P64.solve(w.tol, 100)

    k64, rel64 = solve64()
    t64 = _time(lambda: solve64(), P64.stream, 2)
    phi64 = P64.solution()
    # the FP64-mode kernels of the same level: bytes against the measured HBM rate, FP64-pipe
    # operations against the FP64 issue peak (3 per cell in the half-sweep: int->double of the exact
    # fixed-point neighbour sum, + g, x 1/D; 2 per fine cell in the residual + restriction by the
    # fixed-point walk: int->double of the residual, the children's sum)
    sweep64 = "k_smooth_tma64" if P64.level_sweep_kind(0) == "tma" else "k_smooth_vec<double,2,0>"
    t64_sm = _time(lambda: P64.op_smooth(0, 0), P64.stream, 10)
    t64_rr = _time(lambda: P64.op_residual_restrict(0), P64.stream, 10)
    b64_sm, b64_rr = 0.5 * N * 24, N * 17.0
    out["kernels_fp64"] = {
        "smooth_half_sweep": {"ms": t64_sm, "GB/s": b64_sm / t64_sm / 1e6, "hbm_frac": b64_sm / t64_sm / 1e6 / hbm,
                              "bytes_per_launch": int(b64_sm), "fp64_ops_per_cell": 3,
                              "fp64_frac": 0.5 * N * 3 / t64_sm / 1e9 / FP64_OPS_PEAK, "device_kernel": sweep64,
                              "bound": "integer ALU + FP64 pipe (fixed-point neighbour sum)"},
        "resid_restrict": {"ms": t64_rr, "GB/s": b64_rr / t64_rr / 1e6, "hbm_frac": b64_rr / t64_rr / 1e6 / hbm,
                           "bytes_per_launch": int(b64_rr), "fp64_ops_per_cell": 2,
                           "fp64_frac": N * 2 / t64_rr / 1e9 / FP64_OPS_PEAK, "device_kernel": "k_resid_restrict_walk",
                           "bound": "integer ALU (64-bit fixed-point residual per cell)"},
    }
    err = float(torch.linalg.norm(phi_m - phi64) / torch.linalg.norm(phi64))

    def solve_m():
        P.set_solution(None)
        return P.solve(w.tol, 100)

    km, relm = solve_m()
    tm = _time(lambda: solve_m(), stream, 2)
    tv64 = _time(lambda: P64.vcycle(1), P64.stream, 3)
    tvm = _time(lambda: P.vcycle(1), stream, 3)
    out["time_to_tol"] = {
        "tol": w.tol,
        "mixed": {"ms": tm, "cycles": km, "rel_residual": relm, "solve_mlups": N / tm / 1e3},
        "fp64": {"ms": t64, "cycles": k64, "rel_residual": rel64, "solve_mlups": N / t64 / 1e3},
        "speedup_mixed_vs_fp64": t64 / tm,
        "rel_error_mixed_vs_fp64": err,
    }
    out["vcycle_mlups"] = {"mixed_outer_cycle": N / tvm / 1e3, "fp64_vcycle": N / tv64 / 1e3,
                           "mixed_outer_cycle_ms": tvm, "fp64_vcycle_ms": tv64}
    P64.close()
    try:
        out["time_loop"] = measure_time_loop(P, w, sp, r, q, stream)
    except Exception as e:
        out["time_loop"] = {"error": repr(e)}
    try:  # the same loop with one FP32 V(2,2) per outer step: one cycle per time step, as in Sec. 8.1
        P1 = Poisson(w.dims, h=w.h, bc_type=w.bc_type, bc_value=w.bc_value, precision="mixed", mixed_inner=1)
        d1 = measure_time_loop(P1, w, sp, r, q, P1.stream)
        d1["fp32_cycles_per_outer_step"] = 1
        out["time_loop_one_fp32_cycle"] = d1
        P1.close()
    except Exception as e:
        out["time_loop_one_fp32_cycle"] = {"error": repr(e)}
    try:
        out["time_loop_periodic"] = measure_time_loop_periodic(w, sp)
    except Exception as e:
        out["time_loop_periodic"] = {"error": repr(e)}
    try:
        out["permittivity"] = measure_permittivity(w, sp, t64, k64, hbm)
    except Exception as e:
        out["permittivity"] = {"error": repr(e)}
    try:
        out["poisson_boltzmann"] = measure_pb(w, sp)
    except Exception as e:
        out["poisson_boltzmann"] = {"error": repr(e)}
    try:
        out["batched"] = measure_batched()
    except Exception as e:  # reported, never fatal for the main line
        out["batched"] = {"error": repr(e)}
    try:
        out["adjoint"] = measure_adjoint()
    except Exception as e:
        out["adjoint"] = {"error": repr(e)}
    return out


def measure_time_loop(P, w, sp, r, q, stream, steps: int = 20, vel: float = 0.07):
    """The warm-started time loop of Sec. 8.1 at the bench workload: each time step sets the charge
    of the spheres at their new positions, runs one cycle from the previous step's potential (one
    outer step of the defect correction in mixed precision) and gathers the forces."""
    import torch

    nx, ny, nz = w.dims
    cs = []
    for t in range(steps + 1):
        ct = sp.centers.copy()
        ct[:, 0] += vel * (t + 1)
        cs.append(torch.from_numpy(ct).cuda())
    rho = P.new_field()
    F = torch.empty(sp.count, 3, dtype=torch.float64, device="cuda")
    P.sphere_density(cs[0], r, q, w.subsample, out=rho)
    P.set_rhs(rho)
    P.set_solution(None)
    P.vcycle(5)
    it = iter(cs[1:])

    def tstep():
        ct = next(it)
        P.sphere_density(ct, r, q, w.subsample, out=rho)
        P.set_rhs(rho)
        P.vcycle(1)
        P.force_gather(ct, r, q, w.subsample, out=F)

    ms = _time(tstep, stream, steps - 1)
    rel = P.residual()
    N = nx * ny * nz
    return {"ms_per_step": ms, "mlups": N / ms / 1e3, "steps": steps, "cycles_per_step": 1,
            "first_step_cycles": 5, "sphere_velocity_cells_per_step": vel,
            "rel_residual_after_last_step": rel}


def measure_time_loop_periodic(w, sp, steps: int = 20, vel: float = 0.07):
    """The production mode of Sec. 8.1 with periodic side walls: the workload's spheres in a domain
    periodic along x and y (plates on z), V(3,3) cycles, five at the first time step and one per
    later step from the previous potential, the spheres moving along x across the periodic wall;
    each step sets the charge, runs the cycle (one mixed outer step) and gathers the forces."""
    import torch

    from paper_1410_6609_gb300.solver import Poisson

    nx, ny, nz = w.dims
    N = nx * ny * nz
    bc = (2, 2, 2, 2, 0, 0)
    P = Poisson(w.dims, h=w.h, bc_type=bc, bc_value=(0.0, 0.0, 0.0, 0.0, 0.0, 1.0), precision=w.precision,
                nu1=3, nu2=3)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    r, q = dev(sp.radius), dev(sp.density)
    cs = []
    for t in range(steps + 1):
        ct = sp.centers.copy()
        ct[:, 0] = np.mod(ct[:, 0] + vel * (t + 1) * 40.0, nx * w.h)  # far enough to cross the wall
        cs.append(dev(ct))
    rho = P.new_field()
    F = torch.empty(sp.count, 3, dtype=torch.float64, device="cuda")
    P.sphere_density(cs[0], r, q, w.subsample, out=rho)
    P.set_rhs(rho)
    P.set_solution(None)
    P.vcycle(5)
    it = iter(cs[1:])

    def tstep():
        ct = next(it)
        P.sphere_density(ct, r, q, w.subsample, out=rho)
        P.set_rhs(rho)
        P.vcycle(1)
        P.force_gather(ct, r, q, w.subsample, out=F)

    ms = _time(tstep, P.stream, steps - 1)
    rel = P.residual()
    kind = P.level_sweep_kind(0)
    P.close()
    return {"ms_per_step": ms, "mlups": N / ms / 1e3, "steps": steps, "cycle": "V(3,3)", "cycles_per_step": 1,
            "first_step_cycles": 5, "walls": "periodic x, y; Dirichlet 0 / 1 on z",
            "sphere_velocity_cells_per_step": vel * 40.0, "rel_residual_after_last_step": rel,
            "finest_sweep_kernel": kind}


def measure_permittivity(w, sp, t64_const, k64_const, hbm):
    """The same spheres as dielectric particles (permittivity 2 in a fluid of 80, cells weighted
    by their covered volume) with the workload's charges and walls: the FP64 solve of
    -div(eps grad phi) = rho with Galerkin coarse operators to the workload's tolerance, beside
    the constant-permittivity FP64 solve, and the weighted half-sweep's HBM throughput."""
    import torch

    from paper_1410_6609_gb300.solver import Poisson

    nx, ny, nz = w.dims
    N = nx * ny * nz
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    out = {"tol": w.tol, "particle_eps": 2.0, "fluid_eps": 80.0, "constant_eps_fp64_ms": t64_const,
           "constant_eps_fp64_cycles": k64_const}
    for prec in ("fp64", "mixed"):
        P = Poisson(w.dims, h=w.h, bc_type=w.bc_type, bc_value=w.bc_value, precision=prec)
        c, r = dev(sp.centers), dev(sp.radius)
        vol = P.sphere_density(c, r, torch.ones(sp.count, dtype=torch.float64, device="cuda"), w.subsample)
        torch.cuda.synchronize()
        eps = 80.0 - 78.0 * vol
        torch.cuda.synchronize()
        P.set_permittivity(eps)
        rho = P.sphere_density(c, r, dev(sp.density), w.subsample)
        P.set_rhs(rho)

        def solve():
            P.set_solution(None)
            return P.solve(w.tol, 300)

        k, rel = solve()
        t = _time(solve, P.stream, 2)
        d = {"cycles": k, "rel_residual": rel, "ms": t, "solve_mlups": N / t / 1e3}
        if prec == "fp64":
            t_sw = _time(lambda: P.op_smooth(0, 0), P.stream, 10)
            # a half-sweep reads the other colour, its own right-hand side, 1/D and three weights,
            # the other colour's three weights (the + faces), and writes its colour: 80 B per cell
            # of it in FP64, 40 B in single precision
            bsw = 40.0 * N
            d.update({"half_sweep_ms": t_sw, "half_sweep_GB/s": bsw / t_sw / 1e6,
                      "half_sweep_hbm_frac": bsw / t_sw / 1e6 / hbm, "half_sweep_bytes": int(bsw),
                      "half_sweep_bound": "FP64 pipe (profiles/k_var_smooth_fp64_spheres256.md)"})
        else:
            t_sw = _time(lambda: P.op_smooth(0, 0), P.stream, 10)
            bsw = 20.0 * N
            # the fused residual and restriction reads both colours' potentials, right-hand
            # sides, D and three weights (24 B per fine cell) and writes the coarse right-hand side
            t_rr = _time(lambda: P.op_residual_restrict(0), P.stream, 10)
            brr = 24.5 * N
            d.update({"half_sweep_ms": t_sw, "half_sweep_GB/s": bsw / t_sw / 1e6,
                      "half_sweep_hbm_frac": bsw / t_sw / 1e6 / hbm, "half_sweep_bytes": int(bsw),
                      "resid_restrict_ms": t_rr, "resid_restrict_GB/s": brr / t_rr / 1e6,
                      "resid_restrict_hbm_frac": brr / t_rr / 1e6 / hbm})
        out[prec] = d
        P.close()
    out["speedup_mixed_vs_fp64"] = out["fp64"]["ms"] / out["mixed"]["ms"]
    return out


def measure_pb(w, sp, debye: float = 4.0, charge: float = 4.0):
    """Charged dielectric spheres (permittivity 2, no ions inside) in a 1:1 electrolyte
    (permittivity 80, Debye length `debye` cells) at the workload's size and walls: Newton's
    method for the nonlinear Poisson-Boltzmann equation from zero to the workload's tolerance
    (linearised steps to 1e-3 by V-cycles), with the sphere densities scaled so that the
    potential reaches the nonlinear regime."""
    import torch

    from paper_1410_6609_gb300.solver import Poisson

    nx, ny, nz = w.dims
    N = nx * ny * nz
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    out = {"tol": w.tol, "debye_length_cells": debye, "charge_scale": charge}
    for prec in ("fp64", "mixed"):
        P = Poisson(w.dims, h=w.h, bc_type=w.bc_type, bc_value=w.bc_value, precision=prec)
        c, r = dev(sp.centers), dev(sp.radius)
        vol = P.sphere_density(c, r, torch.ones(sp.count, dtype=torch.float64, device="cuda"), w.subsample)
        torch.cuda.synchronize()
        eps = 80.0 - 78.0 * vol
        k2 = (1.0 - vol) * (80.0 / debye ** 2)
        torch.cuda.synchronize()
        P.set_permittivity(eps)
        P.set_reaction(k2)
        rho = P.sphere_density(c, r, dev(sp.density * charge), w.subsample)

        def solve():
            P.set_rhs(rho)
            P.set_solution(None)
            return P.solve_pb(w.tol, 40, 1e-3, 30)

        it, rel = solve()
        t = _time(solve, P.stream, 1)
        out[prec] = {"newton_steps": it, "rel_residual": rel, "ms": t, "mlups_per_solve": N / t / 1e3,
                     "max_abs_phi_thermal_units": float(P.solution().abs().max())}
        P.close()
    out["speedup_mixed_vs_fp64"] = out["fp64"]["ms"] / out["mixed"]["ms"]
    return out


def measure_batched(tol: float = 1e-9):
    """64 independent charged-sphere systems of 64^3..192^3 solved as one batch (mixed precision)
    vs the same systems solved one after another with single contexts."""
    import torch

    from paper_1410_6609_gb300.batch import BatchPoisson
    from paper_1410_6609_gb300.solver import Poisson

    ws = synth.batched_workloads()
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    rho = []
    for w in ws:
        sp = w.spheres()
        P = Poisson(w.dims, h=w.h, bc_type=w.bc_type, bc_value=w.bc_value)
        rho.append(P.sphere_density(dev(sp.centers), dev(sp.radius), dev(sp.density), w.subsample))
        P.close()
    cells = sum(int(np.prod(w.dims)) for w in ws)
    systems = [dict(dims=w.dims, h=w.h, bc_type=w.bc_type, bc_value=w.bc_value) for w in ws]
    Bt = BatchPoisson(systems, precision="mixed")
    tune = Bt.autotune(reps=2)
    stream = Bt.stream

    def run_batch():
        Bt.set_rhs_all(rho)
        for b in range(len(ws)):
            Bt.set_solution(b, None)
        return Bt.solve(tol, 50)

    cyc, rel = run_batch()
    l0 = Bt.kernel_launches
    t_batch = _time(run_batch, stream, 3)
    launches = (Bt.kernel_launches - l0) // 4
    Bt.close()
    singles = [Poisson(w.dims, h=w.h, bc_type=w.bc_type, bc_value=w.bc_value, precision="mixed") for w in ws]

    def run_singles():
        for b, P in enumerate(singles):
            P.set_rhs(rho[b])
            P.set_solution(None)
            P.solve(tol, 50)

    run_singles()
    t_seq = _time(run_singles, singles[0].stream, 2)
    for P in singles:
        P.close()
    return {"systems": len(ws), "cells": cells, "tol": tol, "tiles": list(tune["tiles"]),
            "batch_ms": t_batch, "batch_mlups": cells / t_batch / 1e3, "max_cycles": max(cyc),
            "max_rel_residual": max(rel), "kernel_launches_per_solve": int(launches),
            "sequential_single_ms": t_seq, "speedup_vs_sequential": t_seq / t_batch}


def measure_adjoint():
    """Adjoint workload: 256^3, 32 spheres; J = sum of z-forces and dJ/d(densities, wall values)
    through the hand-written autograd functions (forward solve + one adjoint solve)."""
    import torch

    from paper_1410_6609_gb300.autograd import z_force_objective
    from paper_1410_6609_gb300.solver import Poisson

    w = synth.WORKLOADS["adjoint256"]
    sp = w.spheres()
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    c, r = dev(sp.centers), dev(sp.radius)
    res = {}
    for prec, tol in (("fp64", 1e-10), ("mixed", 1e-10)):
        P = Poisson(w.dims, h=w.h, bc_type=w.bc_type, bc_value=w.bc_value, precision=prec)

        def grad():
            q = dev(sp.density).requires_grad_(True)
            v = dev(np.array(w.bc_value)).requires_grad_(True)
            J = z_force_objective(P, q, v, c, r, w.subsample, tol=tol)
            J.backward()
            return q.grad, v.grad

        gq, gv = grad()
        t = _time(grad, P.stream, 3)
        res[prec] = {"ms_forward_and_gradient": t, "tol": tol, "dJ_dV_top": float(gv[5])}
        res[prec + "_grad"] = gq
        P.close()
    g64, gm = res.pop("fp64_grad"), res.pop("mixed_grad")
    res["rel_diff_mixed_vs_fp64_grad"] = float(torch.linalg.norm(gm - g64) / torch.linalg.norm(g64))
    return res


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
