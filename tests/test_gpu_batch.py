"""Batched solves over systems of different sizes: bit-identical to single contexts, converged
per system (checked by the CPU oracle), unaffected by the tile shapes the autotuner picks."""
import numpy as np
import pytest
import torch

import oracle
from paper_1410_6609_gb300 import synth
from paper_1410_6609_gb300.batch import BatchPoisson
from paper_1410_6609_gb300.solver import Poisson

pytestmark = pytest.mark.gpu

D, N = 0, 1

# different sizes and level counts: coarsest grids 4^3, 3^3, 6x5x3 and a single-level 4x4x6
SYSTEMS = [
    dict(dims=(32, 32, 32), h=1.0, bc_type=synth.WALL_BC_TYPE, bc_value=synth.wall_bc_value(1.0)),
    dict(dims=(48, 48, 48), h=0.5, bc_type=(D,) * 6, bc_value=(0.0, 0.1, 0.0, 0.0, 0.0, 1.0)),
    dict(dims=(24, 40, 12), h=1.0, bc_type=(D, N, N, D, D, N), bc_value=(0.2, 0.0, -0.1, 0.0, 0.0, 0.3)),
    dict(dims=(64, 32, 48), h=1.0, bc_type=synth.WALL_BC_TYPE, bc_value=synth.wall_bc_value(-0.5)),
    dict(dims=(4, 4, 6), h=1.0, bc_type=(D, N, N, D, D, N), bc_value=(0.0,) * 6),
    dict(dims=(96, 96, 96), h=1.0, bc_type=synth.WALL_BC_TYPE, bc_value=synth.wall_bc_value(1.0)),
]


def _with_defect(defect, make):
    """make() with CCMG_DEFECT=defect in the environment (None: as it is)."""
    import os
    if defect is None:
        return make()
    old = os.environ.get("CCMG_DEFECT")
    os.environ["CCMG_DEFECT"] = defect
    try:
        return make()
    finally:
        if old is None:
            del os.environ["CCMG_DEFECT"]
        else:
            os.environ["CCMG_DEFECT"] = old


def _single(s, precision="mixed", defect=None):
    return _with_defect(defect, lambda: Poisson(s["dims"], h=s["h"], bc_type=s["bc_type"], bc_value=s["bc_value"],
                                                precision=precision))


def rhos():
    return [torch.from_numpy(synth.random_field(s["dims"], 30 + i)).cuda() for i, s in enumerate(SYSTEMS)]


@pytest.mark.parametrize("defect", [None, "walk"])
def test_zero_start_batch_is_bit_identical_to_single_contexts(defect):
    """Solves from the never-written zero iterate (mixed precision): the systems whose finest rows
    are whole 4-float vectors carry their residuals by recurrence (CCMG_DEFECT unset) exactly as
    single contexts do, the others (and all, with CCMG_DEFECT=walk) evaluate them directly; every
    system's cycles, relative residual and iterate equal those of its single context, bit for bit."""
    rho = rhos()
    Bt = _with_defect(defect, lambda: BatchPoisson(SYSTEMS, precision="mixed"))
    for b, r in enumerate(rho):
        Bt.set_rhs(b, r)
    for rep in range(2):  # the second solve after the first left non-zero iterates and flags behind
        Bt.reset_solutions()
        cyc, rel = Bt.solve(1e-9, 50)
    for b, s in enumerate(SYSTEMS):
        P = _single(s, "mixed", defect)
        P.set_rhs(rho[b])
        P.set_solution(None)
        k, r = P.solve(1e-9, 50)
        assert (k, r) == (cyc[b], rel[b]), (b, k, cyc[b], r, rel[b])
        assert torch.equal(P.solution(), Bt.solution(b)), b
        counts = P.outer_counts()
        assert (counts[1] > 0) == (defect is None and s["dims"][0] % 8 == 0 and min(s["dims"]) >= 6), (b, counts)
        P.close()
    # a later fixed number of cycles takes no recurrence step (the flags were reset)
    Bt.reset_solutions()
    Bt.vcycle(2)
    for b, s in enumerate(SYSTEMS[:2]):
        P = _single(s, "mixed", defect)
        P.set_rhs(rho[b])
        P.set_solution(None)
        P.vcycle(2)
        assert torch.equal(P.solution(), Bt.solution(b)), b
        P.close()
    Bt.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batch_is_bit_identical_to_single_contexts(precision):
    tol = 1e-10 if precision == "fp64" else 1e-9
    rho = rhos()
    Bt = BatchPoisson(SYSTEMS, precision=precision)
    for b, r in enumerate(rho):
        Bt.set_rhs(b, r)
    cyc, rel = Bt.solve(tol, 50)
    for b, s in enumerate(SYSTEMS):
        P = _single(s, precision)
        P.set_rhs(rho[b])
        k, r = P.solve(tol, 50)
        assert (k, r) == (cyc[b], rel[b]), (b, k, cyc[b], r, rel[b])
        assert torch.equal(P.solution(), Bt.solution(b)), b
        P.close()
    Bt.close()


def test_batch_converges_per_system_checked_by_oracle():
    rho = rhos()
    Bt = BatchPoisson(SYSTEMS, precision="mixed")
    for b, r in enumerate(rho):
        Bt.set_rhs(b, r)
    cyc, rel = Bt.solve(1e-9, 50)
    assert max(rel) < 1e-9
    for b, s in enumerate(SYSTEMS):
        f = oracle.rhs(rho[b].cpu().numpy(), s["h"], s["bc_type"], s["bc_value"])
        phi = Bt.solution(b).cpu().numpy()
        assert oracle.rel_residual(phi, f, s["h"], s["bc_type"]) < 1.0001e-9, b
    Bt.close()


def test_tiles_change_speed_not_results():
    rho = rhos()
    out = []
    for tiles in [(64, 4, 64, 4), (16, 16, 32, 8), (128, 2, 128, 2)]:
        Bt = BatchPoisson(SYSTEMS, precision="mixed")
        Bt.set_tiles(tiles)
        assert Bt.tiles() == tiles
        for b, r in enumerate(rho):
            Bt.set_rhs(b, r)
        Bt.solve(1e-9, 50)
        out.append([Bt.solution(b) for b in range(len(SYSTEMS))])
        Bt.close()
    for other in out[1:]:
        for a, c in zip(out[0], other):
            assert torch.equal(a, c)


def test_autotune_picks_a_candidate(tmp_path, monkeypatch):
    monkeypatch.setenv("CCMG_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    Bt = BatchPoisson(SYSTEMS[:4], precision="mixed")
    res = Bt.autotune(reps=2)
    assert not res["cached"] and len(res["ms"]) >= 4 and min(res["ms"]) > 0
    assert Bt.tiles() == res["tiles"]
    Bt2 = BatchPoisson(SYSTEMS[:4], precision="mixed")
    res2 = Bt2.autotune(reps=2)
    assert res2["cached"] and Bt2.tiles() == res["tiles"]
    Bt.close()
    Bt2.close()


def test_batched_workload_64_systems():
    """The batched charged-sphere workload: 64 systems of 64^3..192^3 with 20..120 spheres each,
    FP32 cycles inside FP64 defect correction, all to a 1e-9 relative residual in one batch."""
    ws = synth.batched_workloads()
    systems = [dict(dims=w.dims, h=w.h, bc_type=w.bc_type, bc_value=w.bc_value) for w in ws]
    Bt = BatchPoisson(systems, precision="mixed")
    rho = []
    for b, w in enumerate(ws):
        sp = w.spheres()
        P = Poisson(w.dims, h=w.h, bc_type=w.bc_type, bc_value=w.bc_value)
        dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
        rho.append(P.sphere_density(dev(sp.centers), dev(sp.radius), dev(sp.density), w.subsample))
        P.close()
        Bt.set_rhs(b, rho[b])
    cyc, rel = Bt.solve(1e-9, 50)
    assert max(rel) < 1e-9 and max(cyc) <= 6
    for b in (0, 17, 63):  # sampled systems, residual checked by the oracle
        w = ws[b]
        f = oracle.rhs(rho[b].cpu().numpy(), w.h, w.bc_type, w.bc_value)
        assert oracle.rel_residual(Bt.solution(b).cpu().numpy(), f, w.h, w.bc_type) < 1.0001e-9
    Bt.close()


def test_zero_start_without_writing_and_flag_uploads_in_order():
    """set_solution(None) in a mixed batch writes nothing (the first cycle's update stores phi = s e):
    reading a system before any cycle gives zeros, and cycles issued right after the resets (no
    synchronisation between host flag changes and the queued work) match single contexts bit
    for bit, also after a first solve has left non-zero iterates behind."""
    rho = rhos()
    Bt = BatchPoisson(SYSTEMS, precision="mixed")
    for b, r in enumerate(rho):
        Bt.set_rhs(b, r)
    Bt.solve(1e-9, 50)
    Bt.reset_solutions()
    assert not torch.any(Bt.solution(2) != 0)
    Bt.reset_solutions()
    Bt.vcycle(2)
    for b, s in enumerate(SYSTEMS):
        P = _single(s)
        P.set_rhs(rho[b])
        P.set_solution(None)
        P.vcycle(2)
        assert torch.equal(P.solution(), Bt.solution(b)), b
        P.close()
    Bt.close()


# Systems whose finest levels all qualify for the TMA-staged batched sweep (packed rows of whole
# 4-float vectors, next level of half the size with whole vectors), with tiles of 32 packed
# columns x 32 rows left ragged in x (hx 48, 40), in y (80, 40) and in the slabs (136 planes),
# and one system with a zero right-hand side (converged before its first cycle: its work items
# are skipped and its iterate stays zero).
TMA_SYSTEMS = [
    dict(dims=(64, 64, 64), h=1.0, bc_type=synth.WALL_BC_TYPE, bc_value=synth.wall_bc_value(1.0)),
    dict(dims=(96, 80, 48), h=1.0, bc_type=(D, N, N, D, D, N), bc_value=(0.2, 0.0, -0.1, 0.0, 0.0, 0.3)),
    dict(dims=(80, 40, 136), h=0.5, bc_type=(D,) * 6, bc_value=(0.0, 0.1, 0.0, 0.0, 0.0, 1.0)),
    dict(dims=(128, 32, 16), h=1.0, bc_type=synth.WALL_BC_TYPE, bc_value=synth.wall_bc_value(-0.5)),
    dict(dims=(64, 48, 32), h=1.0, bc_type=(D,) * 6, bc_value=(0.0,) * 6),
]


def _solve_batch(systems, rho, sweep):
    import os
    old = os.environ.get("CCMG_SWEEP")
    if sweep:
        os.environ["CCMG_SWEEP"] = sweep
    try:
        Bt = BatchPoisson(systems, precision="mixed")
    finally:
        if old is None:
            os.environ.pop("CCMG_SWEEP", None)
        else:
            os.environ["CCMG_SWEEP"] = old
    for b, r in enumerate(rho):
        Bt.set_rhs(b, r)
    cyc, rel = Bt.solve(1e-9, 50)
    sols = [Bt.solution(b) for b in range(len(systems))]
    Bt.close()
    return cyc, rel, sols


def test_tma_staged_batch_equals_direct_load_batch_and_single_contexts():
    rho = [torch.from_numpy(synth.random_field(s["dims"], 60 + i)).cuda() for i, s in enumerate(TMA_SYSTEMS)]
    rho[-1].zero_()
    ct, rt, st = _solve_batch(TMA_SYSTEMS, rho, None)   # TMA-staged finest-level sweeps
    cv, rv, sv = _solve_batch(TMA_SYSTEMS, rho, "vec")  # direct-load sweeps everywhere
    assert ct == cv and rt == rv
    assert ct[-1] == 0 and not torch.any(st[-1] != 0)
    for b, s in enumerate(TMA_SYSTEMS):
        assert torch.equal(st[b], sv[b]), b
        P = _single(s)
        P.set_rhs(rho[b])
        k, r = P.solve(1e-9, 50)
        assert (k, r) == (ct[b], rt[b]), b
        assert torch.equal(P.solution(), st[b]), b
        P.close()
        if b < len(TMA_SYSTEMS) - 1:
            f = oracle.rhs(rho[b].cpu().numpy(), s["h"], s["bc_type"], s["bc_value"])
            assert oracle.rel_residual(st[b].cpu().numpy(), f, s["h"], s["bc_type"]) < 1.0001e-9, b


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_set_rhs_all_equals_per_system_calls(precision):
    """mg_batch_set_rhs_all (three launches for every system) gives the same solves, bit for bit,
    as set_rhs per system, whether a density sits on a 16-byte boundary (two cells per thread) or
    not (one cell per thread); called twice in a row, the second call's values are the ones
    solved; a wrong count is refused."""
    tol = 1e-10 if precision == "fp64" else 1e-9
    rho = rhos()
    shifted = []
    for r in rho:  # the same values 8 bytes past a 16-byte boundary
        buf = torch.empty(r.numel() + 1, dtype=torch.float64, device="cuda")
        v = buf[1:].view(r.shape)
        v.copy_(r)
        shifted.append(v)
    assert all(t.data_ptr() % 16 == 8 for t in shifted)
    out = []
    for mode in ("each", "all", "all_shifted"):
        Bt = BatchPoisson(SYSTEMS, precision=precision)
        if mode == "each":
            for b, r in enumerate(rho):
                Bt.set_rhs(b, r)
        elif mode == "all":
            Bt.set_rhs_all([r * 2.0 for r in rho])  # overwritten by the next call
            Bt.set_rhs_all(rho)
        else:
            Bt.set_rhs_all(shifted)
        cyc, rel = Bt.solve(tol, 50)
        out.append((cyc, rel, [Bt.solution(b).clone() for b in range(len(SYSTEMS))]))
        if mode == "all":
            with pytest.raises(ValueError):
                Bt.set_rhs_all(rho[:-1])
        Bt.close()
    for o in out[1:]:
        assert o[0] == out[0][0] and o[1] == out[0][1]
        assert all(torch.equal(a, b) for a, b in zip(o[2], out[0][2]))
