"""Periodic walls (Sec. 2.4: the domain is extended cyclically, the neighbour across a periodic
face is the cell at the opposite side) on the GPU against the oracle: every level operation in
FP64 and FP32, V-cycles, the fixed-point FP64 residual against exact rational arithmetic, the
E-field (both stencils), the charge of spheres across periodic walls (bit-exact), forces and the
force adjoint, mixed-precision and batched solves. Tolerances as in the wall-only parity tests.
"""
import os
from fractions import Fraction

import numpy as np
import pytest
import torch

import oracle
from paper_1410_6609_gb300 import synth
from paper_1410_6609_gb300.batch import BatchPoisson
from paper_1410_6609_gb300.solver import Poisson
from test_gpu_parity import _rows_max, cpu, gpu, maxrel, rel
from test_gpu_parity import test_level_operations_match_oracle as _level_operations
from test_gpu_parity import test_single_precision_level_operations_match_oracle as _level_operations_f32
from test_gpu_parity import test_vcycles_match_oracle as _vcycles

pytestmark = pytest.mark.gpu

D, N, P = 0, 1, 2

# a ragged 5-level grid (vector and scalar sweeps, an odd 9x5x3 coarsest grid), a small one whose
# coarsest grid is odd in every axis, and the 32^3 grid; periodic in one, two and all but one axis
CASES = [((144, 80, 48), (P, P, P, P, D, D)), ((12, 10, 14), (P, P, D, N, P, P)), ((32, 32, 32), (D, N, P, P, P, P))]


@pytest.mark.parametrize("dims,bc", CASES)
def test_periodic_level_operations_match_oracle(dims, bc):
    _level_operations(dims, bc)


@pytest.mark.parametrize("dims,bc", CASES[:2])
def test_periodic_single_precision_level_operations_match_oracle(dims, bc):
    _level_operations_f32(dims, bc)


@pytest.mark.parametrize("dims,bc", CASES)
@pytest.mark.parametrize("ncycles", [1, 3])
def test_periodic_vcycles_match_oracle(dims, bc, ncycles):
    _vcycles(dims, bc, ncycles)


def _neighbours(phi, bc):
    """The six neighbour arrays (-x,+x,-y,+y,-z,+z): zero beyond a wall, wrapped across a
    periodic axis."""
    out = []
    for ax, q in ((2, 0), (1, 2), (0, 4)):
        per = bc[q] == P
        for step in (1, -1):  # value of the -e (+e) neighbour: the array shifted forward (back)
            a = np.roll(phi, step, axis=ax)
            if not per:
                idx = [slice(None)] * 3
                idx[ax] = 0 if step == 1 else -1
                a[tuple(idx)] = 0.0
            out.append(a)
    return out


@pytest.mark.parametrize("dims,bc", [((24, 20, 18), (P, P, D, N, P, P)), ((40, 8, 6), (P, P, P, P, D, N))])
def test_periodic_fp64_residual_against_exact_arithmetic(dims, bc):
    """The fixed-point FP64 residual with periodic halos (wrapped columns, rows and planes of the
    tile walk, including ragged tiles) within (8 + D)/32 of an ulp of the largest value among the
    five rows the walk reads for the cell (across a periodic axis the row at the opposite side) or
    of its g, plus half an ulp of itself, from the exact value."""
    rng = np.random.default_rng(12)
    nx, ny, nz = dims
    shape = (nz, ny, nx)
    phi = rng.standard_normal(shape) * np.exp2(rng.integers(-40, 41, shape))
    phi[rng.random(shape) < 0.1] = 0.0
    sh = {D: 1, N: -1, P: 0}
    diag = np.full(shape, 6, dtype=np.int64)
    diag[:, :, 0] += sh[bc[0]]
    diag[:, :, -1] += sh[bc[1]]
    diag[:, 0, :] += sh[bc[2]]
    diag[:, -1, :] += sh[bc[3]]
    diag[0] += sh[bc[4]]
    diag[-1] += sh[bc[5]]
    nbs = _neighbours(phi, bc)
    g = rng.standard_normal(shape) * np.exp2(rng.integers(-40, 41, shape))
    cancel = rng.random(shape) < 0.5
    g[cancel] = (diag * phi - sum(nbs))[cancel]
    Pz = Poisson(dims, h=1.0, bc_type=bc)
    Pz.level_set(0, 0, gpu(phi))
    Pz.level_set(0, 1, gpu(g))
    _, r = Pz.residual(field=True)
    r = cpu(r)
    Pz.close()
    # the closed-form neighbours agree with the oracle's stencil
    assert maxrel(r, oracle.residual(phi, g, 1.0, bc)) < 1e-12 or np.abs(r).max() == 0.0
    big = np.maximum(_rows_max(phi, bc), np.abs(g))
    worst = 0.0
    for idx in np.ndindex(*shape):
        exact = Fraction(g[idx]) + sum(Fraction(float(n[idx])) for n in nbs) - int(diag[idx]) * Fraction(phi[idx])
        bound = Fraction(8 + int(diag[idx]), 32) * Fraction(np.spacing(big[idx])) + Fraction(np.spacing(abs(r[idx]))) / 2
        worst = max(worst, float(abs(Fraction(float(r[idx])) - exact) / bound))
    assert worst <= 1.0, worst


def _straddling_spheres():
    # centres near the periodic x and y walls (and one inside), radii 2..4
    c = np.array([[0.7, 20.3, 30.1], [62.9, 1.2, 11.4], [30.5, 47.4, 20.2], [1.5, 46.8, 40.6], [33.0, 24.0, 24.0]])
    return c, np.array([3.5, 2.5, 4.0, 3.0, 2.0]), np.array([1.0, -0.6, 0.8, -1.2, 0.5])


@pytest.mark.parametrize("sf", [1, 2, 3])
def test_periodic_sphere_density_bit_exact(sf):
    dims = (64, 48, 56)
    bc = (P, P, P, P, D, D)
    c, R, q = _straddling_spheres()
    Pz = Poisson(dims, bc_type=bc)
    got = cpu(Pz.sphere_density(gpu(c), gpu(R), gpu(q), sf))
    ref = oracle.sphere_density((dims[2], dims[1], dims[0]), 1.0, c, R, q, sf, bc)
    assert np.array_equal(got, ref)
    Pz.close()


@pytest.mark.parametrize("h", [1.0, 0.3])
def test_periodic_efield_and_forces_match_oracle(h):
    dims = (64, 48, 56)
    bc = (P, P, P, P, D, D)
    bcv = (0.0, 0.0, 0.0, 0.0, -0.5, 1.0)
    c, R, q = _straddling_spheres()
    c = c * h
    R = R * h
    phi = synth.random_field(dims, 9)
    Pz = Poisson(dims, h=h, bc_type=bc, bc_value=bcv)
    Pz.set_solution(gpu(phi))
    for st in (7, 19):
        Pz.gradient_stencil = st
        E = cpu(Pz.efield())
        assert maxrel(E, oracle.efield(phi, h, bc, bcv, stencil=st)) < 1e-15, st
        F = cpu(Pz.force_gather(gpu(c), gpu(R), gpu(q), 2))
        Fref = oracle.force_gather(phi, h, bc, bcv, c, R, q, 2, stencil=st)
        assert maxrel(F, Fref) < 1e-12, st
    Pz.close()


def test_periodic_adjoint_kernels_match_oracle():
    dims = (64, 48, 56)
    bc = (P, P, P, P, D, N)
    bcv = (0.0, 0.0, 0.0, 0.0, 0.7, 0.2)
    c, R, q = _straddling_spheres()
    wF = np.random.default_rng(3).standard_normal((len(R), 3))
    phi = synth.random_field(dims, 4)
    Pz = Poisson(dims, bc_type=bc, bc_value=bcv)
    Pz.set_solution(gpu(phi))
    gphi, gd, gbc = Pz.force_gather_adjoint(gpu(c), gpu(R), gpu(q), gpu(wF), 2)
    r_gphi, r_gd, r_gbc = oracle.force_gather_adjoint(phi, 1.0, bc, bcv, c, R, q, wF, 2)
    assert maxrel(cpu(gphi), r_gphi) < 1e-13
    assert maxrel(cpu(gd), r_gd) < 1e-12
    assert maxrel(cpu(gbc), r_gbc) < 1e-12 and np.all(cpu(gbc)[:4] == 0.0)
    gfield = synth.random_field(dims, 6)
    got = cpu(Pz.sphere_density_adjoint(gpu(c), gpu(R), gpu(gfield), 2))
    assert maxrel(got, oracle.sphere_density_adjoint(gfield, 1.0, c, R, 2, bc)) < 1e-13
    lam = synth.random_field(dims, 8)
    grho, gbc2 = Pz.rhs_adjoint(gpu(lam))
    r_grho, r_gbc2 = oracle.rhs_adjoint(lam, 1.0, bc)
    assert maxrel(cpu(gbc2), r_gbc2) < 1e-13 and np.all(cpu(gbc2)[:4] == 0.0)
    Pz.close()


@pytest.mark.parametrize("dims,bc", [((64, 64, 64), (P, P, P, P, D, D)), ((64, 60, 64), (D, N, P, P, P, P)),
                                     ((72, 40, 48), (P, P, D, N, P, P))])
def test_periodic_mixed_precision_and_the_staged_sweep(dims, bc):
    """Mixed precision to 1e-9 (checked by the oracle's residual); with the TMA-staged half-sweep
    requested on every level it can run on, the periodic levels take it (wrapped halo rows, columns
    and planes loaded into the staged tiles; ragged tiles in y for 60 rows) and give the same
    iterates as the direct-load sweep."""
    nx, ny, nz = dims
    bcv = (0.0, 0.0, 0.0, 0.0, 0.0, 1.0) if bc[5] == D else (0.0, 0.5, 0.0, 0.2, 0.0, 0.0)
    sp = synth.random_spheres(dims, 20, 4.0, 17)
    rho = oracle.sphere_density((nz, ny, nx), 1.0, sp.centers, sp.radius, sp.density, 2, bc)
    f = oracle.rhs(rho, 1.0, bc, bcv)
    Pz = Poisson(dims, bc_type=bc, bc_value=bcv, precision="mixed")
    Pz.set_rhs(gpu(rho))
    k, r = Pz.solve(1e-9, 50)
    phi = cpu(Pz.solution())
    assert r < 1e-9
    assert oracle.rel_residual(phi, f, 1.0, bc) < 1.0001e-9
    ref64, _, _ = oracle.solve(f, 1.0, bc, tol=1e-12)
    assert rel(phi, ref64) < 1e-7
    assert Pz.level_sweep_kind(0) == "vec"  # too small for the staged sweep by default
    old = os.environ.get("CCMG_SWEEP")
    os.environ["CCMG_SWEEP"] = "tma"
    try:
        Pt = Poisson(dims, bc_type=bc, bc_value=bcv, precision="mixed")
        Pw = Poisson(dims, bc_type=synth.WALL_BC_TYPE, bc_value=bcv, precision="mixed")
    finally:
        if old is None:
            del os.environ["CCMG_SWEEP"]
        else:
            os.environ["CCMG_SWEEP"] = old
    assert Pt.level_sweep_kind(0) == "tma" and Pw.level_sweep_kind(0) == "tma"
    Pt.set_rhs(gpu(rho))
    assert Pt.solve(1e-9, 50) == (k, r)
    assert torch.equal(Pt.solution(), Pz.solution())
    # the staged half-sweep on its own against the direct-load one, both colours
    phi0 = synth.random_field(dims, 5).astype(np.float32).astype(np.float64)
    g0 = (synth.random_field(dims, 6) * 0.1).astype(np.float32).astype(np.float64)
    for colour in (0, 1):
        outs = []
        for ctx in (Pt, Pz):
            ctx.level_set(0, 0, gpu(phi0))
            ctx.level_set(0, 1, gpu(g0))
            ctx.op_smooth(0, colour)
            outs.append(cpu(ctx.level_get(0, 0)))
        assert np.array_equal(outs[0], outs[1]), colour
    for ctx in (Pz, Pt, Pw):
        ctx.close()


@pytest.mark.parametrize("precision,zero_start", [("fp64", False), ("mixed", False), ("mixed", True)])
def test_periodic_batch_is_bit_identical_to_single_contexts(precision, zero_start):
    """Batched solves with periodic axes (and one system without) equal single contexts bit for bit;
    from the never-written zero the mixed solves carry their residuals by recurrence (the batched
    step's periodic variant serving the system without periodic axes too)."""
    systems = [
        dict(dims=(32, 32, 32), h=1.0, bc_type=(P, P, P, P, D, D), bc_value=(0.0, 0.0, 0.0, 0.0, 0.0, 1.0)),
        dict(dims=(48, 40, 24), h=0.5, bc_type=(D, N, P, P, P, P), bc_value=(0.2, -0.1, 0.0, 0.0, 0.0, 0.0)),
        dict(dims=(24, 40, 12), h=1.0, bc_type=(D, N, N, D, D, N), bc_value=(0.2, 0.0, -0.1, 0.0, 0.0, 0.3)),
        dict(dims=(64, 32, 48), h=1.0, bc_type=(P, P, N, N, D, D), bc_value=(0.0, 0.0, 0.1, -0.1, 0.0, 1.0)),
    ]
    tol = 1e-10 if precision == "fp64" else 1e-9
    rho = [torch.from_numpy(synth.random_field(s["dims"], 50 + i)).cuda() for i, s in enumerate(systems)]
    Bt = BatchPoisson(systems, precision=precision)
    for b, r in enumerate(rho):
        Bt.set_rhs(b, r)
    if zero_start:
        Bt.reset_solutions()
    cyc, rels = Bt.solve(tol, 50)
    for b, s in enumerate(systems):
        Pz = Poisson(s["dims"], h=s["h"], bc_type=s["bc_type"], bc_value=s["bc_value"], precision=precision)
        Pz.set_rhs(rho[b])
        if zero_start:
            Pz.set_solution(None)
        k, r = Pz.solve(tol, 50)
        assert (k, r) == (cyc[b], rels[b]), b
        if zero_start:
            assert Pz.outer_counts()[1] >= 1, b  # the recurrence ran
        assert torch.equal(Pz.solution(), Bt.solution(b)), b
        f = oracle.rhs(rho[b].cpu().numpy(), s["h"], s["bc_type"], s["bc_value"])
        assert oracle.rel_residual(cpu(Pz.solution()), f, s["h"], s["bc_type"]) < tol * 1.0001, b
        Pz.close()
    Bt.close()


def test_periodic_static_residual_matches_oracle():
    from paper_1410_6609_gb300 import _lib
    dims = (20, 12, 16)
    bc = (P, P, D, N, P, P)
    phi = synth.random_field(dims, 3)
    f = synth.random_field(dims, 4)
    lib = _lib.load()
    bct = (__import__("ctypes").c_int * 6)(*bc)
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    dphi, df = gpu(phi), gpu(f)
    st = lib.mg_residual_norm_static(dims[0], dims[1], dims[2], 0.5, bct, dphi.data_ptr(), df.data_ptr(),
                                     out.data_ptr(), None)
    assert st == 0
    r = oracle.residual(phi, f, 4.0, bc)
    got = cpu(out)
    assert abs(got[1] - np.linalg.norm(r)) <= 1e-12 * np.linalg.norm(r)
    assert abs(got[0] - np.linalg.norm(r) / np.linalg.norm(f)) <= 1e-12 * got[0]
