"""The mixed-precision outer step with its residual carried by recurrence (mg_op_defect_update and
the solve that uses it; the operator is the folded stencil of Sec. 2.4).

Kernel parity: phi' = phi + s e must equal the oracle bit for bit (the same single FP64 addition of
an exact product); the residual pair hi + lo must lie within the kernel's stated bound of the
oracle's exactly rounded r' = r - s A e, hi must be the float nearest to r'/s' (up to cells within
the bound of a rounding tie), and |lo| <= ulp(hi)/2. Cases: walls of every kind, periodic axes,
the first step from a zero iterate (the pair formed from the right-hand side), and a level large
enough for the kernel's grid-stride loop to wrap. The correction is a smooth field plus noise, so
that A e cancels much of its terms, as the inner cycles' corrections do.

Solves: with the recurrence (the default) against the direct residual after every step
(CCMG_DEFECT=walk): the same number of outer steps, both below the tolerance by the oracle's own
residual, and the returned relative residual always a direct evaluation (equal to mg_residual).
"""
from __future__ import annotations

import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_1410_6609_gb300 import synth  # noqa: E402
from paper_1410_6609_gb300.solver import Poisson  # noqa: E402

pytestmark = pytest.mark.gpu

D, N, PER = 0, 1, 2


def _poisson(dims, defect=None, **kw):
    old = os.environ.get("CCMG_DEFECT")
    if defect is not None:
        os.environ["CCMG_DEFECT"] = defect
    try:
        return Poisson(dims, precision="mixed", **kw)
    finally:
        if defect is not None:
            if old is None:
                del os.environ["CCMG_DEFECT"]
            else:
                os.environ["CCMG_DEFECT"] = old


def _smooth_correction(dims, seed):
    """A smooth field (low modes) plus 1e-3 noise, rounded to float."""
    nx, ny, nz = dims
    rng = np.random.default_rng(seed)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    f = np.zeros((nz, ny, nx))
    for _ in range(4):
        kx, ky, kz = rng.uniform(0.5, 2.5, 3)
        f += rng.standard_normal() * np.sin(np.pi * kx * (x + 0.5) / nx + rng.uniform(0, 6)) \
            * np.sin(np.pi * ky * (y + 0.5) / ny + rng.uniform(0, 6)) * np.sin(np.pi * kz * (z + 0.5) / nz)
    f = 300.0 * f + 1e-3 * rng.standard_normal(f.shape)
    return f.astype(np.float32).astype(np.float64)


def _term_magnitudes(e, bc):
    """Sum over the terms of A e of their magnitudes: six neighbours and (6 + d) |e|."""
    a = np.abs(e)
    tot = np.zeros_like(a)
    nz, ny, nx = a.shape
    n = (nx, ny, nz)
    diag = np.full(a.shape, 6.0)
    for face in range(6):
        axis, step = face // 2, (-1 if face % 2 == 0 else 1)
        nb = np.roll(a, -step, axis=2 - axis)
        idx = np.arange(n[axis])
        edge = (idx == 0) if step < 0 else (idx == n[axis] - 1)
        shape = [1, 1, 1]
        shape[2 - axis] = n[axis]
        edge = np.broadcast_to(edge.reshape(shape), a.shape)
        if bc[face] != PER:
            nb = np.where(edge, 0.0, nb)
            diag = diag + np.where(edge, 1.0 if bc[face] == D else -1.0, 0.0)
        tot += nb
    return tot + diag * a


def _check_step(dims, bc, zero, seed):
    P = _poisson(dims, bc_type=bc)
    rng = np.random.default_rng(seed)
    e = _smooth_correction(dims, seed)
    sc, sn = 2.0 ** -7, 2.0 ** -18
    # a residual that the correction nearly cancels: r = s A e + small rest (what an inner solve
    # leaves), so r' is about 1e-3 of r
    _, Ae = oracle.defect_update(np.zeros(e.shape), e, np.zeros(e.shape), sc, bc)  # = -s A e
    r = -Ae * (1.0 + 1e-3 * rng.standard_normal(e.shape)) + 1e-6 * sc * rng.standard_normal(e.shape)
    phi = np.zeros(e.shape) if zero else rng.standard_normal(e.shape)
    g = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    phi_o, hi, lo, ss = P.op_defect_update(g(phi), g(e), g(r), sc, sn, zero_start=zero)
    phi_o, hi, lo = phi_o.cpu().numpy(), hi.cpu().numpy(), lo.cpu().numpy()
    phi_ref, r_ref = oracle.defect_update(phi, e, r, sc, bc)
    assert np.array_equal(phi_o, phi_ref)
    if zero:  # +0 for a zero product, as the plain first update stores it
        assert not np.any(np.signbit(phi_o) & (phi_o == 0.0))
    # the pair against the exactly rounded recurrence
    err = np.abs((hi + lo) * sn - r_ref)  # hi + lo rounded to double: far below the bound
    bound = sc * (2.0 ** -44 * (np.abs(r) / sc + np.abs(r_ref) / sc) + 2.0 ** -58 * _term_magnitudes(e, bc))
    assert np.all(err <= bound), float(np.max(err / np.maximum(bound, 1e-300)))
    hi_ref = (r_ref / sn).astype(np.float32).astype(np.float64)
    assert np.mean(hi == hi_ref) > 0.999
    ulp = np.spacing(np.abs(hi).astype(np.float32)).astype(np.float64)
    assert np.all(np.abs(hi - hi_ref) <= ulp)
    assert np.all(np.abs(lo) <= 0.5 * ulp)
    want = float(np.sum(hi * hi)) * sn * sn
    assert abs(ss - want) <= 1e-5 * want
    # the step's cancellation was real: |r'| is far below |r|
    assert np.linalg.norm(r_ref) < 1e-2 * np.linalg.norm(r)
    P.close()


@pytest.mark.parametrize("zero", [False, True])
@pytest.mark.parametrize("bc", [
    (D, N, N, D, D, N),
    (PER, PER, N, D, PER, PER),
    (N, N, PER, PER, D, D),
])
def test_defect_update_matches_oracle(bc, zero):
    _check_step((40, 20, 12), bc, zero, 11 + sum(bc))


def test_defect_update_grid_stride():
    """2^21 cells: more items than the kernel's grid has threads, so its loop wraps."""
    _check_step((256, 128, 64), (N, N, N, N, D, D), False, 5)


def test_defect_update_rejects_bad_scales():
    P = _poisson((16, 16, 16))
    f = torch.zeros((16, 16, 16), dtype=torch.float64, device="cuda")
    for sc, sn in ((3.0, 1.0), (1.0, 0.0), (2.0 ** 900, 1.0)):
        with pytest.raises(RuntimeError):
            P.op_defect_update(f, f, f, sc, sn)
    P.close()
    Pw = _poisson((16, 16, 16), defect="walk")
    with pytest.raises(RuntimeError):
        Pw.op_defect_update(f, f, f, 1.0, 1.0)
    Pw.close()


def _solve_pair(dims, bc, bcv, rho, tol):
    out = []
    for defect in (None, "walk"):
        P = _poisson(dims, defect=defect, bc_type=bc, bc_value=bcv)
        P.set_rhs(rho)
        P.set_solution(None)
        k, rel = P.solve(tol, 40)
        cyc, rec, direct = P.outer_counts()
        assert cyc == k
        # a direct evaluation after every step that is not by recurrence (two where a step
        # predicted to end the solve did not: its check leaves out the single-precision copy that
        # the next step then needs), and one before the solve stops after a step by recurrence
        if defect == "walk":
            assert rec == 0 and k <= direct <= 2 * k
        else:  # the first step from zero is by recurrence
            assert rec >= 1 and direct >= 1 and k - rec <= direct <= 2 * (k - rec) + 1
        rel_direct = P.residual()
        out.append((k, rel, rel_direct, P.solution().cpu().numpy()))
        P.close()
    return out


@pytest.mark.parametrize("bc", [synth.WALL_BC_TYPE, (PER, PER, N, N, D, D)])
def test_solve_with_recurrence_matches_direct_residual_solve(bc):
    dims = (64, 64, 64)
    bcv = synth.wall_bc_value(1.0)
    sp = synth.random_spheres(dims, 20, 4.0, 17)
    rho = oracle.sphere_density((64, 64, 64), 1.0, sp.centers, sp.radius, sp.density, 2, bc_type=bc)
    f = oracle.rhs(rho, 1.0, bc, bcv)
    (k, rel, rd, phi), (kw, relw, rdw, phiw) = _solve_pair(dims, bc, bcv, torch.from_numpy(rho).cuda(), 1e-9)
    assert k == kw
    assert rel < 1e-9 and relw < 1e-9
    assert abs(rel - rd) <= 1e-12 * rd  # the returned value is a direct evaluation
    assert oracle.rel_residual(phi, f, 1.0, bc) < 1.0001e-9
    assert np.linalg.norm(phi - phiw) <= 1e-7 * np.linalg.norm(phiw)


def test_recurrence_estimate_is_confirmed_directly():
    """A loose tolerance that the first step's estimate already meets: the solve evaluates the
    residual directly before it stops, and reports that value."""
    dims = (64, 48, 32)
    bc = synth.WALL_BC_TYPE
    rho = torch.from_numpy(synth.random_field(dims, 4)).cuda()
    for tol in (1e-2, 1e-4, 1e-7, 1e-11):
        (k, rel, rd, _), (kw, relw, _, _) = _solve_pair(dims, bc, (0.0,) * 6, rho, tol)
        assert k == kw and rel < tol
        assert abs(rel - rd) <= 1e-12 * rd
