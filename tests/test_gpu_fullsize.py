"""The hot path at the full sizes of the benchmark workloads, in the configuration bench.py times,
checked against the oracle where it finishes in seconds and by properties that hold at any size
elsewhere; plus the degenerate cases of the method (no charge at all, no spheres, the largest
single-GPU grid).

spheres512: 512^3, 1600 spheres, mixed precision to 1e-9 (the benchmark step). The oracle maps
the charges (bit-exact), takes the relative residual of the GPU potential, and computes the
E-field and the forces from it. spheres256: the FP64 step to 1e-10, same checks.
"""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_1410_6609_gb300 import synth  # noqa: E402
from paper_1410_6609_gb300.solver import Poisson  # noqa: E402

pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _step(w):
    """The benchmark step on the GPU: density, RHS, solve from zero, E-field, forces."""
    sp = w.spheres()
    P = Poisson(w.dims, h=w.h, bc_type=w.bc_type, bc_value=w.bc_value, precision=w.precision)
    c, r, q = _dev(sp.centers), _dev(sp.radius), _dev(sp.density)
    rho = P.sphere_density(c, r, q, w.subsample)
    P.set_rhs(rho)
    P.set_solution(None)
    k, rel = P.solve(w.tol, 100)
    E = P.efield()
    F = P.force_gather(c, r, q, w.subsample)
    P.gradient_stencil = 19
    F19 = P.force_gather(c, r, q, w.subsample)
    P.gradient_stencil = 7
    out = dict(sp=sp, rho=rho.cpu().numpy(), k=k, rel=rel, phi=P.solution().cpu().numpy(), F=F.cpu().numpy(),
               F19=F19.cpu().numpy())
    # E-field: all three components at 4096 random cells (the whole field is 3 GB at 512^3)
    rng = np.random.default_rng(0)
    nz, ny, nx = P.shape
    idx = rng.integers(0, nx * ny * nz, 4096)
    Ev = E.reshape(3, -1)[:, torch.from_numpy(idx).cuda()].cpu().numpy()
    out.update(E_idx=idx, E_vals=Ev)
    del E
    # the FP64 residual field of the final iterate at the same cells (h = 1: r = r~)
    _, rf = P.residual(field=True)
    out.update(r_vals=rf.reshape(-1)[torch.from_numpy(idx).cuda()].cpu().numpy())
    del rf
    P.close()
    return out


@pytest.mark.parametrize("name", ["spheres512", "spheres256"])
def test_benchmark_step_at_full_size(name):
    w = synth.WORKLOADS[name]
    g = _step(w)
    sp = g["sp"]
    # charge mapping: bit-exact
    rho_ref = oracle.sphere_density(tuple(reversed(w.dims)), w.h, sp.centers, sp.radius, sp.density, w.subsample)
    assert np.array_equal(g["rho"], rho_ref)
    # the solve: the oracle's relative residual of the GPU potential meets the tolerance (the
    # oracle sums in another order: 1e-3 relative slack on the residual itself)
    f = oracle.rhs(rho_ref, w.h, w.bc_type, w.bc_value)
    rel_ref = oracle.rel_residual(g["phi"], f, w.h, w.bc_type)
    assert g["rel"] < w.tol and rel_ref < w.tol * (1 + 1e-3)
    assert abs(rel_ref - g["rel"]) <= 1e-3 * g["rel"] + 1e-15
    # E-field and forces from the GPU potential, by the oracle
    E_ref = oracle.efield(g["phi"], w.h, w.bc_type, w.bc_value).reshape(3, -1)[:, g["E_idx"]]
    assert np.max(np.abs(g["E_vals"] - E_ref)) <= 1e-14 * np.max(np.abs(E_ref))
    F_ref = oracle.force_gather(g["phi"], w.h, w.bc_type, w.bc_value, sp.centers, sp.radius, sp.density,
                                w.subsample)
    assert np.max(np.abs(g["F"] - F_ref)) <= 1e-12 * np.max(np.abs(F_ref))
    F19_ref = oracle.force_gather(g["phi"], w.h, w.bc_type, w.bc_value, sp.centers, sp.radius, sp.density,
                                  w.subsample, stencil=19)
    assert np.max(np.abs(g["F19"] - F19_ref)) <= 1e-12 * np.max(np.abs(F19_ref))
    # sampled FP64 residuals against exact rational arithmetic on the GPU iterate: within
    # (8 + D)/32 of an ulp of the largest value among the five grid rows the residual walk reads for
    # the cell (rows j-1, j, j+1 of its plane, row j of the planes beside it) or of its f, plus half
    # an ulp of the result
    assert w.h == 1.0
    _assert_exact_residuals(g["phi"], f, w.bc_type, g["E_idx"], g["r_vals"])


def _assert_exact_residuals(phi, f, bc, idx, r_vals):
    from fractions import Fraction
    nz, ny, nx = phi.shape
    sh = {0: 1, 1: -1}
    R = np.abs(phi).max(axis=2)  # largest |phi| of each grid row (walls only: no row beyond them)
    for q, r in zip(idx, r_vals):
        k, rem = divmod(int(q), ny * nx)
        j, i = divmod(rem, nx)
        ops, d = [float(f[k, j, i]), float(phi[k, j, i])], 6
        for (ii, jj, kk, face) in ((i - 1, j, k, 0), (i + 1, j, k, 1), (i, j - 1, k, 2), (i, j + 1, k, 3),
                                   (i, j, k - 1, 4), (i, j, k + 1, 5)):
            if 0 <= ii < nx and 0 <= jj < ny and 0 <= kk < nz:
                ops.append(float(phi[kk, jj, ii]))
            else:
                d += sh[bc[face]]
        exact = Fraction(ops[0]) + sum(Fraction(v) for v in ops[2:]) - d * Fraction(ops[1])
        rows = [R[k, jj] for jj in (j - 1, j, j + 1) if 0 <= jj < ny] + [R[kk, j] for kk in (k - 1, k + 1) if 0 <= kk < nz]
        big = max(max(rows), abs(ops[0]))
        bound = Fraction(8 + d, 32) * Fraction(np.spacing(big)) + Fraction(np.spacing(abs(float(r)))) / 2
        assert abs(Fraction(float(r)) - exact) <= bound, (q, r, float(exact))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_no_charge_and_no_spheres(precision):
    """f = 0: the relative residual is 0 from the start, no cycle runs, phi stays 0; with no
    spheres the density is 0 and the force list is empty."""
    dims = (64, 48, 32)
    P = Poisson(dims, bc_type=synth.WALL_BC_TYPE, bc_value=(0.0,) * 6, precision=precision)
    empty = torch.empty(0, dtype=torch.float64, device="cuda")
    rho = P.sphere_density(empty.reshape(0, 3), empty, empty, 2)
    assert not torch.any(rho != 0)
    P.set_rhs(rho)
    P.set_solution(None)
    k, rel = P.solve(1e-9, 10)
    assert k == 0 and rel == 0.0
    assert not torch.any(P.solution() != 0)
    F = P.force_gather(empty.reshape(0, 3), empty, empty, 2)
    assert F.numel() == 0
    P.close()


def test_largest_grid_one_gpu():
    """1024^3 (2^30 cells, about 27 GB on the device): the mixed-precision step with 12 800 spheres
    reaches the tolerance, the FP64 residual of the result (mg_residual) agrees with the solve's
    own termination value, and the forces equal the oracle's forces of the GPU potential."""
    dims = (1024, 1024, 1024)
    h = 1.0
    bc_type, bc_value = synth.WALL_BC_TYPE, synth.wall_bc_value(1.0)
    sp = synth.random_spheres(dims, 12800, 4.0, 7, h)
    P = Poisson(dims, h=h, bc_type=bc_type, bc_value=bc_value, precision="mixed")
    c, r, q = _dev(sp.centers), _dev(sp.radius), _dev(sp.density)
    rho = P.sphere_density(c, r, q, 2)
    P.set_rhs(rho)
    del rho
    P.set_solution(None)
    k, rel = P.solve(1e-9, 20)
    assert rel < 1e-9 and 2 <= k <= 6
    rel64 = P.residual()
    assert abs(rel64 - rel) <= 1e-6 * rel
    F = P.force_gather(c, r, q, 2).cpu().numpy()
    phi = P.solution().cpu().numpy()
    P.close()
    F_ref = oracle.force_gather(phi, h, bc_type, bc_value, sp.centers, sp.radius, sp.density, 2)
    assert np.max(np.abs(F - F_ref)) <= 1e-12 * np.max(np.abs(F_ref))
