"""mg_adjoint_solve through the C ABI against the oracle.

The adjoint system A lambda = g has homogeneous walls and the operator is symmetric, so the
oracle's lambda is its Algorithm 1 solve of the same g from zero (the operator of Sec. 2.4 with
the walls folded into the diagonal, its Galerkin coarse operators of Sec. 3; for a variable
permittivity the weighted operator). Same start and the same cycle count give the same state, so
the GPU's FP64 lambda must match to 1e-12; in mixed precision the oracle's own residual of the
GPU's lambda must be below the tolerance.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_1410_6609_gb300 import _lib, synth
from paper_1410_6609_gb300.solver import Poisson

pytestmark = pytest.mark.gpu

D, N, PER = 0, 1, 2


def _vp(t):
    return ctypes.c_void_p(t.data_ptr())


def _call(P, g, lam, tol, max_cycles=100):
    k, rel = ctypes.c_int(), ctypes.c_double()
    st = P.lib.mg_adjoint_solve(P.ctx, _vp(g), _vp(lam), tol, max_cycles, ctypes.byref(k), ctypes.byref(rel))
    return st, k.value, rel.value


@pytest.mark.parametrize("dims,h,bc_type,bcv", [
    ((48, 40, 32), 1.0, synth.WALL_BC_TYPE, synth.wall_bc_value(1.0)),
    ((40, 56, 48), 0.25, (N, D, D, N, N, D), (0.3, 2.0, -1.0, 0.5, 0.1, 4.0)),
    ((64, 32, 40), 1.0, (PER, PER, N, N, D, D), (0.0, 0.0, 0.2, 0.0, 0.0, 1.0)),
])
def test_adjoint_solve_fp64_matches_oracle_solve(dims, h, bc_type, bcv):
    nx, ny, nz = dims
    g = synth.random_field(dims, 31)
    P = Poisson(dims, h=h, bc_type=bc_type, bc_value=bcv)
    lam = torch.full((nz, ny, nx), float("nan"), dtype=torch.float64, device="cuda")
    st, k, rel = _call(P, torch.from_numpy(g).cuda(), lam, 1e-10)
    assert st == _lib.MG_OK, P.lib.mg_last_error(P.ctx)
    ref, k_ref, rel_ref = oracle.solve(g, h, bc_type, tol=1e-10)
    assert k == k_ref, (k, k_ref)
    lg = lam.cpu().numpy()
    assert np.linalg.norm(lg - ref) <= 1e-12 * np.linalg.norm(ref)
    assert abs(rel - rel_ref) <= 1e-12  # residuals relative to ||g||: the same state's residual to rounding
    # homogeneous walls: the forward problem's wall values were neither read nor changed, so a
    # forward solve afterwards equals one before
    rho = torch.from_numpy(synth.random_field(dims, 32)).cuda()
    fwd = []
    for _ in range(2):
        P.set_rhs(rho)
        P.set_solution(None)
        P.solve(1e-10, 100)
        fwd.append(P.solution())
        if len(fwd) == 1:
            assert _call(P, torch.from_numpy(g).cuda(), lam, 1e-10)[0] == _lib.MG_OK
    assert torch.equal(fwd[0], fwd[1])
    P.close()


def test_adjoint_solve_weighted_operator_matches_oracle():
    dims = (32, 40, 48)
    nx, ny, nz = dims
    bc_type = (N, N, D, N, D, D)
    rng = np.random.default_rng(7)
    eps = np.where(rng.random((nz, ny, nx)) < 0.3, 2.0, 80.0)
    g = synth.random_field(dims, 33)
    P = Poisson(dims, h=1.0, bc_type=bc_type, bc_value=(0.1, 0.0, 0.0, 0.2, 0.0, 1.0))
    P.set_permittivity(torch.from_numpy(eps).cuda())
    lam = torch.empty((nz, ny, nx), dtype=torch.float64, device="cuda")
    st, k, rel = _call(P, torch.from_numpy(g).cuda(), lam, 1e-10, 200)
    assert st == _lib.MG_OK
    ref, k_ref, _ = oracle.var_solve(g, eps, 1.0, bc_type, tol=1e-10, max_cycles=200)
    assert k == k_ref
    assert np.linalg.norm(lam.cpu().numpy() - ref) <= 1e-12 * np.linalg.norm(ref)
    P.close()


def test_adjoint_solve_mixed_reaches_tolerance_by_oracle_residual():
    dims = (64, 48, 40)
    bc_type = synth.WALL_BC_TYPE
    g = synth.random_field(dims, 34)
    P = Poisson(dims, bc_type=bc_type, bc_value=synth.wall_bc_value(1.0), precision="mixed")
    lam, k, rel = P.adjoint_solve(torch.from_numpy(g).cuda(), 1e-9, 50)
    assert rel < 1e-9
    rel_or = oracle.rel_residual(lam.cpu().numpy(), g, 1.0, bc_type)
    assert rel_or < 1.0001e-9, rel_or
    P.close()


def test_adjoint_solve_reports_a_missed_tolerance_and_rejects_bad_arguments():
    dims = (32, 32, 32)
    P = Poisson(dims)
    g = torch.from_numpy(synth.random_field(dims, 35)).cuda()
    lam = torch.empty_like(g)
    st, k, rel = _call(P, g, lam, 1e-12, 1)
    assert st == _lib.MG_ERR_NOT_CONVERGED and k == 1 and rel > 1e-12
    assert torch.isfinite(lam).all()
    assert P.lib.mg_adjoint_solve(P.ctx, None, _vp(lam), 1e-10, 10, None, None) == _lib.MG_ERR_INVALID
    assert _call(P, g, lam, -1.0)[0] == _lib.MG_ERR_INVALID
    assert _call(P, g, lam, 1e-10, -1)[0] == _lib.MG_ERR_INVALID
    P.close()
