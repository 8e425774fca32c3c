"""Adjoint gradients of J = sum_s F_s,z through the hand-written autograd functions, against the
oracle's gradient and against central finite differences of the GPU forward solve.

J is quadratic in the sphere densities and affine in the wall voltage, so central differences have
no truncation error; with forward solves to a 1e-13 relative residual and step 1e-6 the
differences are accurate to about 1e-7 of the gradient, well inside the 1e-5 bar.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1410_6609_gb300 import synth
from paper_1410_6609_gb300.autograd import z_force_objective
from paper_1410_6609_gb300.solver import Poisson

pytestmark = pytest.mark.gpu


def gpu(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def grads(P, sp, bcv, tol):
    q = gpu(sp.density).requires_grad_(True)
    v = gpu(bcv).requires_grad_(True)
    J = z_force_objective(P, q, v, gpu(sp.centers), gpu(sp.radius), 2, tol=tol)
    J.backward()
    return float(J.detach()), q.grad.cpu().numpy(), v.grad.cpu().numpy()


def test_autograd_matches_oracle_gradient():
    dims = (48, 40, 64)
    nx, ny, nz = dims
    sp = synth.random_spheres(dims, 8, 4.0, seed=5)
    bc = synth.WALL_BC_TYPE
    bcv = np.array(synth.wall_bc_value(1.0))
    P = Poisson(dims, bc_type=bc, bc_value=bcv)
    J, gq, gv = grads(P, sp, bcv, 1e-13)
    wF = np.zeros((sp.count, 3))
    wF[:, 2] = 1.0
    Jr, gqr, gvr, _ = oracle.force_objective_and_grad((nz, ny, nx), 1.0, bc, bcv, sp.centers, sp.radius,
                                                      sp.density, wF, tol=1e-13)
    assert abs(J - Jr) <= 1e-10 * abs(Jr)
    assert np.abs(gq - gqr).max() <= 1e-9 * np.abs(gqr).max()
    assert np.abs(gv - gvr).max() <= 1e-9 * np.abs(gvr).max()
    P.close()


def _fd_check(P_fwd, P_grad, w, sp, bcv, step=1e-6, bar=1e-5):
    c, r = gpu(sp.centers), gpu(sp.radius)
    J, gq, gv = grads(P_grad, sp, bcv, 1e-12)

    def Jof(dens, v):
        with torch.no_grad():
            return float(z_force_objective(P_fwd, gpu(dens), gpu(v), c, r, 2, tol=1e-13, max_cycles=300))

    fd = np.zeros(sp.count)
    for s in range(sp.count):
        dp, dm = sp.density.copy(), sp.density.copy()
        dp[s] += step
        dm[s] -= step
        fd[s] = (Jof(dp, bcv) - Jof(dm, bcv)) / (2 * step)
    vp, vm = bcv.copy(), bcv.copy()
    vp[5] += step
    vm[5] -= step
    fdv = (Jof(sp.density, vp) - Jof(sp.density, vm)) / (2 * step)
    scale = np.abs(fd).max()
    assert np.abs(gq - fd).max() <= bar * scale, np.abs(gq - fd).max() / scale
    assert abs(gv[5] - fdv) <= bar * abs(fdv), abs(gv[5] - fdv) / abs(fdv)
    return J, gq, gv


def test_adjoint256_fp64_and_mixed_vs_finite_differences():
    """Adjoint workload: 256^3, 32 charged spheres, z-wall voltage 1; dJ/d(densities, voltage)."""
    w = synth.WORKLOADS["adjoint256"]
    sp = w.spheres()
    bcv = np.array(w.bc_value)
    P64 = Poisson(w.dims, bc_type=w.bc_type, bc_value=bcv)
    _, gq64, gv64 = _fd_check(P64, P64, w, sp, bcv)
    Pm = Poisson(w.dims, bc_type=w.bc_type, bc_value=bcv, precision="mixed")
    q = gpu(sp.density).requires_grad_(True)
    v = gpu(bcv).requires_grad_(True)
    # FP32 cycles inside FP64 defect correction, refined to a 1e-11 relative residual: dJ/dV is a
    # small number (the total charge nearly cancels), so a 1e-9 solve leaves ~1e-5 relative error
    J = z_force_objective(Pm, q, v, gpu(sp.centers), gpu(sp.radius), 2, tol=1e-11)
    J.backward()
    gqm, gvm = q.grad.cpu().numpy(), v.grad.cpu().numpy()
    # mixed-precision gradient against the FP64 one, which matched the differences
    assert np.abs(gqm - gq64).max() <= 1e-5 * np.abs(gq64).max()
    assert abs(gvm[5] - gv64[5]) <= 1e-5 * abs(gv64[5])
    P64.close()
    Pm.close()
