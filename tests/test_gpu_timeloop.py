"""The warm-started time loop of Sec. 8.1 on the GPU: every time step sets the right-hand side from
the spheres' new positions and runs a fixed number of V(3,3) cycles from the previous step's
potential (five at the first step, one afterwards), then gathers the forces; mg_step_host selects
this mode with a negative tolerance.

Checks: the host-buffer step equals, bit for bit, the same sequence of device calls; the relative
residual after each step stays bounded while the spheres move (FP64: one cycle contracts the
residual left by the step's new charge by its convergence rate, measured near 5e-4 at 128^3 with
spheres moving 0.07 cells per step; mixed precision: one outer step of four FP32 cycles, near
6e-8), and the forces stay close to those of a potential solved to 1e-12 at every step.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1410_6609_gb300 import synth  # noqa: E402
from paper_1410_6609_gb300._lib import MgError  # noqa: E402
from paper_1410_6609_gb300.solver import Poisson  # noqa: E402

pytestmark = pytest.mark.gpu

DIMS = (128, 128, 128)
VEL = 0.07  # cells per step along x


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _solver(prec):
    return Poisson(DIMS, bc_type=synth.WALL_BC_TYPE, bc_value=synth.wall_bc_value(1.0), precision=prec,
                   nu1=3, nu2=3)


@pytest.mark.parametrize("prec,rel_bound,force_bound", [("fp64", 1e-3, 2e-2), ("mixed", 1e-6, 1e-5)])
def test_time_loop_fixed_cycles(prec, rel_bound, force_bound):
    sp = synth.random_spheres(DIMS, 40, 4.0, 5)
    P, Q, R = _solver(prec), _solver(prec), _solver("fp64")
    c = sp.centers.copy()
    try:
        for t in range(12):
            c[:, 0] += VEL
            ncyc = 5 if t == 0 else 1
            F, k, rel = P.step_host(c, sp.radius, sp.density, 2, tol=-1.0, max_cycles=ncyc)
            assert k == ncyc
            # the same step through the device entry points
            rho = Q.sphere_density(_dev(c), _dev(sp.radius), _dev(sp.density), 2)
            Q.set_rhs(rho)
            Q.vcycle(ncyc)
            relq = Q.residual()
            Fq = Q.force_gather(_dev(c), _dev(sp.radius), _dev(sp.density), 2).cpu().numpy()
            assert np.array_equal(F, Fq)
            assert rel == relq
            if t > 0:
                assert rel < rel_bound, (t, rel)
            # a potential solved to 1e-12 for the same charge
            R.set_rhs(rho)
            R.set_solution(None)
            R.solve(1e-12, 100)
            Fr = R.force_gather(_dev(c), _dev(sp.radius), _dev(sp.density), 2).cpu().numpy()
            err = np.abs(F - Fr).max() / np.abs(Fr).max()
            assert err < force_bound, (t, err)
    finally:
        P.close()
        Q.close()
        R.close()


def test_time_loop_zero_cycles_and_bad_arguments():
    sp = synth.random_spheres((64, 64, 64), 6, 4.0, 3)
    P = Poisson((64, 64, 64), bc_type=synth.WALL_BC_TYPE, bc_value=synth.wall_bc_value(1.0))
    try:
        F, k, rel = P.step_host(sp.centers, sp.radius, sp.density, 2, tol=-1.0, max_cycles=0)
        assert k == 0 and rel == pytest.approx(1.0, rel=1e-12)  # zero iterate: the residual is the rhs
        assert np.all(np.isfinite(F))
        with pytest.raises(MgError):
            P.step_host(sp.centers, sp.radius, sp.density, 2, tol=float("nan"), max_cycles=1)
        with pytest.raises(MgError):
            P.step_host(sp.centers, sp.radius, sp.density, 2, tol=-1.0, max_cycles=-1)
    finally:
        P.close()
