"""The warm-started time loop of Sec. 8.1 on the GPU: every time step sets the right-hand side from
the spheres' new positions and runs a fixed number of V(3,3) cycles from the previous step's
potential (five at the first step, one afterwards), then gathers the forces; mg_step_host selects
this mode with a negative tolerance.

Checks: each step against the oracle continuing from its own previous state (the same cycles from
the previous potential, Sec. 8.1); the host-buffer step equals, bit for bit, the same sequence of
device calls; the relative
residual after each step stays bounded while the spheres move (FP64: one cycle contracts the
residual left by the step's new charge by its convergence rate, measured near 5e-4 at 128^3 with
spheres moving 0.07 cells per step; mixed precision: one outer step of four FP32 cycles, near
6e-8), and the forces stay close to those of a potential solved to 1e-12 at every step.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
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


# Sec. 8.1: five cycles at the first time step, then one per step from the previous potential.
# The oracle runs the same cycles from ITS previous state (never from the GPU's), so a fault that
# only the time loop can hit (the warm start's packing of the potential into the checkerboard
# levels, a zero-start flag left set, a stale defect-correction scale) shows up as a difference.
@pytest.mark.parametrize("walls", ["plates", "periodic_xy"])
@pytest.mark.parametrize("vel", [0.07, 2.8])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_time_loop_against_oracle(prec, vel, walls):
    dims = (48, 40, 32)
    nx, ny, nz = dims
    h = 1.0
    if walls == "plates":
        bc, bcv = synth.WALL_BC_TYPE, synth.wall_bc_value(1.0)
    else:
        bc, bcv = (2, 2, 2, 2, 0, 0), (0.0, 0.0, 0.0, 0.0, 0.0, 1.0)
    sp = synth.random_spheres(dims, 6, 3.0, 11)
    P = Poisson(dims, h=h, bc_type=bc, bc_value=bcv, precision=prec, nu1=3, nu2=3)
    phi_or = np.zeros((nz, ny, nx))
    try:
        for t in range(6):
            c = sp.centers.copy()
            if walls == "periodic_xy":  # through the periodic x wall and on
                c[:, 0] = np.mod(c[:, 0] + vel * (t + 1), nx * h)
            else:  # back and forth, the spheres staying inside the walls
                c[:, 0] += vel * (0.5 if t % 2 == 0 else -0.5)
            ncyc = 5 if t == 0 else 1
            F, k, rel = P.step_host(c, sp.radius, sp.density, 2, tol=-1.0, max_cycles=ncyc)
            assert k == ncyc
            phi = P.solution().cpu().numpy()
            rho = oracle.sphere_density((nz, ny, nx), h, c, sp.radius, sp.density, 2, bc_type=bc)
            f = oracle.rhs(rho, h, bc, bcv)
            if prec == "fp64":
                phi_or, _ = oracle.vcycles(phi_or, f, h, bc, ncyc, nu1=3, nu2=3)
                err = np.linalg.norm(phi - phi_or) / np.linalg.norm(phi_or)
                assert err <= 1e-12, (t, err)
            else:
                # single-precision inner cycles round differently from the oracle's (and their
                # coarsest CGs, both in float to 1e-5, reduce in different orders), so the mixed
                # states agree to that level; the GPU's reported FP64 residual is checked against
                # the oracle's residual of the GPU's own potential
                phi_or, _, _ = oracle.solve_mixed(f, h, bc, tol=0.0, max_cycles=ncyc, nu1=3, nu2=3, phi0=phi_or)
                err = np.linalg.norm(phi - phi_or) / np.linalg.norm(phi_or)
                assert err <= 3e-5, (t, err)
                rel_or = oracle.rel_residual(phi, f, h, bc)
                # both relative to ||f||: the same potential's residual agrees to rounding (after
                # the first step's five outer steps it is itself at the rounding level, 1e-15)
                assert abs(rel - rel_or) <= 1e-12, (t, rel, rel_or)
            Fr = oracle.force_gather(phi_or, h, bc, bcv, c, sp.radius, sp.density, 2)
            ferr = np.abs(F - Fr).max() / np.abs(Fr).max()
            assert ferr <= (1e-12 if prec == "fp64" else 3e-5), (t, ferr)
            if prec == "fp64":
                assert abs(rel - oracle.rel_residual(phi_or, f, h, bc)) <= 1e-12
    finally:
        P.close()
