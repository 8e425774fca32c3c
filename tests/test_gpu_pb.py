"""The screened (linearised Poisson-Boltzmann) and nonlinear Poisson-Boltzmann operators on the
GPU against the oracle: coefficients with the reaction term bit for bit, V-cycles (1e-12), the
shifted spectral solution, Newton's method (solution and the oracle's nonlinear residual), the
Gouy-Chapman double layer, and charged dielectric spheres in an electrolyte.
"""
import numpy as np
import pytest

import oracle
import spectral
from paper_1410_6609_gb300 import synth
from paper_1410_6609_gb300._lib import MgError
from paper_1410_6609_gb300.solver import Poisson
from test_gpu_parity import cpu, gpu, rel

pytestmark = pytest.mark.gpu

D, N, P = 0, 1, 2
CASES = [((48, 40, 24), (N, N, N, N, D, D)), ((12, 10, 14), (D, N, P, P, D, N)), ((32, 32, 32), (P, P, P, P, D, D))]


def _fields(dims, seed):
    nx, ny, nz = dims
    rng = np.random.default_rng(seed)
    eps = np.where(rng.random((nz, ny, nx)) < 0.3, 10.0, 1.0) * np.exp(0.1 * rng.standard_normal((nz, ny, nx)))
    k2 = np.where(eps > 5.0, 0.0, rng.random((nz, ny, nx)) * 2.0)  # no ions in the high-eps cells
    return eps, k2


@pytest.mark.parametrize("dims,bc", CASES)
def test_screened_coefficients_and_vcycles(dims, bc):
    h = 0.5
    eps, k2 = _fields(dims, 1)
    bcv = (0.1, -0.2, 0.3, 0.0, -1.0, 1.0)
    rho = synth.random_field(dims, 2)
    Pz = Poisson(dims, h=h, bc_type=bc, bc_value=bcv)
    Pz.set_permittivity(gpu(eps))
    Pz.set_reaction(gpu(k2))
    for l in range(Pz.num_levels):
        ref = oracle.var_coeffs(eps, bc, l, k2=k2, h=h)
        for which in range(4):
            assert np.array_equal(cpu(Pz.level_get(l, 2 + which)), ref[which]), (l, which)
    Pz.set_rhs(gpu(rho))
    Pz.set_solution(None)
    Pz.vcycle(3)
    f = oracle.var_rhs(rho, eps, h, bc, bcv)
    ref = oracle.var_vcycles(np.zeros_like(f), f, eps, h, bc, 3, k2=k2)
    assert rel(cpu(Pz.solution()), ref) < 1e-12
    k, r = Pz.solve(1e-11, 100)
    assert oracle.var_rel_residual(cpu(Pz.solution()), f, eps, h, bc, k2=k2) < 1.0001e-11
    Pz.close()


@pytest.mark.parametrize("kk", [0.05, 3.0])
def test_screened_constant_coefficients_spectral(kk):
    dims = (32, 24, 40)
    nx, ny, nz = dims
    bc = (P, P, N, N, D, D)
    f = synth.random_field(dims, 7)
    Pz = Poisson(dims, h=0.5, bc_type=bc, eps=1.0)
    Pz.set_reaction(gpu(np.full((nz, ny, nx), kk)))
    Pz.set_rhs(gpu(f))
    k, r = Pz.solve(1e-13, 60)
    assert rel(cpu(Pz.solution()), spectral.solve(f, 0.5, bc, shift=kk)) < 1e-11 and k < 20
    Pz.set_reaction(None)
    assert not Pz.has_permittivity  # back to the constant operator
    Pz.close()


def test_pb_newton_matches_oracle():
    dims = (32, 24, 40)
    nx, ny, nz = dims
    bc = (P, P, N, N, D, D)
    bcv = (0.0, 0.0, 0.0, 0.0, 2.0, -1.0)
    eps, k2 = _fields(dims, 3)
    rho = synth.random_field(dims, 4) * 4.0
    Pz = Poisson(dims, bc_type=bc, bc_value=bcv)
    Pz.set_permittivity(gpu(eps))
    Pz.set_reaction(gpu(k2))
    Pz.set_rhs(gpu(rho))
    Pz.set_solution(None)
    it, r = Pz.solve_pb(1e-11, 30, 1e-3, 30)
    phi = cpu(Pz.solution())
    f = oracle.var_rhs(rho, eps, 1.0, bc, bcv)
    _, r_or = oracle.pb_residual(phi, f, eps, k2, 1.0, bc)
    assert r < 1e-11 and r_or < 1.0001e-11 and it <= 12
    assert np.abs(phi).max() > 1.0  # the nonlinear regime
    ref, it_ref, _ = oracle.pb_newton(f, eps, k2, 1.0, bc, tol=1e-12)
    assert rel(phi, ref) < 1e-9
    # warm start from the converged potential: no step is needed
    assert Pz.solve_pb(1e-10, 30, 1e-3, 30)[0] == 0
    Pz.close()


def test_pb_gouy_chapman():
    phi0, kappa, Lz, nz = 2.0, 1.0, 12.0, 96
    h = Lz / nz
    nx, ny = 8, 8
    bc = (P, P, P, P, D, D)

    def gc(z):
        return 4.0 * np.arctanh(np.tanh(phi0 / 4.0) * np.exp(-kappa * z))

    Pz = Poisson((nx, ny, nz), h=h, bc_type=bc, bc_value=(0.0, 0.0, 0.0, 0.0, phi0, gc(Lz)))
    k2 = np.full((nz, ny, nx), kappa ** 2)
    Pz.set_reaction(gpu(k2))
    Pz.set_rhs(gpu(np.zeros((nz, ny, nx))))
    Pz.set_solution(None)
    it, r = Pz.solve_pb(1e-12, 30, 1e-4, 40)
    phi = cpu(Pz.solution())
    f = oracle.var_rhs(np.zeros((nz, ny, nx)), np.ones((nz, ny, nx)), h, bc, (0.0, 0.0, 0.0, 0.0, phi0, gc(Lz)))
    ref, _, _ = oracle.pb_newton(f, np.ones((nz, ny, nx)), k2, h, bc, tol=1e-13)
    assert rel(phi, ref) < 1e-10
    z = (np.arange(nz) + 0.5) * h
    assert np.abs(phi[:, 3, 5] - gc(z)).max() < 7e-3  # second-order discretisation error at h = 1/8
    Pz.close()


def test_charged_dielectric_spheres_in_an_electrolyte():
    """Charged spheres (eps 2, no ions inside) in an electrolyte (eps 80, Debye length 4 cells),
    plates at 0 and 1: Newton converges to 1e-10 by the oracle's nonlinear residual."""
    dims = (64, 48, 56)
    nx, ny, nz = dims
    bc = synth.WALL_BC_TYPE
    bcv = synth.wall_bc_value(1.0)
    sp = synth.random_spheres(dims, 12, 4.0, 9)
    vol = oracle.sphere_density((nz, ny, nx), 1.0, sp.centers, sp.radius, np.ones(sp.count), 2)
    eps = 80.0 - 78.0 * vol
    k2 = (1.0 - vol) * 80.0 / 4.0 ** 2
    rho = oracle.sphere_density((nz, ny, nx), 1.0, sp.centers, sp.radius, sp.density * 40.0, 2)
    Pz = Poisson(dims, bc_type=bc, bc_value=bcv)
    Pz.set_permittivity(gpu(eps))
    Pz.set_reaction(gpu(k2))
    Pz.set_rhs(gpu(rho))
    Pz.set_solution(None)
    it, r = Pz.solve_pb(1e-10, 30, 1e-3, 30)
    f = oracle.var_rhs(rho, eps, 1.0, bc, bcv)
    _, r_or = oracle.pb_residual(cpu(Pz.solution()), f, eps, k2, 1.0, bc)
    assert r < 1e-10 and r_or < 1.0001e-10 and it <= 15
    Pz.close()


def test_pb_mixed_precision_inner_cycles():
    """Newton with the single-precision inner cycle (MG_MIXED): the same converged potential as
    the FP64 Newton solve, checked by the oracle's nonlinear residual."""
    dims = (32, 24, 40)
    bc = (P, P, N, N, D, D)
    bcv = (0.0, 0.0, 0.0, 0.0, 2.0, -1.0)
    eps, k2 = _fields(dims, 3)
    rho = synth.random_field(dims, 4) * 4.0
    f = oracle.var_rhs(rho, eps, 1.0, bc, bcv)
    out = []
    for prec in ("fp64", "mixed"):
        Pz = Poisson(dims, bc_type=bc, bc_value=bcv, precision=prec)
        Pz.set_permittivity(gpu(eps))
        Pz.set_reaction(gpu(k2))
        Pz.set_rhs(gpu(rho))
        Pz.set_solution(None)
        it, r = Pz.solve_pb(1e-10, 30, 1e-3, 30)
        phi = cpu(Pz.solution())
        assert r < 1e-10 and oracle.pb_residual(phi, f, eps, k2, 1.0, bc)[1] < 1.0001e-10 and it <= 12, prec
        out.append(phi)
        Pz.close()
    assert rel(out[1], out[0]) < 1e-8


def test_pb_refusals():
    Pz = Poisson((16, 16, 16))
    with pytest.raises(MgError):
        Pz.solve_pb()  # no reaction term
    Pz.close()
