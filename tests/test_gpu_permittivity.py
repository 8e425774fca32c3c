"""Variable permittivity on the GPU (Sec. 3: Galerkin coarsening with averaging restriction and
constant prolongation extends the solver to discontinuous dielectricity) against the oracle:
the coefficients of every level bit for bit, the smoother's row property, the fused residual and
restriction, the coarse CG, V-cycles (1e-12), solves checked by the oracle's residual, the exact
layered-dielectric potential, and charged dielectric spheres between plates.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1410_6609_gb300 import synth
from paper_1410_6609_gb300._lib import MgError
from paper_1410_6609_gb300.solver import Poisson
from test_gpu_parity import cpu, gpu, maxrel, rel

pytestmark = pytest.mark.gpu

D, N, P = 0, 1, 2
TOL = 1e-12

CASES = [((48, 40, 24), (N, N, N, N, D, D)), ((12, 10, 14), (D, N, P, P, D, N)), ((32, 32, 32), (P, P, P, P, D, D))]


def _eps(dims, seed, lo=1.0, hi=80.0):
    nx, ny, nz = dims
    rng = np.random.default_rng(seed)
    return np.where(rng.random((nz, ny, nx)) < 0.4, hi, lo) * np.exp(0.1 * rng.standard_normal((nz, ny, nx)))


@pytest.mark.parametrize("dims,bc", CASES)
def test_coefficients_bit_exact(dims, bc):
    eps = _eps(dims, 1)
    Pz = Poisson(dims, bc_type=bc)
    Pz.set_permittivity(gpu(eps))
    assert Pz.has_permittivity
    for l in range(Pz.num_levels):
        ref = oracle.var_coeffs(eps, bc, l)
        for which in range(4):
            got = cpu(Pz.level_get(l, 2 + which))
            assert np.array_equal(got, ref[which]), (l, which)
    Pz.close()


@pytest.mark.parametrize("dims,bc", CASES)
def test_level_operations(dims, bc):
    h = 0.5
    eps = _eps(dims, 2)
    Pz = Poisson(dims, h=h, bc_type=bc)
    Pz.set_permittivity(gpu(eps))
    rng = np.random.default_rng(3)
    L = Pz.num_levels
    for l in range(L - 1):
        nx, ny, nz = Pz.level_dims(l)
        c = oracle.level_coeff(h, l)
        phi = rng.standard_normal((nz, ny, nx))
        f = rng.standard_normal((nz, ny, nx)) * c * 40.0
        kk, jj, ii = np.indices(phi.shape)
        for colour in (0, 1):
            Pz.level_set(l, 0, gpu(phi))
            Pz.level_set(l, 1, gpu(f))
            Pz.op_smooth(l, colour)
            got = cpu(Pz.level_get(l, 0))
            # the other colour is unchanged, and every row of this colour now holds exactly
            assert np.array_equal(got[(ii + jj + kk) % 2 != colour], phi[(ii + jj + kk) % 2 != colour])
            r = f - oracle.var_apply(got, eps, h, bc, l)
            assert np.abs(r[(ii + jj + kk) % 2 == colour]).max() < 1e-13 * np.abs(f).max(), (l, colour)
        Pz.level_set(l, 0, gpu(phi))
        Pz.level_set(l, 1, gpu(f))
        Pz.op_residual_restrict(l)
        ref = oracle.restrict(f - oracle.var_apply(phi, eps, h, bc, l))
        assert np.abs(cpu(Pz.level_get(l + 1, 1)) - ref).max() < 1e-13 * np.abs(f).max(), l
    # coarsest-level CG against a dense solve of the Galerkin operator
    nx, ny, nz = Pz.level_dims(L - 1)
    n = nx * ny * nz
    A = np.zeros((n, n))
    for q in range(n):
        e = np.zeros(n)
        e[q] = 1.0
        A[:, q] = oracle.var_apply(e.reshape(nz, ny, nx), eps, h, bc, L - 1).ravel()
    b = rng.standard_normal(n)
    Pz.level_set(L - 1, 1, gpu(b.reshape(nz, ny, nx)))
    Pz.op_coarse_solve()
    assert rel(cpu(Pz.level_get(L - 1, 0)).ravel(), np.linalg.solve(A, b)) < 1e-11
    Pz.close()


@pytest.mark.parametrize("dims,bc", CASES)
@pytest.mark.parametrize("ncycles", [1, 3])
def test_vcycles_match_oracle(dims, bc, ncycles):
    h = 1.0
    bcv = (0.1, -0.2, 0.3, 0.0, -1.0, 1.0)
    eps = _eps(dims, 4, hi=10.0)
    rho = synth.random_field(dims, 5)
    Pz = Poisson(dims, h=h, bc_type=bc, bc_value=bcv)
    Pz.set_permittivity(gpu(eps))
    Pz.set_rhs(gpu(rho))
    f = oracle.var_rhs(rho, eps, h, bc, bcv)
    assert maxrel(cpu(Pz.level_get(0, 1)), f) < 1e-15
    Pz.set_solution(None)
    Pz.vcycle(ncycles)
    ref = oracle.var_vcycles(np.zeros_like(f), f, eps, h, bc, ncycles)
    assert rel(cpu(Pz.solution()), ref) < TOL
    r_rel, r = Pz.residual(field=True)
    r_ref = f - oracle.var_apply(ref, eps, h, bc, 0)
    assert np.linalg.norm(cpu(r) - r_ref) / np.linalg.norm(f) < TOL
    assert abs(r_rel - np.linalg.norm(r_ref) / np.linalg.norm(f)) < TOL
    Pz.close()


def test_constant_permittivity_through_the_weighted_path():
    dims = (32, 32, 32)
    bc = synth.WALL_BC_TYPE
    bcv = synth.wall_bc_value(1.0)
    rho = synth.random_field(dims, 7)
    A = Poisson(dims, bc_type=bc, bc_value=bcv, eps=2.5)
    A.set_rhs(gpu(rho))
    ka, ra = A.solve(1e-12, 50)
    B = Poisson(dims, bc_type=bc, bc_value=bcv, eps=2.5)
    B.set_permittivity(gpu(np.full((32, 32, 32), 2.5)))
    B.set_rhs(gpu(rho))
    kb, rb = B.solve(1e-12, 50)
    assert abs(ka - kb) <= 1 and rel(cpu(B.solution()), cpu(A.solution())) < 1e-12
    B.set_permittivity(None)  # back to the constant operator
    assert not B.has_permittivity
    B.set_rhs(gpu(rho))
    B.set_solution(None)
    assert B.solve(1e-12, 50) == (ka, ra)
    A.close()
    B.close()


@pytest.mark.parametrize("h", [1.0, 0.25])
def test_layered_dielectric_between_plates(h):
    nx, ny, nz = 16, 8, 32
    e1, e2, V = 3.0, 40.0, 2.0
    L = nz * h
    eps = np.empty((nz, ny, nx))
    eps[: nz // 2] = e1
    eps[nz // 2:] = e2
    bc = (N, N, P, P, D, D)
    Pz = Poisson((nx, ny, nz), h=h, bc_type=bc, bc_value=(0.0, 0.0, 0.0, 0.0, 0.0, V))
    Pz.set_permittivity(gpu(eps))
    Pz.set_rhs(gpu(np.zeros((nz, ny, nx))))
    Pz.solve(1e-14, 200)
    q = V / ((L / 2) * (1 / e1 + 1 / e2))
    z = (np.arange(nz) + 0.5) * h
    exact = np.where(z < L / 2, q * z / e1, q * (L / 2) / e1 + q * (z - L / 2) / e2)
    assert np.abs(cpu(Pz.solution()) - exact[:, None, None]).max() < 1e-12 * V
    Pz.close()


def test_charged_dielectric_spheres_between_plates():
    """Charged spheres of permittivity 2 in a fluid of permittivity 80 (the dielectrophoresis
    setting the paper names), plates at 0 and 1: the solve reaches 1e-10 by the oracle's residual,
    and the forces on the spheres match the oracle's gather on the same potential."""
    dims = (64, 48, 56)
    bc = synth.WALL_BC_TYPE
    bcv = synth.wall_bc_value(1.0)
    sp = synth.random_spheres(dims, 12, 4.0, 9)
    vol = oracle.sphere_density((dims[2], dims[1], dims[0]), 1.0, sp.centers, sp.radius, np.ones(sp.count), 2)
    eps = 80.0 - 78.0 * vol  # volume-weighted permittivity of the partly covered cells
    rho = oracle.sphere_density((dims[2], dims[1], dims[0]), 1.0, sp.centers, sp.radius, sp.density, 2)
    Pz = Poisson(dims, bc_type=bc, bc_value=bcv)
    Pz.set_permittivity(gpu(eps))
    Pz.set_rhs(gpu(rho))
    k, r = Pz.solve(1e-10, 200)
    phi = cpu(Pz.solution())
    f = oracle.var_rhs(rho, eps, 1.0, bc, bcv)
    assert r < 1e-10 and oracle.var_rel_residual(phi, f, eps, 1.0, bc) < 1.0001e-10
    assert 5 < k < 60  # the Galerkin cycle converges on the contrast of 40
    F = cpu(Pz.force_gather(gpu(sp.centers), gpu(sp.radius), gpu(sp.density), 2))
    assert maxrel(F, oracle.force_gather(phi, 1.0, bc, bcv, sp.centers, sp.radius, sp.density, 2)) < 1e-12
    Pz.close()


def test_mixed_precision_weighted_operator():
    """The single-precision inner cycle on float copies of the weighted coefficients inside the
    FP64 defect correction: the dielectric-sphere problem reaches 1e-9 by the oracle's residual,
    the float half-sweep satisfies its rows to float rounding, and the coefficients kept for the
    outer residual are the FP64 ones."""
    dims = (64, 48, 56)
    nx, ny, nz = dims
    bc = synth.WALL_BC_TYPE
    bcv = synth.wall_bc_value(1.0)
    sp = synth.random_spheres(dims, 12, 4.0, 9)
    vol = oracle.sphere_density((nz, ny, nx), 1.0, sp.centers, sp.radius, np.ones(sp.count), 2)
    eps = 80.0 - 78.0 * vol
    rho = oracle.sphere_density((nz, ny, nx), 1.0, sp.centers, sp.radius, sp.density, 2)
    M = Poisson(dims, bc_type=bc, bc_value=bcv, precision="mixed")
    M.set_permittivity(gpu(eps))
    for which in range(4):
        assert np.array_equal(cpu(M.level_get(1, 2 + which)), oracle.var_coeffs(eps, bc, 1)[which])
    M.set_rhs(gpu(rho))
    k, r = M.solve(1e-9, 60)
    f = oracle.var_rhs(rho, eps, 1.0, bc, bcv)
    assert r < 1e-9 and oracle.var_rel_residual(cpu(M.solution()), f, eps, 1.0, bc) < 1.0001e-9 and k < 15
    # a float half-sweep on level 1
    rng = np.random.default_rng(5)
    l = 1
    lx, ly, lz = M.level_dims(l)
    c = oracle.level_coeff(1.0, l)
    phi = rng.standard_normal((lz, ly, lx)).astype(np.float32).astype(np.float64)
    g = (rng.standard_normal((lz, ly, lx)) * c * 40).astype(np.float32).astype(np.float64)
    M.level_set(l, 0, gpu(phi))
    M.level_set(l, 1, gpu(g))
    M.op_smooth(l, 0)
    got = cpu(M.level_get(l, 0))
    kk, jj, ii = np.indices(got.shape)
    res = g - oracle.var_apply(got, eps, 1.0, bc, l)
    assert np.abs(res[(ii + jj + kk) % 2 == 0]).max() < 1e-5 * np.abs(g).max()
    M.close()


def test_refusals():
    dims = (16, 16, 16)
    eps = gpu(_eps(dims, 3))
    Pz = Poisson(dims)
    Pz.set_permittivity(eps)
    with pytest.raises(MgError):
        Pz.op_residual_restrict(0, red_only=True)
    Pz.close()
    C = Poisson(dims)
    with pytest.raises(MgError):
        C.level_get(0, 2)  # no permittivity set
    C.close()


def test_vector_and_per_cell_float_sweeps_are_bit_identical():
    """The vectorised single-precision weighted half-sweep against the per-cell one (the process
    environment selects the per-cell kernel for a child process): identical iterates."""
    import subprocess
    import sys
    code = (
        "import numpy as np, torch\n"
        "from paper_1410_6609_gb300 import synth\n"
        "from paper_1410_6609_gb300.solver import Poisson\n"
        "dims = (64, 48, 40)\n"
        "rng = np.random.default_rng(8)\n"
        "eps = np.where(rng.random((40, 48, 64)) < 0.4, 80.0, 1.0)\n"
        "M = Poisson(dims, bc_type=(2, 2, 1, 1, 0, 0), bc_value=(0, 0, 0, 0, 0, 1), precision='mixed')\n"
        "M.set_permittivity(torch.from_numpy(eps).cuda())\n"
        "M.set_rhs(torch.from_numpy(synth.random_field(dims, 3)).cuda())\n"
        "M.set_solution(None)\n"
        "M.vcycle(2)\n"
        "np.save(__import__('sys').argv[1], M.solution().cpu().numpy())\n")
    import os
    import tempfile
    out = []
    with tempfile.TemporaryDirectory() as d:
        for mode in ("", "cell"):
            env = dict(os.environ, CCMG_VAR_SWEEP=mode)
            path = os.path.join(d, f"phi{mode}.npy")
            subprocess.run([sys.executable, "-c", code, path], check=True, env=env,
                           cwd=os.path.dirname(os.path.dirname(__file__)))
            out.append(np.load(path))
    assert np.array_equal(out[0], out[1])


def test_adjoint_with_variable_permittivity():
    """The right-hand-side adjoint of the weighted operator against the oracle, and gradients of
    J = sum of the z-forces through the differentiable chain (densities and wall values, the
    adjoint solve reusing the symmetric weighted operator) against central finite differences."""
    from paper_1410_6609_gb300.autograd import z_force_objective
    dims = (32, 32, 40)
    nx, ny, nz = dims
    bc = (D, N, P, P, D, D)
    bcv = np.array([0.3, 0.0, 0.0, 0.0, -0.5, 1.0])
    eps = _eps(dims, 7, hi=10.0)
    Pz = Poisson(dims, bc_type=bc, bc_value=tuple(bcv))
    Pz.set_permittivity(gpu(eps))
    lam = synth.random_field(dims, 8)
    grho, gbc = Pz.rhs_adjoint(gpu(lam))
    r_grho, r_gbc = oracle.var_rhs_adjoint(lam, eps, 1.0, bc)
    assert np.array_equal(cpu(grho), r_grho)
    assert maxrel(cpu(gbc), r_gbc) < 1e-13
    centers = np.array([[12.3, 16.0, 20.0], [22.0, 9.5, 14.2], [8.4, 24.6, 27.1]])
    radius = np.array([3.0, 2.5, 2.8])
    dens = torch.tensor([1.0, -0.7, 0.4], dtype=torch.float64, device="cuda", requires_grad=True)
    bcv_t = torch.tensor(bcv, dtype=torch.float64, device="cuda", requires_grad=True)
    c, r = gpu(centers), gpu(radius)
    J = z_force_objective(Pz, dens, bcv_t, c, r, 2, tol=1e-13, max_cycles=200)
    J.backward()

    def Jof(d, v):
        with torch.no_grad():
            return float(z_force_objective(Pz, d, v, c, r, 2, tol=1e-13, max_cycles=200))

    step = 1e-3
    for s_ in range(3):
        dp, dm = dens.detach().clone(), dens.detach().clone()
        dp[s_] += step
        dm[s_] -= step
        fd = (Jof(dp, bcv_t.detach()) - Jof(dm, bcv_t.detach())) / (2 * step)
        assert abs(fd - float(dens.grad[s_])) <= 1e-6 * max(1.0, abs(fd)), (s_, fd, float(dens.grad[s_]))
    for q in (0, 5):
        vp, vm = bcv_t.detach().clone(), bcv_t.detach().clone()
        vp[q] += step
        vm[q] -= step
        fd = (Jof(dens.detach(), vp) - Jof(dens.detach(), vm)) / (2 * step)
        assert abs(fd - float(bcv_t.grad[q])) <= 1e-6 * max(1.0, abs(fd)), (q, fd, float(bcv_t.grad[q]))
    Pz.close()
