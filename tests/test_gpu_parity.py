"""Parity of the CUDA path (through the C ABI) with the CPU oracle, kernel by kernel and cycle by
cycle, on seeded inputs. FP64 tolerance: 1e-12 relative in solution and residual (the method is
the same algorithm; only rounding order differs: reciprocal multiply for the diagonal, FMA
contraction, tree reductions). Integer decisions (sub-cell counts) are bit-exact.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1410_6609_gb300 import synth
from paper_1410_6609_gb300.solver import Poisson

pytestmark = pytest.mark.gpu

D, N, PER = 0, 1, 2
TOL = 1e-12


def gpu(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def cpu(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def maxrel(a, b):
    m = np.abs(b).max()
    return np.abs(a - b).max() / (m if m > 0 else 1.0)


# (nx, ny, nz) cases: a ragged multi-block case with 5 levels and an odd coarsest grid, a small
# non-cubic one, and the 32^3 manufactured grid.
CASES = [((144, 80, 48), (N, N, N, N, D, D)), ((12, 10, 14), (D, N, N, D, D, N)), ((32, 32, 32), (D,) * 6)]


@pytest.mark.parametrize("dims,bc", CASES)
def test_level_operations_match_oracle(dims, bc):
    h = 0.5
    P = Poisson(dims, h=h, bc_type=bc)
    L = P.num_levels
    assert [tuple(P.level_dims(l)) for l in range(L)] == oracle.levels(*dims)
    rng = np.random.default_rng(1)
    for l in range(L - 1):
        nx, ny, nz = P.level_dims(l)
        c = oracle.level_coeff(h, l)
        phi = rng.standard_normal((nz, ny, nx))
        f = rng.standard_normal((nz, ny, nx)) * c
        for colour in (0, 1):
            P.level_set(l, 0, gpu(phi))
            P.level_set(l, 1, gpu(f))
            P.op_smooth(l, colour)
            got = cpu(P.level_get(l, 0))
            ref = oracle.rbgs_half(phi, f, c, bc, colour)
            assert maxrel(got, ref) < 1e-14, (l, colour)
        # fused residual + restriction
        P.level_set(l, 0, gpu(phi))
        P.level_set(l, 1, gpu(f))
        P.op_residual_restrict(l)
        got = cpu(P.level_get(l + 1, 1))
        ref = oracle.restrict(oracle.residual(phi, f, c, bc))
        assert maxrel(got, ref) < 1e-13, l
        # prolongation with the x2 correction
        ec = rng.standard_normal(tuple(reversed(P.level_dims(l + 1))))
        P.level_set(l, 0, gpu(phi))
        P.level_set(l + 1, 0, gpu(ec))
        P.op_prolong_correct(l)
        got = cpu(P.level_get(l, 0))
        assert maxrel(got, oracle.prolong_correct(phi, ec, 2.0)) < 1e-15
    # coarsest-grid CG
    nx, ny, nz = P.level_dims(L - 1)
    cL = oracle.level_coeff(h, L - 1)
    b = rng.standard_normal((nz, ny, nx))
    P.level_set(L - 1, 1, gpu(b))
    its = P.op_coarse_solve()
    x_ref, it_ref = oracle.cg(b, cL, bc)
    assert rel(cpu(P.level_get(L - 1, 0)), x_ref) < 1e-12
    assert abs(its - it_ref) <= 2
    P.close()


@pytest.mark.parametrize("dims,bc", CASES)
@pytest.mark.parametrize("ncycles", [1, 3])
def test_vcycles_match_oracle(dims, bc, ncycles):
    nx, ny, nz = dims
    h = 1.0
    bcv = (0.1, -0.2, 0.3, 0.0, -1.0, 1.0)
    rho = synth.random_field(dims, seed=5)
    P = Poisson(dims, h=h, bc_type=bc, bc_value=bcv)
    P.set_rhs(gpu(rho))
    P.set_solution(None)
    P.vcycle(ncycles)
    got = cpu(P.solution())
    f = oracle.rhs(rho, h, bc, bcv)
    ref, _ = oracle.vcycles(np.zeros_like(f), f, h, bc, ncycles)
    assert rel(got, ref) < TOL
    # residual of the same state, relative to ||f||
    r_rel, r = P.residual(field=True)
    r_ref = oracle.residual(ref, f, oracle.level_coeff(h, 0), bc)
    assert np.linalg.norm(cpu(r) - r_ref) / np.linalg.norm(f) < TOL
    assert abs(r_rel - np.linalg.norm(r_ref) / np.linalg.norm(f)) < TOL
    P.close()


def test_manufactured_solution_to_1e10():
    """32^3, h = 1/32, homogeneous Dirichlet, f = 3 pi^2 sin sin sin: V(2,2) over 4 levels to a
    1e-10 relative residual; the O(h^2) error is the closed form (x/sin x)^2 - 1, x = pi h/2."""
    f, h = synth.manufactured_rhs(32)
    P = Poisson((32, 32, 32), h=h, bc_type=(D,) * 6)
    assert P.num_levels == 4 and P.level_dims(3) == (4, 4, 4)
    P.set_rhs(gpu(f))
    k, r = P.solve(1e-10, 50)
    phi = cpu(P.solution())
    ref, k_ref, r_ref = oracle.solve(f, h, (D,) * 6, tol=1e-10)
    assert k == k_ref and r < 1e-10
    assert rel(phi, ref) < TOL
    u = synth.manufactured_exact(32)
    x = np.pi * h / 2
    err = np.linalg.norm(phi - u) / np.linalg.norm(u)
    assert abs(err - ((x / np.sin(x)) ** 2 - 1)) < 1e-6 * err + 1e-9
    P.close()


def _spheres_case(dims, count, seed, R=4.0):
    sp = synth.random_spheres(dims, count, R, seed)
    return sp, gpu(sp.centers), gpu(sp.radius), gpu(sp.density)


@pytest.mark.parametrize("sf", [1, 2, 3])
def test_sphere_density_bit_exact(sf):
    dims = (96, 64, 80)
    sp, c, r, q = _spheres_case(dims, 25, 7, R=3.5)
    P = Poisson(dims, bc_type=synth.WALL_BC_TYPE)
    got = cpu(P.sphere_density(c, r, q, sf))
    ref = oracle.sphere_density((dims[2], dims[1], dims[0]), 1.0, sp.centers, sp.radius, sp.density, sf)
    assert np.array_equal(got, ref)
    P.close()


def test_efield_and_forces_match_oracle():
    dims = (64, 48, 80)
    bc = synth.WALL_BC_TYPE
    bcv = (0.0, 0.0, 0.0, 0.0, 0.0, 1.0)
    sp, c, r, q = _spheres_case(dims, 12, 3)
    phi = synth.random_field(dims, 9)
    P = Poisson(dims, bc_type=bc, bc_value=bcv)
    P.set_solution(gpu(phi))
    E = cpu(P.efield())
    Eref = oracle.efield(phi, 1.0, bc, bcv)
    assert maxrel(E, Eref) < 1e-15
    F = cpu(P.force_gather(c, r, q, 2))
    Fref = oracle.force_gather(phi, 1.0, bc, bcv, sp.centers, sp.radius, sp.density, 2)
    assert maxrel(F, Fref) < 1e-12
    # walls touched by the E-field stencil: Neumann slope and Dirichlet on x
    bc2 = (D, N, N, N, D, D)
    bcv2 = (0.3, -0.7, 0.2, 0.0, -1.0, 1.0)
    P2 = Poisson(dims, bc_type=bc2, bc_value=bcv2)
    P2.set_solution(gpu(phi))
    assert maxrel(cpu(P2.efield()), oracle.efield(phi, 1.0, bc2, bcv2)) < 1e-15
    P.close()
    P2.close()


@pytest.mark.parametrize("h", [0.5, 0.3])
def test_efield_differences_bit_exact(h):
    """The central differences of the E-field, E = (phi(x - 1) - phi(x + 1)) / (2h) per axis, bit for
    bit against the IEEE double subtraction (numpy) on every interior cell, for potentials chosen
    to exercise the rounding of the differences: magnitudes spread over 2^-600 .. 2^600 with zeros of both signs, subnormals, neighbours equal
    or a few ulps apart (cancellation), values near the largest double (overflow to infinity), and
    an infinity. With h = 0.5 the factor 1/(2h) is 1; with h = 0.3 it is a rounded FP64 product.
    Rows of 128 packed columns, so that the warps away from the x walls take the interior path;
    the sign of a zero difference is not compared (the wall path forms it as -(phi(x+1) - phi(x-1)))."""
    dims = (256, 24, 16)
    nx, ny, nz = dims
    rng = np.random.default_rng(31)
    phi = rng.standard_normal((nz, ny, nx)) * np.exp2(rng.integers(-600, 601, (nz, ny, nx)).astype(float))
    u = rng.random(phi.shape)
    phi[u < 0.05] = 0.0
    phi[(u >= 0.05) & (u < 0.08)] = -0.0
    phi[(u >= 0.08) & (u < 0.11)] = rng.integers(-50, 50, int(((u >= 0.08) & (u < 0.11)).sum())) * 5e-324
    # x neighbours two apart equal, or a few ulps apart
    sel = (u >= 0.11) & (u < 0.2)
    kk, jj, ii = np.nonzero(sel)
    ok = ii + 2 < nx
    kk, jj, ii = kk[ok], jj[ok], ii[ok]
    steps = rng.integers(-3, 4, kk.size)
    phi[kk, jj, ii + 2] = phi[kk, jj, ii] + steps * np.spacing(phi[kk, jj, ii])
    big = (u >= 0.2) & (u < 0.22)
    phi[big] = np.sign(rng.standard_normal(int(big.sum()))) * 1.7e308
    phi[nz // 2, ny // 2, nx // 2] = np.inf
    P = Poisson(dims, h=h, bc_type=(D,) * 6)
    P.set_solution(gpu(phi))
    E = cpu(P.efield())
    P.close()
    inv2h = 1.0 / (2.0 * h)
    with np.errstate(over="ignore", invalid="ignore"):
        ref = [(phi[1:-1, 1:-1, :-2] - phi[1:-1, 1:-1, 2:]), (phi[1:-1, :-2, 1:-1] - phi[1:-1, 2:, 1:-1]),
               (phi[:-2, 1:-1, 1:-1] - phi[2:, 1:-1, 1:-1])]
        ref = [r if h == 0.5 else r * inv2h for r in ref]
    for a in range(3):
        got, want = E[a][1:-1, 1:-1, 1:-1], ref[a]
        nan = np.isnan(want)
        assert np.array_equal(np.isnan(got), nan), a
        g_, w_ = np.where(got == 0, 0.0, got)[~nan], np.where(want == 0, 0.0, want)[~nan]
        assert np.array_equal(g_.view(np.uint64), w_.view(np.uint64)), (a, int((g_ != w_).sum()))


@pytest.mark.parametrize("h", [1.0, 0.3])
def test_d3q19_efield_and_forces_match_oracle(h):
    """The D3Q19 gradient (Sec. 2.4) where all 18 neighbours exist, D3Q7 elsewhere: the GPU repeats
    the oracle's per-cell operations, so interior E values are bit-identical; forces (sums over
    cells in another order) to 1e-12. A non-power-of-two h exercises the division path. The
    force adjoint refuses this stencil; other stencil values are rejected."""
    dims = (40, 36, 32)
    bc = (D, N, N, N, D, D)
    bcv = (0.3, -0.7, 0.2, 0.0, -1.0, 1.0)
    sp, c, r, q = _spheres_case(dims, 8, 4)
    phi = synth.random_field(dims, 13)
    P = Poisson(dims, h=h, bc_type=bc, bc_value=bcv)
    assert P.gradient_stencil == 7
    P.gradient_stencil = 19
    assert P.gradient_stencil == 19
    P.set_solution(gpu(phi))
    E = cpu(P.efield())
    Eref = oracle.efield(phi, h, bc, bcv, stencil=19)
    assert np.array_equal(E[:, 1:-1, 1:-1, 1:-1], Eref[:, 1:-1, 1:-1, 1:-1])
    assert maxrel(E, Eref) < 1e-15
    assert maxrel(E, oracle.efield(phi, h, bc, bcv, stencil=7)) > 1e-3  # the stencils differ on this field
    cs, rs = sp.centers * h, sp.radius * h
    F = cpu(P.force_gather(gpu(cs), gpu(rs), q, 2))
    Fref = oracle.force_gather(phi, h, bc, bcv, cs, rs, sp.density, 2, stencil=19)
    assert maxrel(F, Fref) < 1e-12
    with pytest.raises(Exception):
        P.gradient_stencil = 5
    assert P.gradient_stencil == 19
    with pytest.raises(Exception):
        P.force_gather_adjoint(gpu(cs), gpu(rs), q, gpu(np.ones((len(rs), 3))), 2)
    P.gradient_stencil = 7
    assert maxrel(cpu(P.efield()), oracle.efield(phi, h, bc, bcv)) < 1e-15
    P.close()


def test_adjoint_kernels_match_oracle():
    dims = (32, 32, 40)
    bc = (D, N, N, N, D, D)
    bcv = (0.5, 0.1, 0.0, 0.0, 0.0, 1.0)
    # spheres close to the walls so the ghost terms are exercised
    centers = np.array([[2.2, 16.0, 20.0], [16.0, 30.1, 1.7], [20.3, 11.2, 38.4], [12.0, 12.0, 12.0]])
    radius = np.array([2.5, 2.0, 2.2, 3.0])
    dens = np.array([1.0, -0.7, 0.4, 0.9])
    wF = np.random.default_rng(2).standard_normal((4, 3))
    phi = synth.random_field(dims, 4)
    P = Poisson(dims, bc_type=bc, bc_value=bcv)
    P.set_solution(gpu(phi))
    gphi, gd, gbc = P.force_gather_adjoint(gpu(centers), gpu(radius), gpu(dens), gpu(wF), 2)
    r_gphi, r_gd, r_gbc = oracle.force_gather_adjoint(phi, 1.0, bc, bcv, centers, radius, dens, wF, 2)
    assert maxrel(cpu(gphi), r_gphi) < 1e-13
    assert maxrel(cpu(gd), r_gd) < 1e-12
    assert maxrel(cpu(gbc), r_gbc) < 1e-12
    gfield = synth.random_field(dims, 6)
    got = cpu(P.sphere_density_adjoint(gpu(centers), gpu(radius), gpu(gfield), 2))
    assert maxrel(got, oracle.sphere_density_adjoint(gfield, 1.0, centers, radius, 2)) < 1e-13
    lam = synth.random_field(dims, 8)
    grho, gbc2 = P.rhs_adjoint(gpu(lam))
    r_grho, r_gbc2 = oracle.rhs_adjoint(lam, 1.0, bc)
    assert maxrel(cpu(grho), r_grho) == 0.0
    assert maxrel(cpu(gbc2), r_gbc2) < 1e-13
    P.close()


def test_mixed_precision_reaches_tolerance():
    dims = (64, 64, 64)
    bc = synth.WALL_BC_TYPE
    bcv = synth.wall_bc_value(1.0)
    sp = synth.random_spheres(dims, 20, 4.0, 17)
    rho = oracle.sphere_density((64, 64, 64), 1.0, sp.centers, sp.radius, sp.density, 2)
    f = oracle.rhs(rho, 1.0, bc, bcv)
    P = Poisson(dims, bc_type=bc, bc_value=bcv, precision="mixed")
    P.set_rhs(gpu(rho))
    k, r = P.solve(1e-9, 50)
    phi = cpu(P.solution())
    assert r < 1e-9
    assert oracle.rel_residual(phi, f, 1.0, bc) < 1.0001e-9  # checked independently on the CPU
    ref, k_ref, _ = oracle.solve_mixed(f, 1.0, bc, tol=1e-9)
    assert abs(k - k_ref) <= 1
    ref64, _, _ = oracle.solve(f, 1.0, bc, tol=1e-12)
    assert rel(phi, ref64) < 1e-7
    P.close()


def test_step_host_matches_device_path():
    dims = (64, 64, 48)
    bc = synth.WALL_BC_TYPE
    bcv = synth.wall_bc_value(1.0)
    sp, c, r, q = _spheres_case(dims, 10, 23)
    P = Poisson(dims, bc_type=bc, bc_value=bcv)
    F, k, rel_res = P.step_host(sp.centers, sp.radius, sp.density, 2, 1e-10, 50)
    assert rel_res < 1e-10 and k > 0
    P2 = Poisson(dims, bc_type=bc, bc_value=bcv)
    P2.set_rhs(P2.sphere_density(c, r, q, 2))
    P2.solve(1e-10, 50)
    F2 = cpu(P2.force_gather(c, r, q, 2))
    assert np.array_equal(F, F2)
    P.close()
    P2.close()


def test_single_level_grid_is_a_cg_solve():
    dims = (4, 4, 6)  # 4/2 = 2 < 3: the finest grid is the coarsest
    bc = (D, N, N, D, D, N)
    rho = synth.random_field(dims, 2)
    P = Poisson(dims, bc_type=bc)
    assert P.num_levels == 1
    P.set_rhs(gpu(rho))
    k, r = P.solve(1e-12, 5)
    f = oracle.rhs(rho, 1.0, bc, (0.0,) * 6)
    ref, _, _ = oracle.solve(f, 1.0, bc, tol=1e-12)
    assert rel(cpu(P.solution()), ref) < TOL and k == 1
    P.close()


def test_solve_reports_not_converged():
    f, h = synth.manufactured_rhs(32)
    P = Poisson((32, 32, 32), h=h)
    P.set_rhs(gpu(f))
    k, r = P.solve(1e-10, 2, raise_on_fail=False)
    assert k == 2 and r > 1e-10
    from paper_1410_6609_gb300._lib import MgError
    P.set_solution(None)
    with pytest.raises(MgError):
        P.solve(1e-10, 1)
    P.close()


@pytest.mark.parametrize("dims,bc", CASES[:2])
def test_single_precision_level_operations_match_oracle(dims, bc):
    """The FP32 kernels of the mixed-precision inner cycle against the oracle's single-precision
    level operations. Both round in float; the GPU multiplies by 1/(6+d) where the oracle
    divides and contracts with FMA, so agreement is to a few float ulps (rel. 1e-6)."""
    h = 0.5
    P = Poisson(dims, h=h, bc_type=bc, precision="mixed")
    rng = np.random.default_rng(3)
    tol = 1e-6
    for l in range(P.num_levels - 1):
        nx, ny, nz = P.level_dims(l)
        c = oracle.level_coeff(h, l)
        phi = rng.standard_normal((nz, ny, nx)).astype(np.float32).astype(np.float64)
        f = (rng.standard_normal((nz, ny, nx)) * c).astype(np.float32).astype(np.float64)
        for colour in (0, 1):
            P.level_set(l, 0, gpu(phi))
            P.level_set(l, 1, gpu(f))
            P.op_smooth(l, colour)
            assert maxrel(cpu(P.level_get(l, 0)), oracle.rbgs_half_f32(phi, f, c, bc, colour)) < tol
        P.level_set(l, 0, gpu(phi))
        P.level_set(l, 1, gpu(f))
        P.op_residual_restrict(l)
        ref = oracle.restrict_f32(oracle.residual_f32(phi, f, c, bc))
        # the residual cancels O(1) terms to O(1) results: compare against the operands' scale
        assert np.abs(cpu(P.level_get(l + 1, 1)) - ref).max() < tol * 8 * np.abs(f).max()
        # the red-only variant of the cycle: the same restriction with the black residuals dropped
        P.level_set(l, 0, gpu(phi))
        P.level_set(l, 1, gpu(f))
        P.op_residual_restrict(l, red_only=True)
        res = oracle.residual_f32(phi, f, c, bc)
        kk, jj, ii = np.indices(res.shape)
        res[(ii + jj + kk) % 2 == 1] = 0.0
        ref_red = oracle.restrict_f32(res)
        assert np.abs(cpu(P.level_get(l + 1, 1)) - ref_red).max() < tol * 8 * np.abs(f).max()
        assert np.abs(ref_red - ref).max() > 1e-3 * np.abs(ref).max()  # the variants differ on this data
        ec = rng.standard_normal(tuple(reversed(P.level_dims(l + 1)))).astype(np.float32).astype(np.float64)
        P.level_set(l, 0, gpu(phi))
        P.level_set(l + 1, 0, gpu(ec))
        P.op_prolong_correct(l)
        assert maxrel(cpu(P.level_get(l, 0)), oracle.prolong_correct_f32(phi, ec, 2.0)) == 0.0
    # the coarsest CG of the single-precision cycle: in float, to 1e-5 (the GPU reduces in a
    # different order, so the iterates agree to the tolerance, not bit for bit)
    L = P.num_levels
    nx, ny, nz = P.level_dims(L - 1)
    cL = oracle.level_coeff(h, L - 1)
    b = (rng.standard_normal((nz, ny, nx)) * cL).astype(np.float32).astype(np.float64)
    P.level_set(L - 1, 1, gpu(b))
    its = P.op_coarse_solve()
    x = cpu(P.level_get(L - 1, 0))
    x_ref, it_ref = oracle.cg_f32(b, cL, bc)
    x64, _ = oracle.cg(b, cL, bc)
    assert abs(its - it_ref) <= 3, (its, it_ref)
    assert rel(x, x64) < 1e-4 and rel(x_ref.astype(np.float64), x64) < 1e-4
    P.close()


@pytest.mark.parametrize("nu1,nu2,omega,h,eps,bc", [
    (1, 1, 2.0, 1.0, 1.0, (N, N, N, N, D, D)),
    (3, 3, 2.0, 0.3, 2.5, (D,) * 6),                      # V(3,3) (the paper's production cycle), h not a power of 2
    (2, 2, 1.0, 1.0, 1.0, (D, N, N, D, D, N)),            # plain (unmagnified) correction
    (0, 2, 2.0, 1.0, 1.0, (N, N, N, N, N, D)),            # no pre-smoothing; five Neumann walls
    (2, 1, 1.7, 0.125, 78.5, (N, D, N, D, D, N)),
])
def test_cycle_variants_match_oracle(nu1, nu2, omega, h, eps, bc):
    dims = (48, 32, 40)
    bcv = (0.2, -0.1, 0.05, 0.3, -0.4, 0.6)
    rho = synth.random_field(dims, seed=13)
    P = Poisson(dims, h=h, bc_type=bc, bc_value=bcv, nu1=nu1, nu2=nu2, cgc_weight=omega, eps=eps)
    P.set_rhs(gpu(rho))
    P.set_solution(None)
    P.vcycle(3)
    f = oracle.rhs(rho, h, bc, bcv, eps)
    ref, _ = oracle.vcycles(np.zeros_like(f), f, h, bc, 3, nu1=nu1, nu2=nu2, omega=omega)
    assert rel(cpu(P.solution()), ref) < TOL
    rr, r = P.residual(field=True)
    assert np.linalg.norm(cpu(r) - oracle.residual(ref, f, oracle.level_coeff(h, 0), bc)) / np.linalg.norm(f) < TOL
    P.close()


def test_warm_start_continues_the_iteration():
    """mg_set_solution restarts from a given potential (warm start of later time steps): k cycles
    then k more from the saved state equal 2k cycles."""
    dims = (32, 32, 32)
    bc = synth.WALL_BC_TYPE
    rho = synth.random_field(dims, seed=4)
    P = Poisson(dims, bc_type=bc, bc_value=synth.wall_bc_value(1.0))
    P.set_rhs(gpu(rho))
    P.set_solution(None)
    P.vcycle(2)
    mid = P.solution().clone()
    P.vcycle(2)
    full = P.solution().clone()
    P.set_solution(mid)
    P.vcycle(2)
    assert torch.equal(P.solution(), full)
    P.close()


@pytest.mark.parametrize("defect", ["walk", None])
def test_zero_start_without_writing_the_iterate(defect):
    """In mixed precision mg_set_solution(NULL) writes nothing (the first cycle stores phi = s e);
    every call that reads phi before the solve equals that of an explicit zero field, and so does
    the solve where every outer step evaluates its residual directly (CCMG_DEFECT=walk). By
    default a solve from the unwritten zero carries the residual by recurrence (an explicit zero
    field is an iterate like any other and does not), so there the two solves take the same steps
    and agree to rounding."""
    import os

    dims = (64, 48, 32)
    bc = synth.WALL_BC_TYPE
    rho = synth.random_field(dims, seed=8)
    outs = []
    for explicit in (False, True):
        old = os.environ.get("CCMG_DEFECT")
        if defect:
            os.environ["CCMG_DEFECT"] = defect
        try:
            P = Poisson(dims, bc_type=bc, bc_value=synth.wall_bc_value(1.0), precision="mixed")
        finally:
            if defect:
                if old is None:
                    del os.environ["CCMG_DEFECT"]
                else:
                    os.environ["CCMG_DEFECT"] = old
        P.set_rhs(gpu(rho))
        zeros = torch.zeros(tuple(reversed(dims)), dtype=torch.float64, device="cuda")
        P.set_solution(zeros if explicit else None)
        phi0 = P.solution().clone()
        rel0 = P.residual()
        P.set_solution(zeros if explicit else None)
        k, rel = P.solve(1e-9, 20)
        outs.append((phi0, rel0, k, rel, P.solution().clone()))
        P.close()
    (a0, ra0, ka, rela, a), (b0, rb0, kb, relb, b) = outs
    assert torch.equal(a0, b0) and not torch.any(a0 != 0)
    assert ra0 == rb0 and abs(ra0 - 1.0) < 1e-12
    assert ka == kb and rela < 1e-9 and relb < 1e-9
    if defect == "walk":
        assert rela == relb and torch.equal(a, b)
    else:
        assert torch.linalg.norm(a - b) <= 1e-8 * torch.linalg.norm(b)


def _rows_max(phi, bc):
    """Per cell, the largest |phi| over the five grid rows (x lines) that the packed residual walk
    reads for it: rows j-1, j, j+1 of its plane and row j of planes k-1 and k+1, across a periodic
    axis the row at the opposite side, beyond a wall none. The walk's row exponents are taken over
    parts of these rows, so this bounds them from above."""
    R = np.abs(phi).max(axis=2)  # (nz, ny): largest |value| of each row, both colours
    out = R.copy()
    for ax, q in ((1, 2), (0, 4)):  # y rows within the plane, then z neighbours
        for shift in (1, -1):
            nb = np.roll(R, shift, axis=ax)
            if bc[q] != PER:
                if shift == 1:
                    nb[(slice(None),) * ax + (0,)] = 0.0
                else:
                    nb[(slice(None),) * ax + (-1,)] = 0.0
            out = np.maximum(out, nb)
    return np.broadcast_to(out[:, :, None], phi.shape)


def _diag(shape, bc):
    sh = {D: 1, N: -1, PER: 0}
    diag = np.full(shape, 6, dtype=np.int64)
    diag[:, :, 0] += sh[bc[0]]
    diag[:, :, -1] += sh[bc[1]]
    diag[:, 0, :] += sh[bc[2]]
    diag[:, -1, :] += sh[bc[3]]
    diag[0] += sh[bc[4]]
    diag[-1] += sh[bc[5]]
    return diag


def _residual_case(shape, bc, seed):
    """phi and g spread over 2^-40 .. 2^40 with zeros among them, and on half the cells a right-hand
    side that cancels the stencil to its rounding error; the six neighbour fields (zero beyond a
    wall, the opposite side across a periodic axis)."""
    rng = np.random.default_rng(seed)
    phi = rng.standard_normal(shape) * np.exp2(rng.integers(-40, 41, shape))
    phi[rng.random(shape) < 0.1] = 0.0
    diag = _diag(shape, bc)
    p = phi
    for ax, q in ((2, 0), (1, 2), (0, 4)):  # axis 2 is x, 1 is y, 0 is z
        widths = [(0, 0)] * 3
        widths[ax] = (1, 1)
        p = np.pad(p, widths, mode="wrap" if bc[q] == PER else "constant")
    nbs = [p[1:-1, 1:-1, :-2], p[1:-1, 1:-1, 2:], p[1:-1, :-2, 1:-1], p[1:-1, 2:, 1:-1], p[:-2, 1:-1, 1:-1],
           p[2:, 1:-1, 1:-1]]
    g = rng.standard_normal(shape) * np.exp2(rng.integers(-40, 41, shape))
    g[rng.random(shape) < 0.05] = 0.0
    cancel = rng.random(shape) < 0.5
    g[cancel] = (diag * phi - sum(nbs))[cancel]
    return phi, g, diag, nbs


def test_fp64_residual_against_exact_arithmetic_natural_order():
    """The FP64 residual r = g + (sum of the six neighbours) - (6 + d) phi of every cell of a
    single-level (natural order) grid, aligned per cell: within half an ulp of its largest
    operand plus half an ulp of itself from the exact rational value (h = 1, so the scaled and the
    plain residual coincide)."""
    from fractions import Fraction
    dims, bc = (4, 6, 4), (N, D, D, N, N, D)
    shape = tuple(reversed(dims))
    phi, g, diag, nbs = _residual_case(shape, bc, 11)
    P = Poisson(dims, h=1.0, bc_type=bc)
    assert P.num_levels == 1
    P.level_set(0, 0, gpu(phi))
    P.level_set(0, 1, gpu(g))
    _, r = P.residual(field=True)
    r = cpu(r)
    P.close()
    worst = 0.0
    for idx in np.ndindex(*shape):
        ops = [g[idx], phi[idx]] + [float(n[idx]) for n in nbs]
        exact = Fraction(g[idx]) + sum(Fraction(float(n[idx])) for n in nbs) - int(diag[idx]) * Fraction(phi[idx])
        bound = Fraction(np.spacing(max(abs(v) for v in ops))) / 2 + Fraction(np.spacing(abs(r[idx]))) / 2
        err = abs(Fraction(float(r[idx])) - exact)
        worst = max(worst, float(err / bound))
    assert worst <= 1.0, worst


@pytest.mark.parametrize("dims,bc", [((24, 20, 18), (D, N, N, D, D, N)), ((80, 20, 72), (D, N, N, D, D, N)),
                                     ((80, 20, 72), (PER, PER, N, D, PER, PER))])
def test_fp64_residual_against_exact_arithmetic(dims, bc):
    """The FP64 residual of the packed tile walk (each ring row in fixed point at its own
    exponent): within (8 + D)/32 of an ulp of the largest value among the five rows the cell reads
    (or of its g) plus half an ulp of itself from the exact value, which math.fsum rounds once (so
    the bound gains half an ulp of that). Operands spread over 2^-40 .. 2^40, zeros among them,
    right-hand sides that cancel the stencil; a one-tile grid and one of several tiles in every
    direction, ragged in x, y and z (80 x 20 x 72: packed rows of 40 = 32 + 8 columns, rows 8 + 8
    + 4, planes 64 + 8), with walls and with periodic axes (the halo columns, rows and planes of
    the walk then come from the opposite side)."""
    import math
    shape = tuple(reversed(dims))
    phi, g, diag, nbs = _residual_case(shape, bc, 12)
    P_ = Poisson(dims, h=1.0, bc_type=bc)
    assert P_.num_levels > 1
    P_.level_set(0, 0, gpu(phi))
    P_.level_set(0, 1, gpu(g))
    _, r = P_.residual(field=True)
    r = cpu(r)
    P_.close()
    big = np.maximum(_rows_max(phi, bc), np.abs(g)).reshape(-1)
    vals = [g] + nbs + [-phi]
    flat = [v.reshape(-1) for v in vals]
    dflat, rflat = diag.reshape(-1), r.reshape(-1)
    worst = 0.0
    for i in range(rflat.size):
        terms = [float(v[i]) for v in flat[:-1]] + [float(flat[-1][i])] * int(dflat[i])
        ex = math.fsum(terms)
        bound = (8 + int(dflat[i])) / 32 * np.spacing(big[i]) + np.spacing(abs(rflat[i])) / 2 + \
            np.spacing(abs(ex)) / 2
        worst = max(worst, abs(rflat[i] - ex) / bound)
    assert worst <= 1.0, worst


def test_fp64_residual_walk_on_a_smooth_field():
    """On a smooth potential (the case of a solve), where the rows a cell reads hold values of the
    cell's own size, the walk's residual is within an ulp of the largest of the cell's own
    operands (plus half an ulp of itself and of the rounded exact value)."""
    import math
    dims, bc = (96, 40, 24), (N, N, N, N, D, D)
    shape = tuple(reversed(dims))
    zz, yy, xx = np.meshgrid(*(np.arange(n) + 0.5 for n in shape), indexing="ij")
    phi = 1.0 + 0.3 * np.sin(0.05 * xx) * np.cos(0.07 * yy) + zz / shape[0]
    diag = _diag(shape, bc)
    p = np.pad(phi, 1)
    nbs = [p[1:-1, 1:-1, :-2], p[1:-1, 1:-1, 2:], p[1:-1, :-2, 1:-1], p[1:-1, 2:, 1:-1], p[:-2, 1:-1, 1:-1],
           p[2:, 1:-1, 1:-1]]
    g = np.zeros(shape)
    g[:, :, : dims[0] // 2] = (diag * phi - sum(nbs))[:, :, : dims[0] // 2] * 0.999
    P_ = Poisson(dims, h=1.0, bc_type=bc)
    P_.level_set(0, 0, gpu(phi))
    P_.level_set(0, 1, gpu(g))
    _, r = P_.residual(field=True)
    r = cpu(r)
    P_.close()
    ops = np.max(np.abs(np.stack([g, phi] + nbs)), axis=0).reshape(-1)
    vals = [g] + nbs + [-phi]
    flat = [v.reshape(-1) for v in vals]
    dflat, rflat = diag.reshape(-1), r.reshape(-1)
    worst = 0.0
    for i in range(rflat.size):
        terms = [float(v[i]) for v in flat[:-1]] + [float(flat[-1][i])] * int(dflat[i])
        ex = math.fsum(terms)
        bound = np.spacing(ops[i]) + np.spacing(abs(rflat[i])) / 2 + np.spacing(abs(ex)) / 2
        worst = max(worst, abs(rflat[i] - ex) / bound)
    assert worst <= 1.0, worst


@pytest.mark.parametrize("h", [1.0, 0.5])
def test_per_cell_wall_values_match_oracle(h):
    """Wall values per face cell (mg_set_bc_field): the right-hand side equals the oracle's bit for
    bit, the harmonic field a x y + b (per-cell Neumann on x/y, Dirichlet on z) is reproduced by
    the FP64 solve, and the E-field (both stencils) and forces with these ghosts match the oracle;
    clearing a face's array restores its uniform value."""
    nx, ny, nz = 48, 40, 32
    a, b = 0.37, -1.2
    xc, yc = (np.arange(nx) + 0.5) * h, (np.arange(ny) + 0.5) * h
    phi_ex = np.broadcast_to(a * xc[None, None, :] * yc[None, :, None] + b, (nz, ny, nx)).copy()
    fx = np.broadcast_to(a * yc[None, :], (nz, ny))
    fy = np.broadcast_to(a * xc[None, :], (nz, nx))
    fz = a * xc[None, :] * yc[:, None] + b
    field = [-fx, fx, -fy, fy, fz, fz]
    bc = (N, N, N, N, D, D)
    bcv = (0.1, -0.2, 0.3, -0.4, 0.5, -0.6)  # overridden by the arrays
    P = Poisson((nx, ny, nz), h=h, bc_type=bc, bc_value=bcv)
    for q in range(6):
        P.set_bc_field(q, gpu(field[q]))
    rho = synth.random_field((nx, ny, nz), 4) * 0.0
    P.set_rhs(gpu(rho))
    f_ref = oracle.rhs(rho, h, bc, bcv, bc_field=field)
    assert np.array_equal(cpu(P.level_get(0, 1)), f_ref)
    P.set_solution(None)
    k, rel = P.solve(1e-12, 50)
    assert np.abs(cpu(P.solution()) - phi_ex).max() < 1e-9 * np.abs(phi_ex).max()
    # E-field and forces on a random potential with these ghosts
    phi = synth.random_field((nx, ny, nz), 11)
    P.set_solution(gpu(phi))
    sp, c, r, q = _spheres_case((nx, ny, nz), 6, 8)
    cs, rs = sp.centers * h, sp.radius * h
    for stencil in (7, 19):
        P.gradient_stencil = stencil
        E_ref = oracle.efield(phi, h, bc, bcv, stencil=stencil, bc_field=field)
        assert maxrel(cpu(P.efield()), E_ref) < 1e-15
        F_ref = oracle.force_gather(phi, h, bc, bcv, cs, rs, sp.density, 2, stencil=stencil, bc_field=field)
        assert maxrel(cpu(P.force_gather(gpu(cs), gpu(rs), q, 2)), F_ref) < 1e-12
    P.gradient_stencil = 7
    # back to uniform values on the z faces
    P.set_bc_field(4, None)
    P.set_bc_field(5, None)
    field_u = field[:4] + [None, None]
    assert maxrel(cpu(P.efield()), oracle.efield(phi, h, bc, bcv, bc_field=field_u)) < 1e-15
    P.set_rhs(gpu(rho))
    assert np.array_equal(cpu(P.level_get(0, 1)), oracle.rhs(rho, h, bc, bcv, bc_field=field_u))
    with pytest.raises(Exception):
        P.set_bc_field(6, gpu(field[0]))
    P.close()


def test_fp64_residual_walk_non_finite_values():
    """Infinities and a NaN in the iterate: the cells whose rows hold them take the direct FP64
    formula (the walk's fallback); the non-finite pattern equals the oracle's, and every finite
    residual is within the walk's bound of the oracle's FP64 residual."""
    dims, bc = (80, 20, 72), (D, N, N, D, D, N)
    nx, ny, nz = dims
    rng = np.random.default_rng(29)
    phi = rng.standard_normal((nz, ny, nx))
    phi[3, 4, 10] = np.inf
    phi[40, 12, 60] = -np.inf
    phi[66, 17, 33] = np.nan
    g = rng.standard_normal((nz, ny, nx))
    P = Poisson(dims, h=1.0, bc_type=bc)
    assert P.num_levels > 1
    P.level_set(0, 0, gpu(phi))
    P.level_set(0, 1, gpu(g))
    _, r = P.residual(field=True)
    r = cpu(r)
    P.close()
    with np.errstate(invalid="ignore", over="ignore"):
        ref = oracle.residual(phi, g, 1.0, bc)
    assert np.array_equal(np.isnan(r), np.isnan(ref))
    assert np.array_equal(np.isinf(r), np.isinf(ref)) and np.array_equal(r[np.isinf(r)], ref[np.isinf(ref)])
    fin = np.isfinite(ref)
    assert (~fin).sum() >= 3
    assert np.abs(r[fin] - ref[fin]).max() <= 1e-14 * np.abs(ref[fin]).max()
