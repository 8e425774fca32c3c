"""Pins of the CPU oracle against facts fixed by the paper and by mathematics (no GPU).

Each test ties one part of the oracle to something other than the oracle itself: a closed-form
discrete solution, an exact spectral solver, a dense direct solve, a literal Galerkin triple
product, a symmetry, a table of the paper, or brute force on tiny inputs.
"""
import math
import os

import numpy as np
import pytest

import oracle
import spectral
from paper_1410_6609_gb300 import synth

D, N = 0, 1
HERE = os.path.dirname(os.path.abspath(__file__))


def dense(dims, c, bc):
    """Matrix of oracle.apply, column by column (unit vectors)."""
    nx, ny, nz = dims
    n = nx * ny * nz
    A = np.zeros((n, n))
    for q in range(n):
        e = np.zeros(n)
        e[q] = 1.0
        A[:, q] = oracle.apply(e.reshape(nz, ny, nx), c, bc).ravel()
    return A


def injection(fine):
    """Constant prolongation P (fine x coarse): each child takes its parent's value (Sec. 3)."""
    nx, ny, nz = fine
    mx, my, mz = nx // 2, ny // 2, nz // 2
    P = np.zeros((nx * ny * nz, mx * my * mz))
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                P[i + nx * (j + ny * k), i // 2 + mx * (j // 2 + my * (k // 2))] = 1.0
    return P


# ------------------------------------------------------------------------------------------
# Level hierarchy (Sec. 3: coarsen while dims even; 256^3 gives the paper's seven levels)

def test_levels():
    assert oracle.levels(32, 32, 32) == [(32,) * 3, (16,) * 3, (8,) * 3, (4,) * 3]
    assert len(oracle.levels(256, 256, 256)) == 7
    assert oracle.levels(256, 256, 256)[-1] == (4, 4, 4)
    assert len(oracle.levels(512, 512, 512)) == 8
    assert oracle.levels(96, 96, 96)[-1] == (3, 3, 3) and len(oracle.levels(96, 96, 96)) == 6
    assert len(oracle.levels(64, 64, 64)) == 5 and len(oracle.levels(192, 192, 192)) == 7
    assert oracle.levels(48, 40, 64) == [(48, 40, 64), (24, 20, 32), (12, 10, 16), (6, 5, 8)]


# ------------------------------------------------------------------------------------------
# Manufactured solution: sin(pi x) sin(pi y) sin(pi z) is an exact eigenvector of the
# Dirichlet cell-centred operator, so the converged discrete solution is the exact one times
# (x/sin x)^2 with x = pi h / 2. Pins the stencil, the Dirichlet folding and the whole solve.

@pytest.mark.parametrize("n", [32, 64])
def test_manufactured_closed_form(n):
    f, h = synth.manufactured_rhs(n)
    u = synth.manufactured_exact(n)
    phi, k, rel = oracle.solve(f, h, (D,) * 6, tol=1e-12)
    assert rel < 1e-12 and k < 30
    err = np.linalg.norm(phi - u) / np.linalg.norm(u)
    x = np.pi * h / 2
    closed = (x / np.sin(x)) ** 2 - 1.0
    assert abs(err - closed) < 1e-9 * closed + 1e-12
    if n == 32:
        assert abs(closed - 8.0358e-4) < 1e-7  # O(h^2) error at h = 1/32


def test_manufactured_to_tolerance_1e10():
    f, h = synth.manufactured_rhs(32)
    phi, k, rel = oracle.solve(f, h, (D,) * 6, tol=1e-10)
    assert rel < 1e-10 and 5 <= k <= 15


# ------------------------------------------------------------------------------------------
# Exact discrete solutions by the spectral solver (homogeneous BCs, any RHS)

@pytest.mark.parametrize("bc", [(D,) * 6, (N, N, N, N, D, D), (D, N, N, D, D, N), (N, D, D, D, N, D)])
def test_spectral_random_rhs(bc):
    dims = (16, 12, 20)
    f = synth.random_field(dims, seed=7)
    phi, k, rel = oracle.solve(f, 1.0, bc, tol=1e-13, max_cycles=200)
    ex = spectral.solve(f, 1.0, bc)
    assert np.linalg.norm(phi - ex) / np.linalg.norm(ex) < 1e-11


def test_spectral_charged_spheres_between_plates():
    """Charged spheres between grounded plates: the exact discrete potential (spectral) vs the
    oracle's multigrid solve of the subsampled sphere charges."""
    dims = (32, 24, 40)
    sp = synth.random_spheres(dims, 5, 3.0, seed=11)
    rho = oracle.sphere_density((dims[2], dims[1], dims[0]), 1.0, sp.centers, sp.radius, sp.density, 2)
    bc = (N, N, N, N, D, D)
    f = oracle.rhs(rho, 1.0, bc, (0.0,) * 6)
    phi, k, rel = oracle.solve(f, 1.0, bc, tol=1e-13, max_cycles=200)
    ex = spectral.solve(rho, 1.0, bc)
    assert np.linalg.norm(phi - ex) / np.linalg.norm(ex) < 1e-11


# ------------------------------------------------------------------------------------------
# Inhomogeneous BCs: linear potentials are exact discrete solutions (the ghost extrapolation
# of a linear function is exact), so the solve must reproduce them.

def test_plates_linear_potential():
    nx, ny, nz = 12, 10, 24
    V = 1.7
    bc = (N, N, N, N, D, D)
    f = oracle.rhs(np.zeros((nz, ny, nx)), 1.0, bc, (0, 0, 0, 0, 0.0, V))
    phi, k, rel = oracle.solve(f, 1.0, bc, tol=1e-13, max_cycles=200)
    zc = (np.arange(nz) + 0.5) / nz
    ex = np.broadcast_to(V * zc[:, None, None], phi.shape)
    assert np.abs(phi - ex).max() < 1e-11
    assert oracle.rel_residual(np.ascontiguousarray(ex), f, 1.0, bc) < 1e-14


@pytest.mark.parametrize("h", [1.0, 0.25])
def test_neumann_slope_linear_potential(h):
    """phi = s z: Neumann at -z with outward derivative -s, Dirichlet s L at +z."""
    nx, ny, nz = 8, 8, 16
    s = 0.8
    L = nz * h
    bc = (N, N, N, N, N, D)
    f = oracle.rhs(np.zeros((nz, ny, nx)), h, bc, (0, 0, 0, 0, -s, s * L))
    phi, k, rel = oracle.solve(f, h, bc, tol=1e-13, max_cycles=200)
    zc = (np.arange(nz) + 0.5) * h
    assert np.abs(phi - s * zc[:, None, None]).max() < 1e-10
    # and the reverse: Dirichlet 0 at -z, Neumann +s at +z
    bc2 = (N, N, N, N, D, N)
    f2 = oracle.rhs(np.zeros((nz, ny, nx)), h, bc2, (0, 0, 0, 0, 0.0, s))
    phi2, _, _ = oracle.solve(f2, h, bc2, tol=1e-13, max_cycles=200)
    assert np.abs(phi2 - s * zc[:, None, None]).max() < 1e-10


# ------------------------------------------------------------------------------------------
# Dense direct solve at small size: the multigrid fixed point is A^-1 f

@pytest.mark.parametrize("dims,bc", [((8, 6, 10), (D, N, N, D, D, N)), ((8, 8, 8), (N, N, N, N, D, D))])
def test_dense_direct_solve(dims, bc):
    nx, ny, nz = dims
    A = dense(dims, 1.0, bc)
    f = synth.random_field(dims, seed=3)
    x = np.linalg.solve(A, f.ravel()).reshape(nz, ny, nx)
    phi, k, rel = oracle.solve(f, 1.0, bc, tol=1e-13, max_cycles=200)
    assert np.linalg.norm(phi - x) / np.linalg.norm(x) < 1e-12


# ------------------------------------------------------------------------------------------
# Galerkin coarsening: R A_l P (averaging restriction R = P^T/8, constant prolongation P) equals
# the closed-form level-(l+1) operator with half the coefficient (Sec. 3, seven-point stencil
# on all levels).

@pytest.mark.parametrize("bc", [(D, N, N, D, D, N), (D,) * 6, (N, N, N, N, D, D)])
def test_galerkin_closed_form(bc):
    fine = (12, 12, 12)
    c0 = 1.0 / 0.5 ** 2
    A0 = dense(fine, c0, bc)
    P = injection(fine)
    Ac = (P.T / 8.0) @ A0 @ P
    A1 = dense((6, 6, 6), c0 / 2.0, bc)
    assert np.abs(Ac - A1).max() <= 1e-14 * np.abs(A1).max()
    P2 = injection((6, 6, 6))
    A2 = dense((3, 3, 3), c0 / 4.0, bc)
    assert np.abs((P2.T / 8.0) @ A1 @ P2 - A2).max() <= 1e-14 * np.abs(A2).max()
    assert oracle.level_coeff(0.5, 2) == c0 / 4.0


def test_operator_symmetry_all_levels():
    bc = (D, N, N, D, D, N)
    rng = np.random.default_rng(5)
    for l, (nx, ny, nz) in enumerate(oracle.levels(24, 20, 28)):
        c = oracle.level_coeff(0.5, l)
        u = rng.standard_normal((nz, ny, nx))
        v = rng.standard_normal((nz, ny, nx))
        a = np.vdot(u, oracle.apply(v, c, bc))
        b = np.vdot(v, oracle.apply(u, c, bc))
        assert abs(a - b) <= 1e-13 * (abs(a) + abs(b))


# ------------------------------------------------------------------------------------------
# Single-level pieces against their definitions on tiny inputs

def test_rbgs_half_solves_its_rows():
    """After a red half-sweep, every red row of A phi = f holds exactly (up to rounding), and
    the black values are untouched (Sec. 5.3)."""
    dims = (6, 8, 4)
    bc = (D, N, N, D, D, N)
    f = synth.random_field(dims, 1)
    phi = synth.random_field(dims, 2)
    out = oracle.rbgs_half(phi, f, 4.0, bc, 0)
    r = oracle.residual(out, f, 4.0, bc)
    k, j, i = np.indices(phi.shape)
    red = (i + j + k) % 2 == 0
    assert np.abs(r[red]).max() < 1e-13 * np.abs(f).max() * 10
    assert np.array_equal(out[~red], phi[~red])


def test_restrict_prolong_adjoint_pair():
    """Averaging restriction is P^T / 8; prolongation is P (brute force on a tiny grid)."""
    fine = (4, 6, 8)
    r = synth.random_field(fine, 4)
    P = injection(fine)
    assert np.allclose(oracle.restrict(r).ravel(), (P.T / 8.0) @ r.ravel(), rtol=0, atol=1e-15)
    ec = synth.random_field((2, 3, 4), 5)
    phi = synth.random_field(fine, 6)
    out = oracle.prolong_correct(phi, ec, 2.0)
    assert np.allclose(out.ravel(), phi.ravel() + 2.0 * (P @ ec.ravel()), rtol=0, atol=1e-14)


def test_cg_exact_on_coarse_grids():
    bc = (N, N, N, N, D, D)
    for dims in [(4, 4, 4), (3, 3, 3), (6, 5, 8)]:
        nx, ny, nz = dims
        A = dense(dims, 0.125, bc)
        b = synth.random_field(dims, 9)
        x, it = oracle.cg(b, 0.125, bc)
        ex = np.linalg.solve(A, b.ravel()).reshape(nz, ny, nx)
        assert np.linalg.norm(x - ex) / np.linalg.norm(ex) < 1e-12
        assert it <= 2 * b.size
    x, it = oracle.cg(np.zeros((4, 4, 4)), 1.0, bc)
    assert it == 0 and not x.any()


def test_cg_f32_reaches_its_tolerance_against_a_dense_solve():
    """The single-precision CG of the mixed solver's inner cycles: its float solution leaves a
    residual (evaluated in double with the dense matrix) within a few times its 1e-5 tolerance and
    lies within 1e-4 of the dense solve, on walls of every kind and a periodic pair."""
    for dims, bc in [((4, 4, 4), (N, N, N, N, D, D)), ((6, 5, 8), (D, N, N, D, D, N)), ((4, 4, 6), (2, 2, N, N, D, D))]:
        nx, ny, nz = dims
        A = dense(dims, 0.125, bc)
        b = synth.random_field(dims, 9).astype(np.float32).astype(np.float64)
        x, it = oracle.cg_f32(b, 0.125, bc)
        assert x.dtype == np.float32 and 0 < it <= 2 * b.size
        ex = np.linalg.solve(A, b.ravel())
        xd = x.astype(np.float64).ravel()
        assert np.linalg.norm(b.ravel() - A @ xd) <= 5e-5 * np.linalg.norm(b)
        assert np.linalg.norm(xd - ex) <= 1e-4 * np.linalg.norm(ex)
    x, it = oracle.cg_f32(np.zeros((4, 4, 4)), 1.0, (N, N, N, N, D, D))
    assert it == 0 and not x.any()


def test_cg_iterations_grow_with_diameter():
    """CG iterations grow roughly with the coarse-grid diameter (Sec. 8.3, Tab. WeakScalProbSizeCG)."""
    bc = (N, N, N, N, D, D)
    its = []
    for n in (4, 8, 16):
        b = synth.random_field((n, n, n), 1)
        its.append(oracle.cg(b, 1.0, bc, rtol=1e-8)[1])
    assert its[0] < its[1] < its[2]
    assert 1.3 < its[2] / its[1] < 3.0


# ------------------------------------------------------------------------------------------
# Convergence of the cycle: the x2 magnified correction gives a V(2,2) factor near 0.1 and the
# plain correction is far slower (Sec. 3, Braess).

@pytest.mark.parametrize("n,bc", [(32, (D,) * 6), (32, (N, N, N, N, D, D))])
def test_vcycle_convergence_factor(n, bc):
    def factor(omega):
        phi = np.random.default_rng(1).standard_normal((n, n, n))
        f = np.zeros_like(phi)
        r = []
        for _ in range(10):
            r.append(np.linalg.norm(oracle.residual(phi, f, 1.0, bc)))
            phi, _ = oracle.vcycles(phi, f, 1.0, bc, 1, omega=omega)
        return r[-1] / r[-2]
    assert factor(2.0) < 0.15
    assert factor(1.0) > 0.5


# ------------------------------------------------------------------------------------------
# E-field (central differences with BC ghosts) and the Coulomb force

def test_efield_exact_for_linear_potential():
    nx, ny, nz = 6, 5, 12
    V, h = 2.0, 0.5
    bc = (N, N, N, N, D, D)
    zc = (np.arange(nz) + 0.5) * h
    L = nz * h
    phi = np.ascontiguousarray(np.broadcast_to(V * zc[:, None, None] / L, (nz, ny, nx)))
    E = oracle.efield(phi, h, bc, (0, 0, 0, 0, 0, V))
    assert np.abs(E[2] + V / L).max() < 1e-13
    assert np.abs(E[0]).max() == 0.0 and np.abs(E[1]).max() == 0.0
    # Neumann x walls with slope s: phi = s x, E_x = -s everywhere
    s = 0.3
    xc = (np.arange(nx) + 0.5) * h
    phi2 = np.ascontiguousarray(np.broadcast_to(s * xc[None, None, :], (nz, ny, nx)))
    E2 = oracle.efield(phi2, h, (N, N, N, N, N, N), (-s, s, 0, 0, 0, 0))
    assert np.abs(E2[0] + s).max() < 1e-13


def test_force_on_symmetric_sphere_in_uniform_field():
    """A charged sphere at the centre of a plate capacitor: by the reflection symmetry of the
    domain its self-force vanishes, so F = Q_mapped * E_applied exactly, with E_applied = -V/L
    (Sec. 6.3, Coulomb force validation in a homogeneous field)."""
    n = 24
    V = -10.0
    h = 1.0
    bc = (N, N, N, N, D, D)
    bcv = (0, 0, 0, 0, 0.0, V)
    c = np.array([[n / 2, n / 2, n / 2]])
    for sf in (1, 2, 3):
        rho = oracle.sphere_density((n, n, n), h, c, [4.0], [1.5], sf)
        f = oracle.rhs(rho, h, bc, bcv)
        phi, k, rel = oracle.solve(f, h, bc, tol=1e-13, max_cycles=200)
        F = oracle.force_gather(phi, h, bc, bcv, c, [4.0], [1.5], sf)[0]
        Q = rho.sum() * h ** 3
        assert abs(F[2] - Q * (-V / (n * h))) < 1e-9 * abs(Q * V / n)
        assert abs(F[0]) < 1e-9 * abs(Q * V / n) and abs(F[1]) < 1e-9 * abs(Q * V / n)
        assert F[2] > 0  # positive charge, field pointing to +z (V < 0 at the top)


# ------------------------------------------------------------------------------------------
# Subsampling (Sec. 2.4) against brute force and Table ValidPotSubs

def test_sphere_density_brute_force():
    dims = (10, 9, 11)
    nx, ny, nz = dims
    c = np.array([[4.3, 4.1, 5.7], [7.9, 4.6, 3.2]])
    R = np.array([2.5, 1.7])
    dens = np.array([1.25, -0.5])
    for sf in (1, 2, 3):
        rho = oracle.sphere_density((nz, ny, nx), 1.0, c, R, dens, sf)
        ref = np.zeros((nz, ny, nx))
        sub = (2 * np.arange(sf) + 1) / (2 * sf)
        for s in range(2):
            for k in range(nz):
                for j in range(ny):
                    for i in range(nx):
                        X = i + sub[None, None, :]
                        Y = j + sub[None, :, None]
                        Z = k + sub[:, None, None]
                        inside = (X - c[s, 0]) ** 2 + (Y - c[s, 1]) ** 2 + (Z - c[s, 2]) ** 2 <= R[s] ** 2
                        ref[k, j, i] += dens[s] * (inside.sum() / sf ** 3)
        assert np.array_equal(rho, ref)


def _volume_errors(R, sf, npts=11):
    n = int(2 * R + 8)
    V = 4.0 / 3.0 * np.pi * R ** 3
    g = np.linspace(-0.51 / sf, 0.51 / sf, npts)
    out = []
    for dx in g:
        for dy in g:
            for dz in g:
                c = np.array([[n / 2 + dx, n / 2 + dy, n / 2 + dz]])
                rho = oracle.sphere_density((n, n, n), 1.0, c, [R], [1.0], sf)
                out.append((rho.sum() - V) / V)
    return np.array(out)


def test_subsampling_scale_invariance():
    """The mapped volume depends only on R*s_f and shift*s_f: the table's e_rVmax entries with
    equal R*s_f are identical; here the whole error sets coincide."""
    a = _volume_errors(4, 2, npts=5)
    b = _volume_errors(8, 1, npts=5)
    assert np.array_equal(a, b)


def test_subsampling_matches_table():
    rows = np.loadtxt(os.path.join(HERE, "golden", "valid_pot_subs.txt"))
    for R, sf, mean_pct, _ in rows:
        if R not in (4.0, 6.0):
            continue
        ours = 100.0 * np.abs(_volume_errors(R, int(sf))).mean()
        # The paper's shift set is not given exactly; an 11^3 grid of shifts over the same range
        # reproduces the table's means to within a factor 1.4 (measured 1.09 - 1.33).
        assert mean_pct / 1.4 < ours < mean_pct * 1.4, (R, sf, ours, mean_pct)
    # halving with each increment of s_f (Sec. 6.3)
    m = [np.abs(_volume_errors(4, sf)).mean() for sf in (1, 2, 3, 4)]
    assert m[0] > m[1] > m[2] > m[3]


# ------------------------------------------------------------------------------------------
# Adjoint gradient of J = sum_s F_z against finite differences of the forward oracle. J is
# quadratic in the densities and affine in the wall voltage, so central differences have no
# truncation error; the step only scales rounding and solver error.

def test_adjoint_gradient_vs_finite_differences():
    dims = (16, 16, 20)
    nx, ny, nz = dims
    sp = synth.random_spheres(dims, 3, 2.5, seed=21)
    bc = synth.WALL_BC_TYPE
    bcv = np.array(synth.wall_bc_value(1.0))
    wF = np.zeros((3, 3))
    wF[:, 2] = 1.0
    shape = (nz, ny, nx)
    J, gd, gbc, _ = oracle.force_objective_and_grad(shape, 1.0, bc, bcv, sp.centers, sp.radius,
                                                    sp.density, wF, tol=1e-14, max_cycles=300)

    def Jof(dens, v):
        rho = oracle.sphere_density(shape, 1.0, sp.centers, sp.radius, dens, 2)
        f = oracle.rhs(rho, 1.0, bc, v)
        phi, _, _ = oracle.solve(f, 1.0, bc, tol=1e-14, max_cycles=300)
        return oracle.force_gather(phi, 1.0, bc, v, sp.centers, sp.radius, dens, 2)[:, 2].sum()

    step = 1e-3
    for s in range(3):
        dp = sp.density.copy()
        dm = sp.density.copy()
        dp[s] += step
        dm[s] -= step
        fd = (Jof(dp, bcv) - Jof(dm, bcv)) / (2 * step)
        assert abs(fd - gd[s]) <= 1e-7 * max(1.0, abs(fd))
    vp = bcv.copy()
    vm = bcv.copy()
    vp[5] += step
    vm[5] -= step
    fd = (Jof(sp.density, vp) - Jof(sp.density, vm)) / (2 * step)
    assert abs(fd - gbc[5]) <= 1e-7 * max(1.0, abs(fd))
    assert abs(J - Jof(sp.density, bcv)) <= 1e-12 * max(1.0, abs(J))


# ------------------------------------------------------------------------------------------
# Mixed precision: converges to the FP64 tolerance it is asked for and agrees with FP64

@pytest.mark.parametrize("inner", [1, 3])
def test_mixed_precision_defect_correction(inner):
    dims = (32, 32, 32)
    sp = synth.random_spheres(dims, 6, 3.0, seed=8)
    rho = oracle.sphere_density((32, 32, 32), 1.0, sp.centers, sp.radius, sp.density, 2)
    bc = synth.WALL_BC_TYPE
    f = oracle.rhs(rho, 1.0, bc, synth.wall_bc_value(1.0))
    pm, km, relm = oracle.solve_mixed(f, 1.0, bc, tol=1e-9, inner=inner)
    pd, kd, reld = oracle.solve(f, 1.0, bc, tol=1e-9)
    assert relm < 1e-9 and reld < 1e-9
    # each outer step runs `inner` single-precision cycles, each about as effective as an FP64 one
    assert abs(km * inner - kd) <= 3 * inner
    ex = spectral.solve(f, 1.0, bc)  # exact discrete solution (the BC terms are part of f)
    assert np.linalg.norm(pm - pd) / np.linalg.norm(pd) < 1e-7
    assert np.linalg.norm(pm - ex) / np.linalg.norm(ex) < 1e-7


# ------------------------------------------------------------------------------------------
# The D3Q19 gradient (Sec. 2.4, "Coulomb force"): (1/w_1) sum_q w_q phi(x + e_q) e_q / h^2 with
# D3Q19 weights, used where all 18 neighbours exist. Closed forms on polynomial fields; cell
# centres at (i + 1/2) h.

def _centres(n, h):
    return (np.arange(n) + 0.5) * h


def _interior(a):
    return a[..., 1:-1, 1:-1, 1:-1]


@pytest.mark.parametrize("h", [1.0, 0.25])
def test_d3q19_gradient_exact_for_quadratics(h):
    nx, ny, nz = 9, 8, 7
    x, y, z = np.meshgrid(_centres(nx, h), _centres(ny, h), _centres(nz, h), indexing="xy")
    x, y, z = (np.transpose(v, (2, 0, 1)).copy() for v in (x, y, z))  # [nz, ny, nx]
    bc = (D,) * 6
    phi = 0.7 * x - 1.3 * y + 0.4 * z + 0.25 * x * x - 0.5 * y * z + 2.0
    E = oracle.efield(phi, h, bc, (0.0,) * 6, stencil=19)
    ref = [-(0.7 + 0.5 * x), -(-1.3 - 0.5 * z), -(0.4 - 0.5 * y)]
    for a in range(3):
        assert np.abs(_interior(E[a]) - _interior(ref[a])).max() < 1e-12 / h


@pytest.mark.parametrize("h", [1.0, 0.5])
def test_d3q19_gradient_of_x_y2_carries_the_edge_term(h):
    """For phi = x y^2 the D3Q19 x-derivative is y^2 + h^2/3 (the edge directions contribute
    h^2 sum_q w_q e_qx^2 e_qy^2 / w_1 = h^2 (4/36) 3), the y-derivative 2xy and the z-derivative 0
    exactly, while the D3Q7 central difference gives y^2: a dropped or mis-weighted edge term, or
    a wrong sign, fails here."""
    nx, ny, nz = 8, 9, 6
    x, y, z = np.meshgrid(_centres(nx, h), _centres(ny, h), _centres(nz, h), indexing="xy")
    x, y, z = (np.transpose(v, (2, 0, 1)).copy() for v in (x, y, z))
    phi = x * y * y
    bc = (N,) * 4 + (D, D)
    E19 = oracle.efield(phi, h, bc, (0.0,) * 6, stencil=19)
    E7 = oracle.efield(phi, h, bc, (0.0,) * 6, stencil=7)
    scale = np.abs(phi).max() / h
    assert np.abs(_interior(E19[0]) + _interior(y * y + h * h / 3.0)).max() < 1e-13 * scale
    assert np.abs(_interior(E19[1]) + _interior(2 * x * y)).max() < 1e-13 * scale
    assert np.abs(_interior(E19[2])).max() < 1e-13 * scale
    assert np.abs(_interior(E7[0]) + _interior(y * y)).max() < 1e-13 * scale
    # cells without all 18 neighbours take the D3Q7 differences (ghosts included)
    border = np.ones(phi.shape, bool)
    border[1:-1, 1:-1, 1:-1] = False
    assert np.array_equal(E19[:, border], E7[:, border])


def test_d3q19_force_on_symmetric_sphere_in_uniform_field():
    """As for the D3Q7 gradient: the self-force vanishes by reflection symmetry and the applied
    field is linear, so F = Q_mapped * E_applied."""
    n = 24
    V = -10.0
    bc = (N, N, N, N, D, D)
    bcv = (0, 0, 0, 0, 0.0, V)
    c = np.array([[n / 2, n / 2, n / 2]])
    for sf in (1, 2):
        rho = oracle.sphere_density((n, n, n), 1.0, c, [4.0], [1.5], sf)
        f = oracle.rhs(rho, 1.0, bc, bcv)
        phi, _, _ = oracle.solve(f, 1.0, bc, tol=1e-13, max_cycles=200)
        F = oracle.force_gather(phi, 1.0, bc, bcv, c, [4.0], [1.5], sf, stencil=19)[0]
        Q = rho.sum()
        assert abs(F[2] - Q * (-V / n)) < 1e-9 * abs(Q * V / n)
        assert abs(F[0]) < 1e-9 * abs(Q * V / n) and abs(F[1]) < 1e-9 * abs(Q * V / n)


# ------------------------------------------------------------------------------------------
# Boundary values per face cell (the validation runs of Sec. 6.3 prescribe the analytic potential
# on the boundary): each face carries an array over its cells instead of one value.

def _xy_fields(nx, ny, nz, h, a, b):
    xc, yc = (np.arange(nx) + 0.5) * h, (np.arange(ny) + 0.5) * h
    phi = np.broadcast_to(a * xc[None, None, :] * yc[None, :, None] + b, (nz, ny, nx)).copy()
    # faces: 0,1 [nz, ny]; 2,3 [nz, nx]; 4,5 [ny, nx]. Neumann values are outward derivatives.
    fx = np.broadcast_to(a * yc[None, :], (nz, ny))
    fy = np.broadcast_to(a * xc[None, :], (nz, nx))
    fz = a * xc[None, :] * yc[:, None] + b
    return phi, [-fx, fx, -fy, fy, fz, fz]


@pytest.mark.parametrize("h", [1.0, 0.5])
def test_per_cell_boundary_values_reproduce_a_harmonic_field(h):
    """phi = a x y + b is harmonic and its 7-point finite-volume Laplacian vanishes; with Neumann
    values per face cell on the x and y faces (the outward derivative, varying along each face)
    and Dirichlet values per face cell on the z faces, the ghosts are exact, so the discrete
    solution and the E-field (boundary cells included) equal phi and -grad phi: a transposed or
    shifted face index, or a wrong ghost sign, fails here."""
    nx, ny, nz = 12, 10, 8
    a, b = 0.37, -1.2
    phi_ex, field = _xy_fields(nx, ny, nz, h, a, b)
    bc = (N, N, N, N, D, D)
    f = oracle.rhs(np.zeros((nz, ny, nx)), h, bc, (0.0,) * 6, bc_field=field)
    phi, _, _ = oracle.solve(f, h, bc, tol=1e-14, max_cycles=100)
    assert np.abs(phi - phi_ex).max() < 1e-11 * np.abs(phi_ex).max()
    xc, yc = (np.arange(nx) + 0.5) * h, (np.arange(ny) + 0.5) * h
    for stencil in (7, 19):
        E = oracle.efield(phi_ex, h, bc, (0.0,) * 6, stencil=stencil, bc_field=field)
        assert np.abs(E[0] + a * yc[None, :, None]).max() < 1e-12 * a * yc.max()
        assert np.abs(E[1] + a * xc[None, None, :]).max() < 1e-12 * a * xc.max()
        assert np.abs(E[2]).max() < 1e-12 * a * xc.max()
    # the uniform slots still apply to faces without an array
    f2 = oracle.rhs(np.zeros((nz, ny, nx)), h, bc, (0.0, 0.0, 0.0, 0.0, 0.5, -0.5),
                    bc_field=field[:4] + [None, None])
    f3 = oracle.rhs(np.zeros((nz, ny, nx)), h, bc, (0.0,) * 6,
                    bc_field=field[:4] + [np.full((ny, nx), 0.5), np.full((ny, nx), -0.5)])
    assert np.array_equal(f2, f3)


def test_per_cell_dirichlet_values_of_a_linear_field():
    """Dirichlet values per face cell taken from a linear potential on all six faces (each face
    array varies in both of its directions) reproduce the potential exactly."""
    nx, ny, nz, h = 10, 12, 14, 0.25
    xc, yc, zc = ((np.arange(n) + 0.5) * h for n in (nx, ny, nz))
    g = np.array([0.3, -0.8, 0.55])
    lin = lambda x, y, z: g[0] * x + g[1] * y + g[2] * z + 0.1
    X, Y, Z = xc[None, None, :], yc[None, :, None], zc[:, None, None]
    phi_ex = lin(X, Y, Z) + 0 * (X + Y + Z)
    Lx, Ly, Lz = nx * h, ny * h, nz * h
    field = [lin(0.0, yc[None, :], zc[:, None]), lin(Lx, yc[None, :], zc[:, None]),
             lin(xc[None, :], 0.0, zc[:, None]), lin(xc[None, :], Ly, zc[:, None]),
             lin(xc[None, :], yc[:, None], 0.0), lin(xc[None, :], yc[:, None], Lz)]
    bc = (D,) * 6
    f = oracle.rhs(np.zeros((nz, ny, nx)), h, bc, (0.0,) * 6, bc_field=field)
    phi, _, _ = oracle.solve(f, h, bc, tol=1e-14, max_cycles=100)
    assert np.abs(phi - phi_ex).max() < 1e-11 * np.abs(phi_ex).max()


# ------------------------------------------------------------------------------------------
# Periodic boundary conditions (Sec. 2.4: the domain is extended cyclically; the neighbour across
# a periodic axis is the cell at the opposite side)

PER = oracle.PERIODIC


@pytest.mark.parametrize("bc", [(PER, PER, PER, PER, D, D), (PER, PER, N, N, D, N), (D, N, PER, PER, PER, PER),
                                (PER, PER, D, D, PER, PER)])
def test_periodic_spectral_random_rhs(bc):
    """The exact discrete solution by a DFT along the periodic axes and sine/cosine transforms
    along the others."""
    dims = (16, 12, 20)
    f = synth.random_field(dims, seed=7)
    phi, k, rel = oracle.solve(f, 1.0, bc, tol=1e-13, max_cycles=200)
    ex = spectral.solve(f, 1.0, bc)
    assert np.linalg.norm(phi - ex) / np.linalg.norm(ex) < 1e-11


def test_periodic_operator_eigenvector():
    """cos(2 pi m (i+1/2)/n + a) along a periodic axis (a phase that makes it neither a Dirichlet
    nor a Neumann eigenvector) and sin(pi (k+1/2)/nz) between Dirichlet walls: A phi = (sum of
    the 1D eigenvalues) phi exactly, at the wrapped cells too."""
    nx, ny, nz, h = 12, 10, 8, 0.5
    i, j, k = np.arange(nx) + 0.5, np.arange(ny) + 0.5, np.arange(nz) + 0.5
    phi = (np.cos(2 * np.pi * 2 * i / nx + 0.3)[None, None, :] * np.cos(2 * np.pi * 3 * j / ny - 0.7)[None, :, None]
           * np.sin(np.pi * k / nz)[:, None, None])
    lam = ((2 - 2 * np.cos(2 * np.pi * 2 / nx)) + (2 - 2 * np.cos(2 * np.pi * 3 / ny))
           + (2 - 2 * np.cos(np.pi / nz))) / h ** 2
    Aphi = oracle.apply(phi, 1.0 / h ** 2, (PER, PER, PER, PER, D, D))
    assert np.abs(Aphi - lam * phi).max() < 1e-12 * lam
    # a wrong pairing at the wrap (the Neumann shift, or no neighbour) breaks it
    assert np.abs(oracle.apply(phi, 1.0 / h ** 2, (N, N, PER, PER, D, D)) - lam * phi).max() > 1e-3 * lam


@pytest.mark.parametrize("bc", [(PER, PER, D, N, PER, PER), (PER,) * 6, (N, D, PER, PER, D, D)])
def test_periodic_galerkin_closed_form(bc):
    fine = (12, 12, 12)
    c0 = 4.0
    A0 = dense(fine, c0, bc)
    P = injection(fine)
    A1 = dense((6, 6, 6), c0 / 2.0, bc)
    assert np.abs((P.T / 8.0) @ A0 @ P - A1).max() <= 1e-14 * np.abs(A1).max()
    assert np.abs(A0 - A0.T).max() == 0.0


def test_periodic_rhs_has_no_wall_term():
    nx, ny, nz = 6, 4, 8
    rho = synth.random_field((nx, ny, nz), seed=2)
    bcv = (3.0, -1.0, 2.0, 5.0, 0.5, -0.25)
    f = oracle.rhs(rho, 0.5, (PER, PER, PER, PER, D, N), bcv, eps=2.0)
    ref = rho / 2.0
    ref[0] += 2 * 0.5 / 0.25
    ref[-1] += -0.25 / 0.5
    assert np.array_equal(f, ref)


def _dyadic_spheres():
    # centres and radii with few significand bits: shifting a centre by whole cells (h = 1)
    # leaves every sub-cell distance exactly the same
    c = np.array([[0.75, 5.5, 3.25], [9.625, 0.375, 7.5], [4.5, 4.25, 0.5]])
    return c, np.array([2.5, 1.75, 2.25]), np.array([1.25, -0.5, 2.0])


def test_periodic_density_wraps_to_the_opposite_side():
    """A sphere across periodic walls maps the same charges as the sphere moved into the
    interior, the field rolled back: brute force by translation."""
    nx, ny, nz = 10, 9, 11
    c, R, q = _dyadic_spheres()
    bc = (PER,) * 6
    shifts = np.array([[3, 0, 0], [-3, 3, 0], [0, 0, 4]])  # moves sphere s wholly inside
    for s in range(3):
        for sf in (1, 2, 3):
            rho = oracle.sphere_density((nz, ny, nx), 1.0, c[s:s + 1], R[s:s + 1], q[s:s + 1], sf, bc)
            moved = oracle.sphere_density((nz, ny, nx), 1.0, c[s:s + 1] + shifts[s], R[s:s + 1], q[s:s + 1], sf)
            d = shifts[s]
            assert np.array_equal(rho, np.roll(moved, shift=(-d[2], -d[1], -d[0]), axis=(0, 1, 2)))
        # without the periodic axes the charge beyond the walls is lost
        assert oracle.sphere_density((nz, ny, nx), 1.0, c[s:s + 1], R[s:s + 1], q[s:s + 1], 2).sum() != rho.sum()


@pytest.mark.parametrize("stencil", [7, 19])
def test_periodic_efield_closed_form(stencil):
    """phi = cos(2 pi m (i+1/2)/n) along x (periodic): the central difference (and the D3Q19
    gradient, which reduces to it for a function of x alone) is exactly
    -sin(2 pi m/n) sin(2 pi m (i+1/2)/n) / h ... with the wrap at both ends."""
    nx, ny, nz, h, m = 12, 6, 8, 0.5, 1
    xi = 2 * np.pi * m * (np.arange(nx) + 0.5) / nx
    phi = np.ascontiguousarray(np.broadcast_to(np.cos(xi)[None, None, :], (nz, ny, nx)))
    E = oracle.efield(phi, h, (PER,) * 6, (0.0,) * 6, stencil=stencil)
    ex = np.sin(2 * np.pi * m / nx) * np.sin(xi) / h  # -(cos(x+d) - cos(x-d)) / (2h)
    assert np.abs(E[0] - ex[None, None, :]).max() < 1e-14
    assert np.abs(E[1]).max() < 1e-15 and np.abs(E[2]).max() < 1e-15


@pytest.mark.parametrize("stencil", [7, 19])
def test_periodic_force_by_translation(stencil):
    """The force on spheres across periodic walls equals that on the spheres moved into the
    interior with the potential rolled along: the gather and the gradient wrap."""
    nx, ny, nz = 12, 10, 14
    c, R, q = _dyadic_spheres()
    bc = (PER,) * 6
    phi = synth.random_field((nx, ny, nz), seed=9)
    shift = np.array([4, 3, 5])
    F = oracle.force_gather(phi, 1.0, bc, (0.0,) * 6, c, R, q, 2, stencil=stencil)
    rolled = np.roll(phi, shift=(shift[2], shift[1], shift[0]), axis=(0, 1, 2))
    Fm = oracle.force_gather(rolled, 1.0, bc, (0.0,) * 6, c + shift, R, q, 2, stencil=stencil)
    assert np.array_equal(F, Fm)


def test_periodic_adjoint_gradient_vs_finite_differences():
    dims = (12, 12, 16)
    nx, ny, nz = dims
    bc = (PER, PER, PER, PER, D, D)
    bcv = np.array([0.0, 0.0, 0.0, 0.0, 0.0, 1.0])
    c = np.array([[0.5, 6.0, 8.0], [7.0, 11.25, 6.5], [11.5, 0.75, 9.0]])  # across the x and y walls
    R = np.array([2.5, 2.0, 2.25])
    dens = np.array([1.0, -0.75, 0.5])
    wF = np.zeros((3, 3))
    wF[:, 0] = 1.0
    wF[:, 2] = 0.5
    shape = (nz, ny, nx)
    J, gd, gbc, _ = oracle.force_objective_and_grad(shape, 1.0, bc, bcv, c, R, dens, wF, tol=1e-14, max_cycles=300)

    def Jof(dn, v):
        rho = oracle.sphere_density(shape, 1.0, c, R, dn, 2, bc)
        f = oracle.rhs(rho, 1.0, bc, v)
        phi, _, _ = oracle.solve(f, 1.0, bc, tol=1e-14, max_cycles=300)
        return float(np.sum(wF * oracle.force_gather(phi, 1.0, bc, v, c, R, dn, 2)))

    step = 1e-3
    for s in range(3):
        dp, dm = dens.copy(), dens.copy()
        dp[s] += step
        dm[s] -= step
        fd = (Jof(dp, bcv) - Jof(dm, bcv)) / (2 * step)
        assert abs(fd - gd[s]) <= 1e-7 * max(1.0, abs(fd))
    vp, vm = bcv.copy(), bcv.copy()
    vp[5] += step
    vm[5] -= step
    fd = (Jof(dens, vp) - Jof(dens, vm)) / (2 * step)
    assert abs(fd - gbc[5]) <= 1e-7 * max(1.0, abs(fd))
    assert np.all(gbc[:4] == 0.0)


def test_periodic_faces_must_pair():
    with pytest.raises(ValueError):
        oracle.apply(np.zeros((4, 4, 4)), 1.0, (PER, D, D, D, D, D))


# ------------------------------------------------------------------------------------------
# Variable permittivity (Sec. 3: Galerkin coarsening with averaging restriction and constant
# prolongation extends the solver to discontinuous dielectricity): -div(eps grad phi) = rho

def dense_var(eps, h, bc, level, dims, k2=None):
    nx, ny, nz = dims
    n = nx * ny * nz
    A = np.zeros((n, n))
    for q in range(n):
        e = np.zeros(n)
        e[q] = 1.0
        A[:, q] = oracle.var_apply(e.reshape(nz, ny, nx), eps, h, bc, level, k2=k2).ravel()
    return A


def _jumping_eps(dims, seed, lo=1.0, hi=80.0):
    nx, ny, nz = dims
    rng = np.random.default_rng(seed)
    return np.where(rng.random((nz, ny, nx)) < 0.4, hi, lo) * np.exp(0.1 * rng.standard_normal((nz, ny, nx)))


@pytest.mark.parametrize("bc", [(D,) * 6, (N, N, N, N, D, D), (PER, PER, D, N, PER, PER)])
def test_var_constant_permittivity_is_the_constant_operator(bc):
    dims = (16, 12, 20)
    nx, ny, nz = dims
    rho = synth.random_field(dims, 1)
    bcv = (0.1, -0.2, 0.3, 0.0, -1.0, 1.0)
    eps = np.full((nz, ny, nx), 2.5)
    f = oracle.var_rhs(rho, eps, 0.5, bc, bcv)
    assert np.abs(f - 2.5 * oracle.rhs(rho, 0.5, bc, bcv, eps=2.5)).max() <= 1e-12 * np.abs(f).max()
    phi, k, rel = oracle.var_solve(f, eps, 0.5, bc, tol=1e-13, max_cycles=100)
    ref, k_ref, _ = oracle.solve(f / 2.5, 0.5, bc, tol=1e-13, max_cycles=100)
    assert np.linalg.norm(phi - ref) / np.linalg.norm(ref) < 1e-12 and k == k_ref
    Dw = oracle.var_coeffs(eps, bc, 1)
    assert np.all(np.stack(Dw[1:]) == 2.5 / 2.0)  # Galerkin weights, divided by the factor 2


@pytest.mark.parametrize("bc", [(D, N, N, D, D, N), (PER, PER, D, D, N, D), (PER,) * 6])
def test_var_galerkin_closed_form(bc):
    """(1/8) P^T A_l P / omega equals the level-(l+1) operator built from the coarsening formulas
    for a jumping permittivity (two levels; the correction factor omega = 2 sits in the coarse
    diffusion operator); with a reaction term, the coarse reaction is the Galerkin product alone:
    A_{l+1} = R A_diff P / omega + R M P."""
    fine = (12, 12, 12)
    eps = _jumping_eps(fine, 4)
    h = 0.5
    A0 = dense_var(eps, h, bc, 0, fine)
    assert np.abs(A0 - A0.T).max() <= 1e-12 * np.abs(A0).max()
    Pm = injection(fine)
    A1 = dense_var(eps, h, bc, 1, (6, 6, 6))
    assert np.abs((Pm.T / 8.0) @ A0 @ Pm / 2.0 - A1).max() <= 1e-13 * np.abs(A1).max()
    P2 = injection((6, 6, 6))
    A2 = dense_var(eps, h, bc, 2, (3, 3, 3))
    assert np.abs((P2.T / 8.0) @ A1 @ P2 / 2.0 - A2).max() <= 1e-13 * np.abs(A2).max()
    k2 = np.random.default_rng(6).random(eps.shape) * 3.0
    M0 = np.diag(k2.ravel())
    A1r = dense_var(eps, h, bc, 1, (6, 6, 6), k2=k2)
    ref = (Pm.T / 8.0) @ A0 @ Pm / 2.0 + (Pm.T / 8.0) @ M0 @ Pm
    assert np.abs(dense_var(eps, h, bc, 0, fine, k2=k2) - (A0 + M0)).max() <= 1e-13 * np.abs(A0).max()
    assert np.abs(A1r - ref).max() <= 1e-13 * np.abs(ref).max()


def test_var_dense_direct_solve():
    dims = (8, 6, 10)
    nx, ny, nz = dims
    bc = (D, N, PER, PER, D, N)
    eps = _jumping_eps(dims, 5)
    A = dense_var(eps, 1.0, bc, 0, dims)
    f = synth.random_field(dims, 3)
    x = np.linalg.solve(A, f.ravel()).reshape(nz, ny, nx)
    phi, k, rel = oracle.var_solve(f, eps, 1.0, bc, tol=1e-13, max_cycles=300)
    assert np.linalg.norm(phi - x) / np.linalg.norm(x) < 1e-11


@pytest.mark.parametrize("h", [1.0, 0.25])
def test_var_layered_dielectric_between_plates(h):
    """Two dielectric layers between plates at 0 and V (interface on a cell face): the flux is
    constant, so the exact potential is linear in each layer with slopes q/eps1 and q/eps2,
    V = q (L/2) (1/eps1 + 1/eps2). The harmonic-mean face weight and the wall folding reproduce
    it exactly at the cell centres."""
    nx, ny, nz = 6, 4, 16
    e1, e2, V = 3.0, 40.0, 2.0
    L = nz * h
    eps = np.empty((nz, ny, nx))
    eps[: nz // 2] = e1
    eps[nz // 2:] = e2
    bc = (N, N, PER, PER, D, D)
    bcv = (0.0, 0.0, 0.0, 0.0, 0.0, V)
    f = oracle.var_rhs(np.zeros((nz, ny, nx)), eps, h, bc, bcv)
    phi, k, rel = oracle.var_solve(f, eps, h, bc, tol=1e-14, max_cycles=200)
    q = V / ((L / 2) * (1 / e1 + 1 / e2))
    z = (np.arange(nz) + 0.5) * h
    exact = np.where(z < L / 2, q * z / e1, q * (L / 2) / e1 + q * (z - L / 2) / e2)
    assert np.abs(phi - exact[:, None, None]).max() < 1e-12 * V
    # the arithmetic mean at the interface would not reproduce it
    assert abs((phi[nz // 2] - phi[nz // 2 - 1]).max() - q * h * (1 / e1 + 1 / e2) / 2) < 1e-12



# ------------------------------------------------------------------------------------------
# Screened and Poisson-Boltzmann operators (the next application the paper names for the solver
# module): -div(eps grad phi) + k2 phi = rho and -div(eps grad phi) + k2 sinh(phi) = rho

@pytest.mark.parametrize("bc", [(PER, PER, N, N, D, D), (D,) * 6, (N, D, PER, PER, D, N)])
@pytest.mark.parametrize("kk", [0.05, 3.0])
def test_screened_spectral(bc, kk):
    """Constant eps and k2: the exact discrete solution by the sine/cosine/Fourier diagonalisation
    with every eigenvalue shifted by k2 h^2."""
    dims = (16, 12, 20)
    nx, ny, nz = dims
    f = synth.random_field(dims, 7)
    eps = np.full((nz, ny, nx), 1.0)
    k2 = np.full((nz, ny, nx), kk)
    phi, k, rel = oracle.var_solve(f, eps, 0.5, bc, tol=1e-13, max_cycles=100, k2=k2)
    ex = spectral.solve(f, 0.5, bc, shift=kk)
    assert np.linalg.norm(phi - ex) / np.linalg.norm(ex) < 1e-11 and k < 20


def _pb_residual_numpy(phi, f, h, bc, k2):
    """F = f - (-lap_h phi with the homogeneous-wall ghosts folded in) - k2 sinh(phi) for eps = 1,
    written independently of the oracle (ghost cells by padding)."""
    p = np.pad(phi, 1)
    for ax, q in ((2, 0), (1, 2), (0, 4)):
        lo = [slice(None)] * 3
        hi = [slice(None)] * 3
        src_lo = [slice(None)] * 3
        src_hi = [slice(None)] * 3
        lo[ax], hi[ax], src_lo[ax], src_hi[ax] = 0, -1, 1, -2
        if bc[q] == PER:
            src_lo[ax], src_hi[ax] = -2, 1
            p[tuple(lo)] = p[tuple(src_lo)]
            p[tuple(hi)] = p[tuple(src_hi)]
        else:
            sgn_lo = -1.0 if bc[q] == D else 1.0
            sgn_hi = -1.0 if bc[q + 1] == D else 1.0
            p[tuple(lo)] = sgn_lo * p[tuple(src_lo)]
            p[tuple(hi)] = sgn_hi * p[tuple(src_hi)]
    c = p[1:-1, 1:-1, 1:-1]
    lap = (p[1:-1, 1:-1, :-2] + p[1:-1, 1:-1, 2:] + p[1:-1, :-2, 1:-1] + p[1:-1, 2:, 1:-1] + p[:-2, 1:-1, 1:-1]
           + p[2:, 1:-1, 1:-1] - 6 * c) / h ** 2
    return f + lap - k2 * np.sinh(phi)


def test_pb_newton_satisfies_the_discrete_equation():
    """Newton's result satisfies -lap phi + k2 sinh(phi) = f (homogeneous walls, eps = 1) by an
    independent numpy evaluation, converges quadratically, and differs from the linearised
    (Debye-Hueckel) solution at large potential but agrees with it at small potential to O(phi^3)."""
    dims = (16, 12, 20)
    nx, ny, nz = dims
    bc = (PER, PER, N, N, D, D)
    eps = np.ones((nz, ny, nx))
    k2 = np.full((nz, ny, nx), 0.5)
    rho = synth.random_field(dims, 3) * 4.0
    f = oracle.var_rhs(rho, eps, 1.0, bc, (0.0,) * 6)
    phi, it, rel = oracle.pb_newton(f, eps, k2, 1.0, bc, tol=1e-12)
    F = _pb_residual_numpy(phi, f, 1.0, bc, k2)
    assert np.linalg.norm(F) / np.linalg.norm(f) < 1e-11 and it <= 8
    assert np.abs(phi).max() > 1.0  # nonlinear regime
    lin, _, _ = oracle.var_solve(f, eps, 1.0, bc, tol=1e-13, k2=k2)
    assert np.abs(phi - lin).max() > 0.05 * np.abs(lin).max()
    small = f * 1e-3
    phs, _, _ = oracle.pb_newton(small, eps, k2, 1.0, bc, tol=1e-13)
    lns, _, _ = oracle.var_solve(small, eps, 1.0, bc, tol=1e-14, k2=k2)
    assert np.abs(phs - lns).max() < 1e-5 * np.abs(lns).max()
    # quadratic convergence: residual after step n+1 <= C * (after step n)^2
    rels = [oracle.pb_newton(f, eps, k2, 1.0, bc, tol=0.0, max_newton=n)[2] for n in range(1, 5)]
    assert rels[2] < 10 * rels[1] ** 2 * 1e0 + 1e-14 and rels[1] < rels[0]


def test_pb_gouy_chapman_second_order():
    """A charged wall at potential phi0 in a 1:1 electrolyte (planar double layer): the continuum
    solution tanh(phi/4) = tanh(phi0/4) exp(-kappa z) (Gouy-Chapman); with the far wall at its
    exact value the discrete Newton solution converges to it at second order in h."""
    phi0, kappa, Lz = 2.0, 1.0, 12.0

    def gc(z):
        return 4.0 * np.arctanh(np.tanh(phi0 / 4.0) * np.exp(-kappa * z))

    errs = []
    for nz in (48, 96, 192):
        h = Lz / nz
        nx, ny = 4, 4
        bc = (PER, PER, PER, PER, D, D)
        eps = np.ones((nz, ny, nx))
        k2 = np.full((nz, ny, nx), kappa ** 2)
        f = oracle.var_rhs(np.zeros((nz, ny, nx)), eps, h, bc, (0.0, 0.0, 0.0, 0.0, phi0, gc(Lz)))
        phi, it, rel = oracle.pb_newton(f, eps, k2, h, bc, tol=1e-12)
        z = (np.arange(nz) + 0.5) * h
        errs.append(np.abs(phi[:, 0, 0] - gc(z)).max())
    assert errs[0] < 2e-2 and 3.0 < errs[0] / errs[1] < errs[1] / errs[2] < 4.2  # the rate approaches 4


def test_var_rhs_adjoint_is_the_transpose():
    """<lambda, var_rhs(rho, g)> is linear in (rho, g): its gradient by var_rhs_adjoint equals the
    explicit derivatives (random directions, exact in floating point up to rounding)."""
    dims = (8, 6, 10)
    nx, ny, nz = dims
    bc = (D, N, PER, PER, N, D)
    rng = np.random.default_rng(4)
    eps = 1.0 + rng.random((nz, ny, nx)) * 5.0
    lam = rng.standard_normal((nz, ny, nx))
    h = 0.5
    grho, gbc = oracle.var_rhs_adjoint(lam, eps, h, bc)
    rho = rng.standard_normal((nz, ny, nx))
    g = rng.standard_normal(6)
    J = lambda r, v: float(np.sum(lam * oracle.var_rhs(r, eps, h, bc, v)))  # noqa: E731
    assert abs(J(rho, g) - (np.sum(grho * rho) + np.dot(gbc, g))) < 1e-10 * max(1.0, abs(J(rho, g)))
    assert np.all(gbc[2:4] == 0.0)  # periodic faces have no value


def test_oracle_results_do_not_depend_on_the_thread_count():
    """The plane loops run on several threads; every cell takes the same operations and every
    field norm a fixed summation order, so solves, fields and forces are bit-identical for any
    thread count (also for a periodic axis of odd length, where the sweep stays serial)."""
    dims = (40, 36, 28)
    nx, ny, nz = dims
    sp = synth.random_spheres(dims, 5, 3.0, 9)
    bc, bcv = (1, 1, 2, 2, 0, 0), (0.1, -0.2, 0.0, 0.0, 0.0, 1.0)
    out = []
    n0 = oracle.set_threads(0)
    try:
        for t in (1, 3, 8):
            oracle.set_threads(t)
            rho = oracle.sphere_density((nz, ny, nx), 1.0, sp.centers, sp.radius, sp.density, 2, bc_type=bc)
            f = oracle.rhs(rho, 1.0, bc, bcv)
            phi, k, rel = oracle.solve(f, 1.0, bc, tol=1e-10)
            pm, km, relm = oracle.solve_mixed(f, 1.0, bc, tol=1e-9)
            E = oracle.efield(phi, 1.0, bc, bcv)
            F = oracle.force_gather(phi, 1.0, bc, bcv, sp.centers, sp.radius, sp.density, 2)
            odd = oracle.rbgs_half(phi[:, :, :39], f[:, :, :39], 1.0, (2, 2, 0, 0, 0, 0), 0)
            out.append((f, phi, k, rel, pm, km, relm, E, F, odd))
    finally:
        oracle.set_threads(n0)
    for o in out[1:]:
        for a, b in zip(out[0], o):
            assert np.array_equal(a, b)


# --------------------------------------------------------------------------------------------
# The mixed-precision outer step with its residual carried by recurrence (the folded operator of
# Sec. 2.4): pinned to the residual's definition. With dyadic data of few bits every FP64
# operation of oracle.residual is exact, so the recurrence must land exactly on the residual of
# the updated iterate; a wrong sign, a dropped or misplaced neighbour or a wrong wall shift of the
# diagonal breaks the equality.

@pytest.mark.parametrize("bc", [(0, 1, 1, 0, 0, 1), (2, 2, 0, 1, 2, 2), (1, 1, 2, 2, 0, 1), (0, 0, 0, 0, 0, 0)])
def test_defect_update_is_the_residual_of_the_updated_iterate(bc):
    rng = np.random.default_rng(sum(bc) + 7)
    shape = (6, 5, 8)
    phi = rng.integers(-64, 64, shape) / 8.0
    f = rng.integers(-100, 100, shape).astype(np.float64)
    e = rng.integers(-32, 32, shape) / 4.0
    for s in (0.125, 2.0):
        r = oracle.residual(phi, f, 1.0, bc)  # h = 1, level 0: c = 1, scaled = natural units
        phi2, r2 = oracle.defect_update(phi, e, r, s, bc)
        assert np.array_equal(phi2, phi + s * e)
        assert np.array_equal(r2, oracle.residual(phi2, f, 1.0, bc))


def test_defect_update_rounds_once():
    """Non-dyadic data: r' is the exactly rounded value of r + s (sum - D e), checked against
    rational arithmetic cell by cell; a zero correction leaves everything unchanged."""
    from fractions import Fraction

    rng = np.random.default_rng(3)
    shape = (3, 4, 4)
    bc = (0, 1, 2, 2, 1, 0)
    phi = rng.standard_normal(shape)
    e = rng.standard_normal(shape).astype(np.float32)
    r = rng.standard_normal(shape) * 1e-3
    s = 2.0 ** -5
    _, r2 = oracle.defect_update(phi, e, r, s, bc)
    nz, ny, nx = shape
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                acc = Fraction(float(r[k, j, i]))
                d = 6
                for axis, n in ((0, nx), (1, ny), (2, nz)):
                    for step in (-1, 1):
                        q = [i, j, k]
                        q[axis] += step
                        face = 2 * axis + (0 if step < 0 else 1)
                        if 0 <= q[axis] < n or bc[face] == 2:
                            q[axis] %= n
                            acc += Fraction(s) * Fraction(float(e[q[2], q[1], q[0]]))
                        else:
                            d += 1 if bc[face] == 0 else -1
                acc -= Fraction(s) * d * Fraction(float(e[k, j, i]))
                assert r2[k, j, i] == float(acc)
    phi3, r3 = oracle.defect_update(phi, np.zeros(shape), r, s, bc)
    assert np.array_equal(phi3, phi) and np.array_equal(r3, r)


@pytest.mark.parametrize("bc", [(N, N, N, N, D, D), (2, 2, N, D, D, N)])
def test_defect_recurrence_loop_takes_the_direct_loops_steps(bc):
    """The mixed solver's outer loop with the residual carried by recurrence (oracle.defect_update
    after the oracle's single-precision inner cycles, the residual evaluated directly only before
    the loop stops) against the oracle's loop with the direct FP64 residual after every step: the
    same outer steps, both below the tolerance by the direct residual, solutions equal to the inner
    cycles' single precision. The scale rule is the solver's: the largest power of two not above
    the RMS of the previous residual (of f first)."""
    dims = (24, 20, 16)
    nx, ny, nz = dims
    n = nx * ny * nz
    rho = synth.random_field(dims, 21)
    f = oracle.rhs(rho, 1.0, bc, (0.0, 0.0, 0.0, 0.0, 0.0, 1.0))  # h = 1: scaled = natural units
    tol, inner = 1e-9, 4

    def pow2_floor(v):
        m, e = math.frexp(v)  # v = m 2^e, 0.5 <= m < 1
        return math.ldexp(1.0, e - 1)

    phi_d, k_d, rel_d = oracle.solve_mixed(f, 1.0, bc, tol=tol, inner=inner)
    fn = np.linalg.norm(f)
    phi = np.zeros_like(f)
    r = f.copy()
    scale = pow2_floor(fn / math.sqrt(n))
    k = 0
    while True:
        rel = np.linalg.norm(r) / fn  # the recurrence's estimate
        if rel < tol and oracle.rel_residual(phi, f, 1.0, bc) < tol:
            break
        assert k < 20
        e = oracle.vcycles_f32(np.zeros_like(f), (r / scale).astype(np.float32), 1.0, bc, inner)
        r_used = r
        phi, r = oracle.defect_update(phi, e, r, scale, bc)
        scale = pow2_floor(np.linalg.norm(r_used) / math.sqrt(n))
        k += 1
    assert k == k_d and rel_d < tol
    assert oracle.rel_residual(phi, f, 1.0, bc) < tol
    # the carried residual stays the residual of the carried iterate (to FP64 rounding)
    assert np.linalg.norm(r - oracle.residual(phi, f, 1.0, bc)) <= 1e-13 * fn
    assert np.linalg.norm(phi - phi_d) <= 1e-6 * np.linalg.norm(phi_d)
