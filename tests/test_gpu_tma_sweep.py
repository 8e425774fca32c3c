"""The TMA-staged single-precision half-sweep against the vectorised direct-load half-sweep and
against the oracle.

Both evaluate phi_i = (g_i + sum of neighbours) / (6 + d_i) with the same operands in the same
order, so they must agree bit for bit. The TMA kernel marches tiles of 128 x 8 cells through
z-slabs, with the other colour's planes copied into shared memory by tensor-map loads whose
out-of-range elements (the walls) arrive as zeros. The grids here make every edge case of that
scheme occur: rows shorter than a tile and not a multiple of it, row counts that leave a partial
tile, plane counts that leave a partial slab, and mixed Dirichlet/Neumann walls (every diagonal
shift). Both kernels are also checked against the oracle's single-precision sweep, the TMA one
below at the sizes where the cycle runs it (plain, periodic and fused with the prolongation).
"""
from __future__ import annotations

import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402

pytestmark = pytest.mark.gpu

D, N = 0, 1
BC_MIX = (N, D, D, N, D, N)


def _with_sweep(kind, dims, **kw):
    from paper_1410_6609_gb300.solver import Poisson

    old = os.environ.get("CCMG_SWEEP")
    os.environ["CCMG_SWEEP"] = kind
    try:
        return Poisson(dims, precision="mixed", **kw)
    finally:
        if old is None:
            del os.environ["CCMG_SWEEP"]
        else:
            os.environ["CCMG_SWEEP"] = old


def _pair(dims, **kw):
    """Two mixed-precision contexts of the same problem: TMA half-sweeps (on every level the
    kernel can run on) and vectorised ones."""
    return _with_sweep("tma", dims, **kw), _with_sweep("vec", dims, **kw)


def test_default_policy():
    """By default only levels of 2^24 cells per colour and more take the TMA kernel."""
    from paper_1410_6609_gb300.solver import Poisson

    P = Poisson((512, 256, 256), precision="mixed")
    assert [P.level_sweep_kind(l) for l in range(3)] == ["tma", "vec", "vec"]
    P.close()
    P = Poisson((256, 128, 128), precision="fp64")
    assert P.level_sweep_kind(0) == "vec"
    P.close()


@pytest.mark.parametrize("dims", [(200, 88, 72), (256, 64, 96), (128, 160, 40), (512, 24, 48), (72, 84, 40)])
def test_tma_half_sweeps_bit_identical(dims):
    a, b = _pair(dims, bc_type=BC_MIX, bc_value=(0.0, 1.0, -0.5, 0.25, 0.0, 2.0))
    assert a.level_sweep_kind(0) == "tma"
    assert b.level_sweep_kind(0) == "vec"
    nx, ny, nz = dims
    rng = np.random.default_rng(sum(dims))
    phi = torch.from_numpy(rng.standard_normal((nz, ny, nx))).cuda()
    f = torch.from_numpy(rng.standard_normal((nz, ny, nx)) * 3.0).cuda()
    for P in (a, b):
        P.level_set(0, 0, phi)
        P.level_set(0, 1, f)
    for colour in (0, 1, 1, 0, 1, 0):
        a.op_smooth(0, colour)
        b.op_smooth(0, colour)
        torch.cuda.synchronize()
        xa, xb = a.level_get(0, 0), b.level_get(0, 0)
        assert torch.equal(xa, xb), f"colour {colour}: {(xa != xb).sum().item()} cells differ"
    assert not torch.equal(a.level_get(0, 0), phi)  # the sweeps did change the field
    a.close()
    b.close()


def test_wait_timeout_reported_and_context_usable():
    """A half-sweep whose plane copy never arrives: the bounded waits run out, the kernel sets the
    error flag and returns; the host reports MG_ERR_TIMEOUT and the context keeps working."""
    from paper_1410_6609_gb300 import _lib

    dims = (128, 64, 64)
    a, b = _pair(dims)
    assert a.level_sweep_kind(0) == "tma"
    rng = np.random.default_rng(3)
    phi = torch.from_numpy(rng.standard_normal((64, 64, 128))).cuda()
    f = torch.from_numpy(rng.standard_normal((64, 64, 128))).cuda()
    for P in (a, b):
        P.level_set(0, 0, phi)
        P.level_set(0, 1, f)
    before = a.level_get(0, 0)
    st = a.lib.mg_selftest_wait_timeout(a.ctx, 0)
    assert st == _lib.MG_ERR_TIMEOUT, st
    assert "bounded wait" in a.lib.mg_last_error(a.ctx).decode()
    assert torch.equal(a.level_get(0, 0), before)  # no CTA wrote the level
    # the flag was cleared: the sweeps and a solve run normally afterwards
    for colour in (0, 1):
        a.op_smooth(0, colour)
        b.op_smooth(0, colour)
    assert torch.equal(a.level_get(0, 0), b.level_get(0, 0))
    a.set_rhs(f)
    a.set_solution(None)
    k, rel = a.solve(1e-8, 40)
    assert rel < 1e-8
    assert a.lib.mg_selftest_wait_timeout(a.ctx, a.num_levels - 1) == _lib.MG_ERR_INVALID
    a.close()
    b.close()


@pytest.mark.parametrize("dims,tma_levels", [((256, 192, 128), 2), ((144, 84, 16), 1)])
def test_tma_solve_bit_identical(dims, tma_levels):
    """A whole mixed-precision solve equals the vectorised one: TMA half-sweeps and the
    TMA-fused prolongation + black sweep on the finest levels (a partial tile in x and y on the
    second grid)."""
    from paper_1410_6609_gb300 import synth

    a, b = _pair(dims, bc_type=(N, N, N, N, D, D), bc_value=(0, 0, 0, 0, 0.0, 1.0))
    assert [a.level_sweep_kind(l) for l in range(tma_levels + 1)] == ["tma"] * tma_levels + ["vec"]
    sp = synth.random_spheres(dims, 60 if dims[2] > 64 else 6, 4.0, 21, 1.0)
    dev = lambda v: torch.from_numpy(np.ascontiguousarray(v)).cuda()  # noqa: E731
    c, r, q = dev(sp.centers), dev(sp.radius), dev(sp.density)
    out = []
    for P in (a, b):
        rho = P.new_field()
        P.sphere_density(c, r, q, 2, out=rho)
        P.set_rhs(rho)
        P.set_solution(None)
        k, rel = P.solve(1e-9, 30)
        out.append((k, rel, P.solution().clone()))
    assert out[0][0] == out[1][0]
    assert out[0][1] == out[1][1]
    assert out[0][1] < 1e-9
    assert torch.equal(out[0][2], out[1][2])
    a.close()
    b.close()


# ------------------------------------------------------------------------------------------------
# The TMA-staged sweeps against the oracle directly (Sec. 5.3: red-black Gauss-Seidel), at sizes
# where they are the kernel the cycle runs. Both sides round in float; the GPU multiplies by
# 1/(6+d) where the oracle divides, so they agree to a few float ulps (1e-6 relative, the bound of
# the direct-load sweep's oracle test in test_gpu_parity.py).

F32_TOL = 1e-6
PER = 2


def _maxrel(a, b):
    m = np.abs(b).max()
    return np.abs(a - b).max() / (m if m > 0 else 1.0)


def _f32_fields(dims, seed, fscale=3.0):
    nx, ny, nz = dims
    rng = np.random.default_rng(seed)
    phi = rng.standard_normal((nz, ny, nx), dtype=np.float32)
    f = rng.standard_normal((nz, ny, nx), dtype=np.float32) * np.float32(fscale)
    return phi, f


def _check_sweeps_against_oracle(P, phi, f, bc, colours):
    """Each half-sweep from the same state, then the whole sequence from the oracle's own states."""
    dev = lambda a: torch.from_numpy(a.astype(np.float64)).cuda()  # noqa: E731
    c = oracle.level_coeff(1.0, 0)
    for colour in (0, 1):
        P.level_set(0, 0, dev(phi))
        P.level_set(0, 1, dev(f))
        P.op_smooth(0, colour)
        err = _maxrel(P.level_get(0, 0).cpu().numpy(), oracle.rbgs_half_f32(phi, f, c, bc, colour))
        assert err < F32_TOL, (colour, err)
    P.level_set(0, 0, dev(phi))
    ref = phi
    for colour in colours:
        P.op_smooth(0, colour)
        ref = oracle.rbgs_half_f32(ref, f, c, bc, colour)
    err = _maxrel(P.level_get(0, 0).cpu().numpy(), ref)
    assert err < 4 * F32_TOL, err


def test_tma_sweep_against_oracle_where_the_cycle_uses_it():
    """512 x 256 x 256: 2^24 cells per colour, the size from which the default policy stages the
    finest level's sweeps by TMA (the headline workload's finest-level kernel)."""
    from paper_1410_6609_gb300.solver import Poisson

    dims = (512, 256, 256)
    P = Poisson(dims, precision="mixed", bc_type=BC_MIX, bc_value=(0.0, 1.0, -0.5, 0.25, 0.0, 2.0))
    assert P.level_sweep_kind(0) == "tma"
    phi, f = _f32_fields(dims, 41)
    _check_sweeps_against_oracle(P, phi, f, BC_MIX, (0, 1, 1, 0))
    P.close()


@pytest.mark.parametrize("dims,bc", [
    ((520, 16, 16), (PER, PER, PER, PER, D, D)),    # three x tiles, the last one ragged
    ((528, 12, 40), (PER, PER, N, D, D, N)),        # three x tiles, a partial tile in y
    ((264, 40, 72), (N, D, PER, PER, PER, PER)),    # periodic y and z, a partial slab
])
def test_periodic_tma_sweep_against_oracle(dims, bc):
    """The staged sweep on periodic levels (selected by CCMG_SWEEP=tma): wrapped halo rows,
    columns and planes loaded by the threads, with tiles starting beyond x = 0 so that the left
    halo comes through the tensor copy and the wrapped column sits at the last tile's end. Also
    bit-identical to the direct-load sweep."""
    a, b = _pair(dims, bc_type=bc)
    assert a.level_sweep_kind(0) == "tma" and b.level_sweep_kind(0) == "vec"
    phi, f = _f32_fields(dims, sum(dims))
    _check_sweeps_against_oracle(a, phi, f, bc, (0, 1, 0, 1))
    dev = lambda v: torch.from_numpy(v.astype(np.float64)).cuda()  # noqa: E731
    for P in (a, b):
        P.level_set(0, 0, dev(phi))
        P.level_set(0, 1, dev(f))
    for colour in (0, 1, 1, 0):
        a.op_smooth(0, colour)
        b.op_smooth(0, colour)
        assert torch.equal(a.level_get(0, 0), b.level_get(0, 0)), colour
    a.close()
    b.close()


@pytest.mark.parametrize("dims,policy", [((512, 256, 256), None), ((272, 48, 40), "tma")])
def test_fused_prolongation_sweep_against_oracle(dims, policy):
    """The first black post-sweep fused with the prolongation (Sec. 3: phi += 2 P e_c, then the
    black half-sweep), on the TMA-staged kernel: its black cells against the oracle's
    prolong_correct_f32 followed by rbgs_half_f32, its red cells untouched."""
    from paper_1410_6609_gb300.solver import Poisson

    bc = (N, N, N, N, D, D)
    P = _with_sweep(policy, dims, bc_type=bc) if policy else Poisson(dims, precision="mixed", bc_type=bc)
    assert P.prolong_sweep_kind(0) == "tma"
    nx, ny, nz = dims
    phi, f = _f32_fields(dims, 43)
    rng = np.random.default_rng(44)
    ec = rng.standard_normal((nz // 2, ny // 2, nx // 2), dtype=np.float32) * np.float32(0.1)
    dev = lambda v: torch.from_numpy(v.astype(np.float64)).cuda()  # noqa: E731
    P.level_set(0, 0, dev(phi))
    P.level_set(0, 1, dev(f))
    P.level_set(1, 0, dev(ec))
    P.op_prolong_smooth(0)
    out = P.level_get(0, 0).cpu().numpy()
    ref = oracle.rbgs_half_f32(oracle.prolong_correct_f32(phi, ec, 2.0), f, 1.0, bc, 1)
    kk, jj, ii = np.indices(phi.shape)
    black = (ii + jj + kk) % 2 == 1
    assert _maxrel(out[black], ref[black]) < F32_TOL
    assert np.array_equal(out[~black], phi[~black].astype(np.float64))
    # the direct-load fused sweep gives the same bits
    Q = _with_sweep("vec", dims, bc_type=bc)
    assert Q.prolong_sweep_kind(0) == "vec"
    Q.level_set(0, 0, dev(phi))
    Q.level_set(0, 1, dev(f))
    Q.level_set(1, 0, dev(ec))
    Q.op_prolong_smooth(0)
    assert np.array_equal(Q.level_get(0, 0).cpu().numpy()[black], out[black])
    P.close()
    Q.close()


# ------------------------------------------------------------------------------------------------
# The FP64 half-sweep staged the same way (FP64 mode): every landed plane converted once into 64-bit
# fixed point at the plane's largest exponent, the six-neighbour sum formed exactly from there and
# rounded once, then + g and x 1/(6 + d). Against the oracle's FP64 half-sweep, the direct-load FP64
# sweep (which aligns per cell: the two agree to rounding, not bit for bit) and exact arithmetic.
# Tiles of 64 x 8 cells of a colour, ragged in x (hx 100, 68), in y (88, 40) and in the slabs.

def _fp64_pair(dims, **kw):
    from paper_1410_6609_gb300.solver import Poisson

    out = []
    for kind in ("tma", "vec"):
        old = os.environ.get("CCMG_SWEEP")
        os.environ["CCMG_SWEEP"] = kind
        try:
            out.append(Poisson(dims, precision="fp64", **kw))
        finally:
            if old is None:
                del os.environ["CCMG_SWEEP"]
            else:
                os.environ["CCMG_SWEEP"] = old
    return out


@pytest.mark.parametrize("dims", [(200, 88, 72), (256, 64, 96), (136, 40, 32), (512, 24, 48)])
def test_fp64_tma_half_sweeps_match_oracle(dims):
    a, b = _fp64_pair(dims, bc_type=BC_MIX, bc_value=(0.0, 1.0, -0.5, 0.25, 0.0, 2.0))
    assert a.level_sweep_kind(0) == "tma" and b.level_sweep_kind(0) == "vec"
    nx, ny, nz = dims
    rng = np.random.default_rng(sum(dims) + 1)
    phi = rng.standard_normal((nz, ny, nx))
    f = rng.standard_normal((nz, ny, nx)) * 3.0
    for colour in (0, 1):
        for P in (a, b):
            P.level_set(0, 0, torch.from_numpy(phi).cuda())
            P.level_set(0, 1, torch.from_numpy(f).cuda())
            P.op_smooth(0, colour)
        xa, xb = a.level_get(0, 0).cpu().numpy(), b.level_get(0, 0).cpu().numpy()
        ref = oracle.rbgs_half(phi, f, 1.0, BC_MIX, colour)
        assert _maxrel(xa, ref) < 1e-14 and _maxrel(xa, xb) < 1e-14
        kk, jj, ii = np.indices(phi.shape)
        assert np.array_equal(xa[(ii + jj + kk) % 2 != colour], phi[(ii + jj + kk) % 2 != colour])
    a.level_set(0, 0, torch.from_numpy(phi).cuda())
    ref = phi
    for colour in (0, 1, 1, 0, 1, 0):  # the same sequence on both sides
        a.op_smooth(0, colour)
        ref = oracle.rbgs_half(ref, f, 1.0, BC_MIX, colour)
    assert _maxrel(a.level_get(0, 0).cpu().numpy(), ref) < 1e-13
    a.close()
    b.close()


def test_fp64_tma_half_sweep_against_exact_arithmetic():
    """Values spread over 2^-30 .. 2^30 with zeros: each updated cell within the sum's bound of the
    exact (g + S)/(6 + d): S within 7/32 of an ulp of the largest other-colour value in the boxes of
    planes k-1..k+1 the kernel aligns to (bounded here by whole rows: the tile's 8 rows of the cell
    and the row beyond each side) plus half an ulp of itself, then three roundings (+ g,
    1/(6 + d), the product)."""
    import math
    dims = (136, 40, 32)
    bc = BC_MIX
    a, b = _fp64_pair(dims, bc_type=bc)
    b.close()
    nx, ny, nz = dims
    rng = np.random.default_rng(21)
    phi = rng.standard_normal((nz, ny, nx)) * np.exp2(rng.integers(-30, 31, (nz, ny, nx)))
    phi[rng.random(phi.shape) < 0.1] = 0.0
    f = rng.standard_normal((nz, ny, nx)) * np.exp2(rng.integers(-30, 31, (nz, ny, nx)))
    sh = {D: 1, N: -1}
    diag = np.full(phi.shape, 6, dtype=np.int64)
    diag[:, :, 0] += sh[bc[0]]
    diag[:, :, -1] += sh[bc[1]]
    diag[:, 0, :] += sh[bc[2]]
    diag[:, -1, :] += sh[bc[3]]
    diag[0] += sh[bc[4]]
    diag[-1] += sh[bc[5]]
    p = np.pad(phi, 1)
    nbs = [p[1:-1, 1:-1, :-2], p[1:-1, 1:-1, 2:], p[1:-1, :-2, 1:-1], p[1:-1, 2:, 1:-1], p[:-2, 1:-1, 1:-1],
           p[2:, 1:-1, 1:-1]]
    kk, jj, ii = np.indices(phi.shape)
    for colour in (0, 1):
        a.level_set(0, 0, torch.from_numpy(phi).cuda())
        a.level_set(0, 1, torch.from_numpy(f).cuda())
        a.op_smooth(0, colour)
        out = a.level_get(0, 0).cpu().numpy()
        # the largest |value| of the other colour over rows j-1..j+1 of planes k-1..k+1
        oth = np.where((ii + jj + kk) % 2 != colour, np.abs(phi), 0.0)
        R = oth.max(axis=2)  # (nz, ny) row maxima
        big = np.zeros((nz, ny))
        for z in range(nz):
            for y in range(ny):
                y0 = (y // 8) * 8
                big[z, y] = R[max(z - 1, 0):z + 2, max(y0 - 1, 0):y0 + 9].max()
        worst = 0.0
        for idx in zip(*np.nonzero((ii + jj + kk) % 2 == colour)):
            S = math.fsum(float(n[idx]) for n in nbs)
            D_ = int(diag[idx])
            exact = (f[idx] + S) / D_
            sbound = 7 / 32 * np.spacing(big[idx[0], idx[1]]) + np.spacing(abs(S))
            bound = sbound / D_ + 4 * np.spacing(abs(exact)) + np.spacing(abs(f[idx] + S)) / D_
            worst = max(worst, abs(out[idx] - exact) / bound)
        assert worst <= 1.0, (colour, worst)
    a.close()


def test_fp64_tma_default_policy_and_solve():
    """By default FP64 levels of 2^22 cells per colour and more take the staged sweep; a whole FP64
    solve with it takes the direct-load solve's cycles and reaches the same solution to rounding."""
    from paper_1410_6609_gb300 import synth
    from paper_1410_6609_gb300.solver import Poisson

    dims = (256, 256, 128)
    P = Poisson(dims, precision="fp64")
    assert [P.level_sweep_kind(l) for l in range(2)] == ["tma", "vec"]
    P.close()
    a, b = _fp64_pair(dims, bc_type=(N, N, N, N, D, D), bc_value=(0, 0, 0, 0, 0.0, 1.0))
    rho = torch.from_numpy(synth.random_field(dims, 77)).cuda()
    out = []
    for P in (a, b):
        P.set_rhs(rho)
        P.set_solution(None)
        k, rel = P.solve(1e-10, 40)
        out.append((k, rel, P.solution().cpu().numpy()))
    assert out[0][0] == out[1][0] and out[0][1] < 1e-10 and out[1][1] < 1e-10
    assert abs(out[0][1] - out[1][1]) <= 1e-3 * out[1][1]
    assert np.linalg.norm(out[0][2] - out[1][2]) <= 1e-9 * np.linalg.norm(out[1][2])
    a.close()
    b.close()


def test_fp64_tma_wait_timeout_reported_and_context_usable():
    from paper_1410_6609_gb300 import _lib

    dims = (128, 64, 64)
    a, b = _fp64_pair(dims)
    assert a.level_sweep_kind(0) == "tma"
    rng = np.random.default_rng(5)
    phi = torch.from_numpy(rng.standard_normal((64, 64, 128))).cuda()
    f = torch.from_numpy(rng.standard_normal((64, 64, 128))).cuda()
    for P in (a, b):
        P.level_set(0, 0, phi)
        P.level_set(0, 1, f)
    before = a.level_get(0, 0)
    assert a.lib.mg_selftest_wait_timeout(a.ctx, 0) == _lib.MG_ERR_TIMEOUT
    assert torch.equal(a.level_get(0, 0), before)
    for colour in (0, 1):
        a.op_smooth(0, colour)
        b.op_smooth(0, colour)
    assert _maxrel(a.level_get(0, 0).cpu().numpy(), b.level_get(0, 0).cpu().numpy()) < 1e-14
    a.close()
    b.close()


def test_fp64_tma_half_sweep_non_finite_values():
    """An infinity and a NaN in the iterate: the tile planes around them take the direct FP64 sum.
    Infinite and NaN results where the direct-load sweep has them, finite cells within 1e-14."""
    dims = (136, 40, 32)
    a, b = _fp64_pair(dims, bc_type=BC_MIX)
    nx, ny, nz = dims
    rng = np.random.default_rng(23)
    phi = rng.standard_normal((nz, ny, nx))
    phi[10, 20, 32] = np.inf     # a red cell (i + j + k even)
    phi[20, 5, 100] = -np.inf    # a black one
    phi[25, 30, 71] = np.nan     # red
    f = rng.standard_normal((nz, ny, nx))
    for colour in (0, 1):
        for P in (a, b):
            P.level_set(0, 0, torch.from_numpy(phi).cuda())
            P.level_set(0, 1, torch.from_numpy(f).cuda())
            P.op_smooth(0, colour)
        xa, xb = a.level_get(0, 0).cpu().numpy(), b.level_get(0, 0).cpu().numpy()
        assert np.array_equal(np.isnan(xa), np.isnan(xb)) and np.array_equal(np.isinf(xa), np.isinf(xb))
        fin = np.isfinite(xb)
        assert np.array_equal(xa[np.isinf(xa)], xb[np.isinf(xb)])
        assert np.abs(xa[fin] - xb[fin]).max() <= 1e-14 * np.abs(xb[fin]).max()
        assert (~fin).sum() >= 3
    a.close()
    b.close()
