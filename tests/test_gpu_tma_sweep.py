"""The TMA-staged single-precision half-sweep against the vectorised direct-load half-sweep.

Both evaluate phi_i = (g_i + sum of neighbours) / (6 + d_i) with the same operands in the same
order, so they must agree bit for bit. The TMA kernel marches tiles of 128 x 8 cells through
z-slabs, with the other colour's planes copied into shared memory by tensor-map loads whose
out-of-range elements (the walls) arrive as zeros. The grids here make every edge case of that
scheme occur: rows shorter than a tile and not a multiple of it, row counts that leave a partial
tile, plane counts that leave a partial slab, and mixed Dirichlet/Neumann walls (every diagonal
shift). The vectorised kernel is itself checked against the oracle's single-precision sweep in
test_gpu_parity.py.
"""
from __future__ import annotations

import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

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
