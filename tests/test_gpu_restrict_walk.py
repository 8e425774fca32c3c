"""The FP64 residual + restriction by the fixed-point residual walk (FP64 mode, Sec. 3: coarse value
= the mean of the eight children's residuals, with the scaled right-hand sides g_c = 4 x mean).

The walk forms every fine residual of a tile plane in 64-bit fixed point at one exponent per ring
row (the same arithmetic as the outer residual of the mixed path) and adds the eight children of
each coarse cell across lanes, plane pairs and warp pairs. Checked against the oracle's
restrict(residual) and against the direct-load kernel on levels with ragged tiles in x, y and z,
walls and periodic axes (CCMG_RESTRICT=walk puts it on every packed level it can run on), and a
whole FP64 solve with it against the direct-load one.
"""
from __future__ import annotations

import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402

pytestmark = pytest.mark.gpu

D, N, PER = 0, 1, 2


def _with_restrict(kind, dims, **kw):
    from paper_1410_6609_gb300.solver import Poisson

    old = os.environ.get("CCMG_RESTRICT")
    os.environ["CCMG_RESTRICT"] = kind
    try:
        return Poisson(dims, precision="fp64", **kw)
    finally:
        if old is None:
            del os.environ["CCMG_RESTRICT"]
        else:
            os.environ["CCMG_RESTRICT"] = old


def _maxrel(a, b):
    m = np.abs(b).max()
    return np.abs(a - b).max() / (m if m > 0 else 1.0)


@pytest.mark.parametrize("dims,bc", [
    ((80, 20, 72), (D, N, N, D, D, N)),           # packed rows of 40 = 32 + 8, rows 8 + 8 + 4, planes 64 + 8
    ((80, 20, 72), (PER, PER, N, D, PER, PER)),   # the same with periodic x, y and z
    ((144, 80, 48), (N, N, N, N, D, D)),          # two levels wide enough for the walk
])
def test_walk_restriction_matches_oracle(dims, bc):
    h = 0.5
    a = _with_restrict("walk", dims, h=h, bc_type=bc)
    b = _with_restrict("vec", dims, h=h, bc_type=bc)
    rng = np.random.default_rng(sum(dims))
    walked = 0
    for l in range(a.num_levels - 1):
        nx, ny, nz = a.level_dims(l)
        c = oracle.level_coeff(h, l)
        phi = rng.standard_normal((nz, ny, nx))
        f = rng.standard_normal((nz, ny, nx)) * c
        f[rng.random(f.shape) < 0.5] = 0.0  # rows with and without a right-hand side
        out = []
        for P in (a, b):
            P.level_set(l, 0, torch.from_numpy(phi).cuda())
            P.level_set(l, 1, torch.from_numpy(f).cuda())
            P.level_set(l + 1, 1, torch.full(tuple(reversed(P.level_dims(l + 1))), np.nan,
                                             dtype=torch.float64, device="cuda"))
            P.op_residual_restrict(l)
            out.append(P.level_get(l + 1, 1).cpu().numpy())
        ref = oracle.restrict(oracle.residual(phi, f, c, bc))
        assert np.all(np.isfinite(out[0])), l  # every coarse cell written
        assert _maxrel(out[0], ref) < 1e-13, l
        assert _maxrel(out[0], out[1]) < 1e-13, l
        walked += nx // 2 >= 32
    assert walked >= 1
    a.close()
    b.close()


def test_walk_restriction_solve_matches_direct_load():
    """An FP64 solve with the walk's restriction on its wide levels (by default only levels of at
    least 2^25 cells take it) takes the direct-load solve's cycles and reaches the same solution to
    rounding."""
    from paper_1410_6609_gb300 import synth

    dims = (256, 128, 96)
    bc = (N, N, N, N, D, D)
    a = _with_restrict("walk", dims, bc_type=bc, bc_value=(0, 0, 0, 0, 0.0, 1.0))
    b = _with_restrict("vec", dims, bc_type=bc, bc_value=(0, 0, 0, 0, 0.0, 1.0))
    rho = torch.from_numpy(synth.random_field(dims, 78)).cuda()
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
