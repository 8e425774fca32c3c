"""The allocation-free residual norm (mg_residual_norm_static) against the context's residual.

mg_residual_norm_static is for callers that cannot let the library allocate device memory (their
memory belongs to another allocator or pool, or an allocation's device-wide synchronisation is
not acceptable where they run). Its scratch is a static device array shared by all calls. This
file is collected last so that a run that stops at the first failure has run everything else.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_1410_6609_gb300 import _lib, synth
from paper_1410_6609_gb300.solver import Poisson

D, N = 0, 1


def _vp(t):
    return ctypes.c_void_p(t.data_ptr())


def test_rejects_nz_beyond_the_static_limit():
    # argument checks come first; no device work is enqueued for a rejected call
    lib = _lib.load()
    bc = (ctypes.c_int * 6)(*([D] * 6))
    assert lib.mg_residual_norm_static(8, 8, 4097, 1.0, bc, None, None, None, None) == _lib.MG_ERR_INVALID
    assert lib.mg_residual_norm_static(8, 8, 0, 1.0, bc, None, None, None, None) == _lib.MG_ERR_INVALID


@pytest.mark.gpu
def test_static_scratch_residual_matches_context_residual():
    lib = _lib.load()
    dims = (48, 40, 36)
    nx, ny, nz = dims
    bc_type = (N, N, D, N, D, D)
    bcv = (0.2, -0.1, 0.0, 0.3, 0.0, 1.0)
    h = 0.5
    P = Poisson(dims, h=h, bc_type=bc_type, bc_value=bcv)
    rho = torch.from_numpy(synth.random_field(dims, 12)).cuda()
    P.set_rhs(rho)
    P.set_solution(None)
    bc = (ctypes.c_int * 6)(*bc_type)
    out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    stream = ctypes.c_void_p(P.stream.cuda_stream)
    f = P.level_get(0, 1)  # the context's right-hand side with the wall terms, natural order
    for call in range(2):  # two calls in a row on the shared static scratch
        P.vcycle(1)
        rel_ctx, r_ctx = P.residual(field=True)
        phi = P.solution()
        st = lib.mg_residual_norm_static(nx, ny, nz, h, bc, _vp(phi), _vp(f), _vp(out), stream)
        assert st == _lib.MG_OK, call
        torch.cuda.synchronize()
        rel_static, rn_static = out.cpu().numpy()
        assert abs(rel_static - rel_ctx) <= 1e-12 * rel_ctx, (call, rel_static, rel_ctx)
        rn_ctx = float(torch.linalg.norm(r_ctx))
        assert abs(rn_static - rn_ctx) <= 1e-12 * rn_ctx, (call, rn_static, rn_ctx)
    P.close()
