"""C ABI checks that need no GPU: the library builds and loads, exports every symbol the header
declares, and rejects invalid parameters before touching the device."""
import ctypes
import os
import re
import shutil

import pytest

from paper_1410_6609_gb300 import _build, _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ccmg.h")

needs_nvcc = pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                                reason="nvcc not available")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mg_[a-z0-9_]+)\s*\(", text)))


@needs_nvcc
def test_library_exports_every_declared_symbol():
    lib = _lib.load()
    names = declared_functions()
    assert len(names) >= 25
    for n in names:
        assert hasattr(lib, n), n
    # and the binding covers the whole header
    assert set(names) == set(_lib.SIGNATURES), set(names) ^ set(_lib.SIGNATURES)


def test_params_struct_matches_header():
    text = open(HEADER).read()
    body = re.search(r"typedef struct \{(.*?)\} mg_params;", text, flags=re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = re.findall(r"\b([a-z_][a-z0-9_]*)\s*(?:\[6\])?\s*[,;]", body)
    assert fields == [f for f, _ in _lib.MgParams._fields_], fields


def _params(**kw):
    lib = _lib.load()
    p = _lib.MgParams()
    lib.mg_default_params(ctypes.byref(p), 32, 32, 32, 1.0)
    for k, v in kw.items():
        if k in ("bc_type", "bc_value"):
            for q in range(6):
                getattr(p, k)[q] = v[q]
        else:
            setattr(p, k, v)
    return lib, p


@needs_nvcc
@pytest.mark.parametrize("bad", [
    dict(nx=31), dict(ny=2), dict(nz=0), dict(h=0.0), dict(h=-1.0), dict(eps=0.0),
    dict(bc_type=(1, 1, 1, 1, 1, 1)), dict(bc_type=(0, 0, 0, 0, 0, 7)), dict(nu1=-1), dict(nu2=0),
    dict(bc_type=(2, 0, 0, 0, 0, 0)), dict(bc_type=(0, 0, 0, 2, 0, 0)),  # periodic faces unpaired
    dict(bc_type=(2, 2, 2, 2, 2, 2)), dict(bc_type=(2, 2, 1, 1, 2, 2)),  # no Dirichlet face: singular
    dict(nu2=17), dict(prec=5), dict(bc_value=(0, 0, 0, 0, 0, float("nan"))),
    dict(nx=4 * 1024, ny=2 * 5 * 7, nz=2 * 5 * 7),  # coarsest grid too large
])
def test_create_rejects_invalid_params(bad):
    lib, p = _params(**bad)
    ctx = ctypes.c_void_p()
    st = lib.mg_create(ctypes.byref(p), None, ctypes.byref(ctx))
    assert st == _lib.MG_ERR_INVALID
    assert not ctx.value
    assert lib.mg_last_error(None)


@needs_nvcc
def test_null_context_is_invalid():
    lib = _lib.load()
    assert lib.mg_vcycle(None, 1) == _lib.MG_ERR_INVALID
    assert lib.mg_solve(None, 1e-10, 10, None, None) == _lib.MG_ERR_INVALID
    assert lib.mg_adjoint_solve(None, None, None, 1e-10, 10, None, None) == _lib.MG_ERR_INVALID
    assert lib.mg_destroy(None) == _lib.MG_ERR_INVALID
    assert lib.mg_op_defect_update(None, 0, 1.0, 1.0, None, None, None, None, None, None, None) == _lib.MG_ERR_INVALID
    assert lib.mg_op_defect_step(None) == _lib.MG_ERR_INVALID
    assert lib.mg_outer_counts(None, None) == _lib.MG_ERR_INVALID
    assert lib.mg_num_levels(None) == 0


def test_build_script_uses_sm103a():
    assert "arch=compute_103a,code=sm_103a" in " ".join(_build.ARCH)


@needs_nvcc
def test_batch_create_rejects_invalid_params():
    lib = _lib.load()
    arr = (_lib.MgParams * 2)()
    for b in range(2):
        lib.mg_default_params(ctypes.byref(arr[b]), 32, 32, 32, 1.0)
    arr[1].prec = 1  # systems of one batch must share the precision
    h = ctypes.c_void_p()
    assert lib.mg_batch_create(2, arr, None, ctypes.byref(h)) == _lib.MG_ERR_INVALID and not h.value
    assert lib.mg_batch_create(0, arr, None, ctypes.byref(h)) == _lib.MG_ERR_INVALID
    arr[1].prec = 0
    arr[1].nx = 30 + 1  # odd
    assert lib.mg_batch_create(2, arr, None, ctypes.byref(h)) == _lib.MG_ERR_INVALID
    assert b"even" in lib.mg_batch_last_error(None)
    assert lib.mg_batch_solve(None, 1e-9, 10, None, None) == _lib.MG_ERR_INVALID
    assert lib.mg_batch_set_rhs_all(None, None) == _lib.MG_ERR_INVALID


@needs_nvcc
def test_static_residual_rejects_unpaired_periodic_faces():
    lib = _lib.load()
    bc = (ctypes.c_int * 6)(2, 0, 0, 0, 0, 0)
    dummy = ctypes.c_void_p(16)  # never dereferenced: the types are checked first
    st = lib.mg_residual_norm_static(8, 8, 8, 1.0, bc, dummy, dummy, dummy, None)
    assert st == _lib.MG_ERR_INVALID
