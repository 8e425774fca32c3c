"""CPU oracle for the cell-centred multigrid electrostatics solver (arXiv 1410.6609).

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. The product path (``paper_1410_6609_gb300``) never
imports it and shares no code with it.

The arithmetic lives in ``ccmg_oracle.c`` (plain scalar loops, FP64, ``-ffp-contract=off``);
this module only compiles it with gcc, loads it with ctypes and marshals NumPy arrays. The one
exception is ``defect_update`` (NumPy with an exactly rounded ``math.fsum`` per cell).
Arrays are C-ordered ``[nz, ny, nx]`` (x fastest), matching the C layout ``i + nx*(j + ny*k)``.

Every function cites the paper passage it follows (section / equation / algorithm).
Pins that tie the oracle to something other than itself are in ``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = [os.path.join(_HERE, "ccmg_oracle.c"), os.path.join(_HERE, "oracle_level_ops.inc")]
_LIB_PATH = os.path.join(_HERE, "libccmg_oracle.so")
_lock = threading.Lock()
_lib = None

DIRICHLET = 0
NEUMANN = 1
PERIODIC = 2
CG_RTOL = 1e-14


def build(force: bool = False) -> str:
    """Compile the oracle shared library with gcc (plain C11, no FMA contraction), with OpenMP
    across z-planes where the compiler has it (the results do not depend on the thread count;
    without OpenMP the same loops run serially)."""
    newest = max(os.path.getmtime(p) for p in _SRC)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= newest:
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    base = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC", "-o", tmp, _SRC[0]]
    try:
        subprocess.check_call(base + ["-fopenmp", "-lm"], cwd=_HERE, stderr=subprocess.DEVNULL)
    except subprocess.CalledProcessError:
        subprocess.check_call(base + ["-Wno-unknown-pragmas", "-lm"], cwd=_HERE)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def set_threads(n: int) -> int:
    """Threads of the oracle's plane loops (n < 1 keeps the current setting); returns the count in
    effect (1 when the library was built without OpenMP)."""
    return int(_load().ccmg_or_set_threads(int(n)))


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            P = ctypes.c_void_p
            I = ctypes.c_int
            D = ctypes.c_double
            F = ctypes.c_float
            sig = {
                "ccmg_or_levels": (I, [I, I, I, P]),
                "ccmg_or_set_threads": (I, [I]),
                "ccmg_or_apply": (None, [P, P, I, I, I, D, P]),
                "ccmg_or_apply_f": (None, [P, P, I, I, I, F, P]),
                "ccmg_or_rbgs_half_f": (None, [P, P, I, I, I, F, P, I]),
                "ccmg_or_residual_f": (None, [P, P, P, I, I, I, F, P]),
                "ccmg_or_restrict_f": (None, [P, P, I, I, I]),
                "ccmg_or_prolong_correct_f": (None, [P, P, I, I, I, F]),
                "ccmg_or_residual": (None, [P, P, P, I, I, I, D, P]),
                "ccmg_or_rbgs_half": (None, [P, P, I, I, I, D, P, I]),
                "ccmg_or_restrict": (None, [P, P, I, I, I]),
                "ccmg_or_prolong_correct": (None, [P, P, I, I, I, D]),
                "ccmg_or_rhs": (None, [P, P, I, I, I, D, D, P, P]),
                "ccmg_or_rhs_adjoint": (None, [P, P, P, I, I, I, D, D, P]),
                "ccmg_or_cg": (I, [P, P, I, I, I, D, P, D, I]),
                "ccmg_or_cg_f": (I, [P, P, I, I, I, ctypes.c_float, P, D, I]),
                "ccmg_or_vcycles": (I, [P, P, I, I, I, D, P, I, I, D, I]),
                "ccmg_or_rel_residual": (D, [P, P, I, I, I, D, P]),
                "ccmg_or_solve": (I, [P, P, I, I, I, D, P, I, I, D, D, I, P]),
                "ccmg_or_solve_mixed": (I, [P, P, I, I, I, D, P, I, I, D, D, I, I, P]),
                "ccmg_or_vcycles_f": (I, [P, P, I, I, I, D, P, I, I, D, I]),
                "ccmg_or_efield": (None, [P, P, I, I, I, D, P, P]),
                "ccmg_or_efield_stencil": (None, [P, P, I, I, I, D, P, P, I]),
                "ccmg_or_efield_field": (None, [P, P, I, I, I, D, P, P, P, P, I]),
                "ccmg_or_rhs_field": (None, [P, P, I, I, I, D, D, P, P, P, P]),
                "ccmg_or_sphere_density": (None, [P, I, I, I, D, I, P, P, P, I]),
                "ccmg_or_sphere_density_adjoint": (None, [P, P, I, I, I, D, I, P, P, I]),
                "ccmg_or_sphere_density_bc": (None, [P, I, I, I, D, I, P, P, P, I, P]),
                "ccmg_or_sphere_density_adjoint_bc": (None, [P, P, I, I, I, D, I, P, P, I, P]),
                "ccmg_or_force_gather": (None, [P, I, I, I, D, P, P, I, P, P, P, I, P]),
                "ccmg_or_force_gather_stencil": (None, [P, I, I, I, D, P, P, I, P, P, P, I, I, P]),
                "ccmg_or_force_gather_field": (None, [P, I, I, I, D, P, P, P, P, I, P, P, P, I, I, P]),
                "ccmg_or_force_gather_adjoint": (None, [P, I, I, I, D, P, P, I, P, P, P, I, P, P, P, P]),
                "ccmg_or_var_coeffs": (None, [P, P, D, I, I, I, P, D, I, P, P, P, P]),
                "ccmg_or_var_apply": (None, [P, P, P, P, I, I, I, D, P, D, I]),
                "ccmg_or_var_rhs": (None, [P, P, P, I, I, I, D, P, P]),
                "ccmg_or_var_rhs_adjoint": (None, [P, P, P, P, I, I, I, D, P]),
                "ccmg_or_var_vcycles": (None, [P, P, P, P, I, I, I, D, P, I, I, D, I]),
                "ccmg_or_var_solve": (I, [P, P, P, P, I, I, I, D, P, I, I, D, D, I, P]),
                "ccmg_or_var_rel_residual": (D, [P, P, P, P, I, I, I, D, P]),
                "ccmg_or_pb_newton": (I, [P, P, P, P, I, I, I, D, P, I, I, D, D, I, D, I, P]),
                "ccmg_or_pb_residual": (D, [P, P, P, P, I, I, I, D, P, P]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _bc(bc_type) -> np.ndarray:
    """Face types (0:-x 1:+x 2:-y 3:+y 4:-z 5:+z): Dirichlet, Neumann or periodic; a periodic
    face needs its opposite face periodic too (Sec. 2.4: the domain is extended cyclically)."""
    a = np.ascontiguousarray(bc_type, dtype=np.int32)
    assert a.shape == (6,)
    for ax in range(3):
        if (a[2 * ax] == PERIODIC) != (a[2 * ax + 1] == PERIODIC):
            raise ValueError("periodic faces come in pairs")
    return a


def _dims(a: np.ndarray):
    nz, ny, nx = a.shape
    return nx, ny, nz


# --------------------------------------------------------------------------------------------
# Hierarchy and coefficients (Sec. 3)

def levels(nx: int, ny: int, nz: int) -> list[tuple[int, int, int]]:
    """Level dimensions: halve while every dimension is even and its half is >= 3 (Sec. 3)."""
    buf = np.zeros(3 * 32, dtype=np.int32)
    n = _load().ccmg_or_levels(nx, ny, nz, _p(buf))
    return [tuple(int(v) for v in buf[3 * l:3 * l + 3]) for l in range(n)]


def level_coeff(h: float, l: int) -> float:
    """c_l = 1/(2^l h^2): coefficient of the Galerkin operator on level l (Sec. 3)."""
    return 1.0 / (2.0 ** l * h * h)


# --------------------------------------------------------------------------------------------
# Single-level operations (Sec. 2.4 stencil, Sec. 3 transfers, Sec. 5.3 RBGS and CG)

def apply(phi, c: float, bc_type) -> np.ndarray:
    """A_l phi with the folded boundary stencil (Sec. 2.4)."""
    phi = _f64(phi)
    out = np.empty_like(phi)
    _load().ccmg_or_apply(_p(phi), _p(out), *_dims(phi), c, _p(_bc(bc_type)))
    return out


def apply_f32(phi, c: float, bc_type) -> np.ndarray:
    phi = np.ascontiguousarray(phi, dtype=np.float32)
    out = np.empty_like(phi)
    _load().ccmg_or_apply_f(_p(phi), _p(out), *_dims(phi), c, _p(_bc(bc_type)))
    return out


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float32)


def rbgs_half_f32(phi, f, c: float, bc_type, colour: int) -> np.ndarray:
    """Single-precision red/black half-sweep (the mixed-precision inner cycle, Sec. 5.3)."""
    phi = _f32(phi).copy()
    _load().ccmg_or_rbgs_half_f(_p(phi), _p(_f32(f)), *_dims(phi), c, _p(_bc(bc_type)), colour)
    return phi


def residual_f32(phi, f, c: float, bc_type) -> np.ndarray:
    phi = _f32(phi)
    r = np.empty_like(phi)
    _load().ccmg_or_residual_f(_p(phi), _p(_f32(f)), _p(r), *_dims(phi), c, _p(_bc(bc_type)))
    return r


def restrict_f32(r) -> np.ndarray:
    r = _f32(r)
    nz, ny, nx = r.shape
    fc = np.empty((nz // 2, ny // 2, nx // 2), dtype=np.float32)
    _load().ccmg_or_restrict_f(_p(r), _p(fc), nx, ny, nz)
    return fc


def prolong_correct_f32(phi, ec, omega: float = 2.0) -> np.ndarray:
    phi = _f32(phi).copy()
    _load().ccmg_or_prolong_correct_f(_p(phi), _p(_f32(ec)), *_dims(phi), omega)
    return phi


def residual(phi, f, c: float, bc_type) -> np.ndarray:
    """r = f - A_l phi (Sec. 8.3 'Resid')."""
    phi, f = _f64(phi), _f64(f)
    r = np.empty_like(phi)
    _load().ccmg_or_residual(_p(phi), _p(f), _p(r), *_dims(phi), c, _p(_bc(bc_type)))
    return r


def rbgs_half(phi, f, c: float, bc_type, colour: int) -> np.ndarray:
    """One red (colour 0, i+j+k even) or black (colour 1) Gauss-Seidel half-sweep (Sec. 5.3)."""
    phi = _f64(phi).copy()
    f = _f64(f)
    _load().ccmg_or_rbgs_half(_p(phi), _p(f), *_dims(phi), c, _p(_bc(bc_type)), colour)
    return phi


def restrict(r) -> np.ndarray:
    """Averaging restriction: coarse value = mean of the 8 children (Sec. 3)."""
    r = _f64(r)
    nz, ny, nx = r.shape
    fc = np.empty((nz // 2, ny // 2, nx // 2))
    _load().ccmg_or_restrict(_p(r), _p(fc), nx, ny, nz)
    return fc


def prolong_correct(phi, ec, omega: float = 2.0) -> np.ndarray:
    """phi += omega * (constant prolongation of ec) (Sec. 3, magnified correction)."""
    phi = _f64(phi).copy()
    ec = _f64(ec)
    _load().ccmg_or_prolong_correct(_p(phi), _p(ec), *_dims(phi), omega)
    return phi


def _bc_field(shape, bc_field):
    """Per-cell boundary values for the C oracle: one slot per face (faces 0,1 [nz, ny], 2,3
    [nz, nx], 4,5 [ny, nx]; None keeps the face's uniform value) -> (values, mask)."""
    nz, ny, nx = shape
    shapes = [(nz, ny), (nz, ny), (nz, nx), (nz, nx), (ny, nx), (ny, nx)]
    parts, on = [], np.zeros(6, dtype=np.int32)
    for q in range(6):
        v = None if bc_field is None else bc_field[q]
        if v is None:
            parts.append(np.zeros(shapes[q]).ravel())
        else:
            v = np.asarray(v, dtype=np.float64)
            assert v.shape == shapes[q], (q, v.shape, shapes[q])
            parts.append(v.ravel())
            on[q] = 1
    return np.ascontiguousarray(np.concatenate(parts)), on


def rhs(rho, h: float, bc_type, bc_value, eps: float = 1.0, bc_field=None) -> np.ndarray:
    """f = rho/eps with Dirichlet (+2g/h^2) and Neumann (+g/h) face terms (Sec. 2.4, 4.3); g per
    face cell where bc_field gives the face an array (see _bc_field)."""
    rho = _f64(rho)
    f = np.empty_like(rho)
    if bc_field is None:
        _load().ccmg_or_rhs(_p(rho), _p(f), *_dims(rho), h, eps, _p(_bc(bc_type)), _p(_f64(bc_value)))
    else:
        vals, on = _bc_field(rho.shape, bc_field)
        _load().ccmg_or_rhs_field(_p(rho), _p(f), *_dims(rho), h, eps, _p(_bc(bc_type)), _p(_f64(bc_value)),
                                  _p(vals), on.ctypes.data_as(ctypes.c_void_p))
    return f


def rhs_adjoint(lam, h: float, bc_type, eps: float = 1.0):
    """Adjoint of :func:`rhs`: returns (dJ/drho, dJ/dbc_value[6]) given lam = dJ/df."""
    lam = _f64(lam)
    grho = np.empty_like(lam)
    gbc = np.zeros(6)
    _load().ccmg_or_rhs_adjoint(_p(lam), _p(grho), _p(gbc), *_dims(lam), h, eps, _p(_bc(bc_type)))
    return grho, gbc


def cg(b, c: float, bc_type, rtol: float = CG_RTOL, maxit: int | None = None):
    """Unpreconditioned CG from x = 0 on A_l x = b (Sec. 5.3 coarse solver). Returns (x, iters)."""
    b = _f64(b)
    x = np.empty_like(b)
    if maxit is None:
        maxit = 2 * b.size
    it = _load().ccmg_or_cg(_p(x), _p(b), *_dims(b), c, _p(_bc(bc_type)), rtol, maxit)
    return x, it


CG_RTOL_F32 = 1e-5


def cg_f32(b, c: float, bc_type, rtol: float = CG_RTOL_F32, maxit: int | None = None):
    """The same CG in single precision (the coarsest grid of the mixed solver's single-precision
    inner cycles; not in the paper). Returns (x as float32, iters)."""
    b = _f32(b)
    x = np.empty_like(b)
    if maxit is None:
        maxit = 2 * b.size
    it = _load().ccmg_or_cg_f(_p(x), _p(b), *_dims(b), c, _p(_bc(bc_type)), rtol, maxit)
    return x, it


# --------------------------------------------------------------------------------------------
# Cycles and solves (Sec. 3, Sec. 5.3, Algorithm 1)

def vcycles(phi, f, h: float, bc_type, ncycles: int, nu1: int = 2, nu2: int = 2,
            omega: float = 2.0):
    """ncycles V(nu1,nu2)-cycles on A_0 phi = f (f BC-adapted). Returns (phi, last CG iters)."""
    phi = _f64(phi).copy()
    f = _f64(f)
    it = _load().ccmg_or_vcycles(_p(phi), _p(f), *_dims(phi), h, _p(_bc(bc_type)), nu1, nu2, omega,
                                 ncycles)
    return phi, it


def rel_residual(phi, f, h: float, bc_type) -> float:
    """||f - A_0 phi||_2 / ||f||_2 (Algorithm 1 termination quantity)."""
    phi, f = _f64(phi), _f64(f)
    return float(_load().ccmg_or_rel_residual(_p(phi), _p(f), *_dims(phi), h, _p(_bc(bc_type))))


def solve(f, h: float, bc_type, tol: float = 1e-10, max_cycles: int = 100, nu1: int = 2,
          nu2: int = 2, omega: float = 2.0, phi0=None):
    """Algorithm 1: V-cycles while ||r||/||f|| >= tol. Returns (phi, cycles, rel_res)."""
    f = _f64(f)
    phi = np.zeros_like(f) if phi0 is None else _f64(phi0).copy()
    rel = ctypes.c_double()
    k = _load().ccmg_or_solve(_p(phi), _p(f), *_dims(f), h, _p(_bc(bc_type)), nu1, nu2, omega, tol,
                              max_cycles, ctypes.byref(rel))
    return phi, k, rel.value


def defect_update(phi, e, r, s: float, bc_type):
    """One outer step of the mixed-precision defect correction with the residual carried by
    recurrence (not in the paper; its operator is the folded stencil of Sec. 2.4 on a level of
    Sec. 3). Adding s e to the iterate changes the residual by exactly -s A e, so

        phi' = phi + s e                 (s a power of two: s e is exact, one FP64 rounding),
        r'   = r - s A e = r + s (sum of e's six neighbours - (6 + d) e),

    in the scaled units of the level (r = g + sum - D phi, g = f / c_l): a neighbour across a
    periodic face is the cell at the opposite side, a Dirichlet face adds 1 to the diagonal and a
    Neumann face takes 1 from it (the correction has homogeneous walls). e is rounded to float
    first, as the single-precision inner cycles hold it. Every term of r' is then an exact double
    (a float times a small integer times a power of two), and r' is their sum rounded once to the
    nearest double (math.fsum, an exactly rounded summation). Pure-Python loop over the cells:
    small grids only. Returns (phi', r')."""
    phi, r = _f64(phi), _f64(r)
    ev = np.ascontiguousarray(e, dtype=np.float32).astype(np.float64)
    bc = _bc(bc_type)
    nz, ny, nx = ev.shape
    n = (nx, ny, nz)
    terms = [r.copy()]
    diag = np.full(ev.shape, 6.0)
    for face in range(6):
        axis, step = face // 2, (-1 if face % 2 == 0 else 1)
        nb = np.roll(ev, -step, axis=2 - axis)  # nb[cell] = e[cell + step along the axis]
        idx = np.arange(n[axis])
        edge = (idx == 0) if step < 0 else (idx == n[axis] - 1)  # cells whose neighbour is outside
        shape = [1, 1, 1]
        shape[2 - axis] = n[axis]
        edge = np.broadcast_to(edge.reshape(shape), ev.shape)
        if bc[face] != PERIODIC:  # the wrapped value is no neighbour: a wall
            nb = np.where(edge, 0.0, nb)
            diag = diag + np.where(edge, 1.0 if bc[face] == DIRICHLET else -1.0, 0.0)
        terms.append(s * nb)
    terms.append(-s * (diag * ev))
    stack = np.stack(terms, axis=-1).reshape(-1, len(terms))
    r_new = np.array([math.fsum(row) for row in stack]).reshape(ev.shape)
    return phi + s * ev, r_new


def vcycles_f32(phi, f, h: float, bc_type, ncycles: int, nu1: int = 2, nu2: int = 2, omega: float = 2.0):
    """ncycles single-precision V-cycles on A phi = f (the mixed solver's inner cycles; not in the
    paper). Returns phi as float32."""
    phi = _f32(phi).copy()
    _load().ccmg_or_vcycles_f(_p(phi), _p(_f32(f)), *_dims(phi), h, _p(_bc(bc_type)), nu1, nu2, omega, ncycles)
    return phi


def solve_mixed(f, h: float, bc_type, tol: float = 1e-9, max_cycles: int = 100, nu1: int = 2,
                nu2: int = 2, omega: float = 2.0, phi0=None, inner: int = 4):
    """FP64 defect correction around `inner` single-precision V-cycles per outer step.
    Returns (phi, outer iterations, rel_res)."""
    f = _f64(f)
    phi = np.zeros_like(f) if phi0 is None else _f64(phi0).copy()
    rel = ctypes.c_double()
    k = _load().ccmg_or_solve_mixed(_p(phi), _p(f), *_dims(f), h, _p(_bc(bc_type)), nu1, nu2, omega,
                                    tol, max_cycles, inner, ctypes.byref(rel))
    return phi, k, rel.value


# --------------------------------------------------------------------------------------------
# Fields and forces (Sec. 2.4: Eq. ElectrostatForce, central differences, subsampling)

def efield(phi, h: float, bc_type, bc_value, stencil: int = 7, bc_field=None) -> np.ndarray:
    """E = -grad phi; returns [3, nz, ny, nx]. stencil 7: central differences with BC ghost
    values; 19: the D3Q19 gradient (Sec. 2.4) where all 18 neighbours are inside, else 7."""
    phi = _f64(phi)
    E = np.empty((3,) + phi.shape)
    if bc_field is not None:
        vals, on = _bc_field(phi.shape, bc_field)
        _load().ccmg_or_efield_field(_p(phi), _p(E), *_dims(phi), h, _p(_bc(bc_type)), _p(_f64(bc_value)),
                                     _p(vals), on.ctypes.data_as(ctypes.c_void_p), int(stencil))
    elif stencil == 7:
        _load().ccmg_or_efield(_p(phi), _p(E), *_dims(phi), h, _p(_bc(bc_type)), _p(_f64(bc_value)))
    else:
        _load().ccmg_or_efield_stencil(_p(phi), _p(E), *_dims(phi), h, _p(_bc(bc_type)), _p(_f64(bc_value)),
                                       int(stencil))
    return E


def _spheres(centers, radius, density):
    c = _f64(centers).reshape(-1, 3)
    r = _f64(radius).reshape(-1)
    d = _f64(density).reshape(-1)
    assert c.shape[0] == r.shape[0] == d.shape[0]
    return c, r, d


def sphere_density(shape, h: float, centers, radius, density, sf: int = 2, bc_type=None) -> np.ndarray:
    """rho(b) = sum_s density_s * (subsampled overlap fraction of sphere s with cell b); along
    periodic axes of bc_type a sphere's charge reaches the cells at the opposite side."""
    nz, ny, nx = shape
    c, r, d = _spheres(centers, radius, density)
    rho = np.empty((nz, ny, nx))
    bc = None if bc_type is None else _p(_bc(bc_type))
    _load().ccmg_or_sphere_density_bc(_p(rho), nx, ny, nz, h, c.shape[0], _p(c), _p(r), _p(d), sf, bc)
    return rho


def sphere_density_adjoint(gfield, h: float, centers, radius, sf: int = 2, bc_type=None) -> np.ndarray:
    gfield = _f64(gfield)
    c, r, _ = _spheres(centers, radius, np.zeros(len(_f64(radius).reshape(-1))))
    g = np.zeros(c.shape[0])
    bct = None if bc_type is None else _bc(bc_type)
    _load().ccmg_or_sphere_density_adjoint_bc(_p(gfield), _p(g), *_dims(gfield), h, c.shape[0], _p(c),
                                              _p(r), sf, None if bct is None else _p(bct))
    return g


def force_gather(phi, h: float, bc_type, bc_value, centers, radius, density, sf: int = 2, stencil: int = 7,
                 bc_field=None):
    """F_s = h^3 sum_b w_{s,b} density_s E(x_b) (Eq. ElectrostatForce), E by the gradient stencil
    of efield (7 or 19) with its boundary values. Returns [P, 3]."""
    phi = _f64(phi)
    c, r, d = _spheres(centers, radius, density)
    F = np.empty((c.shape[0], 3))
    if bc_field is not None:
        vals, on = _bc_field(phi.shape, bc_field)
        _load().ccmg_or_force_gather_field(_p(phi), *_dims(phi), h, _p(_bc(bc_type)), _p(_f64(bc_value)),
                                           _p(vals), on.ctypes.data_as(ctypes.c_void_p), c.shape[0], _p(c), _p(r),
                                           _p(d), sf, int(stencil), _p(F))
    elif stencil == 7:
        _load().ccmg_or_force_gather(_p(phi), *_dims(phi), h, _p(_bc(bc_type)), _p(_f64(bc_value)),
                                     c.shape[0], _p(c), _p(r), _p(d), sf, _p(F))
    else:
        _load().ccmg_or_force_gather_stencil(_p(phi), *_dims(phi), h, _p(_bc(bc_type)), _p(_f64(bc_value)),
                                             c.shape[0], _p(c), _p(r), _p(d), sf, int(stencil), _p(F))
    return F


def force_gather_adjoint(phi, h: float, bc_type, bc_value, centers, radius, density, wF,
                         sf: int = 2):
    """Adjoint of :func:`force_gather` for J = sum wF * F. Returns (dJ/dphi, dJ/ddensity, dJ/dbc)."""
    phi = _f64(phi)
    c, r, d = _spheres(centers, radius, density)
    wF = _f64(wF).reshape(-1, 3)
    gphi = np.zeros_like(phi)
    gd = np.zeros(c.shape[0])
    gbc = np.zeros(6)
    _load().ccmg_or_force_gather_adjoint(_p(phi), *_dims(phi), h, _p(_bc(bc_type)), _p(_f64(bc_value)),
                                         c.shape[0], _p(c), _p(r), _p(d), sf, _p(wF), _p(gphi), _p(gd),
                                         _p(gbc))
    return gphi, gd, gbc


def force_objective_and_grad(shape, h: float, bc_type, bc_value, centers, radius, density, wF,
                             sf: int = 2, eps: float = 1.0, tol: float = 1e-13, max_cycles: int = 200):
    """J = sum wF * F(density, bc_value) and its gradient by one adjoint solve.

    Chain: density -> rho field (subsampling) -> f = rhs(rho, bc) -> phi = A^-1 f -> F.
    A is symmetric, so the adjoint solve A lam = dJ/dphi reuses the same multigrid (homogeneous
    BCs: the BC values enter only through the RHS). Returns (J, dJ/ddensity[P], dJ/dbc[6], info).
    """
    rho = sphere_density(shape, h, centers, radius, density, sf, bc_type)
    f = rhs(rho, h, bc_type, bc_value, eps)
    phi, k1, rel1 = solve(f, h, bc_type, tol=tol, max_cycles=max_cycles)
    F = force_gather(phi, h, bc_type, bc_value, centers, radius, density, sf)
    J = float(np.sum(_f64(wF).reshape(-1, 3) * F))
    gphi, gdens, gbc = force_gather_adjoint(phi, h, bc_type, bc_value, centers, radius, density, wF, sf)
    lam, k2, rel2 = solve(gphi, h, bc_type, tol=tol, max_cycles=max_cycles)
    grho, gbc_rhs = rhs_adjoint(lam, h, bc_type, eps)
    gdens = gdens + sphere_density_adjoint(grho, h, centers, radius, sf, bc_type)
    return J, gdens, gbc + gbc_rhs, {"phi": phi, "lam": lam, "cycles": (k1, k2), "rel": (rel1, rel2)}


# --------------------------------------------------------------------------------------------
# Variable permittivity (Sec. 3: Galerkin coarsening with averaging restriction and constant
# prolongation extends the solver to discontinuous dielectricity; -div(eps grad phi) = rho, face
# weights the harmonic mean of the two cells' permittivities), with an optional reaction term
# k2 phi (screened / linearised Poisson-Boltzmann operator; k2 >= 0 per cell, None: none). The
# coarse levels carry the diffusion part divided by the correction factor omega (the coarse-grid
# correction itself is not magnified) and the reaction part unmagnified.

def _k2(k2):
    return None if k2 is None else _p(_f64(k2))


def var_coeffs(eps, bc_type, level: int = 0, k2=None, h: float = 1.0, omega: float = 2.0):
    """Scaled weights (D, wx, wy, wz) of level `level` of the hierarchy of eps ([nz, ny, nx])."""
    eps = _f64(eps)
    nx, ny, nz = _dims(eps)
    d = levels(nx, ny, nz)[level]
    out = [np.empty((d[2], d[1], d[0])) for _ in range(4)]
    k2a = None if k2 is None else _f64(k2)
    _load().ccmg_or_var_coeffs(_p(eps), None if k2a is None else _p(k2a), h, nx, ny, nz, _p(_bc(bc_type)), omega,
                               level, *[_p(a) for a in out])
    return tuple(out)


def var_apply(phi, eps, h: float, bc_type, level: int = 0, k2=None, omega: float = 2.0) -> np.ndarray:
    """A_l phi with the coarse operator of level `level` (phi of that level's shape)."""
    eps, phi = _f64(eps), _f64(phi)
    k2a = None if k2 is None else _f64(k2)
    out = np.empty_like(phi)
    _load().ccmg_or_var_apply(_p(phi), _p(out), _p(eps), None if k2a is None else _p(k2a), *_dims(eps), h,
                              _p(_bc(bc_type)), omega, level)
    return out


def var_rhs(rho, eps, h: float, bc_type, bc_value) -> np.ndarray:
    """f = rho plus the wall terms 2 eps g / h^2 (Dirichlet), eps g / h (Neumann)."""
    rho, eps = _f64(rho), _f64(eps)
    f = np.empty_like(rho)
    _load().ccmg_or_var_rhs(_p(rho), _p(eps), _p(f), *_dims(rho), h, _p(_bc(bc_type)), _p(_f64(bc_value)))
    return f


def var_rhs_adjoint(lam, eps, h: float, bc_type):
    """Adjoint of var_rhs: (dJ/drho = lambda, dJ/dbc_value per face)."""
    lam, eps = _f64(lam), _f64(eps)
    grho = np.empty_like(lam)
    gbc = np.zeros(6)
    _load().ccmg_or_var_rhs_adjoint(_p(lam), _p(eps), _p(grho), _p(gbc), *_dims(lam), h, _p(_bc(bc_type)))
    return grho, gbc


def var_vcycles(phi, f, eps, h: float, bc_type, ncycles: int, nu1: int = 2, nu2: int = 2, omega: float = 2.0,
                k2=None):
    phi = _f64(phi).copy()
    f, eps = _f64(f), _f64(eps)
    k2a = None if k2 is None else _f64(k2)
    _load().ccmg_or_var_vcycles(_p(phi), _p(f), _p(eps), None if k2a is None else _p(k2a), *_dims(f), h,
                                _p(_bc(bc_type)), nu1, nu2, omega, ncycles)
    return phi


def var_solve(f, eps, h: float, bc_type, tol: float = 1e-10, max_cycles: int = 100, nu1: int = 2, nu2: int = 2,
              omega: float = 2.0, phi0=None, k2=None):
    """Algorithm 1 with the weighted operators. Returns (phi, cycles, relative residual)."""
    f, eps = _f64(f), _f64(eps)
    k2a = None if k2 is None else _f64(k2)
    phi = np.zeros_like(f) if phi0 is None else _f64(phi0).copy()
    rel = ctypes.c_double()
    k = _load().ccmg_or_var_solve(_p(phi), _p(f), _p(eps), None if k2a is None else _p(k2a), *_dims(f), h,
                                  _p(_bc(bc_type)), nu1, nu2, omega, tol, max_cycles, ctypes.byref(rel))
    return phi, k, rel.value


def var_rel_residual(phi, f, eps, h: float, bc_type, k2=None) -> float:
    k2a = None if k2 is None else _f64(k2)
    return _load().ccmg_or_var_rel_residual(_p(_f64(phi)), _p(_f64(f)), _p(_f64(eps)),
                                            None if k2a is None else _p(k2a), *_dims(_f64(f)), h, _p(_bc(bc_type)))


# --------------------------------------------------------------------------------------------
# Poisson-Boltzmann (the next application the paper names for the solver module):
# -div(eps grad phi) + k2 sinh(phi) = rho by Newton's method

def pb_newton(f, eps, k2, h: float, bc_type, tol: float = 1e-10, max_newton: int = 50, inner_tol: float = 1e-12,
              max_cycles: int = 200, nu1: int = 2, nu2: int = 2, omega: float = 2.0, phi0=None):
    """Newton's method for -div(eps grad phi) + k2 sinh(phi) = f. Returns (phi, steps, ||F||/||f||)."""
    f, eps, k2 = _f64(f), _f64(eps), _f64(k2)
    phi = np.zeros_like(f) if phi0 is None else _f64(phi0).copy()
    rel = ctypes.c_double()
    it = _load().ccmg_or_pb_newton(_p(phi), _p(f), _p(eps), _p(k2), *_dims(f), h, _p(_bc(bc_type)), nu1, nu2,
                                   omega, tol, max_newton, inner_tol, max_cycles, ctypes.byref(rel))
    return phi, it, rel.value


def pb_residual(phi, f, eps, k2, h: float, bc_type):
    """(F, ||F||/||f||) with F = f - A_eps phi - k2 sinh(phi)."""
    phi, f, eps, k2 = _f64(phi), _f64(f), _f64(eps), _f64(k2)
    F = np.empty_like(phi)
    r = _load().ccmg_or_pb_residual(_p(phi), _p(f), _p(eps), _p(k2), *_dims(f), h, _p(_bc(bc_type)), _p(F))
    return F, r
