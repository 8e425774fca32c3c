"""Python face of libccmg: a cell-centred multigrid Poisson solver context on one GPU.

PyTorch provides device memory and the CUDA stream only; every operation runs in the library's
CUDA kernels through the C ABI of ``include/ccmg.h``. Fields are float64 CUDA tensors of shape
``[nz, ny, nx]`` (x fastest), the layout the ABI expects.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib
from ._lib import DIRICHLET, NEUMANN, PERIODIC, MG_FP64, MG_MIXED, MgError  # noqa: F401

PRECISIONS = {"fp64": MG_FP64, "mixed": MG_MIXED}


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def scale_convert(x: torch.Tensor, e: torch.Tensor, y: torch.Tensor, sc: float):
    """The power-of-two products and conversions on caller data (mg_op_scale_convert): returns
    float(x * (1/sc)), fma(sc, double(e), y) and x * sc."""
    lib = _lib.load()
    n = x.numel()
    if not (x.dtype == torch.float64 and y.dtype == torch.float64 and e.dtype == torch.float32):
        raise TypeError("x, y must be float64 and e float32")
    if not (x.is_cuda and e.is_cuda and y.is_cuda) or e.numel() != n or y.numel() != n:
        raise ValueError("x, e, y must be CUDA tensors with the same number of elements")
    x, e, y = x.contiguous(), e.contiguous(), y.contiguous()
    xf = torch.empty(n, dtype=torch.float32, device=x.device)
    yo = torch.empty(n, dtype=torch.float64, device=x.device)
    xs = torch.empty(n, dtype=torch.float64, device=x.device)
    st = lib.mg_op_scale_convert(_ptr(x), _ptr(e), _ptr(y), n, float(sc), _ptr(xf), _ptr(yo), _ptr(xs),
                                 ctypes.c_void_p(torch.cuda.current_stream(x.device).cuda_stream))
    if st != _lib.MG_OK:
        raise MgError(st, "mg_op_scale_convert")
    return xf.view(x.shape), yo.view(x.shape), xs.view(x.shape)


class Poisson:
    """Solver context for -lap(phi) = rho/eps on an nx*ny*nz grid (see include/ccmg.h).

    Work is enqueued on the stream that is current when the context is created.
    """

    def __init__(self, dims, h: float = 1.0, bc_type=(DIRICHLET,) * 6, bc_value=(0.0,) * 6, nu1: int = 2,
                 nu2: int = 2, cgc_weight: float = 2.0, precision: str = "fp64", eps: float = 1.0,
                 mixed_inner: int = 4, device=None):
        if not torch.cuda.is_available():
            raise RuntimeError("libccmg needs a CUDA device; there is no CPU implementation")
        self.lib = _lib.load()
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        nx, ny, nz = (int(v) for v in dims)
        self.dims = (nx, ny, nz)
        self.shape = (nz, ny, nx)
        self.h = float(h)
        self.eps = float(eps)
        self.bc_type = tuple(int(v) for v in bc_type)
        self.bc_value = tuple(float(v) for v in bc_value)
        p = _lib.MgParams()
        self.lib.mg_default_params(ctypes.byref(p), nx, ny, nz, self.h)
        for q in range(6):
            p.bc_type[q] = self.bc_type[q]
            p.bc_value[q] = self.bc_value[q]
        p.nu1, p.nu2, p.cgc_weight = int(nu1), int(nu2), float(cgc_weight)
        p.prec = PRECISIONS[precision]
        p.eps = self.eps
        p.mixed_inner = int(mixed_inner)
        self.mixed_inner = int(mixed_inner)
        self.precision = precision
        self.params = p
        with torch.cuda.device(self.device):
            self.stream = torch.cuda.current_stream(self.device)
            ctx = ctypes.c_void_p()
            st = self.lib.mg_create(ctypes.byref(p), ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(ctx))
            _lib.check(self.lib, None, st, "mg_create")
        self.ctx = ctx

    # -- housekeeping ----------------------------------------------------------------------
    def close(self):
        if getattr(self, "ctx", None):
            self.lib.mg_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _check(self, st, what):
        _lib.check(self.lib, self.ctx, st, what)

    def _field(self, t, name, shape=None):
        shape = self.shape if shape is None else shape
        if not isinstance(t, torch.Tensor) or t.device != self.device or t.dtype != torch.float64:
            raise TypeError(f"{name} must be a float64 tensor on {self.device}")
        if tuple(t.shape) != tuple(shape) and t.numel() != int(np.prod(shape)):
            raise ValueError(f"{name} must have shape {shape}")
        return t.contiguous()

    def new_field(self, *lead):
        return torch.empty(*lead, *self.shape, dtype=torch.float64, device=self.device)

    @property
    def num_levels(self) -> int:
        return self.lib.mg_num_levels(self.ctx)

    def level_sweep_kind(self, level: int) -> str:
        """'tma' or 'vec': the kernel that performs the level's half-sweeps (mg_level_sweep_kind)."""
        k = self.lib.mg_level_sweep_kind(self.ctx, level)
        if k < 0:
            raise ValueError(f"no half-sweeps on level {level}")
        return "tma" if k == 1 else "vec"

    def level_dims(self, level: int):
        d = (ctypes.c_int * 3)()
        self._check(self.lib.mg_level_dims(self.ctx, level, d), "mg_level_dims")
        return tuple(d)

    @property
    def kernel_launches(self) -> int:
        return int(self.lib.mg_kernel_launches(self.ctx))

    # -- problem set-up --------------------------------------------------------------------
    def set_bc_values(self, values):
        v = (ctypes.c_double * 6)(*[float(x) for x in values])
        self._check(self.lib.mg_set_bc_values(self.ctx, v), "mg_set_bc_values")
        self.bc_value = tuple(float(x) for x in values)

    def set_rhs(self, rho):
        rho = self._field(rho, "rho")
        self._check(self.lib.mg_set_rhs(self.ctx, _ptr(rho)), "mg_set_rhs")

    def set_rhs_f(self, f):
        f = self._field(f, "f")
        self._check(self.lib.mg_set_rhs_f(self.ctx, _ptr(f)), "mg_set_rhs_f")

    def set_solution(self, phi=None):
        if phi is not None:
            phi = self._field(phi, "phi")
        self._check(self.lib.mg_set_solution(self.ctx, _ptr(phi)), "mg_set_solution")

    def solution(self, out=None):
        out = self.new_field() if out is None else out
        self._check(self.lib.mg_get_solution(self.ctx, _ptr(out)), "mg_get_solution")
        return out

    # -- iteration -------------------------------------------------------------------------
    def vcycle(self, ncycles: int = 1):
        self._check(self.lib.mg_vcycle(self.ctx, int(ncycles)), "mg_vcycle")

    def solve(self, tol: float = 1e-10, max_cycles: int = 100, raise_on_fail: bool = True):
        k = ctypes.c_int()
        rel = ctypes.c_double()
        st = self.lib.mg_solve(self.ctx, float(tol), int(max_cycles), ctypes.byref(k), ctypes.byref(rel))
        if raise_on_fail:
            self._check(st, "mg_solve")
        return k.value, rel.value

    def outer_counts(self) -> tuple[int, int, int]:
        """(outer cycles run by solve, those that carried the residual by recurrence, direct
        finest-level residual evaluations) since creation (mg_outer_counts)."""
        a = (ctypes.c_longlong * 3)()
        self._check(self.lib.mg_outer_counts(self.ctx, a), "mg_outer_counts")
        return int(a[0]), int(a[1]), int(a[2])

    def residual(self, field: bool = False):
        rel = ctypes.c_double()
        r = self.new_field() if field else None
        self._check(self.lib.mg_residual(self.ctx, ctypes.byref(rel), _ptr(r)), "mg_residual")
        return (rel.value, r) if field else rel.value

    # -- fields and forces -----------------------------------------------------------------
    def efield(self, out=None):
        out = self.new_field(3) if out is None else out
        self._check(self.lib.mg_efield(self.ctx, _ptr(out)), "mg_efield")
        return out

    def set_bc_field(self, face: int, values=None):
        """Wall values per cell of one face (None: back to the face's uniform value); values is a
        float64 tensor on the device of shape [nz, ny] (faces 0, 1), [nz, nx] (2, 3) or [ny, nx] (4, 5)."""
        nx, ny, nz = self.dims
        shapes = [(nz, ny), (nz, ny), (nz, nx), (nz, nx), (ny, nx), (ny, nx)]
        if values is None:
            self._check(self.lib.mg_set_bc_field(self.ctx, int(face), None), "mg_set_bc_field")
            return
        t = self._field(values, "bc field", shapes[int(face)] if 0 <= int(face) < 6 else (0,))
        self._check(self.lib.mg_set_bc_field(self.ctx, int(face), _ptr(t)), "mg_set_bc_field")

    def set_permittivity(self, eps=None):
        """Cell permittivities (float64 tensor [nz, ny, nx] on the device, positive) for
        -div(eps grad phi) = rho with Galerkin coarse operators (see mg_set_permittivity); None
        returns to the constant eps of the constructor."""
        if eps is None:
            self._check(self.lib.mg_set_permittivity(self.ctx, None), "mg_set_permittivity")
            return
        t = self._field(eps, "permittivity").contiguous()
        self._check(self.lib.mg_set_permittivity(self.ctx, _ptr(t)), "mg_set_permittivity")

    @property
    def has_permittivity(self) -> bool:
        return bool(self.lib.mg_has_permittivity(self.ctx))

    def set_reaction(self, k2=None):
        """Reaction coefficients k2 >= 0 per cell (float64 tensor [nz, ny, nx] on the device) for
        -div(eps grad phi) + k2 phi (see mg_set_reaction); None removes the term."""
        if k2 is None:
            self._check(self.lib.mg_set_reaction(self.ctx, None), "mg_set_reaction")
            return
        t = self._field(k2, "reaction").contiguous()
        self._check(self.lib.mg_set_reaction(self.ctx, _ptr(t)), "mg_set_reaction")

    def solve_pb(self, tol: float = 1e-10, max_newton: int = 30, inner_tol: float = 1e-3, max_cycles: int = 30,
                 raise_on_fail: bool = True):
        """Newton's method for -div(eps grad phi) + k2 sinh(phi) = f (see mg_solve_pb); returns
        (Newton steps, ||F|| / ||f||)."""
        k = ctypes.c_int()
        rel = ctypes.c_double()
        st = self.lib.mg_solve_pb(self.ctx, float(tol), int(max_newton), float(inner_tol), int(max_cycles),
                                  ctypes.byref(k), ctypes.byref(rel))
        if st != 0 and (raise_on_fail or st != _lib.MG_ERR_NOT_CONVERGED):
            self._check(st, "mg_solve_pb")
        return k.value, rel.value

    @property
    def gradient_stencil(self) -> int:
        """Gradient of efield / force_gather / step: 7 (D3Q7) or 19 (D3Q19 wherever it fits in the domain)."""
        return int(self.lib.mg_gradient_stencil(self.ctx))

    @gradient_stencil.setter
    def gradient_stencil(self, stencil: int):
        self._check(self.lib.mg_set_gradient_stencil(self.ctx, int(stencil)), "mg_set_gradient_stencil")

    @staticmethod
    def _sph(centers, radius, density=None):
        c = centers.contiguous()
        r = radius.contiguous()
        q = density.contiguous() if density is not None else None
        return c, r, q, int(r.shape[0])

    def sphere_density(self, centers, radius, density, sf: int = 2, out=None):
        c, r, q, P = self._sph(centers, radius, density)
        out = self.new_field() if out is None else out
        self._check(self.lib.mg_sphere_density(self.ctx, P, _ptr(c), _ptr(r), _ptr(q), int(sf), _ptr(out)),
                    "mg_sphere_density")
        return out

    def force_gather(self, centers, radius, density, sf: int = 2, out=None):
        c, r, q, P = self._sph(centers, radius, density)
        out = torch.empty(P, 3, dtype=torch.float64, device=self.device) if out is None else out
        self._check(self.lib.mg_force_gather(self.ctx, P, _ptr(c), _ptr(r), _ptr(q), int(sf), _ptr(out)),
                    "mg_force_gather")
        return out

    def force_gather_adjoint(self, centers, radius, density, wF, sf: int = 2):
        c, r, q, P = self._sph(centers, radius, density)
        wF = wF.contiguous()
        gphi = self.new_field()
        gd = torch.empty(P, dtype=torch.float64, device=self.device)
        gbc = torch.empty(6, dtype=torch.float64, device=self.device)
        self._check(self.lib.mg_force_gather_adjoint(self.ctx, P, _ptr(c), _ptr(r), _ptr(q), int(sf), _ptr(wF),
                                                     _ptr(gphi), _ptr(gd), _ptr(gbc)), "mg_force_gather_adjoint")
        return gphi, gd, gbc

    def sphere_density_adjoint(self, centers, radius, gfield, sf: int = 2):
        c, r, _, P = self._sph(centers, radius)
        gfield = self._field(gfield, "gfield")
        gd = torch.empty(P, dtype=torch.float64, device=self.device)
        self._check(self.lib.mg_sphere_density_adjoint(self.ctx, P, _ptr(c), _ptr(r), int(sf), _ptr(gfield),
                                                       _ptr(gd)), "mg_sphere_density_adjoint")
        return gd

    def rhs_adjoint(self, lam):
        lam = self._field(lam, "lambda")
        grho = self.new_field()
        gbc = torch.empty(6, dtype=torch.float64, device=self.device)
        self._check(self.lib.mg_rhs_adjoint(self.ctx, _ptr(lam), _ptr(grho), _ptr(gbc)), "mg_rhs_adjoint")
        return grho, gbc

    def adjoint_solve(self, g, tol: float = 1e-10, max_cycles: int = 100, out=None, raise_on_fail: bool = True):
        """lambda with A lambda = g, homogeneous walls, from zero (mg_adjoint_solve). Returns
        (lambda, cycles, relative residual); the context then holds g and lambda."""
        g = self._field(g, "g")
        out = self.new_field() if out is None else out
        k = ctypes.c_int()
        rel = ctypes.c_double()
        st = self.lib.mg_adjoint_solve(self.ctx, _ptr(g), _ptr(out), float(tol), int(max_cycles), ctypes.byref(k),
                                       ctypes.byref(rel))
        if raise_on_fail:
            self._check(st, "mg_adjoint_solve")
        return out, k.value, rel.value

    def step_host(self, centers: np.ndarray, radius: np.ndarray, density: np.ndarray, sf: int = 2,
                  tol: float = 1e-10, max_cycles: int = 100, forces: np.ndarray | None = None):
        """One electrostatics step through host buffers (see mg_step_host); tol < 0 runs exactly
        max_cycles cycles from the current potential (the warm-started time loop of Sec. 8.1)."""
        c = np.ascontiguousarray(centers, dtype=np.float64)
        r = np.ascontiguousarray(radius, dtype=np.float64)
        q = np.ascontiguousarray(density, dtype=np.float64)
        P = int(r.shape[0])
        F = np.empty((P, 3)) if forces is None else forces
        k = ctypes.c_int()
        rel = ctypes.c_double()
        vp = ctypes.c_void_p
        st = self.lib.mg_step_host(self.ctx, P, vp(c.ctypes.data), vp(r.ctypes.data), vp(q.ctypes.data), int(sf),
                                   float(tol), int(max_cycles), vp(F.ctypes.data), ctypes.byref(k),
                                   ctypes.byref(rel))
        self._check(st, "mg_step_host")
        return F, k.value, rel.value

    # -- level-wise operations (kernel verification) ---------------------------------------
    def level_set(self, level: int, which: int, t):
        shape = tuple(reversed(self.level_dims(level)))
        t = self._field(t, "level field", shape)
        self._check(self.lib.mg_level_set(self.ctx, level, which, _ptr(t)), "mg_level_set")

    def level_get(self, level: int, which: int):
        shape = tuple(reversed(self.level_dims(level)))
        out = torch.empty(*shape, dtype=torch.float64, device=self.device)
        self._check(self.lib.mg_level_get(self.ctx, level, which, _ptr(out)), "mg_level_get")
        return out

    def op_smooth(self, level: int, colour: int):
        self._check(self.lib.mg_op_smooth(self.ctx, level, colour), "mg_op_smooth")

    def op_residual_restrict(self, level: int, red_only: bool = False):
        if red_only:
            self._check(self.lib.mg_op_residual_restrict_red(self.ctx, level), "mg_op_residual_restrict_red")
        else:
            self._check(self.lib.mg_op_residual_restrict(self.ctx, level), "mg_op_residual_restrict")

    def op_prolong_correct(self, level: int):
        self._check(self.lib.mg_op_prolong_correct(self.ctx, level), "mg_op_prolong_correct")

    def op_prolong_smooth(self, level: int):
        """The cycle's first black post-sweep fused with the prolongation (mg_op_prolong_smooth):
        black cells swept from the corrected red values, red cells left uncorrected."""
        self._check(self.lib.mg_op_prolong_smooth(self.ctx, level), "mg_op_prolong_smooth")

    def prolong_sweep_kind(self, level: int) -> str:
        """'tma' or 'vec': the kernel of the fused prolongation sweep (mg_level_prolong_sweep_kind)."""
        k = self.lib.mg_level_prolong_sweep_kind(self.ctx, level)
        if k < 0:
            raise ValueError(f"no fused prolongation sweep on level {level}")
        return "tma" if k == 1 else "vec"

    def op_defect_update(self, phi, e, r, sc: float, sc_next: float, zero_start: bool = False):
        """One outer mixed-precision step with the residual carried by recurrence
        (mg_op_defect_update): from phi (ignored with zero_start), the correction e and the scaled
        residual r (natural order [nz, ny, nx] float64 CUDA tensors) returns phi + sc e, the new
        scaled residual over sc_next as the float pair (hi, lo) in float64 tensors, and the
        squared norm sum(hi^2) sc_next^2."""
        nx, ny, nz = self.dims
        shape = (nz, ny, nx)
        for t in (e, r) if zero_start else (phi, e, r):
            if t.dtype != torch.float64 or not t.is_cuda or tuple(t.shape) != shape:
                raise ValueError(f"fields must be float64 CUDA tensors of shape {shape}")
        e, r = e.contiguous(), r.contiguous()
        phi = phi.contiguous() if not zero_start else None
        phi_out = torch.empty(shape, dtype=torch.float64, device=e.device)
        hi = torch.empty_like(phi_out)
        lo = torch.empty_like(phi_out)
        ss = ctypes.c_double()
        self._check(self.lib.mg_op_defect_update(self.ctx, 1 if zero_start else 0, float(sc), float(sc_next),
                                                 _ptr(phi), _ptr(e), _ptr(r), _ptr(phi_out), _ptr(hi), _ptr(lo),
                                                 ctypes.byref(ss)), "mg_op_defect_update")
        return phi_out, hi, lo, ss.value

    def op_defect_step(self):
        """Enqueue the recurrence step alone on the current state (mg_op_defect_step; timing)."""
        self._check(self.lib.mg_op_defect_step(self.ctx), "mg_op_defect_step")

    def op_residual_norm(self):
        self._check(self.lib.mg_op_residual_norm(self.ctx), "mg_op_residual_norm")

    def op_coarse_solve(self) -> int:
        it = ctypes.c_int()
        self._check(self.lib.mg_op_coarse_solve(self.ctx, ctypes.byref(it)), "mg_op_coarse_solve")
        return it.value
