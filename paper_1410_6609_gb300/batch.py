"""Many independent Poisson systems of different sizes solved together (libccmg batch ABI).

Every multigrid operation is one kernel launch over all systems; a system drops out of the
captured cycle graph as soon as its own residual meets the tolerance. The tile shapes of the
batched launches are chosen by ``autotune`` (which times the whole batched cycle per candidate);
results are cached per device and batch signature in a JSON file (``$CCMG_AUTOTUNE_CACHE`` or
``~/.cache/ccmg/autotune.json``) so that later runs reuse them.
"""
from __future__ import annotations

import ctypes
import json
import os

import torch

from . import _lib
from .solver import DIRICHLET, PRECISIONS, _ptr


def _cache_path() -> str:
    return os.environ.get("CCMG_AUTOTUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "ccmg",
                                                              "autotune.json"))


class BatchPoisson:
    """B systems; ``systems`` is a list of dicts with keys dims, h, bc_type, bc_value (eps optional)."""

    def __init__(self, systems, precision: str = "mixed", nu1: int = 2, nu2: int = 2, cgc_weight: float = 2.0,
                 mixed_inner: int = 4, device=None):
        if not torch.cuda.is_available():
            raise RuntimeError("libccmg needs a CUDA device; there is no CPU implementation")
        self.lib = _lib.load()
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        self.B = len(systems)
        arr = (_lib.MgParams * self.B)()
        self.shapes = []
        self.systems = []
        for b, sy in enumerate(systems):
            nx, ny, nz = (int(v) for v in sy["dims"])
            p = arr[b]
            self.lib.mg_default_params(ctypes.byref(p), nx, ny, nz, float(sy.get("h", 1.0)))
            bt = sy.get("bc_type", (DIRICHLET,) * 6)
            bv = sy.get("bc_value", (0.0,) * 6)
            for q in range(6):
                p.bc_type[q] = int(bt[q])
                p.bc_value[q] = float(bv[q])
            p.nu1, p.nu2, p.cgc_weight = int(nu1), int(nu2), float(cgc_weight)
            p.prec = PRECISIONS[precision]
            p.eps = float(sy.get("eps", 1.0))
            p.mixed_inner = int(mixed_inner)
            self.shapes.append((nz, ny, nx))
            self.systems.append(dict(dims=(nx, ny, nz), h=p.h, bc_type=tuple(bt), bc_value=tuple(bv)))
        self.precision = precision
        self.key_extra = f"{precision}|V({nu1},{nu2})|w{cgc_weight}|inner{mixed_inner}"
        with torch.cuda.device(self.device):
            self.stream = torch.cuda.current_stream(self.device)
            h = ctypes.c_void_p()
            st = self.lib.mg_batch_create(self.B, arr, ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h))
            if st != 0:
                raise _lib.MgError(st, "mg_batch_create: " + (self.lib.mg_batch_last_error(None) or b"").decode())
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.mg_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, what):
        if st != 0:
            raise _lib.MgError(st, what + ": " + (self.lib.mg_batch_last_error(self.h) or b"").decode())

    def _field(self, b, t):
        if not isinstance(t, torch.Tensor) or t.device != self.device or t.dtype != torch.float64:
            raise TypeError(f"field must be a float64 tensor on {self.device}")
        if t.numel() != int(torch.Size(self.shapes[b]).numel()):
            raise ValueError(f"system {b} needs shape {self.shapes[b]}")
        return t.contiguous()

    @property
    def kernel_launches(self) -> int:
        return int(self.lib.mg_batch_kernel_launches(self.h))

    def set_rhs(self, b: int, rho):
        rho = self._field(b, rho)
        self._check(self.lib.mg_batch_set_rhs(self.h, b, _ptr(rho)), "mg_batch_set_rhs")

    def set_rhs_all(self, rhos):
        """Every system's right-hand side in one call (three launches): rhos[b] as for set_rhs(b)."""
        if len(rhos) != self.B:
            raise ValueError(f"need {self.B} right-hand sides, got {len(rhos)}")
        fields = [self._field(b, r) for b, r in enumerate(rhos)]
        arr = (ctypes.c_void_p * self.B)(*[t.data_ptr() for t in fields])
        self._check(self.lib.mg_batch_set_rhs_all(self.h, arr), "mg_batch_set_rhs_all")

    def set_solution(self, b: int, phi=None):
        if phi is not None:
            phi = self._field(b, phi)
        self._check(self.lib.mg_batch_set_solution(self.h, b, _ptr(phi)), "mg_batch_set_solution")

    def reset_solutions(self):
        for b in range(self.B):
            self.set_solution(b, None)

    def solution(self, b: int):
        out = torch.empty(self.shapes[b], dtype=torch.float64, device=self.device)
        self._check(self.lib.mg_batch_get_solution(self.h, b, _ptr(out)), "mg_batch_get_solution")
        return out

    def vcycle(self, ncycles: int = 1):
        self._check(self.lib.mg_batch_vcycle(self.h, int(ncycles)), "mg_batch_vcycle")

    def solve(self, tol: float = 1e-9, max_cycles: int = 100, raise_on_fail: bool = True):
        cyc = (ctypes.c_int * self.B)()
        rel = (ctypes.c_double * self.B)()
        st = self.lib.mg_batch_solve(self.h, float(tol), int(max_cycles), cyc, rel)
        if raise_on_fail:
            self._check(st, "mg_batch_solve")
        return list(cyc), list(rel)

    def set_tiles(self, tiles):
        t = (ctypes.c_int * 4)(*[int(v) for v in tiles])
        self._check(self.lib.mg_batch_set_tiles(self.h, t), "mg_batch_set_tiles")

    def tiles(self):
        t = (ctypes.c_int * 4)()
        self._check(self.lib.mg_batch_get_tiles(self.h, t), "mg_batch_get_tiles")
        return tuple(t)

    def signature(self) -> str:
        dims = sorted(f"{d[0]}x{d[1]}x{d[2]}" for d in (s["dims"] for s in self.systems))
        hist = {}
        for d in dims:
            hist[d] = hist.get(d, 0) + 1
        name = torch.cuda.get_device_name(self.device)
        return name + "|" + self.key_extra + "|" + ",".join(f"{k}*{v}" for k, v in sorted(hist.items()))

    def autotune(self, reps: int = 3, use_cache: bool = True):
        """Pick tile shapes by timing whole batched cycles (cached per device and batch signature).
        Runs cycles on the current state: call before setting the problem."""
        path = _cache_path()
        key = self.signature()
        cache = {}
        if use_cache and os.path.exists(path):
            try:
                with open(path) as f:
                    cache = json.load(f)
            except (OSError, ValueError):
                cache = {}
            if key in cache:
                self.set_tiles(cache[key]["tiles"])
                return {"tiles": tuple(cache[key]["tiles"]), "cached": True, "ms": cache[key].get("ms")}
        best = (ctypes.c_int * 4)()
        ms = (ctypes.c_double * 16)()
        nc = ctypes.c_int()
        self._check(self.lib.mg_batch_autotune(self.h, int(reps), best, ms, ctypes.byref(nc)), "mg_batch_autotune")
        res = {"tiles": tuple(best), "cached": False, "ms": [ms[i] for i in range(nc.value)]}
        if use_cache:
            cache[key] = {"tiles": list(best), "ms": res["ms"]}
            try:
                os.makedirs(os.path.dirname(path), exist_ok=True)
                tmp = path + f".tmp{os.getpid()}"
                with open(tmp, "w") as f:
                    json.dump(cache, f, indent=1)
                os.replace(tmp, path)
            except OSError:
                pass
        return res
