"""Seeded synthetic inputs for the electrostatics workloads.

This module holds input generation only (random sphere sets, analytic right-hand sides and the
workload table). It contains none of the solver's arithmetic, so both the CUDA path and the CPU
checker draw their inputs from here.

The paper's own workloads are synthetic (charged spheres between walls, Sec. 6 and Sec. 8.1);
no dataset is involved. Every generator takes an explicit seed and uses NumPy's PCG64.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

DIRICHLET = 0
NEUMANN = 1
PERIODIC = 2

# Faces: 0:-x 1:+x 2:-y 3:+y 4:-z 5:+z.
# Electrokinetic cell: phi = 0 at -z, phi = V at +z, zero-flux Neumann on the x and y walls.
WALL_BC_TYPE = (NEUMANN, NEUMANN, NEUMANN, NEUMANN, DIRICHLET, DIRICHLET)


def wall_bc_value(voltage: float = 1.0):
    return (0.0, 0.0, 0.0, 0.0, 0.0, float(voltage))


@dataclass
class Spheres:
    centers: np.ndarray  # [P, 3] (x, y, z) in physical units
    radius: np.ndarray   # [P]
    density: np.ndarray  # [P] uniform volume charge density of each sphere

    @property
    def count(self) -> int:
        return int(self.radius.shape[0])


def random_spheres(dims, count: int, radius: float, seed: int, h: float = 1.0,
                   max_tries: int = 1_000_000) -> Spheres:
    """Non-overlapping spheres at uniform-random positions with N(0,1) charge densities.

    Centres are uniform in [R+2, n-R-2] cells along each axis (continuous), so that every charged
    cell stays at least one cell away from the walls. A candidate is rejected when its distance to
    an accepted centre is below 2R+1 cells. Densities are drawn from N(0,1), then their mean is
    subtracted so that they sum to zero (all spheres share one radius, so the total charge of the
    ideal spheres is zero).
    """
    nx, ny, nz = dims
    rng = np.random.default_rng(seed)
    lo = radius + 2.0
    hi = np.array([nx, ny, nz], dtype=np.float64) - radius - 2.0
    if np.any(hi <= lo):
        raise ValueError("domain too small for the sphere radius")
    centers = np.zeros((count, 3))
    n = 0
    tries = 0
    min_d2 = (2.0 * radius + 1.0) ** 2
    while n < count:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("could not place the requested number of spheres")
        c = lo + rng.random(3) * (hi - lo)
        if n and np.min(np.sum((centers[:n] - c) ** 2, axis=1)) < min_d2:
            continue
        centers[n] = c
        n += 1
    density = rng.standard_normal(count)
    density = density - density.mean()
    return Spheres(centers=centers * h, radius=np.full(count, radius * h), density=density)


def manufactured_rhs(n: int) -> tuple[np.ndarray, float]:
    """f = 3 pi^2 sin(pi x) sin(pi y) sin(pi z) at the cell centres of the unit cube, h = 1/n.

    Returns (f[n, n, n] in [z, y, x] order, h). The exact solution with homogeneous Dirichlet
    walls is sin(pi x) sin(pi y) sin(pi z).
    """
    h = 1.0 / n
    x = (np.arange(n) + 0.5) * h
    s = np.sin(np.pi * x)
    f = 3.0 * np.pi ** 2 * s[:, None, None] * s[None, :, None] * s[None, None, :]
    return np.ascontiguousarray(f), h


def manufactured_exact(n: int) -> np.ndarray:
    h = 1.0 / n
    x = (np.arange(n) + 0.5) * h
    s = np.sin(np.pi * x)
    return np.ascontiguousarray(s[:, None, None] * s[None, :, None] * s[None, None, :])


def random_field(dims, seed: int, dtype=np.float64) -> np.ndarray:
    """Standard-normal field of shape [nz, ny, nx]."""
    nx, ny, nz = dims
    return np.random.default_rng(seed).standard_normal((nz, ny, nx)).astype(dtype)


@dataclass
class Workload:
    name: str
    dims: tuple
    h: float
    bc_type: tuple
    bc_value: tuple
    tol: float
    precision: str           # "fp64" or "mixed"
    sphere_count: int = 0
    sphere_radius: float = 4.0
    seed: int = 0
    subsample: int = 2
    extra: dict = field(default_factory=dict)

    def spheres(self) -> Spheres:
        return random_spheres(self.dims, self.sphere_count, self.sphere_radius, self.seed, self.h)


# The five workloads of the method's hot path: manufactured solution, 256^3 and 512^3
# charged-sphere cells, the batched set and the adjoint case.
WORKLOADS = {
    "manufactured32": Workload("manufactured32", (32, 32, 32), 1.0 / 32, (DIRICHLET,) * 6, (0.0,) * 6,
                               1e-10, "fp64"),
    "spheres256": Workload("spheres256", (256, 256, 256), 1.0, WALL_BC_TYPE, wall_bc_value(1.0), 1e-10,
                           "fp64", sphere_count=200, seed=2),
    "spheres512": Workload("spheres512", (512, 512, 512), 1.0, WALL_BC_TYPE, wall_bc_value(1.0), 1e-9,
                           "mixed", sphere_count=1600, seed=3),
    "adjoint256": Workload("adjoint256", (256, 256, 256), 1.0, WALL_BC_TYPE, wall_bc_value(1.0), 1e-10,
                           "fp64", sphere_count=32, seed=5),
    # the 512^3 setup at 384^3 (same sphere density, 675 spheres): each colour array of the finest
    # single-precision level (113 MB) is about the size of L2, the whole problem about 1.6 GB,
    # which suits detailed hardware-counter captures of the finest-level kernels
    "spheres384": Workload("spheres384", (384, 384, 384), 1.0, WALL_BC_TYPE, wall_bc_value(1.0), 1e-9,
                           "mixed", sphere_count=675, seed=6),
}


def batched_workloads(count: int = 64, seed: int = 4, sizes=(64, 96, 128, 192)) -> list[Workload]:
    """Independent charged-sphere systems of uneven size: sizes uniform from ``sizes``, sphere
    counts uniform in [20, 120]; system b draws its spheres with seed 1000 + b."""
    rng = np.random.default_rng(seed)
    n = rng.choice(np.array(sizes), size=count)
    p = rng.integers(20, 121, size=count)
    out = []
    for b in range(count):
        d = int(n[b])
        out.append(Workload(f"batch{b}", (d, d, d), 1.0, WALL_BC_TYPE, wall_bc_value(1.0), 1e-9, "mixed",
                            sphere_count=int(p[b]), seed=1000 + b))
    return out
