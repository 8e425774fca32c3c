"""Exact discrete solver for the cell-centred 7-point Poisson operator by fast sine/cosine
transforms. Used only to pin the oracle; it shares no code with it.

In one dimension, the cell-centred second difference with a face boundary condition on each
end is diagonalised by a trigonometric transform (Strang, "The discrete cosine transform",
SIAM Review 41, 1999):

    ends (low, high)        basis over cell j = 0..n-1       eigenvalue of -d2 (times h^2)
    Dirichlet, Dirichlet     sin(pi (k+1) (j+1/2) / n)        2 - 2 cos(pi (k+1) / n)   DST-II
    Neumann,   Neumann       cos(pi k (j+1/2) / n)            2 - 2 cos(pi k / n)       DCT-II
    Dirichlet, Neumann       sin(pi (k+1/2) (j+1/2) / n)      2 - 2 cos(pi (k+1/2) / n) DST-IV
    Neumann,   Dirichlet     cos(pi (k+1/2) (j+1/2) / n)      2 - 2 cos(pi (k+1/2) / n) DCT-IV
    periodic,  periodic      exp(2 pi i k j / n)              2 - 2 cos(2 pi k / n)     DFT

(homogeneous conditions; the Dirichlet face value is zero on the face, i.e. the ghost is the
negated cell value; the Neumann ghost equals the cell value; a periodic axis wraps around). The 3D operator is the Kronecker
sum of the three 1D operators, so its eigenvalues are sums of the 1D ones.
"""
from __future__ import annotations

import numpy as np
from scipy import fft

D, N, P = 0, 1, 2


def _axis_transform(lo: int, hi: int):
    if (lo, hi) == (D, D):
        return (lambda a, ax: fft.dst(a, type=2, axis=ax, norm="ortho"),
                lambda a, ax: fft.idst(a, type=2, axis=ax, norm="ortho"),
                lambda n: 2.0 - 2.0 * np.cos(np.pi * (np.arange(n) + 1.0) / n))
    if (lo, hi) == (N, N):
        return (lambda a, ax: fft.dct(a, type=2, axis=ax, norm="ortho"),
                lambda a, ax: fft.idct(a, type=2, axis=ax, norm="ortho"),
                lambda n: 2.0 - 2.0 * np.cos(np.pi * np.arange(n) / n))
    if (lo, hi) == (D, N):
        return (lambda a, ax: fft.dst(a, type=4, axis=ax, norm="ortho"),
                lambda a, ax: fft.idst(a, type=4, axis=ax, norm="ortho"),
                lambda n: 2.0 - 2.0 * np.cos(np.pi * (np.arange(n) + 0.5) / n))
    if (lo, hi) == (N, D):
        return (lambda a, ax: fft.dct(a, type=4, axis=ax, norm="ortho"),
                lambda a, ax: fft.idct(a, type=4, axis=ax, norm="ortho"),
                lambda n: 2.0 - 2.0 * np.cos(np.pi * (np.arange(n) + 0.5) / n))
    if (lo, hi) == (P, P):
        return (lambda a, ax: fft.fft(a, axis=ax, norm="ortho"),
                lambda a, ax: fft.ifft(a, axis=ax, norm="ortho"),
                lambda n: 2.0 - 2.0 * np.cos(2.0 * np.pi * np.arange(n) / n))
    raise ValueError((lo, hi))


def solve(f: np.ndarray, h: float, bc_type, shift: float = 0.0) -> np.ndarray:
    """Exact solution of (A + shift) phi = f (homogeneous face BCs), f in [z, y, x] order."""
    nz, ny, nx = f.shape
    # array axis for x, y, z and the BC pair on that axis
    axes = [(2, nx, bc_type[0], bc_type[1]), (1, ny, bc_type[2], bc_type[3]),
            (0, nz, bc_type[4], bc_type[5])]
    g = np.array(f, dtype=np.float64, copy=True)
    lam = np.zeros(f.shape)
    # the real transforms first, the complex DFT of periodic axes last (transforms along
    # different axes commute); undone in the reverse order
    axes = sorted(axes, key=lambda t: t[2] == P)
    inv = []
    for ax, n, lo, hi in axes:
        fwd, bwd, eig = _axis_transform(lo, hi)
        g = fwd(g, ax)
        shape = [1, 1, 1]
        shape[ax] = n
        lam = lam + eig(n).reshape(shape) / (h * h)
        inv.append((ax, bwd, lo == P))
    lam = lam + shift
    if np.any(lam == 0.0):
        raise ValueError("singular operator (no Dirichlet face)")
    g = g / lam
    for ax, bwd, cplx in reversed(inv):
        if not cplx:
            g = np.real(g)  # the periodic axes are undone: real up to rounding
        g = bwd(g, ax)
    return np.real(g)
