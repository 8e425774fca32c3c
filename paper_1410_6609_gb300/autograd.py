"""Differentiable electrostatics: density -> potential -> Coulomb forces, with hand-written adjoints.

Every forward and backward step runs in libccmg kernels; PyTorch only stores tensors and chains the
backward calls.

  * SphereDensity: per-sphere charge densities q -> rho(b) = sum_s q_s w_{s,b} (subsampled overlap,
    Sec. 2.4). Adjoint: dq_s = sum_b w_{s,b} g(b).
  * PoissonSolve: (rho, wall values) -> phi = A^-1 f(rho, walls) with f = rho/eps + wall terms
    (Sec. 2.4). A is symmetric, so the adjoint is one more solve with the same multigrid:
    A lam = dJ/dphi (homogeneous walls), dJ/drho = lam/eps, dJ/dwall = sum over the wall's cells of
    lam * (2/h^2 Dirichlet, 1/h Neumann).
  * ForceGather: (phi, q, wall values) -> F_s = h^3 q_s sum_b w_{s,b} E(x_b) (Eq. ElectrostatForce,
    central differences). Adjoint: scatter of the differences (ghosts included) plus the explicit
    q_s factor.

J = sum_s F_s,z with gradients w.r.t. the densities and the wall voltage is the adjoint workload.
"""
from __future__ import annotations

import torch

from .solver import Poisson


class SphereDensity(torch.autograd.Function):
    @staticmethod
    def forward(ctx, density, solver: Poisson, centers, radius, sf: int):
        ctx.solver, ctx.sf = solver, sf
        ctx.save_for_backward(centers, radius)
        return solver.sphere_density(centers, radius, density.detach(), sf)

    @staticmethod
    def backward(ctx, g):
        centers, radius = ctx.saved_tensors
        gd = ctx.solver.sphere_density_adjoint(centers, radius, g.contiguous(), ctx.sf)
        return gd, None, None, None, None


class PoissonSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, rho, bc_values, solver: Poisson, tol: float, max_cycles: int):
        ctx.solver, ctx.tol, ctx.max_cycles = solver, tol, max_cycles
        solver.set_bc_values(bc_values.detach().cpu().tolist())
        solver.set_rhs(rho.detach().contiguous())
        solver.set_solution(None)
        solver.solve(tol, max_cycles)
        return solver.solution()

    @staticmethod
    def backward(ctx, gphi):
        P = ctx.solver
        lam, _, _ = P.adjoint_solve(gphi.contiguous(), ctx.tol, ctx.max_cycles)
        grho, gbc = P.rhs_adjoint(lam)
        return grho, gbc, None, None, None


class ForceGather(torch.autograd.Function):
    @staticmethod
    def forward(ctx, phi, density, bc_values, solver: Poisson, centers, radius, sf: int):
        ctx.solver, ctx.sf = solver, sf
        ctx.save_for_backward(phi, density, bc_values, centers, radius)
        solver.set_bc_values(bc_values.detach().cpu().tolist())
        solver.set_solution(phi.detach().contiguous())
        return solver.force_gather(centers, radius, density.detach(), sf)

    @staticmethod
    def backward(ctx, gF):
        phi, density, bc_values, centers, radius = ctx.saved_tensors
        P = ctx.solver
        P.set_bc_values(bc_values.detach().cpu().tolist())
        P.set_solution(phi.detach().contiguous())
        gphi, gd, gbc = P.force_gather_adjoint(centers, radius, density.detach(), gF.contiguous(), ctx.sf)
        return gphi, gd, gbc, None, None, None, None


def coulomb_forces(solver: Poisson, density, bc_values, centers, radius, sf: int = 2, tol: float = 1e-12,
                   max_cycles: int = 200):
    """Forces on all spheres as a differentiable function of their densities and the wall values."""
    rho = SphereDensity.apply(density, solver, centers, radius, sf)
    phi = PoissonSolve.apply(rho, bc_values, solver, tol, max_cycles)
    return ForceGather.apply(phi, density, bc_values, solver, centers, radius, sf)


def z_force_objective(solver: Poisson, density, bc_values, centers, radius, sf: int = 2, tol: float = 1e-12,
                      max_cycles: int = 200):
    """J = sum over spheres of the z-component of the Coulomb force."""
    return coulomb_forces(solver, density, bc_values, centers, radius, sf, tol, max_cycles)[:, 2].sum()
