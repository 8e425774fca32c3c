"""GB300-native cell-centred multigrid solver for the electrostatics step of Bartuschat & Ruede,
"Parallel Multiphysics Simulations of Charged Particles in Microfluidic Flows" (arXiv 1410.6609).

Compute lives in hand-written CUDA kernels for sm_103a behind the C ABI of ``include/ccmg.h``
(``libccmg.so``, built in-tree). ``solver.Poisson`` is the Python face of a solver context,
``autograd`` holds the differentiable operations, ``synth`` the seeded synthetic workloads.
"""

__all__ = ["synth", "solver", "autograd", "batch"]
