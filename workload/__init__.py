"""Seeded synthetic inputs shared by the oracle and the CUDA library.

This package holds only input generation: triangulated surfaces (the
polyhedral surface Gamma_h of the discretisation, Sec. 2.1) and the seeded
random initial data of Sec. 2.2.  It contains none of the method's arithmetic
(no finite-element assembly, no time stepping, no energies), so that the
oracle and the GPU path can consume identical inputs without sharing any code
that computes results.
"""

from .meshes import icosphere, ellipsoid, torus, dziuk, refine, project_dziuk, dziuk_phi, mesh_by_name  # noqa: F401
from .rng import splitmix64, uniform01, onehot_choice, initial_values  # noqa: F401
