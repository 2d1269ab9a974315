"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

Meshes (structured simplicial subdivisions of the unit square and cube, and
a disc wheel with one many-cell centre node),
per-cell log-permeability fields, batch recipes and the paper's
manufactured-solution boundary data. This package performs none of the
method's arithmetic (no assembly, no solve) and imports neither the oracle
nor the CUDA library.
"""
from .meshes import (Mesh, unit_square_tri, unit_cube_kuhn, unit_mesh, dof_count, boundary_facets,
                     disc_wheel, unit_square_quad, unit_cube_hex, tensor_facets, boundary_facets_q1)
from .fields import lognormal_logk, constant_logk, batch_recipe, sample_cells, rng
from .mms import MMSParams, PAPER, exact, boundary_pressures, nodal_exact
from .problems import Problem, mms_problem, heterogeneous_problem, wheel_problem

__all__ = [
    "Mesh", "unit_square_tri", "unit_cube_kuhn", "unit_mesh", "dof_count", "boundary_facets",
    "disc_wheel", "unit_square_quad", "unit_cube_hex", "tensor_facets", "boundary_facets_q1",
    "lognormal_logk", "constant_logk", "batch_recipe", "sample_cells", "rng",
    "MMSParams", "PAPER", "exact", "boundary_pressures", "nodal_exact",
    "Problem", "mms_problem", "heterogeneous_problem", "wheel_problem",
]
