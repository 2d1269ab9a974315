"""CPU oracle for the four-field DPP CG-VMS system. TEST INFRASTRUCTURE ONLY.

This package is the slow, plain, FP64 definition of what the GPU solver
computes. It exists to check the CUDA library. Only the test suite, the smoke
check and the benchmark's CPU-baseline leg may import it. The CUDA library and
its Python binding never import it, and it imports neither of them. The two
share no code; the only common module is the seeded input generator package
``inputs``, which holds no method arithmetic.

What it computes (Joshaghani, Chang, Nakshatrala, Knepley, "Composable block
solvers for the four-field double porosity/permeability model", 2018):
  * assembly.py: the CG-VMS stabilised mixed weak form (Eq.
    "CG_VMS_Weak_form", Section 3.3) on P1 simplices. It is evaluated term by
    term with exact quadrature, then assembled into K and f (Eq.
    "S4_linear_problem", Eqs. "S4_cg_stiffness_matrix" and "S4_cg_rhs",
    Section 4). Pressure data is imposed weakly on the whole boundary, as in the
    paper's appendix CG-VMS listing.
  * q1.py: the same CG-VMS form on Q1 quadrilaterals and hexahedra (the
    paper's QUAD and HEX meshes), with the tensor 2-point Gauss rule.
  * solve.py: an FP64 sparse direct solve of K x = f (SuperLU). The
    preconditioned FGMRES on the GPU reaches this same solution, up to its
    tolerance.
  * iterative.py: the same solution for meshes too large to factor, by a
    flexible GMRES driven to a true residual of 1e-13, preconditioned by the
    Method 2 Schur factorisation with incomplete-LU pieces.
  * errors.py: L2 errors against the manufactured solutions (Section 5,
    "errornorm" against the P1 interpolant), per-field parity norms, and
    mass-balance integrals (Eqs. "DG_GE_Darcy_mass_balance_1/2").
  * blocks.py: the field-split blocks A, B, C, D and the selfp Schur matrices
    S_p1, S_p2 (Eqs. "S4_sp1", "S4_sp2", Section 4.2), by their definitions on
    the assembled K.
  * inner.py: the inner solves of the velocity block A: ILU(0) and the
    Chebyshev-Jacobi polynomial, by their textbook definitions.
  * adjoint.py: the adjoint gradient of J = sum (p1 - p1_obs)^2 with respect to
    the per-cell log k1, log k2 and beta. Cross-checks are complex-step and
    central finite differences.

Every function states which of the paper's passages it follows.
"""
from .quadrature import cell_rule, facet_rule
from .assembly import (Geometry, geometry, element_matrices, element_rhs_body,
                       assemble, assemble_rhs, assemble_rows, slot_index, to_nodal, from_nodal)
from .solve import solve_direct, solve_dense, residual
from .iterative import solve_field_split_gmres
from .errors import (p1_mass_matrix, interp_l2_errors, field_rel_errors, field_slices,
                     mass_balance, FIELDS)
from .blocks import field_split_blocks, selfp_schur
from .inner import ilu0, ilu0_factors, ilu0_solve, chebyshev_jacobi
from .q1 import assemble_q1, q1_mass_matrix, mass_balance_q1, gauss_tensor, q1_basis
from .adjoint import (objective, objective_grad_x, adjoint_solve, adjoint_gradients,
                      complex_step_gradient, fd_gradient)

__all__ = [
    "cell_rule", "facet_rule", "Geometry", "geometry", "element_matrices", "element_rhs_body",
    "assemble", "assemble_rhs", "assemble_rows", "slot_index", "to_nodal", "from_nodal",
    "solve_direct", "solve_dense", "residual", "solve_field_split_gmres",
    "p1_mass_matrix", "interp_l2_errors", "field_rel_errors", "field_slices", "mass_balance",
    "FIELDS", "field_split_blocks", "selfp_schur", "ilu0", "ilu0_factors", "ilu0_solve",
    "chebyshev_jacobi", "assemble_q1", "q1_mass_matrix", "mass_balance_q1", "gauss_tensor",
    "q1_basis",
    "objective", "objective_grad_x", "adjoint_solve", "adjoint_gradients",
    "complex_step_gradient", "fd_gradient",
]
