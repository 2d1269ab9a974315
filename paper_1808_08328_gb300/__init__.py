"""GB300-native solver for the four-field double porosity/permeability (DPP) model.

The CG-VMS P1 assembly, the field-split Schur preconditioner (Section 4.2,
Method 2, of Joshaghani, Chang, Nakshatrala & Knepley, 2018) with
smoothed-aggregation AMG on the selfp Schur blocks, and flexible GMRES all run
as hand-written CUDA kernels in libdpp.so (C ABI in include/dpp.h). This
package holds the ctypes binding (``binding``), the build step (``build``) and a
torch-tensor convenience layer (``system``). torch provides device memory and
streams only.
"""
from . import binding
from .binding import (DppError, DPP_FP64, DPP_MIXED_FP32_FP64, DPP_MEM_DEVICE, DPP_MEM_HOST,
                      dpp_adjoint_solve, dpp_apply_K, dpp_assemble, dpp_destroy_pc,
                      dpp_destroy_problem, dpp_export_pairs, dpp_get_rhs, dpp_last_error,
                      dpp_pc_apply, dpp_pc_export_level, dpp_pc_level_sizes, dpp_pc_opts_default,
                      dpp_problem_desc, dpp_problem_sizes, dpp_setup_pc, dpp_solve,
                      dpp_solve_opts_default, dpp_solve_rhs, dpp_status_string)


def __getattr__(name):
    # torch-dependent helpers are imported lazily so the binding loads without torch
    if name in ("DPPSystem", "DPPSolve", "DPPBatch", "solve_batched"):
        from . import system
        return getattr(system, name)
    raise AttributeError(name)
