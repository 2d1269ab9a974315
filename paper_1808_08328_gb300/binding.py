"""ctypes binding of libdpp (include/dpp.h): argument marshalling only.

Every function here has the name of the C entry point it calls and does no
computation of its own. Device buffers are passed as raw pointers; the
convenience layer in ``system.py`` obtains them from torch tensors. If the
library has not been built, loading raises ``RuntimeError``. There is no CPU
fallback.
"""
from __future__ import annotations

import ctypes as C
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libdpp.so")

DPP_OK = 0
DPP_ERR_INVALID_ARGUMENT = 1
DPP_ERR_OUT_OF_MEMORY = 2
DPP_ERR_CUDA = 3
DPP_ERR_NOT_CONVERGED = 4
DPP_ERR_BREAKDOWN = 5
DPP_ERR_NONFINITE = 6
DPP_ERR_TIMEOUT = 7
DPP_ERR_BAD_STATE = 8

DPP_FP64 = 0
DPP_MIXED_FP32_FP64 = 1
DPP_CELL_SIMPLEX, DPP_CELL_Q1 = 0, 1
DPP_MEM_DEVICE = 0
DPP_MEM_HOST = 1


class dpp_problem_desc(C.Structure):
    _fields_ = [
        ("dim", C.c_int32), ("memory", C.c_int32),
        ("n_nodes", C.c_int64), ("n_cells", C.c_int64), ("n_bfacets", C.c_int64),
        ("coords", C.c_void_p), ("cells", C.c_void_p), ("bfacets", C.c_void_p),
        ("log_k1", C.c_void_p), ("log_k2", C.c_void_p),
        ("mu", C.c_double), ("beta", C.c_double), ("gamma_b", C.c_double * 3),
        ("p01", C.c_void_p), ("p02", C.c_void_p), ("cell_kind", C.c_int32),
    ]


class dpp_pc_opts(C.Structure):
    _fields_ = [
        ("cheb_degree_mass", C.c_int32), ("cheb_degree_amg", C.c_int32),
        ("coarse_max_rows", C.c_int32), ("max_levels", C.c_int32),
        ("strength_theta", C.c_double), ("cheb_ratio", C.c_double),
        ("use_lumped_diag", C.c_int32), ("precision", C.c_int32),
        ("sell_min_rows", C.c_int32), ("spmv_format", C.c_int32),
        ("composition", C.c_int32), ("mass_solver", C.c_int32), ("schedule_tuning", C.c_int32),
        ("smooth_filter", C.c_int32), ("cheb_degree_coarse", C.c_int32),
    ]


class dpp_solve_opts(C.Structure):
    _fields_ = [
        ("rtol", C.c_double), ("restart", C.c_int32), ("max_iters", C.c_int32),
        ("x0_zero", C.c_int32), ("x_memory", C.c_int32), ("check_every", C.c_int32),
        ("inner_rtol", C.c_double), ("wait_budget_cycles", C.c_int64),
        ("reorth_eta", C.c_double), ("matrix_free", C.c_int32),
    ]


class dpp_solve_info(C.Structure):
    _fields_ = [
        ("status", C.c_int32), ("iterations", C.c_int32), ("restarts", C.c_int32),
        ("levels", C.c_int32), ("rel_residual", C.c_double),
        ("ms_assemble", C.c_double), ("ms_setup", C.c_double), ("ms_solve", C.c_double),
    ]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class DppError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{status_name(status)}: {message}")
        self.status = status


_P = C.c_void_p
_SIGS = {
    "dpp_pc_opts_default": (None, [C.POINTER(dpp_pc_opts)]),
    "dpp_solve_opts_default": (None, [C.POINTER(dpp_solve_opts)]),
    "dpp_assemble": (C.c_int, [C.POINTER(dpp_problem_desc), C.c_int32, _P, C.POINTER(_P)]),
    "dpp_setup_pc": (C.c_int, [_P, C.POINTER(dpp_pc_opts), _P, C.POINTER(_P)]),
    "dpp_solve": (C.c_int, [_P, _P, C.POINTER(dpp_solve_opts), _P, C.POINTER(dpp_solve_info), _P]),
    "dpp_solve_rhs": (C.c_int, [_P, _P, C.POINTER(dpp_solve_opts), _P, _P,
                                C.POINTER(dpp_solve_info), _P]),
    "dpp_adjoint_solve": (C.c_int, [_P, _P, C.POINTER(dpp_solve_opts), _P, _P, _P, _P, _P, _P,
                                    C.POINTER(dpp_solve_info), _P]),
    "dpp_solve_batched": (C.c_int, [C.c_int32, C.POINTER(dpp_problem_desc), C.POINTER(dpp_pc_opts),
                                    C.POINTER(dpp_solve_opts), C.POINTER(C.c_void_p),
                                    C.POINTER(dpp_solve_info), _P]),
    "dpp_destroy_problem": (None, [_P]),
    "dpp_destroy_pc": (None, [_P]),
    "dpp_status_string": (C.c_char_p, [C.c_int32]),
    "dpp_last_error": (C.c_char_p, []),
    "dpp_problem_sizes": (C.c_int, [_P, C.POINTER(C.c_int64)]),
    "dpp_apply_K": (C.c_int, [_P, C.c_int32, _P, _P, _P]),
    "dpp_apply_K32": (C.c_int, [_P, C.c_int32, _P, _P, _P]),
    "dpp_apply_K_mf": (C.c_int, [_P, C.c_int32, _P, _P, _P]),
    "dpp_apply_K32_mf": (C.c_int, [_P, C.c_int32, _P, _P, _P]),
    "dpp_get_rhs": (C.c_int, [_P, _P, _P]),
    "dpp_export_pairs": (C.c_int, [_P, _P, _P, _P, _P]),
    "dpp_pc_apply": (C.c_int, [_P, _P, C.c_int32, _P, _P, _P]),
    "dpp_pc_level_sizes": (C.c_int, [_P, C.c_int32, C.POINTER(C.c_int64)]),
    "dpp_pc_export_level": (C.c_int, [_P, C.c_int32, _P, _P, _P, _P, _P, _P, _P]),
    "dpp_pc_hierarchies": (C.c_int, [_P, C.POINTER(C.c_int32)]),
    "dpp_pc_apply_mass": (C.c_int, [_P, _P, _P, _P, _P]),
    "dpp_pc_hierarchy_level_sizes": (C.c_int, [_P, C.c_int32, C.c_int32, C.POINTER(C.c_int64)]),
    "dpp_pc_hierarchy_export_level": (C.c_int, [_P, C.c_int32, C.c_int32, _P, _P, _P, _P, _P, _P,
                                                _P]),
    "dpp_adjoint_gradients_noalloc": (C.c_int, [_P, _P, _P, _P, _P, _P, _P]),
    "dpp_release_cached_memory": (C.c_int, []),
    "dpp_launch_count": (C.c_int64, []),
    "dpp_profile_enable": (C.c_int, [C.c_int32]),
    "dpp_profile_select": (C.c_int, [C.c_char_p]),
    "dpp_profile_read": (C.c_int, [C.c_char_p, C.POINTER(C.c_int64), C.POINTER(C.c_double),
                                   C.POINTER(C.c_double)]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load libdpp.so and declare every entry point's signature."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libdpp is not built ({path} missing); run "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = C.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def exported_symbols() -> list[str]:
    return list(_SIGS)


def status_name(status: int) -> str:
    try:
        return load().dpp_status_string(status).decode()
    except Exception:  # library missing: still give a readable name
        return f"status {status}"


def last_error() -> str:
    return load().dpp_last_error().decode()


def _check(status: int, allow=(DPP_OK,)) -> int:
    if status not in allow:
        raise DppError(status, last_error())
    return status


def _ptr(x) -> int | None:
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()  # torch tensor


# --------------------------------------------------------------------- entry points

def dpp_pc_opts_default() -> dpp_pc_opts:
    o = dpp_pc_opts()
    load().dpp_pc_opts_default(C.byref(o))
    return o


def dpp_solve_opts_default() -> dpp_solve_opts:
    o = dpp_solve_opts()
    load().dpp_solve_opts_default(C.byref(o))
    return o


def dpp_assemble(desc: dpp_problem_desc, precision: int = DPP_FP64, stream: int = 0) -> int:
    h = _P()
    _check(load().dpp_assemble(C.byref(desc), precision, stream or None, C.byref(h)))
    return h.value


def dpp_setup_pc(prob: int, opts: dpp_pc_opts | None = None, stream: int = 0) -> int:
    h = _P()
    _check(load().dpp_setup_pc(prob, C.byref(opts) if opts is not None else None,
                               stream or None, C.byref(h)))
    return h.value


def dpp_solve(prob: int, pc: int, opts: dpp_solve_opts | None, x, stream: int = 0,
              allow=(DPP_OK,)) -> dpp_solve_info:
    info = dpp_solve_info()
    st = load().dpp_solve(prob, pc, C.byref(opts) if opts is not None else None, _ptr(x),
                          C.byref(info), stream or None)
    _check(st, allow)
    return info


def dpp_solve_rhs(prob: int, pc: int, opts: dpp_solve_opts | None, b, x, stream: int = 0,
                  allow=(DPP_OK,)) -> dpp_solve_info:
    info = dpp_solve_info()
    st = load().dpp_solve_rhs(prob, pc, C.byref(opts) if opts is not None else None, _ptr(b),
                              _ptr(x), C.byref(info), stream or None)
    _check(st, allow)
    return info


def dpp_adjoint_solve(prob: int, pc: int, opts: dpp_solve_opts | None, x, dJdx, lam, g1, g2, gb,
                      stream: int = 0, allow=(DPP_OK,)) -> dpp_solve_info:
    info = dpp_solve_info()
    st = load().dpp_adjoint_solve(prob, pc, C.byref(opts) if opts is not None else None, _ptr(x),
                                  _ptr(dJdx), _ptr(lam), _ptr(g1), _ptr(g2), _ptr(gb),
                                  C.byref(info), stream or None)
    _check(st, allow)
    return info


def dpp_solve_batched(descs, pc_opts: dpp_pc_opts | None, opts: dpp_solve_opts | None, xs,
                      stream: int = 0, allow=(DPP_OK,)):
    """Batched solve; descs: list of dpp_problem_desc, xs: list of x buffers."""
    n = len(descs)
    darr = (dpp_problem_desc * n)(*descs)
    xarr = (C.c_void_p * n)(*[_ptr(x) for x in xs])
    infos = (dpp_solve_info * n)()
    st = load().dpp_solve_batched(n, darr, C.byref(pc_opts) if pc_opts is not None else None,
                                  C.byref(opts) if opts is not None else None, xarr, infos,
                                  stream or None)
    _check(st, allow)
    return st, [i.as_dict() for i in infos]


def dpp_destroy_problem(prob: int) -> None:
    if prob:
        load().dpp_destroy_problem(prob)


def dpp_destroy_pc(pc: int) -> None:
    if pc:
        load().dpp_destroy_pc(pc)


def dpp_status_string(status: int) -> str:
    return load().dpp_status_string(status).decode()


def dpp_last_error() -> str:
    return last_error()


def dpp_problem_sizes(prob: int) -> dict:
    out = (C.c_int64 * 6)()
    _check(load().dpp_problem_sizes(prob, out))
    return {"n_nodes": out[0], "n_cells": out[1], "n_pairs": out[2], "values_per_pair": out[3],
            "dim": out[4], "sell_groups": out[5]}


def dpp_apply_K(prob: int, transpose: bool, x, y, stream: int = 0) -> None:
    _check(load().dpp_apply_K(prob, 1 if transpose else 0, _ptr(x), _ptr(y), stream or None))


def dpp_apply_K32(prob: int, transpose: bool, x, y, stream: int = 0) -> None:
    _check(load().dpp_apply_K32(prob, 1 if transpose else 0, _ptr(x), _ptr(y), stream or None))


def dpp_apply_K_mf(prob: int, transpose: bool, x, y, stream: int = 0) -> None:
    _check(load().dpp_apply_K_mf(prob, 1 if transpose else 0, _ptr(x), _ptr(y), stream or None))


def dpp_apply_K32_mf(prob: int, transpose: bool, x, y, stream: int = 0) -> None:
    _check(load().dpp_apply_K32_mf(prob, 1 if transpose else 0, _ptr(x), _ptr(y),
                                   stream or None))


def dpp_get_rhs(prob: int, f, stream: int = 0) -> None:
    _check(load().dpp_get_rhs(prob, _ptr(f), stream or None))


def dpp_export_pairs(prob: int, row_ptr, col, vals, stream: int = 0) -> None:
    _check(load().dpp_export_pairs(prob, _ptr(row_ptr), _ptr(col), _ptr(vals), stream or None))


def dpp_pc_apply(prob: int, pc: int, transpose: bool, r, z, stream: int = 0) -> None:
    _check(load().dpp_pc_apply(prob, pc, 1 if transpose else 0, _ptr(r), _ptr(z), stream or None))


def dpp_pc_apply_mass(prob: int, pc: int, r, z, stream: int = 0) -> None:
    _check(load().dpp_pc_apply_mass(prob, pc, _ptr(r), _ptr(z), stream or None))


def dpp_pc_hierarchies(pc: int) -> int:
    n = C.c_int32(0)
    _check(load().dpp_pc_hierarchies(pc, C.byref(n)))
    return int(n.value)


def dpp_pc_level_sizes(pc: int, level: int, hierarchy: int = 0) -> dict:
    out = (C.c_int64 * 5)()
    _check(load().dpp_pc_hierarchy_level_sizes(pc, hierarchy, level, out))
    return {"rows": out[0], "nnz": out[1], "levels": out[2], "p_cols": out[3], "p_nnz": out[4]}


def dpp_pc_export_level(pc: int, level: int, row_ptr, col, val, p_row_ptr=None, p_col=None,
                        p_val=None, stream: int = 0, hierarchy: int = 0) -> None:
    _check(load().dpp_pc_hierarchy_export_level(pc, hierarchy, level, _ptr(row_ptr), _ptr(col),
                                                _ptr(val), _ptr(p_row_ptr), _ptr(p_col),
                                                _ptr(p_val), stream or None))


def dpp_adjoint_gradients_noalloc(prob: int, x, lam, g1, g2, gb, stream: int = 0) -> None:
    """Adjoint sensitivities with no device allocation (fixed library scratch)."""
    _check(load().dpp_adjoint_gradients_noalloc(prob, _ptr(x), _ptr(lam), _ptr(g1), _ptr(g2),
                                                _ptr(gb), stream or None))


def dpp_release_cached_memory() -> None:
    _check(load().dpp_release_cached_memory())


def dpp_launch_count() -> int:
    return int(load().dpp_launch_count())


def dpp_profile_enable(on: bool) -> None:
    _check(load().dpp_profile_enable(1 if on else 0))


def dpp_profile_select(families=None) -> None:
    """Time only these families (an iterable of names); None times every family."""
    arg = ",".join(families).encode() if families else None
    _check(load().dpp_profile_select(arg))


def dpp_profile_read(family: str) -> dict:
    n = C.c_int64()
    ms = C.c_double()
    by = C.c_double()
    _check(load().dpp_profile_read(family.encode(), C.byref(n), C.byref(ms), C.byref(by)))
    return {"launches": n.value, "ms": ms.value, "alg_bytes": by.value}
