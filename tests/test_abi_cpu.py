"""Host-side checks of the C ABI (no GPU needed).

The library must build, load, and export every entry point declared in
include/dpp.h. On a machine without a CUDA device, a call that needs the GPU
must fail with DPP_ERR_CUDA and must not fall back to the CPU.
"""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    from paper_1808_08328_gb300 import binding
    return binding


def _declared():
    src = open(os.path.join(ROOT, "include", "dpp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dpp_[A-Za-z_0-9]+)\s*\(", src)))


def test_header_declares_the_entry_points():
    names = _declared()
    for n in ("dpp_assemble", "dpp_setup_pc", "dpp_solve", "dpp_adjoint_solve",
              "dpp_destroy_problem", "dpp_destroy_pc", "dpp_status_string", "dpp_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    so = C.CDLL(lib.LIB_PATH)
    for n in _declared():
        assert hasattr(so, n), n
    assert sorted(lib.exported_symbols()) == _declared()


def test_defaults_and_status_strings(lib):
    o = lib.dpp_pc_opts_default()
    assert o.cheb_degree_mass == 2 and o.cheb_degree_amg == 2 and o.precision == lib.DPP_FP64
    assert o.cheb_ratio == 10.0
    s = lib.dpp_solve_opts_default()
    assert s.rtol == 1e-10 and s.restart == 30 and s.x0_zero == 1
    assert lib.dpp_status_string(lib.DPP_ERR_NOT_CONVERGED) == "DPP_ERR_NOT_CONVERGED"
    assert lib.dpp_status_string(99) == "DPP_ERR_UNKNOWN"


def test_struct_layouts_match_header(lib):
    # sizes fixed by the C declarations (x86-64 and aarch64 share this ABI)
    assert C.sizeof(lib.dpp_problem_desc) == 4 + 4 + 3 * 8 + 5 * 8 + 2 * 8 + 3 * 8 + 2 * 8 + 8
    assert C.sizeof(lib.dpp_pc_opts) == 4 * 4 + 2 * 8 + 9 * 4 + 4   # padded to 8 bytes
    assert C.sizeof(lib.dpp_solve_opts) == 8 + 5 * 4 + 4 + 8 + 8 + 8 + 4 + 4   # padded to 8
    assert C.sizeof(lib.dpp_solve_info) == 4 * 4 + 4 * 8


def test_invalid_arguments_are_rejected_on_the_host(lib):
    d = lib.dpp_problem_desc()
    d.dim = 4
    with pytest.raises(lib.DppError) as e:
        lib.dpp_assemble(d)
    assert e.value.status == lib.DPP_ERR_INVALID_ARGUMENT
    assert "dim" in lib.dpp_last_error()


def test_no_cpu_fallback_without_a_device(lib):
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    import inputs
    p = inputs.mms_problem(2, 2)
    keep = [np.ascontiguousarray(a) for a in (p.mesh.coords, p.mesh.cells, p.mesh.bfacets,
                                               p.logk1, p.logk2, p.p01, p.p02)]
    d = lib.dpp_problem_desc()
    d.dim, d.memory = 2, lib.DPP_MEM_HOST
    d.n_nodes, d.n_cells, d.n_bfacets = p.mesh.n_nodes, p.mesh.n_cells, p.mesh.n_bfacets
    d.coords, d.cells, d.bfacets, d.log_k1, d.log_k2, d.p01, d.p02 = [a.ctypes.data for a in keep]
    d.mu, d.beta = 1.0, 1.0
    with pytest.raises(lib.DppError) as e:
        lib.dpp_assemble(d)
    assert e.value.status == lib.DPP_ERR_CUDA
    assert "no CUDA device" in lib.dpp_last_error()
