"""SELL-32 AMG SpMV against the CSR path and the oracle.

Level matrices with many rows also get a SELL-32 copy (slices of 32 rows,
column-major), and the autotuner may run their SpMVs in it. The default
threshold (65536 rows) is above every other GPU test's level sizes, so these
tests lower it (sell_min_rows) and force the format (spmv_format = 2), and
compare with the CSR-only preconditioner (spmv_format = 1):
  * one preconditioner application, FP64: the two formats sum each row in a
    different order, so they agree to rounding, 1e-12 relative in the 2-norm;
  * FP64 and mixed-precision solves against the oracle's direct solve at the
    solver's bar: per-field relative L2 error <= 1e-8 at relative residual
    1e-10.
"""
import numpy as np
import pytest

import inputs
import oracle
from oracle.assembly import assemble_problem

from gpu_helpers import needs_gpu, system_cls, torch

pytestmark = [pytest.mark.gpu, needs_gpu]

CASES = [(2, 40, 1024), (3, 9, 512)]


@pytest.fixture(scope="module")
def DPPSystem():
    return system_cls()


@pytest.mark.parametrize("dim,n,min_rows", CASES)
def test_sell_pc_apply_matches_csr(DPPSystem, dim, n, min_rows):
    P = inputs.heterogeneous_problem(dim, n, seed=21)
    s_csr = DPPSystem.from_problem(P).setup_pc(spmv_format=1)
    s_sell = DPPSystem.from_problem(P).setup_pc(spmv_format=2, sell_min_rows=min_rows)
    r = torch.tensor(inputs.rng(22).standard_normal((P.mesh.n_nodes, 2 * dim + 2)), device="cuda")
    for tr in (False, True):
        z1 = s_csr.pc_apply(r, transpose=tr)
        z2 = s_sell.pc_apply(r, transpose=tr)
        assert float(torch.linalg.norm(z1 - z2) / torch.linalg.norm(z1)) <= 1e-12
    s_csr.close()
    s_sell.close()


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
@pytest.mark.parametrize("dim,n,min_rows", CASES)
def test_sell_solve_matches_oracle(DPPSystem, dim, n, min_rows, precision):
    P = inputs.heterogeneous_problem(dim, n, seed=23, beta=1.0)
    K, f = assemble_problem(P)
    x_ref = oracle.to_nodal(oracle.solve_direct(K, f, coords=P.mesh.coords), P.mesh.n_nodes)
    s = DPPSystem.from_problem(P, precision=precision).setup_pc(
        precision=precision, spmv_format=2, sell_min_rows=min_rows)
    x, info = s.solve(rtol=1e-10)
    assert info["status"] == 0 and info["rel_residual"] <= 1e-10
    xg = x.cpu().numpy()
    assert oracle.residual(K, oracle.from_nodal(xg), f) <= 1.5e-10
    err = oracle.field_rel_errors(xg, x_ref)
    assert max(err.values()) <= 1e-8, err
    s.close()
