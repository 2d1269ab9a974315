"""The matrix-free (element-by-element) K apply against the oracle.

dpp_apply_K_mf evaluates K x cell by cell from the geometry and k, with no
assembled values. Tolerances:
  * FP64: K x and K^T x match the oracle's assembled K to 1e-12 relative to
    ||K||_inf ||x||_inf (the geometry is recomputed per cell, and the terms
    are added in another order than in the assembly);
  * FP32 (dpp_apply_K32_mf): matches the FP32 operator of the assembled pair
    values (dpp_apply_K32) and the oracle to 2e-5 of the same scale. FP32 unit
    roundoff is 6e-8, and each row sums up to about 24 cells of roughly 20
    terms each;
  * two applies are bit-identical (fixed-order gather, no atomics);
  * solves with the matrix-free inner operator (matrix_free = 1), FP64 and
    mixed, reach the oracle's solution to 1e-8 relative L2 per field.
"""
import numpy as np
import pytest

import inputs
import oracle
from oracle.assembly import assemble_problem

from gpu_helpers import needs_gpu, system_cls, torch

pytestmark = [pytest.mark.gpu, needs_gpu]

CASES = [("het2d_n33", lambda: inputs.heterogeneous_problem(2, 33, seed=1, beta=1.0)),
         ("het3d_n7", lambda: inputs.heterogeneous_problem(3, 7, seed=2, beta=0.5)),
         ("wheel2d_s70", lambda: inputs.wheel_problem(70, 4, seed=2, beta=0.8)),
         ("mms3d_n5_gb", lambda: inputs.mms_problem(3, 5).with_(gamma_b=np.array([1.0, 2.0, 0.5])))]


@pytest.fixture(scope="module")
def DPPSystem():
    return system_cls()


def _scale(K, xn):
    return abs(K).sum(axis=1).max() * np.abs(xn).max()


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_matrix_free_fp64_matches_oracle(DPPSystem, name, make):
    P = make()
    K, _ = assemble_problem(P)
    s = DPPSystem.from_problem(P)
    xn = inputs.rng(3).standard_normal((P.mesh.n_nodes, 2 * P.dim + 2))
    x = torch.tensor(xn, device="cuda")
    for tr in (False, True):
        y = s.apply_K_mf(x, transpose=tr).cpu().numpy()
        ref = oracle.to_nodal((K.T if tr else K) @ oracle.from_nodal(xn), P.mesh.n_nodes)
        assert np.abs(y - ref).max() <= 1e-12 * _scale(K, xn)
        y2 = s.apply_K_mf(x, transpose=tr).cpu().numpy()
        assert np.array_equal(y, y2)
    s.close()


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_matrix_free_fp32_matches_assembled_fp32(DPPSystem, name, make):
    P = make()
    K, _ = assemble_problem(P)
    s = DPPSystem.from_problem(P, precision=1)
    xn = inputs.rng(4).standard_normal((P.mesh.n_nodes, 2 * P.dim + 2)).astype(np.float32)
    x = torch.tensor(xn, device="cuda")
    for tr in (False, True):
        y_mf = s.apply_K32_mf(x, transpose=tr).cpu().numpy()
        y_as = s.apply_K32(x, transpose=tr).cpu().numpy()
        ref = oracle.to_nodal((K.T if tr else K) @ oracle.from_nodal(xn.astype(np.float64)),
                              P.mesh.n_nodes)
        sc = _scale(K, xn)
        assert np.abs(y_mf - y_as).max() <= 2e-5 * sc
        assert np.abs(y_mf - ref).max() <= 2e-5 * sc
    s.close()


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
@pytest.mark.parametrize("dim,n", [(2, 32), (3, 9)])
def test_matrix_free_solve_matches_oracle(DPPSystem, dim, n, precision):
    P = inputs.heterogeneous_problem(dim, n, seed=0, beta=1.0)
    K, f = assemble_problem(P)
    x_ref = oracle.to_nodal(oracle.solve_direct(K, f, coords=P.mesh.coords), P.mesh.n_nodes)
    s = DPPSystem.from_problem(P, precision=precision).setup_pc(precision=precision)
    x, info = s.solve(rtol=1e-10, matrix_free=1)
    assert info["status"] == 0 and info["rel_residual"] <= 1e-10
    xg = x.cpu().numpy()
    assert oracle.residual(K, oracle.from_nodal(xg), f) <= 1.5e-10
    err = oracle.field_rel_errors(xg, x_ref)
    assert max(err.values()) <= 1e-8, err
    s.close()
