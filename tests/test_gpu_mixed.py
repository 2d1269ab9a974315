"""Mixed precision (FP32 values and preconditioner inside FP64 FGMRES with
refinement) against the oracle.

The solution must meet the same bar as the FP64 path: per-field relative L2
error <= 1e-8 against the oracle's direct solve, at a true FP64 relative
residual <= 1e-10 (recomputed by the oracle). The FP32 operator itself is
compared with the oracle's K at FP32 tolerance: 1e-6 relative to
||K||_inf ||x||_inf, several float ulps over rows of about 15 pairs.
"""
import numpy as np
import pytest

import inputs
import oracle
from oracle.assembly import assemble_problem

from gpu_helpers import needs_gpu, system_cls, torch

pytestmark = [pytest.mark.gpu, needs_gpu]

MIXED = 1


@pytest.fixture(scope="module")
def DPPSystem():
    return system_cls()


@pytest.mark.parametrize("dim,n", [(2, 9), (3, 5)])
def test_apply_K32_matches_oracle(DPPSystem, dim, n):
    P = inputs.heterogeneous_problem(dim, n, seed=11)
    K, _ = assemble_problem(P)
    s = DPPSystem.from_problem(P, precision=MIXED)
    xn = inputs.rng(12).standard_normal((P.mesh.n_nodes, 2 * dim + 2)).astype(np.float32)
    for tr in (False, True):
        y = s.apply_K32(torch.tensor(xn, device="cuda"), transpose=tr).cpu().numpy()
        ref = oracle.to_nodal((K.T if tr else K) @ oracle.from_nodal(xn.astype(np.float64)),
                              P.mesh.n_nodes)
        scale = abs(K).sum(axis=1).max() * np.abs(xn).max()
        assert np.abs(y - ref).max() <= 1e-6 * scale
    s.close()


SOLVES = [("het2d_n32", lambda: inputs.heterogeneous_problem(2, 32, seed=0, beta=1.0)),
          ("het3d_n8", lambda: inputs.heterogeneous_problem(3, 8, seed=0, beta=1.0)),
          ("mms3d_n10", lambda: inputs.mms_problem(3, 10))]


@pytest.mark.parametrize("name,make", SOLVES, ids=[c[0] for c in SOLVES])
def test_mixed_solve_matches_oracle(DPPSystem, name, make):
    P = make()
    K, f = assemble_problem(P)
    x_ref = oracle.to_nodal(oracle.solve_direct(K, f, coords=P.mesh.coords), P.mesh.n_nodes)
    s = DPPSystem.from_problem(P, precision=MIXED).setup_pc(precision=MIXED)
    x, info = s.solve(rtol=1e-10)
    assert info["status"] == 0 and info["rel_residual"] <= 1e-10
    xg = x.cpu().numpy()
    assert oracle.residual(K, oracle.from_nodal(xg), f) <= 1.5e-10
    err = oracle.field_rel_errors(xg, x_ref)
    assert max(err.values()) <= 1e-8, err
    s.close()


def test_mixed_adjoint_matches_fp64_adjoint(DPPSystem):
    P = inputs.heterogeneous_problem(2, 12, seed=2, beta=0.8)
    ref = DPPSystem.from_problem(P).setup_pc()
    mix = DPPSystem.from_problem(P, precision=MIXED).setup_pc(precision=MIXED)
    x, _ = ref.solve(rtol=1e-12)
    g = torch.zeros_like(x)
    g[:, 2] = 1.0
    _, g1, g2, gb, _ = ref.adjoint(x, g, rtol=1e-12)
    _, h1, h2, hb, info = mix.adjoint(x, g, rtol=1e-12)
    assert info["status"] == 0
    sc = max(g1.abs().max().item(), g2.abs().max().item())
    assert torch.allclose(h1, g1, rtol=0, atol=1e-8 * sc)
    assert torch.allclose(h2, g2, rtol=0, atol=1e-8 * sc)
    assert abs(hb.item() - gb.item()) <= 1e-8 * abs(gb.item())
    ref.close()
    mix.close()
