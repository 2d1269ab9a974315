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


@pytest.mark.parametrize("dim,n,opts", [(2, 40, {"coarse_max_rows": 64}), (3, 20, {})],
                         ids=["2d40_multilevel", "3d20_onepass"])
def test_fp32_hierarchy_matches_its_definitions(DPPSystem, dim, n, opts):
    # The mixed mode builds S_p and every level in FP32 (FP32 pair values,
    # FP32 accumulators in the FP64 path's summation order). Level 0 must be the
    # selfp Schur matrices of the oracle's K, and every coarser level the
    # Galerkin product P^T A P of the exported FP32 level, both to FP32
    # rounding: 1e-5 of the largest entry (sums of up to ~700 products). Two
    # setups are bit-identical.
    import scipy.sparse as sp
    from gpu_helpers import csr_from_export
    P = inputs.heterogeneous_problem(dim, n, seed=8, beta=1.0)
    K, _ = assemble_problem(P)
    S1, S2 = oracle.selfp_schur(K, P.mesh.n_nodes, dim)
    ref0 = sp.block_diag([S1, S2]).tocsr()
    s1 = DPPSystem.from_problem(P, precision=MIXED).setup_pc(precision=MIXED, **opts)
    s2 = DPPSystem.from_problem(P, precision=MIXED).setup_pc(precision=MIXED, **opts)
    sz, (rp, col, val), _ = s1.level(0, with_p=False)
    S = csr_from_export(rp, col, val, ref0.shape)
    assert abs(S - ref0).max() <= 1e-5 * abs(ref0).max()
    assert np.array_equal(val.cpu().numpy(), val.cpu().numpy().astype(np.float32))  # FP32 values
    nlev = sz["levels"]
    assert nlev >= 2
    for l in range(nlev - 1):
        szl, (rp, col, val), (prp, pcol, pval) = s1.level(l)
        A = csr_from_export(rp, col, val, (szl["rows"], szl["rows"]))
        Pm = csr_from_export(prp, pcol, pval, (szl["rows"], szl["p_cols"]))
        sz2, (rp2, col2, val2), _ = s1.level(l + 1, with_p=False)
        Ac = csr_from_export(rp2, col2, val2, (sz2["rows"], sz2["rows"]))
        ref = (Pm.T @ A @ Pm).tocsr()
        assert abs(Ac - ref).max() <= 1e-5 * abs(ref).max(), l
        assert abs(Ac - Ac.T).max() <= 1e-5 * abs(Ac).max(), l
    for l in range(nlev):
        a = s1.level(l, with_p=False)[1]
        b = s2.level(l, with_p=False)[1]
        for u, v in zip(a, b):
            assert torch.equal(u, v), f"level {l} differs between two setups"
    # the FP64 entry point of a mixed preconditioner returns its FP32 result, widened
    r = torch.tensor(inputs.rng(3).standard_normal((P.mesh.n_nodes, 2 * dim + 2)), device="cuda")
    z = s1.pc_apply(r)
    assert torch.isfinite(z).all()
    assert np.array_equal(z.cpu().numpy(), z.cpu().numpy().astype(np.float32).astype(np.float64))
    assert torch.equal(z, s2.pc_apply(r))
    s1.close()
    s2.close()
