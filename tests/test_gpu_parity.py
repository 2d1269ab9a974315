"""GPU parity: every CUDA stage of the solver path against the CPU oracle.

Everything goes through the C ABI (ctypes binding). Tolerances:
  * assembly (pair values, load vector): 1e-13 relative to the largest entry.
    Both sides sum the same closed-form terms in different orders.
  * K x, K^T x: 1e-13 relative to ||K||_inf ||x||_inf.
  * S_p and the Galerkin products: 1e-12 relative to the largest entry.
  * solves: per-field relative L2 error <= 1e-8 at a true relative residual
    <= 1e-10.
The inputs are seeded synthetic meshes and fields (the ``inputs`` package).
Sizes span several SELL slices with a ragged last slice (n_nodes not a
multiple of 32). They include 2D and 3D, and homogeneous and log-normal
permeabilities.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import inputs
import oracle
from oracle.assembly import assemble_problem

from gpu_helpers import csr_from_export, needs_gpu, pairs_to_slot_major, system_cls, torch

pytestmark = [pytest.mark.gpu, needs_gpu]

CASES = [("mms2d_n7", lambda: inputs.mms_problem(2, 7)),
         ("het2d_n32", lambda: inputs.heterogeneous_problem(2, 32, seed=1, beta=1.0)),
         ("het3d_n5", lambda: inputs.heterogeneous_problem(3, 5, seed=2, beta=0.5)),
         ("mms3d_n6", lambda: inputs.mms_problem(3, 6)),
         # a node in 70 cells: the assembly's per-pair cell masks cover 64
         # cells, the rest take the tail loop
         ("wheel2d_s70", lambda: inputs.wheel_problem(70, 4, seed=2, beta=0.8)),
         # a constant body force gamma*b: the load's k-weighted pressure rows
         ("het2d_n13_gb", lambda: _with_gb(inputs.heterogeneous_problem(2, 13, seed=3, beta=1.2),
                                           [1.5, -0.7])),
         ("het3d_n5_gb", lambda: _with_gb(inputs.heterogeneous_problem(3, 5, seed=4, beta=0.9),
                                          [0.4, -1.1, 2.0]))]


def _with_gb(P, gb):
    return P.with_(gamma_b=np.asarray(gb, dtype=np.float64))


@pytest.fixture(scope="module")
def DPPSystem():
    return system_cls()


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_assembled_K_matches_oracle(DPPSystem, name, make):
    P = make()
    K, f = assemble_problem(P)
    s = DPPSystem.from_problem(P)
    rp, col, vals = s.export_pairs()
    Kg = pairs_to_slot_major(rp.cpu(), col.cpu(), vals.cpu(), P.mesh.n_nodes, P.dim)
    diff = abs(Kg - K)
    assert diff.max() <= 1e-13 * abs(K).max(), diff.max()
    f_gpu = oracle.from_nodal(s.rhs().cpu().numpy())
    assert np.abs(f_gpu - f).max() <= 1e-13 * max(np.abs(f).max(), 1e-300)
    s.close()


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_apply_K_and_transpose_match_oracle(DPPSystem, name, make):
    P = make()
    K, _ = assemble_problem(P)
    s = DPPSystem.from_problem(P)
    rng = inputs.rng(3)
    xn = rng.standard_normal((P.mesh.n_nodes, 2 * P.dim + 2))
    x = torch.tensor(xn, device="cuda")
    for tr in (False, True):
        y = s.apply_K(x, transpose=tr).cpu().numpy()
        ref = oracle.to_nodal((K.T if tr else K) @ oracle.from_nodal(xn), P.mesh.n_nodes)
        scale = abs(K).sum(axis=1).max() * np.abs(xn).max()
        assert np.abs(y - ref).max() <= 1e-13 * scale
    s.close()


def test_assembly_is_bit_reproducible(DPPSystem):
    P = inputs.heterogeneous_problem(3, 6, seed=4)
    a = DPPSystem.from_problem(P)
    b = DPPSystem.from_problem(P)
    va, vb = a.export_pairs()[2], b.export_pairs()[2]
    assert torch.equal(va, vb)
    assert torch.equal(a.rhs(), b.rhs())
    a.close()
    b.close()


@pytest.mark.parametrize("dim,n", [(2, 9), (3, 4)])
def test_selfp_schur_matches_definition(DPPSystem, dim, n):
    P = inputs.heterogeneous_problem(dim, n, seed=5, beta=2.0)
    K, _ = assemble_problem(P)
    S1, S2 = oracle.selfp_schur(K, P.mesh.n_nodes, dim)
    ref = sp.block_diag([S1, S2]).tocsr()
    s = DPPSystem.from_problem(P).setup_pc()
    sz, (rp, col, val), _ = s.level(0, with_p=False)
    S = csr_from_export(rp, col, val, ref.shape)
    assert abs(S - ref).max() <= 1e-12 * abs(ref).max()
    s.close()


def test_selfp_schur_wide_rows_match_definition(DPPSystem):
    # The wheel's centre and first-ring rows of S_p have 75 to 141 columns,
    # more than the one-pass staging rows hold (64 in 2D): the two-pass path.
    P = inputs.wheel_problem(70, 4, seed=6, beta=1.5)
    K, _ = assemble_problem(P)
    S1, S2 = oracle.selfp_schur(K, P.mesh.n_nodes, 2)
    ref = sp.block_diag([S1, S2]).tocsr()
    assert np.diff(ref.indptr).max() > 64
    s = DPPSystem.from_problem(P).setup_pc()
    sz, (rp, col, val), _ = s.level(0, with_p=False)
    S = csr_from_export(rp, col, val, ref.shape)
    assert abs(S - ref).max() <= 1e-12 * abs(ref).max()
    s.close()


@pytest.mark.parametrize("smooth_filter", [0, 1], ids=["A", "filtered"])
def test_amg_levels_are_galerkin_products(DPPSystem, smooth_filter):
    P = inputs.heterogeneous_problem(2, 40, seed=6)
    s = DPPSystem.from_problem(P).setup_pc(coarse_max_rows=64, smooth_filter=smooth_filter)
    nlev = s.level(0)[0]["levels"]
    assert nlev >= 2
    for l in range(nlev - 1):
        sz, (rp, col, val), (prp, pcol, pval) = s.level(l)
        A = csr_from_export(rp, col, val, (sz["rows"], sz["rows"]))
        Pm = csr_from_export(prp, pcol, pval, (sz["rows"], sz["p_cols"]))
        sz2, (rp2, col2, val2), _ = s.level(l + 1, with_p=False)
        Ac = csr_from_export(rp2, col2, val2, (sz2["rows"], sz2["rows"]))
        ref = (Pm.T @ A @ Pm).tocsr()
        assert abs(Ac - ref).max() <= 1e-12 * abs(ref).max()
        # smoothed aggregation keeps constants in the range of P (up to the smoothing)
        assert Pm.shape[1] < Pm.shape[0]
    s.close()


def test_galerkin_products_3d_are_exact_and_deterministic(DPPSystem):
    # 3D 20^3 cubes: 18,522 level-0 rows, so every row of A P and P^T (A P)
    # takes the warp-per-row product kernels (no block-per-row path); two
    # setups must give bit-identical coarse matrices (fixed summation order).
    P = inputs.heterogeneous_problem(3, 20, seed=8, beta=1.0)
    s1 = DPPSystem.from_problem(P).setup_pc()
    s2 = DPPSystem.from_problem(P).setup_pc()
    sz, (rp, col, val), (prp, pcol, pval) = s1.level(0)
    assert sz["rows"] >= 16384
    A = csr_from_export(rp, col, val, (sz["rows"], sz["rows"]))
    Pm = csr_from_export(prp, pcol, pval, (sz["rows"], sz["p_cols"]))
    sz1, (rp1, col1, val1), _ = s1.level(1, with_p=False)
    Ac = csr_from_export(rp1, col1, val1, (sz1["rows"], sz1["rows"]))
    ref = (Pm.T @ A @ Pm).tocsr()
    ref.sort_indices()
    assert abs(Ac - ref).max() <= 1e-12 * abs(ref).max()
    # S_p is symmetric, and so is the coarse operator (to rounding)
    assert abs(Ac - Ac.T).max() <= 1e-13 * abs(Ac).max()
    for l in range(1, sz["levels"]):
        a = s1.level(l, with_p=False)[1]
        b = s2.level(l, with_p=False)[1]
        for u, v in zip(a, b):
            assert torch.equal(u, v), f"level {l} differs between two setups"
    s1.close()
    s2.close()


def test_release_cached_memory_keeps_live_handles(DPPSystem):
    from paper_1808_08328_gb300 import binding as B
    P = inputs.heterogeneous_problem(2, 24, seed=3, beta=1.0)
    s = DPPSystem.from_problem(P).setup_pc()
    x0, _ = s.solve(rtol=1e-10)
    tmp = DPPSystem.from_problem(inputs.heterogeneous_problem(2, 30, seed=4)).setup_pc()
    tmp.close()
    B.dpp_release_cached_memory()
    x1, info = s.solve(rtol=1e-10)
    assert info["status"] == 0
    assert torch.equal(x0, x1)
    s.close()
    B.dpp_release_cached_memory()


SOLVES = [("het2d_n32", lambda: inputs.heterogeneous_problem(2, 32, seed=0, beta=1.0)),
          ("mms2d_n32", lambda: inputs.mms_problem(2, 32)),
          ("het3d_n8", lambda: inputs.heterogeneous_problem(3, 8, seed=0, beta=1.0)),
          ("mms3d_n10", lambda: inputs.mms_problem(3, 10)),
          ("wheel2d_s70", lambda: inputs.wheel_problem(70, 4, seed=0, beta=1.0)),
          ("het3d_n9_gb", lambda: _with_gb(inputs.heterogeneous_problem(3, 9, seed=1, beta=1.0),
                                           [0.8, 0.3, -1.4]))]


@pytest.mark.parametrize("name,make", SOLVES, ids=[c[0] for c in SOLVES])
def test_fp64_solve_matches_oracle(DPPSystem, name, make):
    P = make()
    K, f = assemble_problem(P)
    x_ref = oracle.to_nodal(oracle.solve_direct(K, f, coords=P.mesh.coords), P.mesh.n_nodes)
    s = DPPSystem.from_problem(P).setup_pc()
    x, info = s.solve(rtol=1e-10)
    assert info["status"] == 0 and info["rel_residual"] <= 1e-10
    xg = x.cpu().numpy()
    # the residual claimed by the library, recomputed by the oracle
    assert oracle.residual(K, oracle.from_nodal(xg), f) <= 1.5e-10
    err = oracle.field_rel_errors(xg, x_ref)
    assert max(err.values()) <= 1e-8, err
    s.close()


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_reorthogonalisation_threshold_keeps_the_solution(DPPSystem, precision):
    # eta = 1: a second Gram-Schmidt pass at every step; eta = 0: never. Both
    # must reach the bar, and the solutions agree to well below it.
    P = inputs.heterogeneous_problem(3, 8, seed=5, beta=1.0)
    s = DPPSystem.from_problem(P, precision=precision).setup_pc(precision=precision)
    xa, ia = s.solve(rtol=1e-10, reorth_eta=1.0)
    xb, ib = s.solve(rtol=1e-10, reorth_eta=0.0)
    assert ia["status"] == 0 and ib["status"] == 0
    assert abs(ia["iterations"] - ib["iterations"]) <= 1
    err = oracle.field_rel_errors(xb.cpu().numpy(), xa.cpu().numpy())
    assert max(err.values()) <= 1e-8, err
    s.close()


def test_pc_apply_is_linear_and_transpose_consistent(DPPSystem):
    P = inputs.heterogeneous_problem(2, 16, seed=7)
    s = DPPSystem.from_problem(P).setup_pc()
    rng = inputs.rng(8)
    a = torch.tensor(rng.standard_normal((P.mesh.n_nodes, 6)), device="cuda")
    b = torch.tensor(rng.standard_normal((P.mesh.n_nodes, 6)), device="cuda")
    za, zb, zab = s.pc_apply(a), s.pc_apply(b), s.pc_apply(2.0 * a - 3.0 * b)
    assert torch.allclose(zab, 2.0 * za - 3.0 * zb, rtol=1e-10, atol=1e-12 * zab.abs().max())
    # preconditioner of K^T: same as that of K with B, C negated -> differs from P^-1
    zt = s.pc_apply(a, transpose=True)
    assert not torch.allclose(zt, za)
    s.close()


@pytest.mark.parametrize("dim,n,gb", [(2, 10, None), (2, 10, [1.7, -0.9]),
                                      (3, 5, [0.6, -1.2, 0.9])],
                         ids=["2d", "2d_gb", "3d_gb"])
def test_adjoint_matches_oracle(DPPSystem, dim, n, gb):
    # With a body force the load depends on log k, so the gradient carries the
    # -lambda^T df/dlog k term as well as the K sensitivities.
    P = inputs.heterogeneous_problem(dim, n, seed=1, beta=1.3)
    Pobs = inputs.heterogeneous_problem(dim, n, seed=2, beta=1.3)
    if gb is not None:
        P, Pobs = _with_gb(P, gb), _with_gb(Pobs, gb)
    K, f = assemble_problem(P)
    Ko, fo = assemble_problem(Pobs)
    xn = oracle.to_nodal(oracle.solve_direct(K, f), P.mesh.n_nodes)
    p1_obs = oracle.to_nodal(oracle.solve_direct(Ko, fo), P.mesh.n_nodes)[:, dim]
    g = oracle.objective_grad_x(xn, p1_obs)
    lam_ref = oracle.adjoint_solve(K, g)
    g1r, g2r, gbr = oracle.adjoint_gradients(P, xn, lam_ref)
    s = DPPSystem.from_problem(P).setup_pc()
    x, _ = s.solve(rtol=1e-13)
    assert oracle.field_rel_errors(x.cpu().numpy(), xn)["p1"] <= 1e-10
    gx = torch.tensor(oracle.objective_grad_x(x.cpu().numpy(), p1_obs), device="cuda")
    lam, g1, g2, gb, info = s.adjoint(x, gx, rtol=1e-13)
    assert info["status"] == 0
    sc = max(abs(g1r).max(), abs(g2r).max())
    assert np.abs(g1.cpu().numpy() - g1r).max() <= 1e-8 * sc
    assert np.abs(g2.cpu().numpy() - g2r).max() <= 1e-8 * sc
    assert abs(gb.item() - gbr) <= 1e-8 * abs(gbr)
    s.close()


def test_error_paths(DPPSystem):
    from paper_1808_08328_gb300 import binding as B
    P = inputs.mms_problem(2, 4)
    bad = P.mesh.cells.copy()
    bad[3, 1] = P.mesh.n_nodes + 5
    with pytest.raises(B.DppError) as e:
        DPPSystem(P.mesh.coords, bad, P.mesh.bfacets, P.logk1, P.logk2, 1.0, 1.0, [0, 0],
                  P.p01, P.p02)
    assert e.value.status == B.DPP_ERR_INVALID_ARGUMENT
    lk = P.logk1.copy()
    lk[0] = np.nan
    with pytest.raises(B.DppError) as e:
        DPPSystem(P.mesh.coords, P.mesh.cells, P.mesh.bfacets, lk, P.logk2, 1.0, 1.0, [0, 0],
                  P.p01, P.p02)
    assert e.value.status == B.DPP_ERR_NONFINITE
    s = DPPSystem.from_problem(inputs.heterogeneous_problem(2, 16, seed=3)).setup_pc()
    x, info = s.solve(check=False, max_iters=1, restart=1)
    assert info["status"] == B.DPP_ERR_NOT_CONVERGED and info["iterations"] == 1
    s.close()


def test_filtered_smoothing_keeps_only_strong_couplings(DPPSystem):
    # smooth_filter = 1 smooths P0 with A^F (the strong entries of A and the
    # diagonal): every nonzero of P is then within one strong edge of its
    # aggregate, so level 0's P is sparser than with the full A; no row of P
    # is empty.
    P = inputs.heterogeneous_problem(3, 10, seed=4, beta=1.0)
    nnz = {}
    for f in (0, 1):
        s = DPPSystem.from_problem(P).setup_pc(smooth_filter=f)
        sz, (rp, col, val), (prp, pcol, pval) = s.level(0)
        nnz[f] = sz["p_nnz"]
        Pm = csr_from_export(prp, pcol, pval, (sz["rows"], sz["p_cols"]))
        assert (np.diff(Pm.indptr) > 0).all()
        s.close()
    assert nnz[1] < 0.6 * nnz[0], nnz
