"""The Q1 (QUAD, HEX) CG-VMS path against the oracle.

cell_kind = DPP_CELL_Q1 assembles the paper's equal-order [Q1 + Q1]^2
discretisation (Table "ELE_level_discretization") on quadrilaterals and
hexahedra. Tolerances as for simplices:
  * pair values, the load vector, K x and K^T x: 1e-13 relative (the cell
    integrals use the same 2-point tensor rule on both sides, summed in
    another order), also on cells with moved interior nodes (non-affine) and
    with a body force;
  * S_p: 1e-12 relative to its largest entry;
  * solves, FP64 and mixed, both compositions: 1e-8 relative L2 per field at
    a true residual of 1e-10;
  * the adjoint gradient: 1e-8 relative against the oracle adjoint;
  * behaviour: the iteration count on the homogeneous 3D MMS problem at
    h = 1/16 lies within half to twice the paper's CG-VMS HEX KSP counts
    (16-21, golden ksp_band_hex.txt);
  * the paths that take simplices only (matrix-free apply, batched solve,
    allocation-free gradients) reject Q1 problems with an error.
"""
import os

import numpy as np
import pytest
import scipy.sparse as sp

import inputs
import oracle
from oracle.assembly import assemble_problem

from gpu_helpers import csr_from_export, needs_gpu, pairs_to_slot_major, system_cls, torch

pytestmark = [pytest.mark.gpu, needs_gpu]


def _moved(P, seed=7):
    m = P.mesh
    X = m.coords.copy()
    inner = np.all((X > 1e-12) & (X < 1 - 1e-12), axis=1)
    X[inner] += inputs.rng(seed).uniform(-0.2, 0.2, size=(inner.sum(), m.dim)) / m.n
    return P.with_(mesh=inputs.Mesh(m.dim, X, m.cells, m.bfacets, m.n, kind=m.kind))


CASES = [("quad_n13", lambda: inputs.heterogeneous_problem(2, 13, seed=1, beta=1.0, kind="q1")),
         ("hex_n5", lambda: inputs.heterogeneous_problem(3, 5, seed=2, beta=0.5, kind="q1")),
         ("hex_n4_moved_gb", lambda: _moved(inputs.heterogeneous_problem(3, 4, seed=3, beta=1.2,
                                                                        kind="q1")).with_(
             gamma_b=np.array([0.4, -1.1, 2.0]))),
         ("quad_n9_moved_gb", lambda: _moved(inputs.mms_problem(2, 9, kind="q1")).with_(
             gamma_b=np.array([1.5, -0.7])))]


@pytest.fixture(scope="module")
def DPPSystem():
    return system_cls()


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_q1_assembly_matches_oracle(DPPSystem, name, make):
    P = make()
    K, f = assemble_problem(P)
    s = DPPSystem.from_problem(P)
    rp, col, vals = s.export_pairs()
    Kg = pairs_to_slot_major(rp.cpu(), col.cpu(), vals.cpu(), P.mesh.n_nodes, P.dim)
    assert abs(Kg - K).max() <= 1e-13 * abs(K).max()
    f_gpu = oracle.from_nodal(s.rhs().cpu().numpy())
    assert np.abs(f_gpu - f).max() <= 1e-13 * max(np.abs(f).max(), 1e-300)
    xn = inputs.rng(3).standard_normal((P.mesh.n_nodes, 2 * P.dim + 2))
    x = torch.tensor(xn, device="cuda")
    scale = abs(K).sum(axis=1).max() * np.abs(xn).max()
    for tr in (False, True):
        y = s.apply_K(x, transpose=tr).cpu().numpy()
        ref = oracle.to_nodal((K.T if tr else K) @ oracle.from_nodal(xn), P.mesh.n_nodes)
        assert np.abs(y - ref).max() <= 1e-13 * scale
    s.close()


def test_q1_selfp_matches_definition(DPPSystem):
    P = inputs.heterogeneous_problem(3, 4, seed=5, beta=2.0, kind="q1")
    K, _ = assemble_problem(P)
    S1, S2 = oracle.selfp_schur(K, P.mesh.n_nodes, 3)
    ref = sp.block_diag([S1, S2]).tocsr()
    s = DPPSystem.from_problem(P).setup_pc()
    sz, (rp, col, val), _ = s.level(0, with_p=False)
    S = csr_from_export(rp, col, val, ref.shape)
    assert abs(S - ref).max() <= 1e-12 * abs(ref).max()
    s.close()


SOLVES = [("quad_n24", lambda: inputs.heterogeneous_problem(2, 24, seed=0, beta=1.0, kind="q1")),
          ("hex_n8", lambda: inputs.heterogeneous_problem(3, 8, seed=0, beta=1.0, kind="q1")),
          ("hex_mms_n10", lambda: inputs.mms_problem(3, 10, kind="q1"))]


@pytest.mark.parametrize("composition", [0, 1], ids=["field", "scale"])
@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
@pytest.mark.parametrize("name,make", SOLVES, ids=[c[0] for c in SOLVES])
def test_q1_solve_matches_oracle(DPPSystem, name, make, precision, composition):
    P = make()
    K, f = assemble_problem(P)
    x_ref = oracle.to_nodal(oracle.solve_direct(K, f, coords=P.mesh.coords), P.mesh.n_nodes)
    s = DPPSystem.from_problem(P, precision=precision).setup_pc(precision=precision,
                                                               composition=composition)
    x, info = s.solve(rtol=1e-10)
    assert info["status"] == 0 and info["rel_residual"] <= 1e-10
    xg = x.cpu().numpy()
    assert oracle.residual(K, oracle.from_nodal(xg), f) <= 1.5e-10
    err = oracle.field_rel_errors(xg, x_ref)
    assert max(err.values()) <= 1e-8, err
    s.close()


def test_q1_adjoint_matches_oracle(DPPSystem):
    P = inputs.heterogeneous_problem(3, 4, seed=1, beta=1.3, kind="q1").with_(
        gamma_b=np.array([0.6, -1.2, 0.9]))
    Pobs = inputs.heterogeneous_problem(3, 4, seed=2, beta=1.3, kind="q1").with_(
        gamma_b=np.array([0.6, -1.2, 0.9]))
    K, f = assemble_problem(P)
    Ko, fo = assemble_problem(Pobs)
    xn = oracle.to_nodal(oracle.solve_direct(K, f), P.mesh.n_nodes)
    p1_obs = oracle.to_nodal(oracle.solve_direct(Ko, fo), P.mesh.n_nodes)[:, 3]
    lam_ref = oracle.adjoint_solve(K, oracle.objective_grad_x(xn, p1_obs))
    g1r, g2r, gbr = oracle.adjoint_gradients(P, xn, lam_ref)
    s = DPPSystem.from_problem(P).setup_pc()
    x, _ = s.solve(rtol=1e-13)
    gx = torch.tensor(oracle.objective_grad_x(x.cpu().numpy(), p1_obs), device="cuda")
    lam, g1, g2, gb, info = s.adjoint(x, gx, rtol=1e-13)
    assert info["status"] == 0
    sc = max(abs(g1r).max(), abs(g2r).max())
    assert np.abs(g1.cpu().numpy() - g1r).max() <= 1e-8 * sc
    assert np.abs(g2.cpu().numpy() - g2r).max() <= 1e-8 * sc
    assert abs(gb.item() - gbr) <= 1e-8 * abs(gbr)
    s.close()


def test_q1_hex_iterations_in_the_papers_band(DPPSystem):
    band = {}
    with open(os.path.join(os.path.dirname(__file__), "golden", "ksp_band_hex.txt")) as fh:
        for line in fh:
            line = line.split("#")[0].strip()
            if line:
                n, lo, hi = (int(v) for v in line.split())
                band[n] = (lo, hi)
    lo, hi = band[16]
    s = DPPSystem.from_problem(inputs.mms_problem(3, 16, kind="q1")).setup_pc()
    for rtol in (1e-5, 1e-7):
        x, info = s.solve(rtol=rtol)
        assert info["status"] == 0
        assert 0.5 * lo <= info["iterations"] <= 2 * hi, (rtol, info["iterations"])
    s.close()


def test_q1_rejected_where_only_simplices_are_supported(DPPSystem):
    from paper_1808_08328_gb300 import binding as B
    from paper_1808_08328_gb300.system import solve_batched
    P = inputs.heterogeneous_problem(2, 6, seed=1, kind="q1")
    s = DPPSystem.from_problem(P).setup_pc()
    x = torch.zeros((P.mesh.n_nodes, 6), dtype=torch.float64, device="cuda")
    with pytest.raises(B.DppError) as e:
        s.apply_K_mf(x)
    assert e.value.status == B.DPP_ERR_BAD_STATE
    with pytest.raises(B.DppError) as e:
        B.dpp_adjoint_gradients_noalloc(s.prob, x, x, torch.zeros(P.mesh.n_cells, device="cuda",
                                                                   dtype=torch.float64),
                                        torch.zeros(P.mesh.n_cells, device="cuda",
                                                    dtype=torch.float64),
                                        torch.zeros(1, device="cuda", dtype=torch.float64))
    assert e.value.status == B.DPP_ERR_BAD_STATE
    s.close()
    xs, infos, st = solve_batched([inputs.heterogeneous_problem(2, 6, seed=2),
                                   P], rtol=1e-10)
    assert infos[0]["status"] == 0
    assert infos[1]["status"] == B.DPP_ERR_INVALID_ARGUMENT
