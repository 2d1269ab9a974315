"""Pins for the oracle's Q1 (QUAD, HEX) CG-VMS assembly.

  * DoF counts against the paper's QUAD and HEX columns (golden file).
  * The tensor 2-point rule integrates Q1 products exactly on a box cell
    (closed form: the tensor product of the 1D P1 mass matrix).
  * Patch tests on meshes whose interior nodes are moved (non-affine cells):
    p = a.x + c with u_i = (k_i/mu)(gamma b - a) is reproduced exactly, with
    and without a body force, and a constant pressure gives u = 0. The rule
    integrates every term that such fields produce exactly, so a wrong sign,
    a dropped term or a wrong facet normal fails.
  * Sparse against dense LU; the block identity K_pu = -K_up^T.
  * MMS convergence rate 2 in every field (Sections 5.1, 5.2 use the same
    meshes for QUAD/HEX as for TRI/TET).
  * The mass-balance invariant (q = 1 is in the Q1 space).
"""
import os

import numpy as np
import pytest

import inputs
import oracle
from oracle.assembly import assemble_problem

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.split("#")[0].strip()
            if line:
                rows.append([int(v) for v in line.split()])
    return rows


def test_q1_dof_counts_match_paper_tables():
    for dim, n, dof in _load("dof_tables_q1.txt"):
        if (n + 1) ** dim <= 40000:
            assert inputs.unit_mesh(dim, n, "q1").n_dofs == dof
        assert inputs.dof_count(dim, n) == dof


@pytest.mark.parametrize("dim", [2, 3])
def test_q1_mesh_partitions_the_box(dim):
    m = inputs.unit_mesh(dim, 3, "q1")
    w, phi, grad, det = oracle.q1.q1_geometry(m.coords, m.cells)
    assert np.all(det > 0)
    assert np.isclose(w.sum(), 1.0)
    assert m.n_cells == 3 ** dim and m.n_bfacets == 2 * dim * 3 ** (dim - 1)


@pytest.mark.parametrize("dim", [2, 3])
def test_q1_rule_integrates_mass_exactly(dim):
    h = 0.37
    coords = np.array([[h * ((v >> k) & 1) for k in range(dim)] for v in range(1 << dim)], float)
    cells = np.arange(1 << dim)[None, :]
    M = oracle.q1_mass_matrix(coords, cells).toarray()
    nv = 1 << dim
    ref = np.empty((nv, nv))
    for a in range(nv):
        for b in range(nv):
            ref[a, b] = h ** dim * np.prod([(1 / 3 if ((a >> k) & 1) == ((b >> k) & 1) else 1 / 6)
                                            for k in range(dim)])
    assert np.allclose(M, ref, rtol=1e-14, atol=0)


def _patch(dim, n, a, c, gb, k1=2.0, k2=0.05, beta=3.0, mu=1.3):
    m = inputs.unit_mesh(dim, n, "q1")
    X = m.coords.copy()
    inner = np.all((X > 1e-12) & (X < 1 - 1e-12), axis=1)
    X[inner] += inputs.rng(7).uniform(-0.2, 0.2, size=(inner.sum(), dim)) / n
    m.coords = X
    p0 = X @ a + c
    return inputs.Problem(m, np.full(m.n_cells, np.log(k1)), np.full(m.n_cells, np.log(k2)), mu,
                          beta, np.asarray(gb, float), p0, p0.copy())


@pytest.mark.parametrize("dim,n", [(2, 4), (3, 3)])
@pytest.mark.parametrize("with_gb", [False, True])
def test_q1_linear_patch_is_reproduced_exactly(dim, n, with_gb):
    a = np.array([0.7, -1.1, 0.4][:dim])
    gb = np.array([1.9, 0.6, -1.3][:dim]) if with_gb else np.zeros(dim)
    P = _patch(dim, n, a, 0.3, gb)
    K, f = assemble_problem(P)
    xn = oracle.to_nodal(oracle.solve_direct(K, f), P.mesh.n_nodes)
    d, mu = dim, P.mu
    assert np.allclose(xn[:, d], P.mesh.coords @ a + 0.3, atol=1e-11)
    assert np.allclose(xn[:, 2 * d + 1], P.mesh.coords @ a + 0.3, atol=1e-11)
    assert np.allclose(xn[:, :d], (2.0 / mu) * (gb - a)[None, :], atol=1e-10)
    assert np.allclose(xn[:, d + 1:2 * d + 1], (0.05 / mu) * (gb - a)[None, :], atol=1e-11)


@pytest.mark.parametrize("dim,n", [(2, 4), (3, 2)])
def test_q1_constant_pressure_gives_zero_velocity(dim, n):
    P = _patch(dim, n, np.zeros(dim), 1.5, np.zeros(dim), k1=1.0, k2=0.1, beta=1.0)
    K, f = assemble_problem(P)
    xn = oracle.to_nodal(oracle.solve_direct(K, f), P.mesh.n_nodes)
    assert np.allclose(xn[:, dim], 1.5, atol=1e-12)
    assert np.allclose(xn[:, :dim], 0.0, atol=1e-11)


@pytest.mark.parametrize("dim,n", [(2, 4), (3, 2)])
def test_q1_sparse_lu_matches_dense_lu_and_block_identity(dim, n):
    P = inputs.heterogeneous_problem(dim, n, seed=3, beta=2.5, kind="q1")
    K, f = assemble_problem(P)
    x1 = oracle.solve_direct(K, f)
    x2 = oracle.solve_dense(K, f)
    assert np.allclose(x1, x2, rtol=1e-12, atol=1e-12 * np.abs(x2).max())
    b = oracle.field_split_blocks(K, P.mesh.n_nodes, dim)
    for i in ("1", "2"):
        assert abs(b[f"K{i}pu"] + b[f"K{i}up"].T).max() < 1e-14


def _rates(dim, ns):
    errs = []
    for n in ns:
        P = inputs.mms_problem(dim, n, kind="q1")
        K, f = assemble_problem(P)
        xn = oracle.to_nodal(oracle.solve_direct(K, f, coords=P.mesh.coords), P.mesh.n_nodes)
        M = oracle.q1_mass_matrix(P.mesh.coords, P.mesh.cells)
        errs.append(oracle.interp_l2_errors(xn, inputs.nodal_exact(P.mesh.coords), M))
    return {fld: np.log(errs[-2][fld] / errs[-1][fld]) / np.log(ns[-1] / ns[-2])
            for fld in oracle.FIELDS}


def test_q1_mms_rate_2d():
    for fld, r in _rates(2, [8, 16, 32]).items():
        assert abs(r - 2.0) < 0.25, (fld, r)


def test_q1_mms_rate_3d():
    for fld, r in _rates(3, [4, 8]).items():
        assert abs(r - 2.0) < 0.35, (fld, r)


@pytest.mark.parametrize("dim,n", [(2, 6), (3, 3)])
def test_q1_mass_balance_invariant(dim, n):
    P = inputs.heterogeneous_problem(dim, n, seed=4, beta=1.7, kind="q1")
    P = P.with_(gamma_b=np.linspace(1.0, -0.5, dim))
    K, f = assemble_problem(P)
    xn = oracle.to_nodal(oracle.solve_direct(K, f), P.mesh.n_nodes)
    b1, b2 = oracle.mass_balance_q1(xn, P.mesh.coords, P.mesh.cells, P.mu, P.beta)
    scale = np.abs(xn).max()
    assert abs(b1) < 1e-11 * scale and abs(b2) < 1e-11 * scale
