"""Pins for the CPU oracle: facts fixed by the paper and by the mathematics.

Each check is chosen so that a plausible mistake fails it: a dropped
stabilisation term, a wrong sign, a transposed block, a bad boundary normal, or
a wrong quadrature.
  * DoF counts against the paper's tables (golden file).
  * Quadrature against closed-form simplex integrals.
  * Linear and constant patch tests: CG-VMS is consistent, and P1 reproduces
    a linear pressure with a constant Darcy velocity exactly (also on a disc
    wheel mesh with slanted boundary normals and a 70-cell node).
  * Sparse LU against dense LU.
  * Block-structure identities of K (Eq. "S4_cg_stiffness_matrix").
  * MMS convergence rate 2 in every field (Sections 5.1 and 5.2, slope
    alpha/d = 1 in 2D and 2/3 in 3D).
  * The mass-balance invariant (Eqs. "DG_GE_Darcy_mass_balance_1/2" with q = 1).
  * Network swap symmetry, and decoupling at beta = 0.
  * Wathen's element bound for the Jacobi-scaled P1 mass matrix.
  * The selfp Schur blocks on the constant pressure, in closed form from the
    mesh alone (divergence theorem on the boundary facets).
"""
import os

import numpy as np
import pytest
import scipy.sparse as sp

import inputs
import oracle
from oracle.assembly import assemble_problem, geometry
from oracle.quadrature import cell_rule, facet_rule

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.split("#")[0].strip()
            if line:
                rows.append([int(v) for v in line.split()])
    return rows


def _solve(P, coords=True):
    K, f = assemble_problem(P)
    x = oracle.solve_direct(K, f, coords=P.mesh.coords if coords else None)
    return K, f, oracle.to_nodal(x, P.mesh.n_nodes)


# --------------------------------------------------------------------------- meshes

def test_dof_counts_match_paper_tables():
    for dim, n, dof in _load("dof_tables.txt"):
        assert inputs.dof_count(dim, n) == dof
        if (n + 1) ** dim <= 40000:
            assert inputs.unit_mesh(dim, n).n_dofs == dof


@pytest.mark.parametrize("dim,n", [(2, 3), (3, 2)])
def test_mesh_is_a_conforming_partition(dim, n):
    m = inputs.unit_mesh(dim, n)
    g = geometry(m.coords, m.cells)
    assert np.all(g.vol > 0)
    assert np.isclose(g.vol.sum(), 1.0)                      # tiles the unit square / cube
    # boundary measure = perimeter / surface area
    X = m.coords[m.bfacets]
    if dim == 2:
        meas = np.linalg.norm(X[:, 1] - X[:, 0], axis=1)
        assert np.isclose(meas.sum(), 4.0)
    else:
        meas = 0.5 * np.linalg.norm(np.cross(X[:, 1] - X[:, 0], X[:, 2] - X[:, 0]), axis=1)
        assert np.isclose(meas.sum(), 6.0)
    assert m.n_cells == (2 if dim == 2 else 6) * n ** dim


def test_disc_wheel_is_a_conforming_partition_of_its_polygon():
    S, R = 70, 3
    m = inputs.disc_wheel(S, R)
    g = geometry(m.coords, m.cells)
    assert np.all(g.vol > 0)
    assert np.isclose(g.vol.sum(), 0.5 * S * np.sin(2 * np.pi / S))    # the polygon's area
    assert m.n_nodes == 1 + S * R and m.n_cells == S * (2 * R - 1)
    assert m.n_bfacets == S                                             # the rim edges only
    assert np.allclose(np.linalg.norm(m.coords[m.bfacets], axis=2), 1.0)
    assert np.bincount(m.cells.ravel()).max() == S                      # the centre node


# --------------------------------------------------------------------------- quadrature

@pytest.mark.parametrize("dim", [2, 3])
def test_cell_rule_integrates_p1_products_exactly(dim):
    # int_K lambda_a lambda_b = |K| (1 + delta_ab) / ((d+1)(d+2)); int_K lambda_a = |K|/(d+1)
    lam, w = cell_rule(dim)
    nv = dim + 1
    M = np.einsum("q,qa,qb->ab", w, lam, lam)
    ref = (np.ones((nv, nv)) + np.eye(nv)) / ((dim + 1) * (dim + 2))
    assert np.allclose(M, ref, rtol=0, atol=1e-15)
    assert np.allclose(w @ lam, 1.0 / nv)


@pytest.mark.parametrize("dim", [2, 3])
def test_facet_rule_integrates_p1_products_exactly(dim):
    lam, w = facet_rule(dim)
    nf = dim
    M = np.einsum("q,qa,qb->ab", w, lam, lam)
    ref = (np.ones((nf, nf)) + np.eye(nf)) / (dim * (dim + 1))
    assert np.allclose(M, ref, rtol=0, atol=1e-15)


# --------------------------------------------------------------------------- patch tests

def _linear_problem(dim, n, a, c1, c2, k1, k2, beta, perturb=True, gamma_b=None):
    m = inputs.unit_mesh(dim, n)
    if perturb:  # move interior nodes so the patch test is not a structured-mesh accident
        rng = inputs.rng(7)
        X = m.coords.copy()
        inner = np.all((X > 1e-12) & (X < 1 - 1e-12), axis=1)
        X[inner] += rng.uniform(-0.2, 0.2, size=(inner.sum(), dim)) / n
        m.coords = X
    p01 = m.coords @ a + c1
    p02 = m.coords @ a + c2
    gb = np.zeros(dim) if gamma_b is None else np.asarray(gamma_b, dtype=np.float64)
    return inputs.Problem(m, np.full(m.n_cells, np.log(k1)), np.full(m.n_cells, np.log(k2)),
                          1.3, beta, gb, p01, p02)


@pytest.mark.parametrize("dim,n", [(2, 4), (3, 3)])
def test_linear_patch_is_reproduced_exactly(dim, n):
    a = np.array([0.7, -1.1, 0.4][:dim])
    P = _linear_problem(dim, n, a, 0.3, 0.3, k1=2.0, k2=0.05, beta=3.0)
    _, _, xn = _solve(P, coords=False)
    mu = P.mu
    d = dim
    assert np.allclose(xn[:, d], P.mesh.coords @ a + 0.3, atol=1e-11)
    assert np.allclose(xn[:, 2 * d + 1], P.mesh.coords @ a + 0.3, atol=1e-11)
    assert np.allclose(xn[:, :d], -(2.0 / mu) * a[None, :], atol=1e-10)
    assert np.allclose(xn[:, d + 1:2 * d + 1], -(0.05 / mu) * a[None, :], atol=1e-11)


@pytest.mark.parametrize("dim,n", [(2, 4), (3, 3)])
def test_body_force_patch_is_reproduced_exactly(dim, n):
    # Darcy's law with a constant body force (Eqs. "DG_GE_Darcy_BLM_1/2"):
    # mu/k_i u_i + grad p_i = gamma b. With p1 = p2 = a.x + c there is no mass
    # transfer, so u_i = (k_i/mu)(gamma b - a) is constant and divergence-free:
    # an exact solution in P1 for constant k. CG-VMS is consistent, so the
    # discrete solution reproduces it only if the load vector carries the
    # body-force terms of Eq. "S4_cg_rhs" with the right weights and signs:
    # 1/2 (w; gamma b) on the velocity rows and 1/2 (grad q; k/mu gamma b) on
    # the pressure rows. A dropped 1/2 or a flipped sign of either term breaks it.
    a = np.array([0.7, -1.1, 0.4][:dim])
    gb = np.array([1.9, 0.6, -1.3][:dim])
    P = _linear_problem(dim, n, a, -0.2, -0.2, k1=2.0, k2=0.05, beta=3.0, gamma_b=gb)
    K, f, xn = _solve(P, coords=False)
    mu, d = P.mu, dim
    assert np.abs(f).max() > 0.1
    assert np.allclose(xn[:, d], P.mesh.coords @ a - 0.2, atol=1e-11)
    assert np.allclose(xn[:, 2 * d + 1], P.mesh.coords @ a - 0.2, atol=1e-11)
    assert np.allclose(xn[:, :d], (2.0 / mu) * (gb - a)[None, :], atol=1e-10)
    assert np.allclose(xn[:, d + 1:2 * d + 1], (0.05 / mu) * (gb - a)[None, :], atol=1e-11)
    # gamma b = a: the body force balances the pressure gradient and u = 0
    P0 = _linear_problem(dim, n, a, 0.5, 0.5, k1=2.0, k2=0.05, beta=3.0, gamma_b=a)
    _, _, x0 = _solve(P0, coords=False)
    assert np.allclose(x0[:, :d], 0.0, atol=1e-11)
    assert np.allclose(x0[:, d + 1:2 * d + 1], 0.0, atol=1e-11)


def test_linear_patch_on_the_disc_wheel():
    # The wheel's rim facets have 70 different outward normals (the box meshes
    # only axis-aligned ones), and its centre node lies in 70 cells. P1 must
    # still reproduce p = a.x + c with u = -(k/mu) a exactly.
    a = np.array([0.9, -0.6])
    W = inputs.wheel_problem(70, 3, seed=0)
    m = W.mesh
    P = inputs.Problem(m, np.full(m.n_cells, np.log(1.7)), np.full(m.n_cells, np.log(0.2)),
                       1.3, 2.0, np.zeros(2), m.coords @ a - 0.4, m.coords @ a - 0.4)
    _, _, xn = _solve(P, coords=False)
    assert np.allclose(xn[:, 2], m.coords @ a - 0.4, atol=1e-11)
    assert np.allclose(xn[:, 5], m.coords @ a - 0.4, atol=1e-11)
    assert np.allclose(xn[:, :2], -(1.7 / 1.3) * a[None, :], atol=1e-10)
    assert np.allclose(xn[:, 3:5], -(0.2 / 1.3) * a[None, :], atol=1e-10)


@pytest.mark.parametrize("dim,n", [(2, 4), (3, 2)])
def test_constant_pressure_gives_zero_velocity(dim, n):
    P = _linear_problem(dim, n, np.zeros(dim), 1.5, 1.5, k1=1.0, k2=0.1, beta=1.0)
    _, _, xn = _solve(P, coords=False)
    d = dim
    assert np.allclose(xn[:, d], 1.5, atol=1e-12)
    assert np.allclose(xn[:, 2 * d + 1], 1.5, atol=1e-12)
    assert np.allclose(xn[:, :d], 0.0, atol=1e-11)
    assert np.allclose(xn[:, d + 1:2 * d + 1], 0.0, atol=1e-11)


# --------------------------------------------------------------------------- linear algebra

@pytest.mark.parametrize("dim,n", [(2, 3), (2, 4), (3, 2)])
def test_sparse_lu_matches_dense_lu(dim, n):
    P = inputs.heterogeneous_problem(dim, n, seed=3, beta=2.5)
    K, f = assemble_problem(P)
    x1 = oracle.solve_direct(K, f)
    x2 = oracle.solve_dense(K, f)
    x3 = oracle.solve_direct(K, f, coords=P.mesh.coords)
    assert np.allclose(x1, x2, rtol=1e-12, atol=1e-12 * np.abs(x2).max())
    assert np.allclose(x3, x2, rtol=1e-12, atol=1e-12 * np.abs(x2).max())


@pytest.mark.parametrize("dim,n", [(2, 4), (3, 2)])
def test_block_structure_identities(dim, n):
    P = inputs.heterogeneous_problem(dim, n, seed=1, beta=0.7)
    K, _ = assemble_problem(P)
    b = oracle.field_split_blocks(K, P.mesh.n_nodes, dim)
    # K_pu = -K_up^T exactly, for both networks
    for i in ("1", "2"):
        assert abs(b[f"K{i}pu"] + b[f"K{i}up"].T).max() < 1e-14
    # the symmetric part of K is blockdiag(A, D): A SPD, D symmetric semi-definite
    Kd = K.toarray()
    S = 0.5 * (Kd + Kd.T)
    A, D = b["A"].toarray(), b["D"].toarray()
    nu = A.shape[0]
    perm = np.concatenate([
        np.concatenate([np.arange(s * P.mesh.n_nodes, (s + 1) * P.mesh.n_nodes)
                        for s in list(range(dim)) + list(range(dim + 1, 2 * dim + 1))]),
        np.arange(dim * P.mesh.n_nodes, (dim + 1) * P.mesh.n_nodes),
        np.arange((2 * dim + 1) * P.mesh.n_nodes, (2 * dim + 2) * P.mesh.n_nodes)])
    Sp = S[np.ix_(perm, perm)]
    assert abs(Sp[:nu, nu:]).max() < 1e-14
    assert np.linalg.eigvalsh(A).min() > 0
    # D is only semi-definite: p1 = p2 = const is its one null vector (no gradient,
    # no transfer). K stays nonsingular because B maps that vector to the boundary
    # flux term, which is non-zero.
    evd = np.linalg.eigvalsh(D)
    assert evd[0] > -1e-13 * evd[-1] and evd[1] > 1e-6 * evd[-1]
    ones = np.ones(D.shape[0])
    assert np.linalg.norm(D @ ones) < 1e-13 * np.linalg.norm(D)
    assert np.linalg.norm(b["B"] @ ones) > 1e-3
    assert np.allclose(A, A.T, atol=1e-15) and np.allclose(D, D.T, atol=1e-15)
    # K^T is K with the B and C blocks negated
    Kt = Kd.T[np.ix_(perm, perm)]
    Kp = Kd[np.ix_(perm, perm)].copy()
    Kp[:nu, nu:] *= -1.0
    Kp[nu:, :nu] *= -1.0
    assert np.allclose(Kt, Kp, atol=1e-14)


def test_selfp_schur_is_spd_and_has_two_ring_pattern():
    P = inputs.heterogeneous_problem(2, 6, seed=2)
    K, _ = assemble_problem(P)
    S1, S2 = oracle.selfp_schur(K, P.mesh.n_nodes, 2)
    for S in (S1, S2):
        Sd = S.toarray()
        assert np.allclose(Sd, Sd.T, atol=1e-13 * abs(Sd).max())
        assert np.linalg.eigvalsh(Sd).min() > 0
    # 2-ring: the pattern of G^2 for the node graph G
    m = P.mesh
    nv = 3
    r = np.repeat(m.cells, nv, axis=1).ravel()
    c = np.tile(m.cells, (1, nv)).ravel()
    G = sp.csr_matrix((np.ones(r.size), (r, c)), shape=(m.n_nodes,) * 2)
    G2 = (G @ G).astype(bool)
    assert ((abs(S1) > 0).astype(bool) > G2).nnz == 0


def _boundary_facets_with_normals(coords, cells, d):
    """Facets of the unit box mesh that belong to one cell, with |F| and the
    outward normal of the box face they lie on."""
    from itertools import combinations
    count = {}
    for c in cells:
        for f in combinations(sorted(int(v) for v in c), d):
            count[f] = count.get(f, 0) + 1
    out = []
    for f, k in count.items():
        if k != 1:
            continue
        X = coords[list(f)]
        n = np.zeros(d)
        for ax in range(d):
            if np.all(np.abs(X[:, ax]) < 1e-12):
                n[ax] = -1.0
            elif np.all(np.abs(X[:, ax] - 1.0) < 1e-12):
                n[ax] = 1.0
        assert np.abs(n).sum() == 1.0, "a boundary facet off the box faces"
        if d == 2:
            area = np.linalg.norm(X[1] - X[0])
        else:
            area = 0.5 * np.linalg.norm(np.cross(X[1] - X[0], X[2] - X[0]))
        out.append((f, area, n))
    return out


@pytest.mark.parametrize("dim,n", [(2, 6), (3, 3)])
def test_selfp_schur_constant_mode_closed_form(dim, n):
    # S_pi = D_ii - C_i diag(A_i)^-1 B_i with C_i = -B_i^T (Section 4.2). On the
    # constant pressure 1:
    #   * L 1 = 0 and 1^T M 1 = |Omega| = 1, so 1^T D_ii 1 = beta/mu;
    #   * (B_i 1)_a = sum_b K_up(a, b) = -int_Omega grad phi_a
    #     = -sum over boundary facets F of a of |F|/d n_F (divergence theorem);
    #   * diag(A_i)_a = sum over the cells of a of mu/(2 k_i) 2|K|/((d+1)(d+2)).
    # So 1^T S_pi 1 = beta/mu + sum_a |(B_i 1)_a|^2 / diag(A_i)_a. A dropped D
    # term, a wrong Schur sign, a lumped or mis-scaled diag(A) or a wrong B
    # all change it.
    from math import factorial
    mu, beta = 1.3, 0.7
    P = inputs.heterogeneous_problem(dim, n, seed=5, beta=beta, mu=mu)
    m = P.mesh
    K, _ = assemble_problem(P)
    S = oracle.selfp_schur(K, m.n_nodes, dim)
    X, C = m.coords, m.cells
    vol = np.abs(np.linalg.det(X[C[:, 1:]] - X[C[:, :1]])) / factorial(dim)
    b1 = np.zeros((m.n_nodes, dim))
    for f, area, nrm in _boundary_facets_with_normals(X, C, dim):
        for v in f:
            b1[v] -= area / dim * nrm
    one = np.ones(m.n_nodes)
    for Si, lk in zip(S, (P.logk1, P.logk2)):
        w = mu / (2.0 * np.exp(lk)) * 2.0 * vol / ((dim + 1) * (dim + 2))
        dA = np.zeros(m.n_nodes)
        for j in range(dim + 1):
            np.add.at(dA, C[:, j], w)
        expected = beta / mu + float(np.sum(b1 ** 2 / dA[:, None]))
        got = float(one @ (Si @ one))
        assert abs(got - expected) <= 1e-12 * expected, (got, expected)


# --------------------------------------------------------------------------- MMS

def _rates(dim, ns):
    errs = []
    for n in ns:
        P = inputs.mms_problem(dim, n)
        _, _, xn = _solve(P)
        M = oracle.p1_mass_matrix(P.mesh.coords, P.mesh.cells)
        errs.append(oracle.interp_l2_errors(xn, inputs.nodal_exact(P.mesh.coords), M))
    out = {}
    for fld in oracle.FIELDS:
        out[fld] = [np.log(errs[i][fld] / errs[i + 1][fld]) / np.log(ns[i + 1] / ns[i])
                    for i in range(len(ns) - 1)]
    return out


def test_mms_rate_2d():
    rates = _rates(2, [8, 16, 32])
    for fld, r in rates.items():
        assert abs(r[-1] - 2.0) < 0.2, (fld, r)


def test_mms_rate_3d():
    rates = _rates(3, [4, 8])
    for fld, r in rates.items():
        assert abs(r[-1] - 2.0) < 0.3, (fld, r)


def test_mms_solution_satisfies_strong_form():
    # u_i = -(k_i/mu) grad p_i and div u1 = -beta/mu (p1 - p2), by centred differences
    prm = inputs.PAPER
    rng = inputs.rng(5)
    for dim in (2, 3):
        x = rng.uniform(0.2, 0.8, size=(20, dim))
        h = 1e-5
        u1, p1, u2, p2 = inputs.exact(x, prm)
        div1 = np.zeros(20)
        for k in range(dim):
            e = np.zeros(dim)
            e[k] = h
            _, p1p, _, _ = inputs.exact(x + e, prm)
            _, p1m, _, _ = inputs.exact(x - e, prm)
            assert np.allclose(-(prm.k1 / prm.mu) * (p1p - p1m) / (2 * h), u1[:, k], rtol=1e-7)
            u1p = inputs.exact(x + e, prm)[0][:, k]
            u1m = inputs.exact(x - e, prm)[0][:, k]
            div1 += (u1p - u1m) / (2 * h)
        assert np.allclose(div1, -prm.beta / prm.mu * (p1 - p2), rtol=1e-6)


# --------------------------------------------------------------------------- invariants

@pytest.mark.parametrize("dim,n,gb", [(2, 8, 0.0), (3, 3, 0.0), (2, 0, 0.0), (2, 8, 1.5),
                                      (3, 3, -0.8)])
def test_mass_balance_invariant(dim, n, gb):
    # n = 0: the disc wheel (70 thin cells around its centre). A body force
    # does not change the invariant: its pressure-row load 1/2 (grad q; k/mu
    # gamma b) vanishes for q = 1.
    P = (inputs.heterogeneous_problem(dim, n, seed=4, beta=1.7) if n else
         inputs.wheel_problem(70, 3, seed=4, beta=1.7))
    P = P.with_(gamma_b=gb * np.linspace(1.0, -0.5, dim))
    _, _, xn = _solve(P)
    b1, b2 = oracle.mass_balance(xn, P.mesh.coords, P.mesh.cells, P.mu, P.beta)
    scale = np.abs(xn).max()
    assert abs(b1) < 1e-11 * scale and abs(b2) < 1e-11 * scale


def _weighted_mass(dim, n, seed):
    m = inputs.unit_mesh(dim, n)
    geom = geometry(m.coords, m.cells)
    lam, wq = cell_rule(dim)
    wts = np.exp(inputs.rng(seed).normal(0, 1, m.n_cells))
    Me = np.einsum("c,c,q,qa,qb->cab", wts, geom.vol, wq, lam, lam)
    nv = dim + 1
    r = np.repeat(m.cells, nv, axis=1).ravel()
    c = np.tile(m.cells, (1, nv)).ravel()
    return sp.csr_matrix((Me.ravel(), (r, c)), shape=(m.n_nodes,) * 2)


@pytest.mark.parametrize("dim,n", [(2, 5), (3, 3)])
def test_ilu0_reproduces_the_matrix_on_its_pattern(dim, n):
    # the defining property of ILU(0): (L U)_ij = A_ij wherever A has an entry
    M = _weighted_mass(dim, n, 12)
    LU = oracle.ilu0(M)
    L, U = oracle.ilu0_factors(LU)
    assert np.array_equal(LU.indptr, sp.csr_matrix(M).indptr)
    prod = (L @ U).tocsr()
    Mc = sp.csr_matrix(M)
    rows = np.repeat(np.arange(Mc.shape[0]), np.diff(Mc.indptr))
    assert np.allclose(np.asarray(prod[rows, Mc.indices]).ravel(), Mc.data, rtol=1e-13, atol=0)
    # the product has fill outside the pattern, so ILU(0) is not the exact LU here
    assert (abs(prod - Mc) > 1e-12 * abs(Mc).max()).nnz > 0


def test_ilu0_of_a_tridiagonal_matrix_is_the_exact_lu():
    # a 1D P1 mass matrix with random cell weights: LU has no fill, so ILU(0) is exact
    n = 40
    w = np.exp(inputs.rng(13).normal(0, 1, n - 1))
    h = 1.0 / (n - 1)
    main = np.zeros(n)
    main[:-1] += 2 * w * h / 6
    main[1:] += 2 * w * h / 6
    T = sp.diags([w * h / 6, main, w * h / 6], [-1, 0, 1], format="csr")
    r = inputs.rng(14).standard_normal(n)
    x = oracle.ilu0_solve(oracle.ilu0(T), r)
    assert np.allclose(x, np.linalg.solve(T.toarray(), r), rtol=1e-12, atol=1e-12 * abs(x).max())


@pytest.mark.parametrize("dim,n", [(2, 5), (3, 2)])
def test_chebyshev_jacobi_degree_one_and_error_bound(dim, n):
    M = _weighted_mass(dim, n, 15)
    r = inputs.rng(16).standard_normal(M.shape[0])
    lo, hi = 0.5, 0.5 * (dim + 2)                     # Wathen's interval
    theta, delta = 0.5 * (hi + lo), 0.5 * (hi - lo)
    # degree 1 is the scaled Jacobi step D^-1 r / theta
    x1 = oracle.chebyshev_jacobi(M, r, 1, lo, hi)
    assert np.allclose(x1, r / M.diagonal() / theta, rtol=1e-12)
    # degree k: the error in the M-norm is at most 1 / T_k(theta/delta) of the exact solve's norm
    xs = np.linalg.solve(M.toarray(), r)
    Md = M.toarray()
    nrm = lambda e: np.sqrt(e @ Md @ e)
    for k in (2, 3, 5):
        xk = oracle.chebyshev_jacobi(M, r, k, lo, hi)
        bound = 1.0 / np.cosh(k * np.arccosh(theta / delta))
        assert nrm(xk - xs) <= bound * nrm(xs) * (1 + 1e-10)
        assert nrm(xk - xs) >= 1e-6 * bound * nrm(xs)  # an approximation, not the exact solve


@pytest.mark.parametrize("dim,n,gb", [(2, 12, 0.0), (3, 5, 0.0), (3, 4, 1.2)])
def test_field_split_gmres_reaches_the_direct_solution(dim, n, gb):
    # The oracle for meshes too large to factor: flexible GMRES to a true
    # residual of 1e-13. It must land on the sparse-LU solution.
    P = inputs.heterogeneous_problem(dim, n, seed=6, beta=1.4)
    P = P.with_(gamma_b=gb * np.linspace(1.0, -0.5, dim))
    K, f = assemble_problem(P)
    x, it, res = oracle.solve_field_split_gmres(K, f, P.mesh.n_nodes, dim)
    assert res <= 1e-13 and oracle.residual(K, x, f) <= 1e-13
    assert it < 60
    xd = oracle.solve_dense(K, f) if K.shape[0] < 3000 else oracle.solve_direct(K, f)
    err = oracle.field_rel_errors(oracle.to_nodal(x, P.mesh.n_nodes),
                                  oracle.to_nodal(xd, P.mesh.n_nodes))
    assert max(err.values()) <= 1e-11, err


def test_swap_symmetry_and_beta_zero_decoupling():
    m = inputs.unit_mesh(2, 6)
    lk, _ = inputs.lognormal_logk(m.n_cells, 9)
    p0, _ = inputs.boundary_pressures(m.coords)
    P = inputs.Problem(m, lk, lk.copy(), 1.0, 2.0, np.zeros(2), p0, p0.copy())
    _, _, xn = _solve(P)
    assert np.allclose(xn[:, :3], xn[:, 3:], atol=1e-12 * abs(xn).max())
    # beta = 0: network 1 does not see network 2's data
    lk1, lk2 = inputs.lognormal_logk(m.n_cells, 10)
    q1, q2 = inputs.boundary_pressures(m.coords)
    Pa = inputs.Problem(m, lk1, lk2, 1.0, 0.0, np.zeros(2), q1, q2)
    Pb = inputs.Problem(m, lk1, lk2 + 1.0, 1.0, 0.0, np.zeros(2), q1, -q2)
    _, _, xa = _solve(Pa)
    _, _, xb = _solve(Pb)
    assert np.allclose(xa[:, :3], xb[:, :3], atol=1e-12 * abs(xa).max())
    assert not np.allclose(xa[:, 3:], xb[:, 3:])


@pytest.mark.parametrize("dim,n", [(2, 5), (3, 2), (2, 0)])
def test_wathen_bound_for_jacobi_scaled_mass(dim, n):
    # eig(diag(M)^-1 M) lies in [1/2, (d+2)/2] for any positive per-cell weights
    # and any simplices (n = 0: the disc wheel, with its thin centre cells)
    m = inputs.unit_mesh(dim, n) if n else inputs.disc_wheel(70, 3)
    geom = geometry(m.coords, m.cells)
    lam, wq = cell_rule(dim)
    wts = np.exp(inputs.rng(11).normal(0, 2, m.n_cells))
    Me = np.einsum("c,c,q,qa,qb->cab", wts, geom.vol, wq, lam, lam)
    nv = dim + 1
    r = np.repeat(m.cells, nv, axis=1).ravel()
    c = np.tile(m.cells, (1, nv)).ravel()
    M = sp.csr_matrix((Me.ravel(), (r, c)), shape=(m.n_nodes,) * 2).toarray()
    Dm = np.diag(1.0 / np.sqrt(np.diag(M)))
    ev = np.linalg.eigvalsh(Dm @ M @ Dm)
    assert ev.min() >= 0.5 - 1e-12
    assert ev.max() <= (dim + 2) / 2 + 1e-12
