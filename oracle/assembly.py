"""Plain CG-VMS P1 assembly of K and f (oracle; test infrastructure only).

The element matrix comes from evaluating, term by term at exact quadrature
points, the stabilised bilinear form of Eq. "CG_VMS_Weak_form" (Section 3.3):

  B_stab = (w1; mu/k1 u1) - (div w1; p1) + (q1; div u1)
         + (w2; mu/k2 u2) - (div w2; p2) + (q2; div u2)
         + (q1 - q2; beta/mu (p1 - p2))
         - 1/2 (mu/k1 w1 - grad q1; k1/mu (mu/k1 u1 + grad p1))
         - 1/2 (mu/k2 w2 - grad q2; k2/mu (mu/k2 u2 + grad p2))

The Galerkin part is B_Gal of Eq. "VMS_classical_mixed_formulation". The
linear functional is

  L_stab = (w1; gb) - (w1.n; p01)_G + (w2; gb) - (w2.n; p02)_G
         - 1/2 (mu/k1 w1 - grad q1; k1/mu gb) - 1/2 (mu/k2 w2 - grad q2; k2/mu gb)

Here gb is the constant gamma*b. The pressure data p0i enters through its P1
interpolant, on every boundary facet. This is the weak imposition of the
paper's appendix CG-VMS listing (bcs = [], ds(1..6) terms). The per-block form
of the result is Eqs. "S4_cg_stiffness_matrix" and "S4_cg_rhs".

Unknown numbering: slot-major. Global index = s * n_nodes + a, where the slot
s runs over [u1_0 .. u1_{d-1}, p1, u2_0 .. u2_{d-1}, p2] and a is the node.
``to_nodal`` converts to the node-interleaved layout [n_nodes, 2d+2].
"""
from __future__ import annotations

from dataclasses import dataclass
from math import factorial

import numpy as np
import scipy.sparse as sp

from .quadrature import cell_rule, facet_rule


@dataclass
class Geometry:
    vol: np.ndarray    # [C] cell measure |K|
    grad: np.ndarray   # [C, nv, d] gradients of the barycentric coordinates


def geometry(coords: np.ndarray, cells: np.ndarray) -> Geometry:
    """Cell measure and constant basis gradients of P1 simplices."""
    X = coords[cells]                     # [C, nv, d]
    d = X.shape[2]
    J = np.transpose(X[:, 1:, :] - X[:, :1, :], (0, 2, 1))   # columns x_a - x_0
    det = np.linalg.det(J)
    vol = np.abs(det) / factorial(d)
    Jinv = np.linalg.inv(J)               # row a-1 is grad lambda_a
    g = np.empty((X.shape[0], d + 1, d))
    g[:, 1:, :] = Jinv
    g[:, 0, :] = -Jinv.sum(axis=1)
    return Geometry(vol, g)


def slot_index(d: int):
    """Slot numbers of the four fields in one node's [2d+2] block."""
    return {"u1": list(range(d)), "p1": [d], "u2": list(range(d + 1, 2 * d + 1)), "p2": [2 * d + 1]}


def _local_fields(d: int, lam: np.ndarray, grad: np.ndarray):
    """Values of every local mixed basis function at the quadrature points.

    Local DoF i = s * nv + a (slot s, vertex a). Returns, for each field,
    the value at the quadrature points and the gradient or divergence
    (constant on a P1 cell). Shapes: vectors [C, n_e, Q, d], scalars [C, n_e, Q].
    """
    C, nv, _ = grad.shape
    Q = lam.shape[0]
    ns = 2 * d + 2
    ne = ns * nv
    U = [np.zeros((C, ne, Q, d)), np.zeros((C, ne, Q, d))]
    DIVU = [np.zeros((C, ne, Q)), np.zeros((C, ne, Q))]
    P = [np.zeros((C, ne, Q)), np.zeros((C, ne, Q))]
    GP = [np.zeros((C, ne, Q, d)), np.zeros((C, ne, Q, d))]
    for net, off in ((0, 0), (1, d + 1)):
        for a in range(nv):
            for k in range(d):
                i = (off + k) * nv + a           # velocity component k at vertex a
                U[net][:, i, :, k] = lam[:, a][None, :]
                DIVU[net][:, i, :] = grad[:, a, k][:, None]
            i = (off + d) * nv + a               # pressure at vertex a
            P[net][:, i, :] = lam[:, a][None, :]
            GP[net][:, i, :, :] = grad[:, a, None, :]
    return U, DIVU, P, GP


def element_matrices(geom: Geometry, k1, k2, mu: float, beta, d: int):
    """Element matrices [C, n_e, n_e] of B_stab (row = test, column = trial).

    k1, k2 are per-cell permeabilities and may be complex (complex-step use);
    beta may be complex too.
    """
    lam, wq = cell_rule(d)
    U, DIVU, P, GP = _local_fields(d, lam, geom.grad)
    w = geom.vol[:, None] * wq[None, :]                       # [C, Q]
    dt = np.result_type(k1, k2, beta, np.float64)

    def inner(X, Y):
        if X.ndim == 4:
            return np.einsum("cq,ciqk,cjqk->cij", w, X, Y)
        return np.einsum("cq,ciq,cjq->cij", w, X, Y)

    a = [mu / np.asarray(k1, dtype=dt), mu / np.asarray(k2, dtype=dt)]  # mu k^-1
    K = np.zeros((geom.vol.shape[0],) + (U[0].shape[1],) * 2, dtype=dt)
    for n in range(2):
        an = a[n][:, None, None, None]
        K += inner(U[n], an * U[n])                        # (w; mu/k u)
        K -= inner(DIVU[n], P[n])                          # -(div w; p)
        K += inner(P[n], DIVU[n])                          # (q; div u)
        K -= 0.5 * inner(an * U[n] - GP[n], (1.0 / an) * (an * U[n] + GP[n]))
    K += inner(P[0] - P[1], (beta / mu) * (P[0] - P[1]))   # (q1 - q2; beta/mu (p1 - p2))
    return K


def element_rhs_body(geom: Geometry, k1, k2, mu: float, gamma_b: np.ndarray, d: int):
    """Volume part of L_stab per element [C, n_e] (the gamma*b terms)."""
    lam, wq = cell_rule(d)
    U, DIVU, P, GP = _local_fields(d, lam, geom.grad)
    w = geom.vol[:, None] * wq[None, :]
    dt = np.result_type(k1, k2, np.float64)
    gb = np.asarray(gamma_b, dtype=np.float64)[None, None, None, :]
    a = [mu / np.asarray(k1, dtype=dt), mu / np.asarray(k2, dtype=dt)]
    F = np.zeros(U[0].shape[:2], dtype=dt)
    for n in range(2):
        an = a[n][:, None, None, None]
        F += np.einsum("cq,ciqk->ci", w, U[n] * gb)                           # (w; gb)
        F -= 0.5 * np.einsum("cq,ciqk->ci", w, (an * U[n] - GP[n]) * ((1.0 / an) * gb))
    return F


def _global_rows(cells: np.ndarray, n_nodes: int, d: int) -> np.ndarray:
    nv = d + 1
    ns = 2 * d + 2
    s = np.repeat(np.arange(ns), nv)            # slot of local DoF i = s*nv + a
    a = np.tile(np.arange(nv), ns)              # vertex of local DoF i
    return s[None, :] * n_nodes + cells[:, a]   # [C, n_e]


def facet_cells(cells: np.ndarray, bfacets: np.ndarray):
    """For each boundary facet: owning cell and the local vertex opposite it."""
    d = cells.shape[1] - 1
    nv = d + 1
    keys, owner, opp = [], [], []
    for drop in range(nv):
        keep = [v for v in range(nv) if v != drop]
        f = np.sort(cells[:, keep].astype(np.int64), axis=1)
        key = np.zeros(f.shape[0], dtype=np.int64)
        for c in range(d):
            key = key * (1 << 21) + f[:, c]
        keys.append(key)
        owner.append(np.arange(cells.shape[0]))
        opp.append(np.full(cells.shape[0], drop))
    keys = np.concatenate(keys)
    owner = np.concatenate(owner)
    opp = np.concatenate(opp)
    order = np.argsort(keys, kind="stable")
    keys, owner, opp = keys[order], owner[order], opp[order]
    fb = np.sort(bfacets.astype(np.int64), axis=1)
    kb = np.zeros(fb.shape[0], dtype=np.int64)
    for c in range(d):
        kb = kb * (1 << 21) + fb[:, c]
    pos = np.searchsorted(keys, kb)
    if np.any(pos >= keys.size) or np.any(keys[np.minimum(pos, keys.size - 1)] != kb):
        raise ValueError("a boundary facet is not a face of any cell")
    return owner[pos], opp[pos]


def _facet_normals(coords, cells, bfacets):
    """Unit outward normals and measures of the boundary facets."""
    d = coords.shape[1]
    owner, opp = facet_cells(cells, bfacets)
    Xf = coords[bfacets]                                   # [F, d, d]
    xo = coords[cells[owner, opp]]                         # opposite vertex
    if d == 2:
        t = Xf[:, 1] - Xf[:, 0]
        n = np.stack([t[:, 1], -t[:, 0]], axis=1)
        meas = np.linalg.norm(t, axis=1)
    else:
        n = np.cross(Xf[:, 1] - Xf[:, 0], Xf[:, 2] - Xf[:, 0])
        meas = 0.5 * np.linalg.norm(n, axis=1)
    n = n / np.linalg.norm(n, axis=1)[:, None]
    flip = np.einsum("fk,fk->f", n, xo - Xf[:, 0]) > 0.0   # must point away from the cell
    n[flip] *= -1.0
    return n, meas


def assemble_rhs(coords, cells, bfacets, geom: Geometry, k1, k2, mu, gamma_b, p01, p02):
    """Global load vector f (slot-major), Eq. "S4_cg_rhs"."""
    n_nodes, d = coords.shape
    ns = 2 * d + 2
    dt = np.result_type(k1, k2, np.float64)
    f = np.zeros(ns * n_nodes, dtype=dt)
    rows = _global_rows(cells, n_nodes, d)
    Fe = element_rhs_body(geom, k1, k2, mu, gamma_b, d)
    np.add.at(f, rows.ravel(), Fe.ravel())
    if bfacets.shape[0]:
        n, meas = _facet_normals(coords, cells, bfacets)
        lam, wq = facet_rule(d)                            # [Q, d] barycentric on the facet
        for net, p0, off in ((0, p01, 0), (1, p02, d + 1)):
            p0h = lam @ p0[bfacets].T                      # [Q, F] interpolant at quad points
            for a in range(d):                             # facet vertex a
                # -(w . n; p0h)_F with w = phi_a e_k
                integral = meas * np.einsum("q,q,qf->f", wq, lam[:, a], p0h)
                for k in range(d):
                    np.add.at(f, (off + k) * n_nodes + bfacets[:, a], -n[:, k] * integral)
    return f


def assemble(coords, cells, bfacets, logk1, logk2, mu, beta, gamma_b, p01, p02,
             chunk: int = 8192, with_rhs: bool = True):
    """Global K (CSR, slot-major) and f, Eq. "S4_linear_problem".

    logk1, logk2 are natural-log permeabilities (may be complex for
    complex-step derivatives).
    """
    coords = np.asarray(coords, dtype=np.float64)
    cells = np.asarray(cells, dtype=np.int64)
    n_nodes, d = coords.shape
    N = (2 * d + 2) * n_nodes
    k1 = np.exp(np.asarray(logk1))
    k2 = np.exp(np.asarray(logk2))
    dt = np.result_type(k1, k2, beta, np.float64)
    geom = geometry(coords, cells)
    K = sp.csr_matrix((N, N), dtype=dt)
    for s in range(0, cells.shape[0], chunk):
        e = slice(s, min(s + chunk, cells.shape[0]))
        g = Geometry(geom.vol[e], geom.grad[e])
        Ke = element_matrices(g, k1[e], k2[e], mu, beta, d)
        rows = _global_rows(cells[e], n_nodes, d)
        ne = rows.shape[1]
        r = np.repeat(rows, ne, axis=1).ravel()
        c = np.tile(rows, (1, ne)).ravel()
        K = K + sp.csr_matrix((Ke.ravel(), (r, c)), shape=(N, N))
    K.sum_duplicates()
    K.sort_indices()
    f = None
    if with_rhs:
        f = assemble_rhs(coords, cells, np.asarray(bfacets, dtype=np.int64), geom, k1, k2, mu,
                         gamma_b, np.asarray(p01), np.asarray(p02))
    return K, f


def assemble_problem(problem, **kw):
    """K and f of a problem: P1 on simplices, or Q1 (oracle/q1.py) on tensor-product cells."""
    m = problem.mesh
    if getattr(m, "kind", "simplex") == "q1":
        from .q1 import assemble_q1
        return assemble_q1(m.coords, m.cells, m.bfacets, problem.logk1, problem.logk2, problem.mu,
                           problem.beta, problem.gamma_b, problem.p01, problem.p02, **kw)
    return assemble(m.coords, m.cells, m.bfacets, problem.logk1, problem.logk2, problem.mu,
                    problem.beta, problem.gamma_b, problem.p01, problem.p02, **kw)


def to_nodal(x: np.ndarray, n_nodes: int) -> np.ndarray:
    """Slot-major vector -> node-interleaved [n_nodes, 2d+2]."""
    return np.ascontiguousarray(np.asarray(x).reshape(-1, n_nodes).T)


def from_nodal(xn: np.ndarray) -> np.ndarray:
    """Node-interleaved [n_nodes, 2d+2] -> slot-major vector."""
    return np.ascontiguousarray(np.asarray(xn).T).ravel()


def assemble_rows(problem, nodes):
    """Exact rows of K and entries of f for the given nodes (oracle, sampled check).

    Only the cells and boundary facets that touch the sampled nodes are
    assembled. The sampled rows receive every contribution they have, so they
    equal the rows of the full system. Returns (K_rows CSR [len(nodes)*ns,
    ns*n_nodes] in slot-major numbering, f_rows, row_ids).
    """
    m = problem.mesh
    nodes = np.asarray(nodes, dtype=np.int64)
    cmask = np.isin(m.cells, nodes).any(axis=1)
    fmask = np.isin(m.bfacets, nodes).any(axis=1)
    K, f = assemble(m.coords, m.cells[cmask], m.bfacets[fmask], problem.logk1[cmask],
                    problem.logk2[cmask], problem.mu, problem.beta, problem.gamma_b, problem.p01,
                    problem.p02)
    n = m.n_nodes
    ns = 2 * m.dim + 2
    rows = (np.arange(ns)[:, None] * n + nodes[None, :]).ravel()
    return K[rows], f[rows], rows
