"""CG-VMS assembly on Q1 quadrilaterals and hexahedra (oracle; test infrastructure only).

The paper's CG-VMS formulation uses equal-order [Q1 + Q1]^2 on QUAD and HEX
meshes (Table "ELE_level_discretization"). The bilinear form and the linear
functional are those of Eq. "CG_VMS_Weak_form" (Section 3.3), written out
term by term as in assembly.py:

  B_stab = sum_i (w_i; mu/k_i u_i) - (div w_i; p_i) + (q_i; div u_i)
           - 1/2 (mu/k_i w_i - grad q_i; k_i/mu (mu/k_i u_i + grad p_i))
         + (q1 - q2; beta/mu (p1 - p2)),
  L_stab = sum_i (w_i; gb) - (w_i.n; p0i)_G - 1/2 (mu/k_i w_i - grad q_i; k_i/mu gb).

Here they are evaluated on tensor-product cells with the isoparametric Q1 map
x(xi) = sum_v x_v phi_v(xi), xi in [0,1]^d, and phi_v the tensor product of
(1 - xi_k) and xi_k. Vertex v of a cell lies at the corner with coordinate
bits (v & 1, (v >> 1) & 1, (v >> 2) & 1). Cell integrals use the tensor
2-point Gauss rule (2^d points), facet integrals the same rule in d-1
dimensions. On parallelepipeds this is exact for every term. On general
cells it is the standard rule for Q1, and it still integrates exactly the
terms that a linear pressure field with a constant velocity produces (the
patch tests). Unknown numbering and the node-interleaved conversion are
those of assembly.py.
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse as sp

from inputs.meshes import tensor_facets


def gauss_tensor(dim: int):
    """Points [Q, dim] in [0,1]^dim and weights [Q] (summing to 1) of the 2-point rule."""
    g = 0.5 / np.sqrt(3.0)
    pts = np.array(list(itertools.product([0.5 - g, 0.5 + g], repeat=dim)))
    return pts, np.full(pts.shape[0], 1.0 / pts.shape[0])


def q1_basis(xi: np.ndarray):
    """Values [Q, nv] and reference gradients [Q, nv, dim] of the Q1 basis at xi [Q, dim]."""
    Q, dim = xi.shape
    nv = 1 << dim
    phi = np.ones((Q, nv))
    dphi = np.ones((Q, nv, dim))
    for v in range(nv):
        for k in range(dim):
            bit = (v >> k) & 1
            f = xi[:, k] if bit else 1.0 - xi[:, k]
            df = 1.0 if bit else -1.0
            phi[:, v] *= f
            for j in range(dim):
                dphi[:, v, j] *= (df if j == k else f)
    return phi, dphi


def q1_geometry(coords, cells):
    """Quadrature weights times |det J| [C, Q], basis values [Q, nv], physical gradients [C, Q, nv, d]."""
    d = coords.shape[1]
    xi, wq = gauss_tensor(d)
    phi, dphi = q1_basis(xi)
    X = coords[cells]                                   # [C, nv, d]
    J = np.einsum("cvr,qvk->cqrk", X, dphi)             # dx_r / dxi_k
    det = np.linalg.det(J)
    Jinv = np.linalg.inv(J)                             # dxi_k / dx_r
    grad = np.einsum("qvk,cqkr->cqvr", dphi, Jinv)
    return np.abs(det) * wq[None, :], phi, grad, det


def _fields(d, phi, grad):
    C, Q, nv, _ = grad.shape
    ns = 2 * d + 2
    ne = ns * nv
    U = [np.zeros((C, ne, Q, d)), np.zeros((C, ne, Q, d))]
    DIVU = [np.zeros((C, ne, Q)), np.zeros((C, ne, Q))]
    P = [np.zeros((C, ne, Q)), np.zeros((C, ne, Q))]
    GP = [np.zeros((C, ne, Q, d)), np.zeros((C, ne, Q, d))]
    for net, off in ((0, 0), (1, d + 1)):
        for a in range(nv):
            for k in range(d):
                i = (off + k) * nv + a
                U[net][:, i, :, k] = phi[None, :, a]
                DIVU[net][:, i, :] = grad[:, :, a, k]
            i = (off + d) * nv + a
            P[net][:, i, :] = phi[None, :, a]
            GP[net][:, i, :, :] = grad[:, :, a, :]
    return U, DIVU, P, GP


def element_matrices_q1(w, phi, grad, k1, k2, mu, beta, d):
    """Element matrices [C, n_e, n_e] of B_stab (row = test, column = trial)."""
    U, DIVU, P, GP = _fields(d, phi, grad)
    dt = np.result_type(k1, k2, beta, np.float64)

    def inner(X, Y):
        if X.ndim == 4:
            return np.einsum("cq,ciqk,cjqk->cij", w, X, Y)
        return np.einsum("cq,ciq,cjq->cij", w, X, Y)

    a = [mu / np.asarray(k1, dtype=dt), mu / np.asarray(k2, dtype=dt)]
    K = np.zeros((w.shape[0],) + (U[0].shape[1],) * 2, dtype=dt)
    for n in range(2):
        an = a[n][:, None, None, None]
        K += inner(U[n], an * U[n])
        K -= inner(DIVU[n], P[n])
        K += inner(P[n], DIVU[n])
        K -= 0.5 * inner(an * U[n] - GP[n], (1.0 / an) * (an * U[n] + GP[n]))
    K += inner(P[0] - P[1], (beta / mu) * (P[0] - P[1]))
    return K


def element_rhs_body_q1(w, phi, grad, k1, k2, mu, gamma_b, d):
    """Volume part of L_stab per element [C, n_e]."""
    U, DIVU, P, GP = _fields(d, phi, grad)
    dt = np.result_type(k1, k2, np.float64)
    gb = np.asarray(gamma_b, dtype=np.float64)[None, None, None, :]
    a = [mu / np.asarray(k1, dtype=dt), mu / np.asarray(k2, dtype=dt)]
    F = np.zeros(U[0].shape[:2], dtype=dt)
    for n in range(2):
        an = a[n][:, None, None, None]
        F += np.einsum("cq,ciqk->ci", w, U[n] * gb)
        F -= 0.5 * np.einsum("cq,ciqk->ci", w, (an * U[n] - GP[n]) * ((1.0 / an) * gb))
    return F


def _global_rows(cells, n_nodes, d):
    nv = cells.shape[1]
    ns = 2 * d + 2
    s = np.repeat(np.arange(ns), nv)
    a = np.tile(np.arange(nv), ns)
    return s[None, :] * n_nodes + cells[:, a]


def facet_owners_q1(cells, bfacets, d):
    """Owning cell of each boundary facet (by its sorted node set)."""
    faces = tensor_facets(d)
    keyof = lambda f: tuple(sorted(int(v) for v in f))
    table = {}
    for c in range(cells.shape[0]):
        for f in faces:
            table[keyof(cells[c, f])] = c
    own = np.empty(bfacets.shape[0], dtype=np.int64)
    for i, f in enumerate(bfacets):
        k = keyof(f)
        if k not in table:
            raise ValueError("a boundary facet is not a face of any cell")
        own[i] = table[k]
    return own


def assemble_rhs_q1(coords, cells, bfacets, w, phi, grad, k1, k2, mu, gamma_b, p01, p02):
    """Global load vector f (slot-major), Eq. "S4_cg_rhs", on Q1 cells."""
    n_nodes, d = coords.shape
    ns = 2 * d + 2
    dt = np.result_type(k1, k2, np.float64)
    f = np.zeros(ns * n_nodes, dtype=dt)
    rows = _global_rows(cells, n_nodes, d)
    np.add.at(f, rows.ravel(), element_rhs_body_q1(w, phi, grad, k1, k2, mu, gamma_b, d).ravel())
    if bfacets.shape[0] == 0:
        return f
    own = facet_owners_q1(cells, bfacets, d)
    centre = coords[cells[own]].mean(axis=1)            # a point inside the owner cell
    s, ws = gauss_tensor(d - 1)
    psi, dpsi = q1_basis(s)                              # [S, nf], [S, nf, d-1]
    Xf = coords[bfacets]                                 # [F, nf, d]
    xs = np.einsum("sa,far->fsr", psi, Xf)
    T = np.einsum("sak,far->fskr", dpsi, Xf)             # tangents [F, S, d-1, d]
    if d == 2:
        nrm = np.stack([T[:, :, 0, 1], -T[:, :, 0, 0]], axis=-1)
    else:
        nrm = np.cross(T[:, :, 0, :], T[:, :, 1, :])
    dA = np.linalg.norm(nrm, axis=-1)                    # [F, S]
    nrm = nrm / dA[..., None]
    out = np.einsum("fsr,fsr->fs", nrm, xs - centre[:, None, :]) < 0.0
    nrm[out] *= -1.0
    for net, p0, off in ((0, p01, 0), (1, p02, d + 1)):
        p0h = np.einsum("sa,fa->fs", psi, p0[bfacets])
        for a in range(bfacets.shape[1]):
            for k in range(d):
                val = -np.einsum("s,fs,fs,fs->f", ws, dA, nrm[:, :, k], psi[None, :, a] * p0h)
                np.add.at(f, (off + k) * n_nodes + bfacets[:, a], val)
    return f


def assemble_q1(coords, cells, bfacets, logk1, logk2, mu, beta, gamma_b, p01, p02,
                chunk: int = 2048, with_rhs: bool = True):
    """Global K (CSR, slot-major) and f on Q1 cells, Eq. "S4_linear_problem"."""
    coords = np.asarray(coords, dtype=np.float64)
    cells = np.asarray(cells, dtype=np.int64)
    n_nodes, d = coords.shape
    N = (2 * d + 2) * n_nodes
    k1 = np.exp(np.asarray(logk1))
    k2 = np.exp(np.asarray(logk2))
    dt = np.result_type(k1, k2, beta, np.float64)
    w, phi, grad, _ = q1_geometry(coords, cells)
    R, Cc, V = [], [], []
    for s0 in range(0, cells.shape[0], chunk):
        e = slice(s0, min(s0 + chunk, cells.shape[0]))
        Ke = element_matrices_q1(w[e], phi, grad[e], k1[e], k2[e], mu, beta, d)
        rows = _global_rows(cells[e], n_nodes, d)
        ne = rows.shape[1]
        R.append(np.repeat(rows, ne, axis=1).ravel())
        Cc.append(np.tile(rows, (1, ne)).ravel())
        V.append(Ke.ravel())
    K = sp.csr_matrix((np.concatenate(V).astype(dt), (np.concatenate(R), np.concatenate(Cc))),
                      shape=(N, N))
    K.sum_duplicates()
    K.sort_indices()
    f = None
    if with_rhs:
        f = assemble_rhs_q1(coords, cells, np.asarray(bfacets, dtype=np.int64), w, phi, grad, k1,
                            k2, mu, gamma_b, np.asarray(p01), np.asarray(p02))
    return K, f


def q1_mass_matrix(coords, cells):
    """Scalar Q1 mass matrix M_ab = int phi_a phi_b by the 2-point tensor rule."""
    w, phi, _, _ = q1_geometry(np.asarray(coords, dtype=np.float64), np.asarray(cells))
    Me = np.einsum("cq,qa,qb->cab", w, phi, phi)
    nv = cells.shape[1]
    r = np.repeat(cells, nv, axis=1).ravel()
    c = np.tile(cells, (1, nv)).ravel()
    n = coords.shape[0]
    return sp.csr_matrix((Me.ravel(), (r, c)), shape=(n, n))


def mass_balance_q1(xh, coords, cells, mu, beta):
    """(int div u1h + beta/mu int (p1h-p2h), int div u2h - beta/mu int (p1h-p2h)) on Q1 cells."""
    d = coords.shape[1]
    w, phi, grad, _ = q1_geometry(np.asarray(coords, dtype=np.float64), np.asarray(cells))
    u1 = xh[:, 0:d][cells]
    u2 = xh[:, d + 1:2 * d + 1][cells]
    div1 = np.einsum("cvk,cqvk->cq", u1, grad)
    div2 = np.einsum("cvk,cqvk->cq", u2, grad)
    dp = np.einsum("qv,cv->cq", phi, (xh[:, d] - xh[:, 2 * d + 1])[cells])
    i1, i2, ip = (float(np.sum(w * div1)), float(np.sum(w * div2)), float(np.sum(w * dp)))
    return i1 + beta / mu * ip, i2 - beta / mu * ip
