"""Adjoint gradients of a pressure-misfit objective (oracle; test infrastructure only).

The system K(theta) x = f(theta) is the CG-VMS system of Eq. "S4_linear_problem",
on simplices (assembly.py) or Q1 cells (q1.py).
theta is one of: a per-cell log k1, a per-cell log k2, or beta. The objective is
J(x) = sum over nodes (p1 - p1_obs)^2. The adjoint identity gives
    dJ/dtheta = -lambda^T (dK/dtheta x - df/dtheta),  with  K^T lambda = dJ/dx.
K^T is applied by a sparse LU transposed solve.

The per-cell derivative of the element matrix is a complex-step derivative of
the oracle's own element routine (Martins, Sturdza & Alonso, ACM TOMS 29(3),
2003): d/dt F(t) = Im F(t + i h) / h with h = 1e-30. The element routine is
analytic in log k and beta, since it uses exp and products but no
conjugation. So this is exact to rounding. Two independent checks of the
whole chain are provided: a global complex-step derivative (a complex sparse
LU solve) and a central finite difference.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .assembly import (Geometry, assemble, element_matrices, element_rhs_body, geometry,
                       _global_rows, from_nodal, to_nodal)
from .solve import lu

CS_H = 1e-30


def objective(xn: np.ndarray, p1_obs: np.ndarray) -> float:
    d = (xn.shape[1] - 2) // 2
    r = xn[:, d] - p1_obs
    return r @ r


def objective_grad_x(xn: np.ndarray, p1_obs: np.ndarray) -> np.ndarray:
    """dJ/dx in node-interleaved layout: 2 (p1 - p1_obs) on the p1 slot."""
    d = (xn.shape[1] - 2) // 2
    g = np.zeros_like(xn)
    g[:, d] = 2.0 * (xn[:, d] - p1_obs)
    return g


def adjoint_solve(K, g_nodal: np.ndarray) -> np.ndarray:
    """lambda with K^T lambda = g (node-interleaved in and out)."""
    n = g_nodal.shape[0]
    lam = lu(K).solve(from_nodal(g_nodal), trans="T")
    return to_nodal(lam, n)


def adjoint_gradients(problem, xn: np.ndarray, lamn: np.ndarray, chunk: int = 8192):
    """(dJ/dlogk1 [C], dJ/dlogk2 [C], dJ/dbeta) from the forward x and adjoint lambda."""
    m = problem.mesh
    if getattr(m, "kind", "simplex") == "q1":
        return _adjoint_gradients_q1(problem, xn, lamn, chunk)
    d = m.dim
    coords, cells = m.coords, m.cells.astype(np.int64)
    n = m.n_nodes
    x = from_nodal(xn)
    lam = from_nodal(lamn)
    geom = geometry(coords, cells)
    k1 = np.exp(problem.logk1)
    k2 = np.exp(problem.logk2)
    g1 = np.zeros(m.n_cells)
    g2 = np.zeros(m.n_cells)
    gb = 0.0
    ih = 1j * CS_H
    for s in range(0, m.n_cells, chunk):
        e = slice(s, min(s + chunk, m.n_cells))
        g = Geometry(geom.vol[e], geom.grad[e])
        rows = _global_rows(cells[e], n, d)
        xe, le = x[rows], lam[rows]                              # [c, n_e]
        for which, out in ((1, g1), (2, g2)):
            kk1 = np.exp(problem.logk1[e] + (ih if which == 1 else 0.0))
            kk2 = np.exp(problem.logk2[e] + (ih if which == 2 else 0.0))
            dK = element_matrices(g, kk1, kk2, problem.mu, problem.beta, d).imag / CS_H
            dF = element_rhs_body(g, kk1, kk2, problem.mu, problem.gamma_b, d).imag / CS_H
            out[e] = -np.einsum("ci,cij,cj->c", le, dK, xe) + np.einsum("ci,ci->c", le, dF)
        dKb = element_matrices(g, k1[e], k2[e], problem.mu, problem.beta + ih, d).imag / CS_H
        gb += -float(np.einsum("ci,cij,cj->", le, dKb, xe))
    return g1, g2, gb


def _adjoint_gradients_q1(problem, xn, lamn, chunk):
    """The same gradients on Q1 cells (element routines of q1.py, complex step)."""
    from .q1 import element_matrices_q1, element_rhs_body_q1, q1_geometry
    from .q1 import _global_rows as rows_q1
    m = problem.mesh
    d = m.dim
    cells = m.cells.astype(np.int64)
    x = from_nodal(xn)
    lam = from_nodal(lamn)
    w, phi, grad, _ = q1_geometry(np.asarray(m.coords, dtype=np.float64), cells)
    k1 = np.exp(problem.logk1)
    k2 = np.exp(problem.logk2)
    g1 = np.zeros(m.n_cells)
    g2 = np.zeros(m.n_cells)
    gb = 0.0
    ih = 1j * CS_H
    for s0 in range(0, m.n_cells, chunk):
        e = slice(s0, min(s0 + chunk, m.n_cells))
        rows = rows_q1(cells[e], m.n_nodes, d)
        xe, le = x[rows], lam[rows]
        for which, out in ((1, g1), (2, g2)):
            kk1 = np.exp(problem.logk1[e] + (ih if which == 1 else 0.0))
            kk2 = np.exp(problem.logk2[e] + (ih if which == 2 else 0.0))
            dK = element_matrices_q1(w[e], phi, grad[e], kk1, kk2, problem.mu, problem.beta, d)
            dF = element_rhs_body_q1(w[e], phi, grad[e], kk1, kk2, problem.mu, problem.gamma_b, d)
            out[e] = (-np.einsum("ci,cij,cj->c", le, dK.imag / CS_H, xe)
                      + np.einsum("ci,ci->c", le, dF.imag / CS_H))
        dKb = element_matrices_q1(w[e], phi, grad[e], k1[e], k2[e], problem.mu,
                                  problem.beta + ih, d).imag / CS_H
        gb += -float(np.einsum("ci,cij,cj->", le, dKb, xe))
    return g1, g2, gb


def _solve_J(problem, p1_obs, logk1, logk2, beta):
    m = problem.mesh
    if getattr(m, "kind", "simplex") == "q1":
        from .q1 import assemble_q1
        K, f = assemble_q1(m.coords, m.cells, m.bfacets, logk1, logk2, problem.mu, beta,
                           problem.gamma_b, problem.p01, problem.p02)
    else:
        K, f = assemble(m.coords, m.cells, m.bfacets, logk1, logk2, problem.mu, beta,
                        problem.gamma_b, problem.p01, problem.p02)
    x = lu(K).solve(f)
    xn = to_nodal(x, m.n_nodes)
    d = m.dim
    r = xn[:, d] - p1_obs
    return np.sum(r * r)


def complex_step_gradient(problem, p1_obs, which: str, index: int = 0) -> float:
    """dJ/dtheta by a complex-step global solve; which in {'logk1','logk2','beta'}."""
    lk1 = problem.logk1.astype(np.complex128)
    lk2 = problem.logk2.astype(np.complex128)
    beta = complex(problem.beta)
    if which == "logk1":
        lk1[index] += 1j * CS_H
    elif which == "logk2":
        lk2[index] += 1j * CS_H
    elif which == "beta":
        beta += 1j * CS_H
    else:
        raise ValueError(which)
    return float(np.imag(_solve_J(problem, p1_obs, lk1, lk2, beta)) / CS_H)


def fd_gradient(problem, p1_obs, which: str, index: int = 0, h: float = 1e-6) -> float:
    """Central finite difference (J(t+h) - J(t-h)) / 2h with direct solves."""
    vals = []
    for sgn in (1.0, -1.0):
        lk1 = problem.logk1.copy()
        lk2 = problem.logk2.copy()
        beta = problem.beta
        if which == "logk1":
            lk1[index] += sgn * h
        elif which == "logk2":
            lk2[index] += sgn * h
        elif which == "beta":
            beta += sgn * h
        else:
            raise ValueError(which)
        vals.append(float(_solve_J(problem, p1_obs, lk1, lk2, beta)))
    return (vals[0] - vals[1]) / (2.0 * h)
