"""Error norms and balance integrals (oracle; test infrastructure only).

  * interp_l2_errors: the L2 error against the P1 interpolant of the exact
    solution. It is what the paper's appendix listing computes with
    ``errornorm(interpolate(exact), solution)``. The difference of two P1
    functions is integrated exactly through the P1 mass matrix.
  * field_rel_errors: relative per-field parity norm between two nodal
    solutions. For a field f in {u1, p1, u2, p2} it is
    ||x_f - y_f||_2 / ||y_f||_2 over all nodal values, counting every
    velocity component.
  * mass_balance: the integrals of Eqs. "DG_GE_Darcy_mass_balance_1/2"
    tested with q = 1. The P1 space contains q = 1 when pressure data is
    imposed weakly, so for the discrete solution
    int div u1 + beta/mu int (p1 - p2) = 0 and int div u2 - beta/mu int (p1 - p2) = 0.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .assembly import geometry
from .quadrature import cell_rule

FIELDS = ("u1", "p1", "u2", "p2")


def field_slices(d: int):
    return {"u1": slice(0, d), "p1": slice(d, d + 1), "u2": slice(d + 1, 2 * d + 1),
            "p2": slice(2 * d + 1, 2 * d + 2)}


def p1_mass_matrix(coords, cells):
    """Scalar P1 mass matrix by quadrature: M_ab = int phi_a phi_b."""
    d = coords.shape[1]
    geom = geometry(coords, cells)
    lam, wq = cell_rule(d)
    Me = np.einsum("c,q,qa,qb->cab", geom.vol, wq, lam, lam)
    nv = d + 1
    r = np.repeat(cells, nv, axis=1).ravel()
    c = np.tile(cells, (1, nv)).ravel()
    n = coords.shape[0]
    return sp.csr_matrix((Me.ravel(), (r, c)), shape=(n, n))


def interp_l2_errors(xh: np.ndarray, x_exact_nodal: np.ndarray, M) -> dict:
    """Per-field L2 error ||I_h f - f_h|| with the P1 mass matrix M."""
    d = (xh.shape[1] - 2) // 2
    out = {}
    for name, sl in field_slices(d).items():
        e = x_exact_nodal[:, sl] - xh[:, sl]
        out[name] = float(np.sqrt(sum(e[:, k] @ (M @ e[:, k]) for k in range(e.shape[1]))))
    return out


def field_rel_errors(x: np.ndarray, y: np.ndarray) -> dict:
    """Relative L2 (nodal) difference per field; y is the reference."""
    d = (y.shape[1] - 2) // 2
    out = {}
    for name, sl in field_slices(d).items():
        den = np.linalg.norm(y[:, sl])
        out[name] = float(np.linalg.norm(x[:, sl] - y[:, sl]) / (den if den > 0 else 1.0))
    return out


def mass_balance(xh: np.ndarray, coords, cells, mu: float, beta: float):
    """(int div u1h + beta/mu int (p1h-p2h), int div u2h - beta/mu int (p1h-p2h))."""
    d = coords.shape[1]
    geom = geometry(coords, cells)
    sl = field_slices(d)
    u1 = xh[:, sl["u1"]][cells]          # [C, nv, d]
    u2 = xh[:, sl["u2"]][cells]
    div1 = np.einsum("cak,cak->c", u1, geom.grad)          # constant per cell
    div2 = np.einsum("cak,cak->c", u2, geom.grad)
    dp = (xh[:, d] - xh[:, 2 * d + 1])[cells].mean(axis=1)  # P1 mean over the cell
    i_div1 = float(np.sum(geom.vol * div1))
    i_div2 = float(np.sum(geom.vol * div2))
    i_dp = float(np.sum(geom.vol * dp))
    return i_div1 + beta / mu * i_dp, i_div2 - beta / mu * i_dp
