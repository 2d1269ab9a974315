"""Field-split blocks and selfp Schur matrices (oracle; test infrastructure only).

Section 4.2 (Method 2, splitting by fields) regroups K as [[A, B], [C, D]]:
  * A = blockdiag(K1_uu, K2_uu), the velocities of both networks;
  * B = blockdiag(K1_up, K2_up);
  * C = blockdiag(K1_pu, K2_pu);
  * D = [[K1_pp, K12_pp], [K21_pp, K2_pp]], the two pressures.
Its Schur preconditioner S_p = D - C diag(A)^-1 B has the diagonal blocks of
Eqs. "S4_sp1" and "S4_sp2":
  S_pi = Ki_pp - Ki_pu diag(Ki_uu)^-1 Ki_up.
In the printed S_p matrix the inverse on diag(K_uu) is missing. The line
above it and Eqs. "S4_sp1/S4_sp2" both carry it, and this module follows
them. The additive split keeps only these two diagonal blocks.
These are computed here by their definitions, as products of extracted
sub-matrices.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def _sel(n_nodes: int, slots):
    return np.concatenate([np.arange(s * n_nodes, (s + 1) * n_nodes) for s in slots])


def field_split_blocks(K, n_nodes: int, d: int):
    """Return dict with A, B, C, D and the per-network sub-blocks (slot-major K)."""
    K = sp.csr_matrix(K)
    u1 = _sel(n_nodes, range(d))
    p1 = _sel(n_nodes, [d])
    u2 = _sel(n_nodes, range(d + 1, 2 * d + 1))
    p2 = _sel(n_nodes, [2 * d + 1])
    u = np.concatenate([u1, u2])
    p = np.concatenate([p1, p2])
    sub = lambda r, c: K[r][:, c]
    return {
        "A": sub(u, u), "B": sub(u, p), "C": sub(p, u), "D": sub(p, p),
        "K1uu": sub(u1, u1), "K1up": sub(u1, p1), "K1pu": sub(p1, u1), "K1pp": sub(p1, p1),
        "K2uu": sub(u2, u2), "K2up": sub(u2, p2), "K2pu": sub(p2, u2), "K2pp": sub(p2, p2),
        "K12pp": sub(p1, p2), "K21pp": sub(p2, p1),
    }


def selfp_schur(K, n_nodes: int, d: int):
    """(S_p1, S_p2) = K_pp - K_pu diag(K_uu)^-1 K_up for each network."""
    b = field_split_blocks(K, n_nodes, d)
    out = []
    for i in ("1", "2"):
        dinv = sp.diags(1.0 / b[f"K{i}uu"].diagonal())
        S = b[f"K{i}pp"] - b[f"K{i}pu"] @ dinv @ b[f"K{i}up"]
        S = sp.csr_matrix(S)
        S.sum_duplicates()
        S.sort_indices()
        out.append(S)
    return tuple(out)
