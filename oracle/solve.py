"""FP64 direct solves of K x = f (oracle; test infrastructure only).

The GPU path's preconditioned FGMRES (Section 4.2, Method 2) converges to the
solution of the assembled system K x = f (Eq. "S4_linear_problem"). The
oracle computes that solution by its definition, with a sparse LU
factorisation (SuperLU, through scipy).

Two orderings:
  * default: SuperLU's own column ordering with partial pivoting;
  * with node coordinates: a geometric nested-dissection ordering of the nodes
    (recursive bisection by the median lattice plane; George, SIAM J. Numer.
    Anal. 10, 1973). A node's DoFs stay together. The factorisation then runs
    without pivoting. That is valid here: the symmetric part of the CG-VMS K
    is blockdiag(A, D) with A and D SPD, so every leading principal minor of K
    is non-zero. The relative residual is checked after the solve, and the
    solve falls back to partial pivoting if it is above 1e-12.
A permutation does not change the solution; it only cuts the fill on 3D meshes.
``solve_dense`` is the textbook dense LU (LAPACK through numpy), used as an
independent check on tiny meshes.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def lu(K):
    return spla.splu(sp.csc_matrix(K), permc_spec="MMD_AT_PLUS_A")


def nested_dissection(coords: np.ndarray, leaf: int = 8) -> np.ndarray:
    """Node order: the two halves first (recursively), then the separator plane."""
    out = []

    def rec(idx):
        if idx.size <= leaf:
            out.extend(idx.tolist())
            return
        X = coords[idx]
        ax = int(np.argmax(X.max(0) - X.min(0)))
        v = X[:, ax]
        vals = np.unique(v)
        if vals.size < 3:
            out.extend(idx.tolist())
            return
        mid = vals[vals.size // 2]
        rec(idx[v < mid])
        rec(idx[v > mid])
        out.extend(idx[v == mid].tolist())
    rec(np.arange(coords.shape[0]))
    return np.asarray(out, dtype=np.int64)


def solve_direct(K, f, trans: bool = False, coords: np.ndarray | None = None):
    """Solve K x = f (or K^T x = f) by sparse LU."""
    f = np.asarray(f)
    if coords is None:
        return lu(K).solve(f, trans="T" if trans else "N")
    n = coords.shape[0]
    ns = K.shape[0] // n
    order = nested_dissection(coords)
    perm = (np.arange(ns)[None, :] * n + order[:, None]).ravel()
    Kp = sp.csc_matrix(sp.csr_matrix(K)[perm][:, perm])
    fac = spla.splu(Kp, permc_spec="NATURAL", diag_pivot_thresh=0.0,
                    options=dict(SymmetricMode=True))
    y = fac.solve(f[perm], trans="T" if trans else "N")
    x = np.empty_like(y)
    x[perm] = y
    Kt = K.T if trans else K
    if np.linalg.norm(f - Kt @ x) > 1e-12 * np.linalg.norm(f):
        return lu(K).solve(f, trans="T" if trans else "N")
    return x


def solve_dense(K, f):
    return np.linalg.solve(K.toarray() if sp.issparse(K) else K, f)


def residual(K, x, f):
    """Relative residual ||f - K x||_2 / ||f||_2."""
    r = f - K @ x
    return float(np.linalg.norm(r) / np.linalg.norm(f))
