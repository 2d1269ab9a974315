"""The inner solves of the velocity block A (oracle; test infrastructure only).

Section 4.2 (and 4.1 per network) approximates A^-1, where A =
blockdiag(K1_uu, K2_uu) holds the two weighted mass matrices, by one sweep of
a simple preconditioner. Two are defined here by their textbook definitions,
for the parity tests of the GPU inner solves:

  * ilu0 / ilu0_solve: the incomplete LU factorisation with zero fill,
    ILU(0) (Saad, "Iterative Methods for Sparse Linear Systems", 2nd ed.,
    Section 10.3), in the matrix's own (natural) row order. This is the
    paper's ILU(0) / block-Jacobi sub-solver. L is unit lower triangular and U
    upper triangular, both on A's sparsity pattern. The defining property,
    (L U)_ij = A_ij for every (i, j) in the pattern, is pinned in the tests.
  * chebyshev_jacobi: the degree-k Chebyshev polynomial preconditioner with
    Jacobi scaling on an interval [lo, hi] that contains the spectrum of
    D^-1 M. It is written in closed form, not as a recurrence:
    x = (I - R_k(D^-1 M)) M^-1 r, with the residual polynomial
    R_k(t) = T_k((theta - t)/delta) / T_k(theta/delta), theta = (hi + lo)/2,
    delta = (hi - lo)/2 (Saad, Section 12.3). Dense matrices, small meshes only.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
from numpy.polynomial import chebyshev as npcheb


def ilu0(A):
    """ILU(0) of a square CSR matrix; returns the factors packed on A's pattern."""
    A = sp.csr_matrix(A, dtype=np.float64, copy=True)
    A.sort_indices()
    n = A.shape[0]
    ip, ix, v = A.indptr, A.indices, A.data
    where = [dict(zip(ix[ip[i]:ip[i + 1]].tolist(), range(ip[i], ip[i + 1]))) for i in range(n)]
    for i in range(n):
        for p in range(ip[i], ip[i + 1]):
            k = ix[p]
            if k >= i:
                break
            v[p] /= v[where[k][k]]                     # l_ik = a_ik / u_kk
            for q in range(ip[k], ip[k + 1]):          # a_ij -= l_ik u_kj on the pattern
                j = ix[q]
                if j > k and j in where[i]:
                    v[where[i][j]] -= v[p] * v[q]
    return A


def ilu0_factors(LU):
    """(L, U) as separate sparse matrices from the packed factors."""
    L = sp.tril(LU, k=-1, format="csr") + sp.identity(LU.shape[0], format="csr")
    U = sp.triu(LU, k=0, format="csr")
    return L, U


def ilu0_solve(LU, r):
    """(L U)^-1 r by forward and backward substitution."""
    L, U = ilu0_factors(LU)
    y = sp.linalg.spsolve_triangular(L, r, lower=True)
    return sp.linalg.spsolve_triangular(U, y, lower=False)


def chebyshev_jacobi(M, r, degree: int, lo: float, hi: float):
    """x = (I - R_k(D^-1 M)) M^-1 r for the Chebyshev residual polynomial on [lo, hi]."""
    M = M.toarray() if sp.issparse(M) else np.asarray(M)
    n = M.shape[0]
    DM = M / np.diag(M)[:, None]                      # D^-1 M
    theta, delta = 0.5 * (hi + lo), 0.5 * (hi - lo)
    Tk = np.zeros(degree + 1)
    Tk[degree] = 1.0                                   # T_k in the Chebyshev basis
    X = (theta * np.eye(n) - DM) / delta
    # T_k(X) from the defining relation T_{j+1} = 2 X T_j - T_{j-1} (T_0 = I, T_1 = X)
    T0, T1 = np.eye(n), X
    if degree == 0:
        Tm = T0
    else:
        for _ in range(degree - 1):
            T0, T1 = T1, 2.0 * X @ T1 - T0
        Tm = T1
    R = Tm / npcheb.chebval(theta / delta, Tk)
    return (np.eye(n) - R) @ np.linalg.solve(M, r)
