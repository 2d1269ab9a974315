"""FP64 iterative solve of K x = f for meshes too large to factor (oracle; test
infrastructure only).

A sparse LU of the whole CG-VMS system (Eq. "S4_linear_problem") takes
minutes at 24^3 cells and is out of reach on the 3D benchmark meshes. This
module reaches the same solution another way. It runs flexible GMRES(m)
(right preconditioning with the preconditioned vectors kept, Saad, SIAM J.
Sci. Comput. 14(2), 1993; Arnoldi and Givens steps as in Saad & Schultz,
SIAM J. Sci. Stat. Comput. 7(3), 1986) on K. It stops when the TRUE residual
||f - K x||_2 / ||f||_2 is far below the GPU path's tolerance. The
preconditioner only decides how fast that happens, never what the answer is.
It is the Schur-complement factorisation of Section 4.2 (Method 2, splitting
by fields), with library factorisations for its pieces:
  * A = blockdiag(K1_uu, K2_uu) has no coupling between velocity components
    or networks, so it is solved block by block. Each n x n component block
    gets an incomplete LU (scipy's spilu, threshold drop_tol); identical
    blocks share one factorisation;
  * the pressure Schur block is the selfp matrix of Eqs. "S4_sp1" and
    "S4_sp2", S_pi = Ki_pp - Ki_pu diag(Ki_uu)^-1 Ki_up, one per network
    (the additive split of Method 2), each with an incomplete LU;
  * z = P^-1 r: y_u = A^-1 r_u; y_p = S_p^-1 (r_p - C y_u);
    z_u = A^-1 (r_u - B y_p); z_p = y_p.
The steps are library primitives: sparse products, sparse triangular solves
and dot products. Tests pin the result against the direct solve on meshes
small enough to factor.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .blocks import field_split_blocks


def _same(a, b) -> bool:
    return (a.shape == b.shape and a.nnz == b.nnz and np.array_equal(a.indptr, b.indptr)
            and np.array_equal(a.indices, b.indices) and np.array_equal(a.data, b.data))


class SchurFieldSplit:
    """The Method 2 block preconditioner with incomplete-LU pieces."""

    def __init__(self, K, n_nodes: int, d: int, drop_tol: float = 1e-4, fill_factor: float = 10.0):
        n = n_nodes
        self.n, self.d = n, d
        u_slots = list(range(d)) + list(range(d + 1, 2 * d + 1))
        p_slots = [d, 2 * d + 1]
        self.iu = np.concatenate([np.arange(s * n, (s + 1) * n) for s in u_slots])
        self.ip = np.concatenate([np.arange(s * n, (s + 1) * n) for s in p_slots])
        b = field_split_blocks(K, n, d)
        self.B, self.C = b["B"].tocsr(), b["C"].tocsr()
        A = b["A"].tocsr()
        ilu = lambda M: spla.spilu(sp.csc_matrix(M), drop_tol=drop_tol, fill_factor=fill_factor)
        blocks = [A[k * n:(k + 1) * n, k * n:(k + 1) * n].tocsr() for k in range(2 * d)]
        self.A_f = []
        for k, Ak in enumerate(blocks):
            prev = next((j for j in range(k) if _same(blocks[j], Ak)), None)
            self.A_f.append(self.A_f[prev] if prev is not None else ilu(Ak))
        Dinv = sp.diags(1.0 / A.diagonal())
        S = (b["D"] - self.C @ Dinv @ self.B).tocsr()
        self.S_f = [ilu(S[:n, :n]), ilu(S[n:, n:])]

    def _ainv(self, r):
        n = self.n
        return np.concatenate([f.solve(r[k * n:(k + 1) * n]) for k, f in enumerate(self.A_f)])

    def apply(self, r):
        n = self.n
        r_u, r_p = r[self.iu], r[self.ip]
        y_u = self._ainv(r_u)
        t_p = r_p - self.C @ y_u
        y_p = np.concatenate([self.S_f[0].solve(t_p[:n]), self.S_f[1].solve(t_p[n:])])
        z_u = self._ainv(r_u - self.B @ y_p)
        z = np.empty_like(r)
        z[self.iu] = z_u
        z[self.ip] = y_p
        return z


def gmres_right(K, f, apply_pc, tol: float = 1e-13, restart: int = 100, max_iters: int = 2000):
    """Flexible right-preconditioned GMRES(m) from x0 = 0; stops on the true relative residual.

    Returns (x, iterations, true relative residual).
    """
    f = np.asarray(f, dtype=np.float64)
    fnorm = np.linalg.norm(f)
    x = np.zeros_like(f)
    if fnorm == 0.0:
        return x, 0, 0.0
    it = 0
    r = f.copy()
    beta = fnorm
    while it < max_iters:
        m = restart
        V = np.zeros((m + 1, f.size))
        Z = np.zeros((m, f.size))
        H = np.zeros((m + 1, m))
        cs, sn = np.zeros(m), np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        k = 0
        for j in range(m):
            Z[j] = apply_pc(V[j])
            w = K @ Z[j]
            for i in range(j + 1):              # modified Gram-Schmidt
                H[i, j] = V[i] @ w
                w -= H[i, j] * V[i]
            hn = np.linalg.norm(w)
            H[j + 1, j] = hn
            if hn > 0.0:
                V[j + 1] = w / hn
            for i in range(j):                  # earlier rotations on the new column
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            rho = np.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / rho, H[j + 1, j] / rho
            H[j, j], H[j + 1, j] = rho, 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            it += 1
            k = j + 1
            if abs(g[j + 1]) <= 0.1 * tol * fnorm or hn == 0.0:   # target met, or exact subspace
                break
        y = np.linalg.solve(np.triu(H[:k, :k]), g[:k])
        x += Z[:k].T @ y
        r = f - K @ x
        beta = np.linalg.norm(r)
        if beta <= tol * fnorm:
            break
    return x, it, float(beta / fnorm)


def solve_field_split_gmres(K, f, n_nodes: int, d: int, tol: float = 1e-13, restart: int = 100):
    """Solve K x = f (slot-major) by flexible GMRES with the field-split preconditioner.

    Returns (x, iterations, true relative residual).
    """
    pc = SchurFieldSplit(K, n_nodes, d)
    K = sp.csr_matrix(K)
    return gmres_right(K, f, pc.apply, tol=tol, restart=restart)
