"""Pins for the oracle adjoint: complex-step and central finite differences.

The objective is J = sum over nodes (p1 - p1_obs)^2. p1_obs is the oracle's p1
for log-k fields drawn from the next seed. The adjoint gradient (transpose solve
plus per-cell element sensitivities) must agree with
  * the global complex-step derivative (Martins et al., ACM TOMS 2003), to
    1e-9 relative: both are exact up to rounding. With and without a body
    force, which makes the load vector depend on log k;
  * central differences with h = 1e-6, to 1e-5 relative to the largest
    sampled gradient entry: the FD truncation and cancellation error is
    about 1e-10 |J| / h.
"""
import numpy as np
import pytest

import inputs
import oracle
from oracle.assembly import assemble_problem


def _setup(dim, n, seed=0, gamma_b=None, kind="simplex"):
    P = inputs.heterogeneous_problem(dim, n, seed=seed, beta=1.3, kind=kind)
    Pobs = inputs.heterogeneous_problem(dim, n, seed=seed + 1, beta=1.3, kind=kind)
    if gamma_b is not None:
        P = P.with_(gamma_b=np.asarray(gamma_b, dtype=np.float64))
        Pobs = Pobs.with_(gamma_b=np.asarray(gamma_b, dtype=np.float64))
    K, f = assemble_problem(P)
    Kobs, fobs = assemble_problem(Pobs)
    xn = oracle.to_nodal(oracle.solve_direct(K, f), P.mesh.n_nodes)
    p1_obs = oracle.to_nodal(oracle.solve_direct(Kobs, fobs), P.mesh.n_nodes)[:, dim]
    g = oracle.objective_grad_x(xn, p1_obs)
    lam = oracle.adjoint_solve(K, g)
    return P, p1_obs, oracle.adjoint_gradients(P, xn, lam)


@pytest.mark.parametrize("dim,n,gamma_b,kind", [(2, 5, None, "simplex"), (3, 2, None, "simplex"),
                                                (2, 5, [2.0, -1.5], "simplex"),
                                                (3, 2, [0.5, 1.0, -2.0], "simplex"),
                                                (2, 4, [1.0, -0.5], "q1"), (3, 2, None, "q1")])
def test_adjoint_matches_complex_step(dim, n, gamma_b, kind):
    # With a body force the load depends on k (1/2 (grad q; k/mu gamma b)), so
    # the adjoint's -lambda^T df/dlog k term is exercised too. The Q1 cases
    # check the element sensitivities of q1.py the same way.
    P, p1_obs, (g1, g2, gb) = _setup(dim, n, gamma_b=gamma_b, kind=kind)
    cells = inputs.sample_cells(P.mesh.n_cells, 4, seed=2)
    for c in cells:
        cs1 = oracle.complex_step_gradient(P, p1_obs, "logk1", int(c))
        cs2 = oracle.complex_step_gradient(P, p1_obs, "logk2", int(c))
        assert abs(g1[c] - cs1) <= 1e-9 * max(abs(cs1), 1e-300) + 1e-14 * abs(g1).max()
        assert abs(g2[c] - cs2) <= 1e-9 * max(abs(cs2), 1e-300) + 1e-14 * abs(g2).max()
    csb = oracle.complex_step_gradient(P, p1_obs, "beta")
    assert abs(gb - csb) <= 1e-9 * abs(csb)


def test_adjoint_matches_central_differences():
    P, p1_obs, (g1, g2, gb) = _setup(2, 6, seed=3)
    cells = inputs.sample_cells(P.mesh.n_cells, 5, seed=5)
    fd1 = np.array([oracle.fd_gradient(P, p1_obs, "logk1", int(c)) for c in cells])
    fd2 = np.array([oracle.fd_gradient(P, p1_obs, "logk2", int(c)) for c in cells])
    scale = max(abs(fd1).max(), abs(fd2).max())
    assert np.allclose(g1[cells], fd1, rtol=0, atol=1e-5 * scale)
    assert np.allclose(g2[cells], fd2, rtol=0, atol=1e-5 * scale)
    fdb = oracle.fd_gradient(P, p1_obs, "beta")
    assert abs(gb - fdb) <= 1e-5 * abs(fdb)
