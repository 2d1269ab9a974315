"""Quadrature rules on simplices (oracle; test infrastructure only).

Every integrand of the P1 CG-VMS form is a polynomial of degree at most two on
each cell or facet, so degree-2 rules integrate it exactly.

  * Triangle: the three interior points with barycentric coordinates
    (2/3, 1/6, 1/6) and its permutations, with equal weights (Strang & Fix).
  * Tetrahedron: the four points (a, b, b, b) and its permutations, where
    a = (5 + 3 sqrt 5)/20 and b = (5 - sqrt 5)/20, with equal weights.
  * Segment (a 2D boundary facet): two-point Gauss-Legendre, exact to degree 3.

Each rule returns barycentric coordinates [Q, nv] and weights [Q] that sum to 1.
A physical integral is the weighted sum times the simplex measure.
"""
from __future__ import annotations

import numpy as np


def _perms(first: float, rest: float, nv: int) -> np.ndarray:
    pts = np.full((nv, nv), rest)
    np.fill_diagonal(pts, first)
    return pts


def cell_rule(dim: int):
    if dim == 2:
        lam = _perms(2.0 / 3.0, 1.0 / 6.0, 3)
        return lam, np.full(3, 1.0 / 3.0)
    if dim == 3:
        s5 = np.sqrt(5.0)
        lam = _perms((5.0 + 3.0 * s5) / 20.0, (5.0 - s5) / 20.0, 4)
        return lam, np.full(4, 0.25)
    raise ValueError("dim must be 2 or 3")


def facet_rule(dim: int):
    """Rule on a boundary facet of a dim-dimensional cell (dimension dim-1)."""
    if dim == 2:
        g = 0.5 / np.sqrt(3.0)
        lam = np.array([[0.5 + g, 0.5 - g], [0.5 - g, 0.5 + g]])
        return lam, np.full(2, 0.5)
    if dim == 3:
        return cell_rule(2)
    raise ValueError("dim must be 2 or 3")
