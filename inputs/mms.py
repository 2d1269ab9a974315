"""The paper's manufactured solutions, used as boundary data and for errors.

2D: Section 5.1 (two-dimensional study), analytic u1, p1, u2, p2 with
eta = sqrt(beta (k1 + k2) / (k1 k2)). 3D: Section 5.2 (three-dimensional
study). The printed 3D p2 carries mu/(beta k1); the appendix CG-VMS listing
(its boundary expressions use the factor 10 = 1/(beta k2)) and the 2D
formula both give mu/(beta k2), which is also the value that satisfies the
PDE. That reading is used here.

Both solutions satisfy the strong form with gamma*b = 0. The default
parameters are the paper's: mu = beta = k1 = 1, k2 = 0.1 (Tables "2D
dataset" and "3D dataset").
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class MMSParams:
    mu: float = 1.0
    beta: float = 1.0
    k1: float = 1.0
    k2: float = 0.1

    @property
    def eta(self) -> float:
        return float(np.sqrt(self.beta * (self.k1 + self.k2) / (self.k1 * self.k2)))


PAPER = MMSParams()


def exact(x: np.ndarray, prm: MMSParams = PAPER):
    """Exact (u1 [n,d], p1 [n], u2 [n,d], p2 [n]) at points x [n, d]."""
    x = np.asarray(x, dtype=np.float64)
    d = x.shape[1]
    mu, beta, k1, k2, eta = prm.mu, prm.beta, prm.k1, prm.k2, prm.eta
    pi = np.pi
    ex = np.exp(pi * x[:, 0])
    if d == 2:
        y = x[:, 1]
        s = ex * np.sin(pi * y)
        ey = np.exp(eta * y)
        p1 = mu / pi * s - mu / (beta * k1) * ey
        p2 = mu / pi * s + mu / (beta * k2) * ey
        u1 = -k1 * np.stack([s, ex * np.cos(pi * y) - eta / (beta * k1) * ey], axis=1)
        u2 = -k2 * np.stack([s, ex * np.cos(pi * y) + eta / (beta * k2) * ey], axis=1)
        return u1, p1, u2, p2
    if d == 3:
        y, z = x[:, 1], x[:, 2]
        s = ex * (np.sin(pi * y) + np.sin(pi * z))
        ey, ez = np.exp(eta * y), np.exp(eta * z)
        p1 = mu / pi * s - mu / (beta * k1) * (ey + ez)
        p2 = mu / pi * s + mu / (beta * k2) * (ey + ez)
        u1 = -k1 * np.stack([s,
                             ex * np.cos(pi * y) - eta / (beta * k1) * ey,
                             ex * np.cos(pi * z) - eta / (beta * k1) * ez], axis=1)
        u2 = -k2 * np.stack([s,
                             ex * np.cos(pi * y) + eta / (beta * k2) * ey,
                             ex * np.cos(pi * z) + eta / (beta * k2) * ez], axis=1)
        return u1, p1, u2, p2
    raise ValueError("dimension must be 2 or 3")


def boundary_pressures(coords: np.ndarray, prm: MMSParams = PAPER):
    """Nodal pressure data (p01, p02) from the exact solution at every node.

    Only boundary-facet nodes are read by the weak boundary term; interior
    values are carried along for convenience.
    """
    _, p1, _, p2 = exact(coords, prm)
    return p1.copy(), p2.copy()


def nodal_exact(coords: np.ndarray, prm: MMSParams = PAPER) -> np.ndarray:
    """Exact solution in node-interleaved layout [n_nodes, 2d+2]."""
    u1, p1, u2, p2 = exact(coords, prm)
    return np.concatenate([u1, p1[:, None], u2, p2[:, None]], axis=1)
