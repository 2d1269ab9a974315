"""Problem descriptions: a mesh plus material data and boundary data.

The fields mirror the C-ABI problem descriptor: coordinates, cells, boundary
facets carrying pressure data, per-cell natural-log permeabilities, mu, beta,
the constant body force gamma*b and nodal boundary pressures p01, p02.

Workloads:
  * mms_problem: the paper's homogeneous MMS problems (Sections 5.1, 5.2):
    k1 = 1, k2 = 0.1, mu = beta = 1, gamma*b = 0, exact-solution pressure data
    on the whole boundary.
  * heterogeneous_problem: the same boundary data (computed with the fixed
    constants k1 = 1, k2 = 0.1, beta = 1) with seeded log-normal per-cell
    permeabilities and a chosen beta.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace

import numpy as np

from .fields import constant_logk, lognormal_logk
from .meshes import Mesh, disc_wheel, unit_mesh
from .mms import PAPER, MMSParams, boundary_pressures


@dataclass
class Problem:
    mesh: Mesh
    logk1: np.ndarray
    logk2: np.ndarray
    mu: float
    beta: float
    gamma_b: np.ndarray
    p01: np.ndarray
    p02: np.ndarray
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def dim(self) -> int:
        return self.mesh.dim

    @property
    def n_dofs(self) -> int:
        return self.mesh.n_dofs

    def with_(self, **kw) -> "Problem":
        return replace(self, **kw)


def mms_problem(dim: int, n: int, prm: MMSParams = PAPER, kind: str = "simplex") -> Problem:
    mesh = unit_mesh(dim, n, kind)
    lk1, lk2 = constant_logk(mesh.n_cells, prm.k1, prm.k2)
    p01, p02 = boundary_pressures(mesh.coords, prm)
    return Problem(mesh, lk1, lk2, prm.mu, prm.beta, np.zeros(dim), p01, p02,
                   name=f"mms{dim}d_n{n}" + ("_q1" if kind == "q1" else ""))


def heterogeneous_problem(dim: int, n: int, seed: int = 0, beta: float = 1.0,
                          mu: float = 1.0, kind: str = "simplex") -> Problem:
    mesh = unit_mesh(dim, n, kind)
    lk1, lk2 = lognormal_logk(mesh.n_cells, seed)
    p01, p02 = boundary_pressures(mesh.coords, PAPER)
    return Problem(mesh, lk1, lk2, mu, beta, np.zeros(dim), p01, p02,
                   name=f"het{dim}d_n{n}_s{seed}" + ("_q1" if kind == "q1" else ""),
                   meta={"seed": seed})


def wheel_problem(sectors: int = 70, rings: int = 4, seed: int = 0, beta: float = 1.0,
                  mu: float = 1.0) -> Problem:
    """Log-normal fields on the disc wheel mesh, with the paper's boundary
    pressures evaluated at the rim nodes."""
    mesh = disc_wheel(sectors, rings)
    lk1, lk2 = lognormal_logk(mesh.n_cells, seed)
    p01, p02 = boundary_pressures(mesh.coords, PAPER)
    return Problem(mesh, lk1, lk2, mu, beta, np.zeros(2), p01, p02,
                   name=f"wheel_s{sectors}_r{rings}_s{seed}", meta={"seed": seed})
