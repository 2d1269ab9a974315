"""Seeded per-cell permeability fields and batch recipes.

Random numbers come from numpy's PCG64 with a fixed seed; both the oracle and
the GPU path receive the drawn arrays as inputs. Nothing here performs the
method's arithmetic.

The 3D heterogeneous workloads use log k1 ~ N(0, 1) and log k2 ~ N(-3, 1),
i.i.d. per cell. The batched 2D workload uses per-instance grid sizes
N ~ U{16..128}, the same log-normal fields, and beta log-uniform in
[0.1, 10].
"""
from __future__ import annotations

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def lognormal_logk(n_cells: int, seed: int, mean1: float = 0.0, mean2: float = -3.0,
                   sigma: float = 1.0) -> tuple[np.ndarray, np.ndarray]:
    """Two i.i.d. normal log-permeability fields (natural log) of length n_cells."""
    g = rng(seed)
    logk1 = g.normal(mean1, sigma, n_cells).astype(np.float64)
    logk2 = g.normal(mean2, sigma, n_cells).astype(np.float64)
    return logk1, logk2


def constant_logk(n_cells: int, k1: float = 1.0, k2: float = 0.1) -> tuple[np.ndarray, np.ndarray]:
    """Homogeneous fields: the paper's k1 = 1, k2 = 0.1."""
    return (np.full(n_cells, np.log(k1), dtype=np.float64),
            np.full(n_cells, np.log(k2), dtype=np.float64))


def batch_recipe(n_inst: int, seed: int, nmin: int = 16, nmax: int = 128):
    """Per-instance (N_i, field seed, beta_i) for the batched 2D workload."""
    g = rng(seed)
    ns = g.integers(nmin, nmax + 1, size=n_inst)
    betas = 10.0 ** g.uniform(-1.0, 1.0, size=n_inst)
    seeds = [seed + 1 + i for i in range(n_inst)]
    return [(int(ns[i]), int(seeds[i]), float(betas[i])) for i in range(n_inst)]


def sample_cells(n_cells: int, count: int, seed: int) -> np.ndarray:
    """Cells drawn uniformly without replacement (finite-difference checks)."""
    return np.sort(rng(seed).choice(n_cells, size=count, replace=False)).astype(np.int64)
