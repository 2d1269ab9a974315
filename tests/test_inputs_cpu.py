"""The seeded input recipe that both the oracle and the CUDA path consume.

These pin the distributions the workloads are stated with (log k1 ~ N(0, 1),
log k2 ~ N(-3, 1) i.i.d. per cell; batched 2D grids N ~ U{16..128} with beta
log-uniform in [0.1, 10]) and that a seed always gives the same arrays.
"""
import numpy as np
import pytest

import inputs
from inputs.fields import batch_recipe, lognormal_logk, sample_cells


def test_lognormal_fields_have_the_stated_moments_and_are_independent():
    n = 400_000
    k1, k2 = lognormal_logk(n, seed=11)
    tol = 5.0 / np.sqrt(n)  # five standard errors of the mean
    assert abs(k1.mean() - 0.0) < tol and abs(k2.mean() + 3.0) < tol
    assert abs(k1.std() - 1.0) < 0.01 and abs(k2.std() - 1.0) < 0.01
    assert abs(np.corrcoef(k1, k2)[0, 1]) < tol
    # normal tails: about 4.55% of draws beyond two standard deviations
    assert abs(np.mean(np.abs(k1) > 2.0) - 0.0455) < 0.002


def test_fields_are_reproducible_per_seed():
    a1, a2 = lognormal_logk(1000, seed=5)
    b1, b2 = lognormal_logk(1000, seed=5)
    c1, _ = lognormal_logk(1000, seed=6)
    assert np.array_equal(a1, b1) and np.array_equal(a2, b2)
    assert not np.array_equal(a1, c1)


def test_batch_recipe_sizes_and_betas():
    scipy_stats = pytest.importorskip("scipy.stats")
    rec = batch_recipe(20_000, seed=3)
    ns = np.array([r[0] for r in rec])
    betas = np.array([r[2] for r in rec])
    seeds = [r[1] for r in rec]
    assert ns.min() == 16 and ns.max() == 128 and len(np.unique(ns)) == 113
    assert abs(ns.mean() - 72.0) < 1.0
    lb = np.log10(betas)
    assert lb.min() >= -1.0 and lb.max() < 1.0
    assert scipy_stats.kstest(lb, "uniform", args=(-1.0, 2.0)).pvalue > 1e-3
    assert len(set(seeds)) == len(seeds)  # every instance draws its own field


def test_benchmark_batch_size():
    """The 256-instance batch (seed 0) that the batched benchmark solves."""
    rec = batch_recipe(256, seed=0)
    dofs = sum(6 * (n + 1) ** 2 for n, _, _ in rec)
    assert dofs == 10_462_734
    assert rec == batch_recipe(256, seed=0)


def test_benchmark_mesh_sizes():
    """The 3D 64^3 Kuhn mesh: 274,625 nodes, 1,572,864 tetrahedra, 2,197,000 DoF."""
    assert inputs.dof_count(3, 64) == 2_197_000
    m = inputs.unit_mesh(3, 8)
    assert m.coords.shape == (9 ** 3, 3) and m.cells.shape == (6 * 8 ** 3, 4)


def test_sampled_cells_are_distinct_and_sorted():
    c = sample_cells(1000, 20, seed=4)
    assert len(np.unique(c)) == 20 and np.all(np.diff(c) > 0)
    assert c.min() >= 0 and c.max() < 1000
