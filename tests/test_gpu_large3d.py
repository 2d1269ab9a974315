"""Per-field parity on large 3D meshes, and the preconditioner's behaviour band.

  * 3D 32^3 Kuhn mesh (35,937 nodes, 287,496 DoF) with the benchmark's
    log-normal recipe: the GPU solution in FP64 and in mixed precision, at a
    true relative residual of 1e-10, against the oracle to 1e-8 relative L2
    per field. A sparse LU of this system is out of reach in test time (its
    cost grows roughly with the square of the size: 140 s at 24^3). So the
    reference is the oracle's flexible GMRES, driven to a true residual of
    1e-13. The oracle tests pin it to the direct solve on smaller meshes.
    The SELL-32 level-0 path and the mirrored Galerkin product are both on,
    as in the benchmark: level 0 has 71,874 rows.
  * The paper's KSP counts for CG-VMS TET with the field split (Section 5.2,
    Tables "Strong_CGVMS_hsize" and "Strong_CGVMS_DoF", golden file
    ksp_band.txt): 12-15 iterations at h = 1/16 and 13-16 at h = 1/28 on the
    homogeneous 3D MMS problem. The paper's tolerance is unstated (1e-5 in its
    listings, 1e-7 in its text), and its inner solvers differ from ours
    (BoomerAMG and ILU there, SA-AMG and Chebyshev here). So the check is a
    loose band, half to twice the paper's range, at both tolerances. It
    tests behaviour only: it does not enter parity.
"""
import os

import numpy as np
import pytest

import inputs
import oracle
from oracle.assembly import assemble_problem

from gpu_helpers import needs_gpu, system_cls

pytestmark = [pytest.mark.gpu, needs_gpu]

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def cube32():
    P = inputs.heterogeneous_problem(3, 32, seed=0, beta=1.0)
    K, f = assemble_problem(P)
    x, it, res = oracle.solve_field_split_gmres(K, f, P.mesh.n_nodes, 3)
    assert res <= 1e-13
    return P, K, f, oracle.to_nodal(x, P.mesh.n_nodes)


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_cube32_solution_matches_oracle_per_field(cube32, precision):
    P, K, f, x_ref = cube32
    s = system_cls().from_problem(P, precision=precision).setup_pc(precision=precision)
    assert s.level(0, with_p=False)[0]["rows"] >= 65536   # SELL-32 level 0, as in the bench
    x, info = s.solve(rtol=1e-10)
    assert info["status"] == 0 and info["rel_residual"] <= 1e-10
    xg = x.cpu().numpy()
    assert oracle.residual(K, oracle.from_nodal(xg), f) <= 1.5e-10
    err = oracle.field_rel_errors(xg, x_ref)
    assert max(err.values()) <= 1e-8, err
    s.close()


def _band():
    out = {}
    with open(os.path.join(GOLDEN, "ksp_band.txt")) as fh:
        for line in fh:
            line = line.split("#")[0].strip()
            if line:
                n, lo, hi = (int(v) for v in line.split())
                out[n] = (lo, hi)
    return out


@pytest.mark.parametrize("n", [16, 28])
def test_ksp_iterations_fall_in_the_papers_band(n):
    lo, hi = _band()[n]
    P = inputs.mms_problem(3, n)
    s = system_cls().from_problem(P).setup_pc()
    its = {}
    for rtol in (1e-5, 1e-7):
        x, info = s.solve(rtol=rtol)
        assert info["status"] == 0
        its[rtol] = info["iterations"]
        assert 0.5 * lo <= info["iterations"] <= 2 * hi, (n, rtol, info["iterations"], (lo, hi))
    assert its[1e-5] <= its[1e-7]
    s.close()
