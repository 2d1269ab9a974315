"""Every public preconditioner and solver option away from its default, on the GPU.

Each option changes how the preconditioner or the Krylov method works, never
the solution: a solve with it must still reach the oracle's solution to 1e-8
relative L2 per field at a true relative residual of 1e-10. Covered:
  * use_lumped_diag = 1 (row-sum lumping in S_p and in the mass Chebyshev
    interval [1/(d+2), 1]);
  * cheb_degree_amg 1 and 3 (both parities of the smoother's start buffer),
    cheb_degree_mass 1 and 3, cheb_ratio 20;
  * strength_theta 0 and 0.08, max_levels 2, coarse_max_rows 64;
  * max_levels 1: the coarsest level is S_p itself, blocks of 343 and 625
    rows, inverted by the cooperative Gauss-Jordan (one grid barrier per pivot);
  * smooth_filter = 1 (prolongator smoothed with the filtered matrix A^F);
  * cheb_degree_coarse 1 and 3 (a separate smoother degree below the finest level);
  * inner_rtol 1e-2 and 1e-6 of the mixed mode; restart 5;
  * x0_zero = 0: from a perturbed oracle solution, and from the oracle
    solution itself (converged before the first iteration).
"""
import numpy as np
import pytest

import inputs
import oracle
from oracle.assembly import assemble_problem

from gpu_helpers import needs_gpu, system_cls, torch

pytestmark = [pytest.mark.gpu, needs_gpu]

PROBS = {"het2d_n24": lambda: inputs.heterogeneous_problem(2, 24, seed=3, beta=1.5),
         "het3d_n6": lambda: inputs.heterogeneous_problem(3, 6, seed=4, beta=0.7)}


@pytest.fixture(scope="module")
def refs():
    out = {}
    for name, make in PROBS.items():
        P = make()
        K, f = assemble_problem(P)
        x = oracle.to_nodal(oracle.solve_direct(K, f, coords=P.mesh.coords), P.mesh.n_nodes)
        out[name] = (P, K, f, x)
    return out


def _check(ref, x, info):
    P, K, f, x_ref = ref
    assert info["status"] == 0 and info["rel_residual"] <= 1e-10
    xg = x.cpu().numpy()
    assert oracle.residual(K, oracle.from_nodal(xg), f) <= 1.5e-10
    err = oracle.field_rel_errors(xg, x_ref)
    assert max(err.values()) <= 1e-8, err


PC_OPTS = [dict(use_lumped_diag=1), dict(cheb_degree_amg=1), dict(cheb_degree_amg=3),
           dict(cheb_degree_mass=1), dict(cheb_degree_mass=3), dict(cheb_ratio=20.0),
           dict(strength_theta=0.0), dict(strength_theta=0.08), dict(max_levels=2),
           dict(max_levels=1), dict(coarse_max_rows=64), dict(smooth_filter=1),
           dict(cheb_degree_coarse=1), dict(cheb_degree_coarse=3)]


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
@pytest.mark.parametrize("opts", PC_OPTS, ids=[",".join(f"{k}={v}" for k, v in o.items())
                                               for o in PC_OPTS])
@pytest.mark.parametrize("name", sorted(PROBS))
def test_pc_option_keeps_the_solution(refs, name, opts, precision):
    ref = refs[name]
    s = system_cls().from_problem(ref[0], precision=precision).setup_pc(precision=precision, **opts)
    x, info = s.solve(rtol=1e-10)
    _check(ref, x, info)
    s.close()


@pytest.mark.parametrize("solve_opts", [dict(inner_rtol=1e-2), dict(inner_rtol=1e-6),
                                        dict(restart=5)],
                         ids=["inner_rtol=1e-2", "inner_rtol=1e-6", "restart=5"])
@pytest.mark.parametrize("name", sorted(PROBS))
def test_solve_option_keeps_the_solution(refs, name, solve_opts):
    ref = refs[name]
    s = system_cls().from_problem(ref[0], precision=1).setup_pc(precision=1)
    x, info = s.solve(rtol=1e-10, **solve_opts)
    _check(ref, x, info)
    if "restart" in solve_opts:
        assert info["restarts"] >= 2
    s.close()


@pytest.mark.parametrize("name", sorted(PROBS))
def test_initial_guess_is_used(refs, name):
    P, K, f, x_ref = refs[name]
    s = system_cls().from_problem(P).setup_pc()
    x0 = x_ref * (1.0 + 1e-3 * inputs.rng(9).standard_normal(x_ref.shape))
    x, info = s.solve(x0=torch.tensor(x0, device="cuda"), rtol=1e-10)
    _check(refs[name], x, info)
    _, cold = s.solve(rtol=1e-10)
    assert info["iterations"] < cold["iterations"]
    # from the solution itself: converged before the first iteration
    xs, info0 = s.solve(x0=torch.tensor(x_ref, device="cuda"), rtol=1e-8)
    assert info0["status"] == 0 and info0["iterations"] == 0
    assert np.array_equal(xs.cpu().numpy(), x_ref)
    s.close()


@pytest.mark.parametrize("name", sorted(PROBS))
def test_exact_pressure_solve_needs_no_more_iterations(refs, name):
    # max_levels = 1 replaces the V-cycle on blockdiag(S_p1, S_p2) by its exact
    # inverse (the coarsest-level Gauss-Jordan on blocks of 343 / 625 rows), so
    # the factorisation can only get closer to the selfp one: a wrong inverse
    # would show as more iterations than the multilevel default.
    ref = refs[name]
    P = ref[0]
    s = system_cls().from_problem(P).setup_pc(max_levels=1)
    x, info = s.solve(rtol=1e-10)
    _check(ref, x, info)
    assert info["levels"] == 1
    s.close()
    s = system_cls().from_problem(P).setup_pc()
    _, info_ml = s.solve(rtol=1e-10)
    s.close()
    assert info_ml["levels"] >= 2
    assert info["iterations"] <= info_ml["iterations"], (info, info_ml)
