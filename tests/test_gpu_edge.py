"""Edge cases of the method and of its inputs, on the GPU.

  * the smallest meshes (one square or cube: 2 triangles, 6 Kuhn tetrahedra,
    1 quadrilateral, 1 hexahedron), where the AMG hierarchy is a single level
    solved directly: FP64 and mixed solves against the oracle's direct solve;
  * beta = 0, where the two networks decouple (the coupling block vanishes),
    and mu != 1: against the oracle;
  * zero data (p01 = p02 = 0, gamma_b = 0): the solution is exactly zero,
    reached before the first iteration;
  * a zero-volume cell: rejected with DPP_ERR_INVALID_ARGUMENT before any
    solve, in the single and in the batched entry point;
  * a batch with no valid instance: DPP_ERR_INVALID_ARGUMENT, and every
    instance's info carries its own status.
"""
import numpy as np
import pytest

import inputs
import oracle
from oracle.assembly import assemble_problem

from gpu_helpers import needs_gpu, system_cls, torch

pytestmark = [pytest.mark.gpu, needs_gpu]


def _ref(P):
    K, f = assemble_problem(P)
    return K, f, oracle.to_nodal(oracle.solve_direct(K, f), P.mesh.n_nodes)


def _check(P, x, info, K, f, x_ref):
    assert info["status"] == 0 and info["rel_residual"] <= 1e-10, info
    xg = x.cpu().numpy()
    assert oracle.residual(K, oracle.from_nodal(xg), f) <= 1.5e-10
    err = oracle.field_rel_errors(xg, x_ref)
    assert max(err.values()) <= 1e-8, err


SMALLEST = {
    "tri_n1": lambda: inputs.heterogeneous_problem(2, 1, seed=1, beta=1.0),
    "kuhn_n1": lambda: inputs.heterogeneous_problem(3, 1, seed=1, beta=1.0),
    "quad_n1": lambda: inputs.heterogeneous_problem(2, 1, seed=1, beta=1.0, kind="q1"),
    "hex_n1": lambda: inputs.heterogeneous_problem(3, 1, seed=1, beta=1.0, kind="q1"),
}


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
@pytest.mark.parametrize("name", sorted(SMALLEST))
def test_smallest_meshes_match_oracle(name, precision):
    P = SMALLEST[name]()
    K, f, x_ref = _ref(P)
    s = system_cls().from_problem(P, precision=precision).setup_pc(precision=precision)
    x, info = s.solve(rtol=1e-10)
    assert info["levels"] == 1
    _check(P, x, info, K, f, x_ref)
    s.close()


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
@pytest.mark.parametrize("dim,n,beta,mu", [(2, 20, 0.0, 1.0), (3, 6, 0.0, 1.0), (3, 6, 2.0, 2.5)],
                         ids=["2d_beta0", "3d_beta0", "3d_mu2.5"])
def test_decoupled_networks_and_viscosity(dim, n, beta, mu, precision):
    P = inputs.heterogeneous_problem(dim, n, seed=7, beta=beta, mu=mu)
    K, f, x_ref = _ref(P)
    s = system_cls().from_problem(P, precision=precision).setup_pc(precision=precision)
    x, info = s.solve(rtol=1e-10)
    _check(P, x, info, K, f, x_ref)
    s.close()
    if beta == 0.0 and precision == 0:
        # with beta = 0 network 1 does not see network 2's data
        lk2 = P.logk2 + 1.0
        P2 = P.with_(logk2=lk2, p02=2.0 * P.p02)
        s2 = system_cls().from_problem(P2).setup_pc()
        x2, info2 = s2.solve(rtol=1e-12)
        s2.close()
        d = P.mesh.dim
        a = x[:, : d + 1].cpu().numpy()
        b = x2[:, : d + 1].cpu().numpy()
        assert np.abs(a - b).max() <= 1e-8 * np.abs(a).max()


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_zero_data_gives_zero_solution(precision):
    P = inputs.heterogeneous_problem(3, 5, seed=2, beta=1.0)
    P = P.with_(p01=np.zeros_like(P.p01), p02=np.zeros_like(P.p02))
    s = system_cls().from_problem(P, precision=precision).setup_pc(precision=precision)
    x, info = s.solve(rtol=1e-10)
    assert info["status"] == 0 and info["iterations"] == 0 and info["rel_residual"] == 0.0
    assert torch.count_nonzero(x).item() == 0
    s.close()


def _collapsed(P):
    """The same mesh with node 4 moved onto node 0: the cells holding both have no area."""
    m = P.mesh
    X = m.coords.copy()
    X[4] = X[0]
    return P.with_(mesh=inputs.Mesh(m.dim, X, m.cells, m.bfacets, m.n))


def test_zero_volume_cell_is_rejected():
    from paper_1808_08328_gb300 import binding as B
    from paper_1808_08328_gb300.system import solve_batched
    P = inputs.heterogeneous_problem(2, 2, seed=3, beta=1.0)
    bad = _collapsed(P)
    with pytest.raises(B.DppError) as e:
        system_cls().from_problem(bad)
    assert e.value.status == B.DPP_ERR_INVALID_ARGUMENT
    # in a batch only that instance fails
    good = inputs.heterogeneous_problem(2, 6, seed=4, beta=1.0)
    xs, infos, st = solve_batched([good, bad, good], rtol=1e-10)
    assert st != 0
    assert infos[1]["status"] == B.DPP_ERR_INVALID_ARGUMENT
    assert infos[0]["status"] == 0 and infos[2]["status"] == 0


def test_batch_without_a_valid_instance():
    from paper_1808_08328_gb300 import binding as B
    from paper_1808_08328_gb300.system import DPPBatch
    system_cls()
    P = inputs.heterogeneous_problem(2, 4, seed=3, beta=1.0)
    bt = DPPBatch([P, P])
    bt.descs[0].mu = -1.0                        # invalid viscosity
    bt.descs[1].n_cells = 0                      # no cells
    po = B.dpp_pc_opts_default()
    so = B.dpp_solve_opts_default()
    st, infos = B.dpp_solve_batched(bt.descs, po, so, bt.xs, 0, allow=tuple(range(9)))
    assert st == B.DPP_ERR_INVALID_ARGUMENT
    assert [i["status"] for i in infos] == [B.DPP_ERR_INVALID_ARGUMENT] * 2
