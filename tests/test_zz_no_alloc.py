"""The allocation-free adjoint-sensitivity entry point against dpp_adjoint_solve.

dpp_adjoint_gradients_noalloc exists for callers that must not allocate device
memory, such as custom calls inside a JAX/XLA graph or processes whose
memory another framework's pool owns. It reuses one fixed library array as
scratch. This test calls it through the C ABI twice in a row, on the forward
solution and adjoint of one problem. Both calls must reproduce the per-cell
gradients and dJ/dbeta that dpp_adjoint_solve wrote. They agree to 1e-12
relative: only the summation order of the beta term differs. The file is
named so that pytest collects it last.
"""
import numpy as np
import pytest

import inputs
import oracle

from gpu_helpers import needs_gpu, system_cls, torch

pytestmark = [pytest.mark.gpu, needs_gpu]


@pytest.mark.parametrize("dim,n,gb", [(2, 12, None), (3, 6, None), (3, 5, [0.3, -1.0, 0.8])])
def test_noalloc_gradients_match_adjoint_solve(dim, n, gb):
    from paper_1808_08328_gb300 import binding as B
    DPPSystem = system_cls()
    P = inputs.heterogeneous_problem(dim, n, seed=4, beta=1.7)
    if gb is not None:  # a body force: the load's log-k derivative enters too
        P = P.with_(gamma_b=np.asarray(gb, dtype=np.float64))
    s = DPPSystem.from_problem(P).setup_pc()
    x, info = s.solve(rtol=1e-12)
    assert info["status"] == 0
    p1_obs = np.zeros(P.mesh.n_nodes)
    gx = torch.tensor(oracle.objective_grad_x(x.cpu().numpy(), p1_obs), device="cuda")
    lam, g1, g2, gb, ainfo = s.adjoint(x, gx, rtol=1e-12)
    assert ainfo["status"] == 0
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):
        h1 = torch.full_like(g1, float("nan"))
        h2 = torch.full_like(g2, float("nan"))
        hb = torch.full_like(gb, float("nan"))
        B.dpp_adjoint_gradients_noalloc(s.prob, x, lam, h1, h2, hb, stream)
        torch.cuda.synchronize()
        sc = max(g1.abs().max().item(), g2.abs().max().item())
        assert torch.allclose(h1, g1, rtol=0, atol=1e-12 * sc)
        assert torch.allclose(h2, g2, rtol=0, atol=1e-12 * sc)
        assert abs(hb.item() - gb.item()) <= 1e-12 * abs(gb.item())
    s.close()


def test_noalloc_rejects_null_arguments():
    from paper_1808_08328_gb300 import binding as B
    DPPSystem = system_cls()
    s = DPPSystem.from_problem(inputs.mms_problem(2, 4))
    z = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(B.DppError) as e:
        B.dpp_adjoint_gradients_noalloc(s.prob, None, z, z, z, z)
    assert e.value.status == B.DPP_ERR_INVALID_ARGUMENT
    s.close()
