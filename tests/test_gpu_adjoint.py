"""Adjoint gradients through torch.autograd on the 3D 32^3 workload (287,496 DoF).

J = sum over nodes (p1 - p1_obs)^2, where p1_obs is the FP64 GPU solution for
log-k fields drawn from the next seed (a seeded reference field). The
gradient with respect to the per-cell log k1, log k2 and beta comes from
DPPSolve.backward, that is the transpose solve plus the cell sensitivity
kernel. It is checked against central differences with h = 1e-6 on 20
random cells (seed 2), and on beta. Each difference takes two forward solves
of the perturbed system. The bar is 1e-6 relative to the largest sampled
finite difference. Each perturbed forward solution is formed as
x_base + d, where d solves K_pert d = f_pert - K_pert x_base (dpp_solve_rhs) to 1e-10
relative to that small right-hand side. The base solution's error, and the
rounding in the rows the perturbation does not touch, are then common to both
sides of a difference and cancel. A plain re-solve of K_pert x = f_pert cannot
resolve a one-cell change of size h: its residual floor (about 3e-15 ||f||) is
about 1e-6 of that change. J(+h) - J(-h) is formed as sum (p1+ - p1-)(p1+ + p1- - 2 p1_obs),
an exact identity. It avoids the cancellation between two large sums of squares,
whose rounding floor (eps |J| / h, about 1e-5 of the largest gradient here) would
otherwise exceed the bar.
"""
import numpy as np
import pytest

import inputs

from gpu_helpers import needs_gpu, system_cls, torch

pytestmark = [pytest.mark.gpu, needs_gpu]

H = 1e-6
RTOL = 1e-13


def test_adjoint_autograd_matches_central_differences():
    DPPSystem = system_cls()
    from paper_1808_08328_gb300.system import DPPSolve
    P = inputs.heterogeneous_problem(3, 32, seed=0, beta=1.0)
    Pobs = inputs.heterogeneous_problem(3, 32, seed=1, beta=1.0)
    so = DPPSystem.from_problem(Pobs).setup_pc()
    xo, _ = so.solve(rtol=RTOL)
    p1_obs = xo[:, 3].clone()
    so.close()
    m = P.mesh
    mesh = dict(coords=m.coords, cells=m.cells, bfacets=m.bfacets, mu=P.mu, gamma_b=P.gamma_b,
                p01=P.p01, p02=P.p02)
    dev = torch.device("cuda")
    lk1 = torch.tensor(P.logk1, device=dev, requires_grad=True)
    lk2 = torch.tensor(P.logk2, device=dev, requires_grad=True)
    beta = torch.tensor([P.beta], device=dev, dtype=torch.float64, requires_grad=True)
    opts = {"solve": {"rtol": RTOL, "max_iters": 2000}}
    x = DPPSolve.apply(lk1, lk2, beta, mesh, opts)
    J = ((x[:, 3] - p1_obs) ** 2).sum()
    J.backward()

    x_base = x.detach().clone()

    def dp1_of(l1, l2, b):
        """p1 correction d of the perturbed system relative to x_base."""
        s = DPPSystem(m.coords, m.cells, m.bfacets, l1, l2, P.mu, b, P.gamma_b, P.p01, P.p02)
        s.setup_pc()
        r = s.rhs() - s.apply_K(x_base)
        d, info = s.solve_rhs(r, rtol=1e-10, max_iters=2000)
        assert info["status"] == 0
        s.close()
        return d[:, 3].clone()

    p1_base = x_base[:, 3]

    def central(dp, dm):
        # J(+) - J(-) = sum (p1+ - p1-)(p1+ + p1- - 2 p1_obs) with p1+- = p1_base + d+-
        return float(((dp - dm) * (2.0 * (p1_base - p1_obs) + dp + dm)).sum()) / (2 * H)

    cells = inputs.sample_cells(m.n_cells, 20, seed=2)
    base1, base2 = P.logk1.copy(), P.logk2.copy()
    fd, ad = [], []
    for c in cells:
        for which, base, grad in ((1, base1, lk1.grad), (2, base2, lk2.grad)):
            lp, lm = base.copy(), base.copy()
            lp[c] += H
            lm[c] -= H
            if which == 1:
                fd.append(central(dp1_of(lp, base2, P.beta), dp1_of(lm, base2, P.beta)))
            else:
                fd.append(central(dp1_of(base1, lp, P.beta), dp1_of(base1, lm, P.beta)))
            ad.append(float(grad[c]))
    fd_b = central(dp1_of(base1, base2, P.beta + H), dp1_of(base1, base2, P.beta - H))
    fd, ad = np.array(fd), np.array(ad)
    scale = np.abs(fd).max()
    assert scale > 0
    assert np.abs(ad - fd).max() <= 1e-6 * scale, (np.abs(ad - fd).max() / scale)
    assert abs(float(beta.grad[0]) - fd_b) <= 1e-6 * abs(fd_b)
