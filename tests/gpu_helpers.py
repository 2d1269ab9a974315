"""Shared helpers for the GPU parity tests (test code only)."""
from __future__ import annotations

import numpy as np
import pytest
import scipy.sparse as sp

torch = pytest.importorskip("torch")

needs_gpu = pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")


def system_cls():
    import __graft_entry__ as g
    g.build()
    from paper_1808_08328_gb300.system import DPPSystem
    return DPPSystem


def pairs_to_slot_major(rp, col, vals, n_nodes, dim):
    """Scalar K (slot-major numbering, like the oracle) from exported pair values."""
    rp = np.asarray(rp, dtype=np.int64)
    col = np.asarray(col, dtype=np.int64)
    vals = np.asarray(vals)
    rows = np.repeat(np.arange(n_nodes), np.diff(rp))
    N = n_nodes
    d = dim
    R, Cc, V = [], [], []

    def put(rs, cs, v):
        R.append(rs * N + rows)
        Cc.append(cs * N + col)
        V.append(v)

    m1, m2 = vals[:, 0], vals[:, 1]
    bu = vals[:, 2:2 + d]
    cu = vals[:, 2 + d:2 + 2 * d]
    d1, d2, e = vals[:, 2 + 2 * d], vals[:, 3 + 2 * d], vals[:, 4 + 2 * d]
    for k in range(d):
        put(k, k, m1)
        put(d + 1 + k, d + 1 + k, m2)
        put(k, d, bu[:, k])
        put(d + 1 + k, 2 * d + 1, bu[:, k])
        put(d, k, cu[:, k])
        put(2 * d + 1, d + 1 + k, cu[:, k])
    put(d, d, d1)
    put(2 * d + 1, 2 * d + 1, d2)
    put(d, 2 * d + 1, e)
    put(2 * d + 1, d, e)
    ns = 2 * d + 2
    return sp.csr_matrix((np.concatenate(V), (np.concatenate(R), np.concatenate(Cc))),
                         shape=(ns * N, ns * N))


def csr_from_export(rp, col, val, shape):
    return sp.csr_matrix((val.cpu().numpy(), col.cpu().numpy(), rp.cpu().numpy()), shape=shape)
