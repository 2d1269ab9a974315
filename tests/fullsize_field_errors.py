"""Per-field error of the benchmark solutions against the FP64 oracle (3D 64^3).

The benchmark workload (3D 64^3 Kuhn mesh, 2,197,000 DoF, log-normal k) is far
too large for a sparse LU. The oracle's reference solution there is its
flexible GMRES with the exact-structure field-split preconditioner, driven to
a true residual of 1e-13 (oracle/iterative.py, pinned to the direct solve in
tests/test_oracle.py). It takes tens of minutes on one CPU core, so the work
is split into two steps that can run on different hosts:

  python tests/fullsize_field_errors.py solve DIR     # needs a GPU
      FP64 and mixed-precision solves at rtol 1e-10 through the C ABI, exactly
      as bench.py runs them; writes DIR/x_fp64.npy, DIR/x_mixed.npy, DIR/info.json
  python tests/fullsize_field_errors.py compare DIR   # CPU only
      assembles the same seeded problem, solves it with the oracle, and prints
      one JSON line with each field's relative L2 error (nodal values, every
      velocity component) and the oracle's own true residual. The oracle's
      solution is saved in DIR and reused by later comparisons.

No value in the comparison comes from the GPU except the solutions under test.
"""
from __future__ import annotations

import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import inputs  # noqa: E402

WORKLOAD = dict(dim=3, n=64, seed=0, beta=1.0)


def problem():
    return inputs.heterogeneous_problem(WORKLOAD["dim"], WORKLOAD["n"], seed=WORKLOAD["seed"],
                                        beta=WORKLOAD["beta"])


def solve(out_dir: str) -> None:
    import torch

    import __graft_entry__ as g
    g.build()
    from paper_1808_08328_gb300.system import DPPSystem
    os.makedirs(out_dir, exist_ok=True)
    P = problem()
    info_all = {}
    for name, prec in (("fp64", 0), ("mixed", 1)):
        s = DPPSystem.from_problem(P, precision=prec).setup_pc(precision=prec)
        x, info = s.solve(rtol=1e-10)
        torch.cuda.synchronize()
        np.save(os.path.join(out_dir, f"x_{name}.npy"), x.cpu().numpy())
        info_all[name] = info
        s.close()
    with open(os.path.join(out_dir, "info.json"), "w") as fh:
        json.dump({"workload": WORKLOAD, "solve": info_all}, fh)
    print(json.dumps(info_all))


def compare(out_dir: str) -> None:
    import oracle
    from oracle.assembly import assemble_problem
    P = problem()
    t0 = time.time()
    K, f = assemble_problem(P)
    t1 = time.time()
    # the oracle's solution is kept in DIR (x_oracle.npy, oracle.json) and reused
    ref_x, ref_meta = os.path.join(out_dir, "x_oracle.npy"), os.path.join(out_dir, "oracle.json")
    if os.path.exists(ref_x) and os.path.exists(ref_meta):
        x = np.load(ref_x)
        with open(ref_meta) as fh:
            meta = json.load(fh)
        it, solve_s = meta["iterations"], meta["solve_s"]
    else:
        x, it, _ = oracle.solve_field_split_gmres(K, f, P.mesh.n_nodes, P.dim)
        solve_s = time.time() - t1
        np.save(ref_x, x)
        with open(ref_meta, "w") as fh:
            json.dump({"iterations": it, "solve_s": solve_s}, fh)
    res = oracle.residual(K, x, f)
    x_ref = oracle.to_nodal(x, P.mesh.n_nodes)
    with open(os.path.join(out_dir, "info.json")) as fh:
        info = json.load(fh)
    line = {"workload": WORKLOAD, "dofs": P.n_dofs, "oracle": {
        "method": "flexible GMRES, field-split Schur preconditioner (incomplete-LU pieces)",
        "iterations": it, "true_rel_residual": res, "assemble_s": t1 - t0, "solve_s": solve_s}}
    for name in ("fp64", "mixed"):
        xg = np.load(os.path.join(out_dir, f"x_{name}.npy"))
        line[name] = {"field_rel_l2": oracle.field_rel_errors(xg, x_ref),
                      "rel_residual_recomputed": oracle.residual(K, oracle.from_nodal(xg), f),
                      "gpu_iterations": info["solve"][name]["iterations"],
                      "gpu_rel_residual": info["solve"][name]["rel_residual"]}
    print(json.dumps(line))


if __name__ == "__main__":
    if len(sys.argv) != 3 or sys.argv[1] not in ("solve", "compare"):
        sys.exit(__doc__)
    (solve if sys.argv[1] == "solve" else compare)(sys.argv[2])
