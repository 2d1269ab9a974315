"""Time one operator of the solver on a seeded workload (for profiling).

Usage:
  python -m paper_1808_08328_gb300.kernel_probe --op apply_K32_mf --dim 3 --n 64 --reps 20

Operators: apply_K, apply_K32, apply_K_mf, apply_K32_mf, pc_apply, pc_apply_mass.
The workload is the log-normal recipe of the benchmark (3D Kuhn tetrahedra or
2D triangles, N cells per edge, seed 0). The operator runs `--warmup` times,
then `--reps` times between CUDA events on the library's stream; the mean time
per call and the algorithmic bytes per call (from the library's own profiling
records) are printed as one JSON line. Under a profiler, give `--reps` a small
value and filter the kernel by name.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

FAMILY = {"apply_K": "apply_K", "apply_K32": "apply_K_fp32", "apply_K_mf": "apply_K_mf",
          "apply_K32_mf": "apply_K_mf_fp32", "pc_apply": None, "pc_apply_mass": None}


def main(argv=None) -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--op", default="apply_K32_mf", choices=sorted(FAMILY))
    ap.add_argument("--dim", type=int, default=3)
    ap.add_argument("--n", type=int, default=64)
    ap.add_argument("--reps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--mass-solver", type=int, default=0)
    args = ap.parse_args(argv)

    import torch

    import inputs
    from paper_1808_08328_gb300 import binding as B
    from paper_1808_08328_gb300.system import DPPSystem

    P = inputs.heterogeneous_problem(args.dim, args.n, seed=0, beta=1.0)
    fp32 = args.op in ("apply_K32", "apply_K32_mf")
    s = DPPSystem.from_problem(P, precision=1 if fp32 else 0)
    if args.op.startswith("pc_"):
        s.setup_pc(mass_solver=args.mass_solver)
    x = torch.randn((P.mesh.n_nodes, 2 * P.dim + 2), dtype=torch.float64, device="cuda")
    op = getattr(s, args.op)
    for _ in range(args.warmup):
        op(x)
    fam = FAMILY[args.op]
    if fam:
        B.dpp_profile_select([fam])
        B.dpp_profile_enable(True)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.reps):
        op(x)
    e1.record(stream)
    torch.cuda.synchronize()
    line = {"op": args.op, "dim": args.dim, "n": args.n, "dofs": P.n_dofs, "reps": args.reps,
            "ms_per_call_wall": e0.elapsed_time(e1) / args.reps}
    if fam:
        rec = B.dpp_profile_read(fam)
        B.dpp_profile_enable(False)
        B.dpp_profile_select(None)
        if rec["launches"]:
            kms = rec["ms"] / rec["launches"]
            line.update(kernel_ms=kms, alg_bytes=rec["alg_bytes"] / rec["launches"],
                        gbs=rec["alg_bytes"] / rec["launches"] / (kms * 1e-3) / 1e9)
    print(json.dumps(line))
    s.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
