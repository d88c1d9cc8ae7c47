"""Profiling harness: setup plus a few V-cycles of a benchmark workload inside a
cudaProfilerStart/Stop region, for `ncu --profile-from-start off`.

    python -m paper_2107_00820_gb300.profile_run --workload sinker3d_32 --vcycles 1 --prec fp32
    python -m paper_2107_00820_gb300.profile_run --workload batch64 --vcycles 1 --batch-mode merged
    python -m paper_2107_00820_gb300.profile_run --workload sinker3d_q3_24 --n 12 --levels 3 --setup

Only the region (the V-cycles, optionally one setup) is profiled; problem
generation and the context's own setup run before it.  batch64: the 64 uneven
instances of the batched sweep, their FP32 cycles as one batched call (merged
launches or the graph of the instances' own cycles).
"""
from __future__ import annotations

import argparse
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    import torch

    import bench
    from paper_2107_00820_gb300 import Context, alstokes as A

    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="sinker3d_32", choices=sorted(bench.WORKLOADS) + ["batch64"])
    ap.add_argument("--batch-mode", default="merged", choices=["merged", "branches"])
    ap.add_argument("--vcycles", type=int, default=1)
    ap.add_argument("--prec", default="fp32", choices=["fp32", "fp64", "both"])
    ap.add_argument("--setup", action="store_true", help="profile one coefficient setup instead")
    ap.add_argument("--n", type=int, default=None, help="cells per direction (default: the workload's)")
    ap.add_argument("--levels", type=int, default=None, help="levels (default: the workload's)")
    args = ap.parse_args()
    if args.workload == "batch64":
        batch_region(args)
        return
    spec = bench.WORKLOADS[args.workload]
    pb = bench.make_problem(spec, args.n, args.levels)
    mu = [torch.as_tensor(m, device="cuda") for m in pb.mu]
    tensor = spec.get("kind") == "tensor"
    mue = [torch.as_tensor(m, device="cuda") for m in pb.meta["mu_eff"]] if tensor else None
    ctx = Context(pb.d, pb.n, pb.levels, mu, pb.gamma, mu_eff=mue, mode=A.ALS_MODE_MIXED, sweeps=spec["sweeps"],
                  schur=A.ALS_SCHUR_P2 if spec.get("schur") == "P2" else A.ALS_SCHUR_P1, order=spec.get("order", 2))
    nu = ctx.nu()
    vecs = {}
    if args.prec in ("fp32", "both"):
        vecs[A.ALS_PREC_FP32] = torch.randn(nu, dtype=torch.float32, device="cuda")
    if args.prec in ("fp64", "both"):
        vecs[A.ALS_PREC_FP64] = torch.randn(nu, dtype=torch.float64, device="cuda")
    outs = {p: torch.zeros_like(b) for p, b in vecs.items()}
    for p, b in vecs.items():           # capture the V-cycle graphs before the region
        ctx.vcycle(b, outs[p], p)
    torch.cuda.synchronize()
    torch.cuda.cudart().cudaProfilerStart()
    if args.setup:
        ctx.update_coefficients(mu, mue)
    else:
        for _ in range(args.vcycles):
            for p, b in vecs.items():
                ctx.vcycle(b, outs[p], p)
    torch.cuda.synchronize()
    torch.cuda.cudart().cudaProfilerStop()
    ctx.close()
    print("profile region done")


def batch_region(args):
    import torch

    from paper_2107_00820_gb300 import Batch, alstokes as A
    from synthetic.problems import batch_instances

    pbs = batch_instances(32, 32, seed=0)
    opts = {"mode": A.ALS_MODE_MIXED, "schur": A.ALS_SCHUR_P2, "sweeps": 5}
    inst = [{"dim": pb.d, "n": pb.n, "levels": pb.levels, "coeffs": [torch.as_tensor(m, device="cuda") for m in pb.mu],
             "gamma": pb.gamma, "options": opts} for pb in pbs]
    batch = Batch(inst)
    batch.set_mode(A.ALS_BATCH_MERGED if args.batch_mode == "merged" else A.ALS_BATCH_BRANCHES)
    b = [torch.randn(s[0], dtype=torch.float32, device="cuda") for s in batch.shapes]
    x = [torch.zeros_like(t) for t in b]
    batch.vcycle(b, x, A.ALS_PREC_FP32)   # tuning and capture before the region
    torch.cuda.synchronize()
    torch.cuda.cudart().cudaProfilerStart()
    for _ in range(args.vcycles):
        batch.vcycle(b, x, A.ALS_PREC_FP32)
    torch.cuda.synchronize()
    torch.cuda.cudart().cudaProfilerStop()
    batch.close()
    print("profile region done")


if __name__ == "__main__":
    main()
