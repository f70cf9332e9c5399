"""Short, profiler-friendly runs of the draw (for ncu and similar tools).

    python -m paper_1810_12437_gb300.profile_draw --workload single --iters 6
    python -m paper_1810_12437_gb300.profile_draw --workload batched --iters 4

`single` draws chain 0 of the batched workload alone (n=5e5, p=5e4), `batched`
draws all 16 chains; both stop after --iters CG iterations (tol 0) and run
with per-kernel timing on (plain launches, one kernel per launch), then print
the per-kernel averages.  --full instead runs every chain to the stop rule
(tol 1e-6), as a whole draw of the benchmark does.  --small uses a 20x smaller
design (n=25,000, p=2,500) of the same recipe; --rg fixes the batched path's
RHS group width (otherwise it is autotuned).

`uneven` runs one uneven-batch draw of 16 problems of the uneven recipe
(n ~ logU[5e3, 6e4], p ~ logU[1e3, 1e4]) to the stop rule (tol 1e-6) in the
persistent kernel, and prints the iteration total and the statuses.
"""
import os
import argparse
import json

import numpy as np
import torch

from . import _native as pb
from . import inputs


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", choices=["single", "batched", "uneven"], default="single")
    ap.add_argument("--iters", type=int, default=6)
    ap.add_argument("--precision", default="fp32_refined")
    ap.add_argument("--small", action="store_true")
    ap.add_argument("--full", action="store_true", help="run to the stop rule (tol 1e-6)")
    ap.add_argument("--rg", type=int, default=0, help="batched RHS group width (1, 2, 4, 8; 0: autotune)")
    args = ap.parse_args(argv)
    if args.rg:
        os.environ["PCG_BETA_BATCH_RG"] = str(args.rg)
    dev = torch.device("cuda:0")
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(dev)
    kw = dict(n=25_000, p=2_500) if args.small else {}
    tol, max_iter = (1e-6, 20_000) if args.full else (0.0, args.iters)
    if args.workload == "uneven":
        probs = inputs.config4(nprob=16, n_range=(5_000, 60_000), p_range=(1_000, 10_000))
        dp = [dict(X=pb.DeviceDesign.from_host(P.X, dev), omega=T(P.omega), z=T(P.z), lam=T(P.lam),
                   tau=float(P.tau), eta=T(P.eta), delta=T(P.delta)) for P in probs]
        ctx = pb.Context(precision=args.precision)
        res = pb.pcg_draw_beta_uneven(ctx, dp, tol=1e-6, max_iter=20_000)
        torch.cuda.synchronize()
        print(json.dumps({"problems": len(dp), "nnz": int(sum(P.X.nnz for P in probs)),
                          "iters": int(sum(r.iters for r in res)), "status": [int(r.status) for r in res]}))
        return
    if args.workload == "single":
        P = inputs.config3(nrhs=1, **kw)
        X = pb.DeviceDesign.from_host(P.X, dev)
        ctx = pb.Context(precision=args.precision, profile=True, reliable_k=50 if args.full else 0)
        pb.pcg_draw_beta(ctx, X, T(P.omega[0]), T(P.z[0]), T(P.lam[0]), float(P.tau[0]), T(P.eta[0]),
                         T(P.delta[0]), tol=tol, max_iter=max_iter)
    else:
        P = inputs.config3(**kw)
        X = pb.DeviceDesign.from_host(P.X, dev)
        ctx = pb.Context(precision=args.precision, profile=True, reliable_k=50 if args.full else 0)
        pb.pcg_draw_beta_batched(ctx, X, T(P.omega), T(P.z), T(P.lam), T(P.tau), T(P.eta), T(P.delta),
                                 tol=tol, max_iter=max_iter)
    torch.cuda.synchronize()
    table = pb.profile_table(ctx)
    print(json.dumps({k: {"avg_us": round(v[0] / v[1] * 1e3, 2), "launches": v[1]} for k, v in table.items()}))


if __name__ == "__main__":
    main()
