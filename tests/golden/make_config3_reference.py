"""Writes tests/golden/config3_oracle.json: the CPU oracle's full draws for the
16 chains of the batched workload (n = 5e5, p = 5e4, log10 r ~ U(-4.5, -1.5),
tol 1e-6 on the paper's RMS rule).

Only ``oracle/`` computes here.  For each chain the file keeps the iteration
count, the final stop quantity, ||beta||_2 and beta at 64 seeded sampled
coordinates, plus a fingerprint of the generated design so that a test can
tell whether its inputs are the ones this file was made from.

Run:  python tests/golden/make_config3_reference.py [--procs 8]
(about 16 x 6 CPU-minutes of single-threaded oracle work).
"""
import argparse
import hashlib
import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

OUT = os.path.join(HERE, "config3_oracle.json")
NSAMPLE = 64


def design_fingerprint(X):
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(X.col_ptr).tobytes())
    h.update(np.ascontiguousarray(X.row_idx[:: max(1, X.nnz // 100_000)]).tobytes())
    return h.hexdigest()[:32]


def sample_indices(p):
    return np.sort(np.random.default_rng(12437).choice(p, size=NSAMPLE, replace=False))


def run_chain(r):
    from oracle import oracle as O
    from paper_1810_12437_gb300 import inputs
    P = inputs.config3()
    t0 = time.time()
    beta, k, res, st = O.draw_beta_cg(P.X, P.omega[r], P.z[r], P.lam[r], float(P.tau[r]), P.eta[r],
                                      P.delta[r], tol=1e-6, stop_rule=O.STOP_RMS, max_iter=20_000)
    idx = sample_indices(P.X.p)
    return dict(chain=r, iters=int(k), resid=float(res), status=int(st),
                beta_norm=float(np.linalg.norm(beta)), sample_idx=idx.tolist(),
                beta_sample=[float(x) for x in beta[idx]], seconds=time.time() - t0)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--procs", type=int, default=8)
    args = ap.parse_args()
    from paper_1810_12437_gb300 import inputs
    P = inputs.config3()
    meta = dict(workload="config3 n=500000 p=50000 R=16", n=P.X.n, p=P.X.p, nnz=P.X.nnz,
                design_fingerprint=design_fingerprint(P.X), tol=1e-6, stop_rule="paper_rms",
                tau=[float(t) for t in P.tau])
    del P
    ctx = mp.get_context("spawn")
    with ctx.Pool(args.procs) as pool:
        chains = pool.map(run_chain, range(16))
    meta["chains"] = sorted(chains, key=lambda c: c["chain"])
    with open(OUT, "w") as f:
        json.dump(meta, f, indent=1)
    print("wrote", OUT, [c["iters"] for c in meta["chains"]])


if __name__ == "__main__":
    main()
