"""Writes tests/golden/config3_oracle.json: the CPU oracle's full draws for the
16 chains of the batched workload (n = 5e5, p = 5e4, log10 r ~ U(-4.5, -1.5),
tol 1e-6 on the paper's RMS rule).

Only ``oracle/`` computes here.  For each chain the file keeps the iteration
count, the final stop quantity, ||beta||_2 and beta at 64 seeded sampled
coordinates, plus a fingerprint of the generated design so that a test can
tell whether its inputs are the ones this file was made from.  Three runs of
the oracle are kept:

* ``chains``: plain left-to-right sums (the oracle's default arithmetic);
* ``compensated``: the same draws with every sum of the products and dot
  products accumulated by compensated summation;
* ``compensated_ulp``: the compensated draws on omega and lambda perturbed by
  about one unit in the last place (``inputs.perturb_ulps``, seeds 9100 + 2r
  and 9101 + 2r for chain r), which measures how far the iteration count of
  these ill-conditioned systems moves under rounding alone;
* ``f32x2`` and ``f32x2_ulp``: the same two compensated runs with the
  products' operands and results held as float pairs (the oracle's
  ``vec="f32x2"`` storage, about 48 bits): the reference band of the
  double-float and fixed-point products.

Run:  python tests/golden/make_config3_reference.py [--procs 8] [--part all|plain|compensated|f32x2]
(plain: about 16 x 6 CPU-minutes; each compensated run about 16 x 10 CPU-minutes).
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


_P = None


def _problem():
    global _P
    if _P is None:
        from paper_1810_12437_gb300 import inputs
        _P = inputs.config3()
    return _P


def run_chain(job):
    r, kind = job
    from oracle import oracle as O
    from paper_1810_12437_gb300 import inputs
    P = _problem()
    omega, lam = P.omega[r], P.lam[r]
    sums = "plain" if kind == "plain" else "compensated"
    vec = "f32x2" if kind.startswith("f32x2") else "f64"
    if kind.endswith("_ulp"):
        omega = inputs.perturb_ulps(omega, 9100 + 2 * r)
        lam = inputs.perturb_ulps(lam, 9101 + 2 * r)
    t0 = time.time()
    beta, k, res, st = O.draw_beta_cg(P.X, omega, P.z[r], lam, float(P.tau[r]), P.eta[r],
                                      P.delta[r], tol=1e-6, stop_rule=O.STOP_RMS, max_iter=20_000,
                                      sums=sums, vec=vec)
    idx = sample_indices(P.X.p)
    return kind, dict(chain=r, iters=int(k), resid=float(res), status=int(st),
                      beta_norm=float(np.linalg.norm(beta)), sample_idx=idx.tolist(),
                      beta_sample=[float(x) for x in beta[idx]], seconds=time.time() - t0)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--procs", type=int, default=8)
    ap.add_argument("--part", choices=["all", "plain", "compensated", "f32x2"], default="all")
    args = ap.parse_args()
    from paper_1810_12437_gb300 import inputs
    P = inputs.config3()
    meta = dict(workload="config3 n=500000 p=50000 R=16", n=P.X.n, p=P.X.p, nnz=P.X.nnz,
                design_fingerprint=design_fingerprint(P.X), tol=1e-6, stop_rule="paper_rms",
                tau=[float(t) for t in P.tau])
    del P
    if os.path.exists(OUT):
        old = json.load(open(OUT))
        if old.get("design_fingerprint") == meta["design_fingerprint"]:
            for key in ("chains", "compensated", "compensated_ulp", "f32x2", "f32x2_ulp"):
                if key in old:
                    meta[key] = old[key]
    kinds = {"all": ["plain", "compensated", "compensated_ulp", "f32x2", "f32x2_ulp"],
             "plain": ["plain"], "compensated": ["compensated", "compensated_ulp"],
             "f32x2": ["f32x2", "f32x2_ulp"]}[args.part]
    # longest chains first, so that the pool's tail is short
    order = list(range(16))
    if "chains" in meta:
        order = sorted(range(16), key=lambda r: -meta["chains"][r]["iters"])
    jobs = [(r, kd) for r in order for kd in kinds]
    ctx = mp.get_context("spawn")
    with ctx.Pool(args.procs) as pool:
        out = pool.map(run_chain, jobs, chunksize=1)
    for kd in kinds:
        key = "chains" if kd == "plain" else kd
        meta[key] = sorted([c for k2, c in out if k2 == kd], key=lambda c: c["chain"])
    with open(OUT, "w") as f:
        json.dump(meta, f, indent=1)
    for kd in ("chains", "compensated", "compensated_ulp", "f32x2", "f32x2_ulp"):
        if kd in meta:
            print(kd, [c["iters"] for c in meta[kd]])


if __name__ == "__main__":
    main()
