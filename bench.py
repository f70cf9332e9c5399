#!/usr/bin/env python
"""Benchmark of the conditional beta draw on GB300.

Workload (one step): 16 conditional draws of beta ~ N(Phi^-1 X^T Omega z,
Phi^-1) sharing one synthetic binary design X with n = 500,000 rows and
p = 50,000 columns (column rates log10 r ~ U(-4.5, -1.5), about 1.15e8
nonzeros), each chain with its own omega, lambda, tau, eta and delta;
right-hand sides by Eq. 2.3 and prior-preconditioned CG to the paper's RMS
rule 1e-6 (Eq. S2), one batched launch (CUDA graph) per step.  Products in
double-float arithmetic (pairs of floats, about 48 bits: float64-like
iteration counts at float32 instruction rates) with float64 CG scalars and
vectors; PCG_BENCH_PRECISION=fx64 selects 64-bit fixed-point products (each
staged tile scaled by a power of two, exact integer sums) and
PCG_BENCH_PRECISION=fp32_refined float32 products with float64 reliable
updates instead.

Printed (rank 0, one JSON line): beta-draws/s of the whole job, the
end-to-end rate through the public API with host buffers, the roofline of the
dominant kernel against the measured HBM peak, the oracle on the host cores,
the plain single-RHS rate on the same GPU, clocks and kernel launch counts.

`--impl reference` times the CPU oracle instead (the reference arm): each
step is a bounded sample of the same workload (every chain's right-hand side
plus a few CG iterations, the chains on all host cores at once), projected
to whole draws/s with the oracle's own iteration counts for these chains
(tests/golden/config3_oracle.json, written by a script that runs only the
oracle); the line says so ("projected": true) and gives the sample's wall
time per step.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "beta-draws/sec and SpMV HBM GB/s vs peak at n=5e5,p=5e4; batched/adjoint vs plain PCG"
UNIT = "beta-draws/s"
NRHS = 16
TOL = 1e-6
PRECISION = os.environ.get("PCG_BENCH_PRECISION", "df32")
RELIABLE_K = 50
# arithmetic of the products per precision: float pairs, 64-bit integer sums of
# fixed-point tiles (vectors as float pairs), float64, float32
DTYPES = {"df32": "f32x2", "fx64": "int64", "fp64": "f64"}
WORKLOAD = ("16 chains sharing binary X, n=500000, p=50000, log10 r_j~U(-4.5,-1.5), "
            "per-chain omega~U(.05,.25), half-Cauchy lambda (2% x100), log10 tau~U(-3.5,-2.5), "
            "paper RMS stop 1e-6")
GOLDEN3 = os.path.join(ROOT, "tests", "golden", "config3_oracle.json")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the single-RHS comparator, e2e and CPU baseline legs")
    ap.add_argument("--small", action="store_true", help="debug: a 20x smaller design")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the uneven-batch and adjoint comparisons")
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.lines = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.gpu)], stdout=subprocess.PIPE,
                stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(ms, world, device=None):
    """Max of a per-rank time over all ranks (the job's step time)."""
    if world <= 1:
        return float(ms)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world, ms_per_step):
    """Whole-job draws/s: every rank draws NRHS chains per step."""
    return world * NRHS / (ms_per_step / 1e3)


def make_workload(rank, small):
    from paper_1810_12437_gb300 import inputs
    if small:
        return inputs.config3(nrhs=NRHS, n=25_000, p=2_500, seed_offset=rank)
    return inputs.config3(nrhs=NRHS, seed_offset=rank)


def tile_geometry(n, p, RG, vsize=4):
    """Tile widths of the shared-memory tiled products (the library's rule:
    220 KB of staged values including one zero sentinel slot, at most 65528
    per 16-bit offset, a multiple of 8)."""
    w = min((220 * 1024 - RG * vsize) // (RG * vsize), 65528) & ~7
    wc, wr = min(w, p), min(w, n)
    return (p + wc - 1) // wc, (n + wr - 1) // wr


def bytes_per_launch(kernel, n, p, nnz, RP, RG=1):
    """Algorithmic bytes of one launch (per RHS group for the tiled kernels):
    every stored index read once (2 bytes, pad slots not counted), chunk
    bounds and segment orders once, every gathered vector read once (it is
    staged on chip), every output written once.  Values are 4 bytes in the
    float32 kernels and 8 bytes in the double-float and fixed-point ones (pairs
    of floats in global memory)."""
    vs = 8 if kernel.endswith(("df32", "fx64")) else 4
    pair = PRECISION in ("df32", "fx64")
    if kernel in ("bt_csr_f32", "t_csr_f32", "bt_csr_df32", "t_csr_df32", "bt_csr_fx64", "t_csr_fx64"):
        Tc, _ = tile_geometry(n, p, RG, vs)
        return 2 * nnz + 4 * (Tc * n + 1) + 4 * n + vs * RG * (p + Tc * n)
    if kernel in ("bt_u", "t_u"):
        Tc, _ = tile_geometry(n, p, RG, 8 if pair else 4)
        v = 8 if pair else 4
        return v * RG * (Tc * n + n + n)
    if kernel in ("bt_csc_f32", "t_csc_f32", "bt_csc_df32", "t_csc_df32", "bt_csc_fx64", "t_csc_fx64"):
        _, Tr = tile_geometry(n, p, RG, vs)
        return 2 * nnz + 4 * (Tr * p + 1) + 4 * p + vs * RG * (n + Tr * p)
    if kernel == "bt_fin":
        return None
    if kernel == "b_csr_f32":
        return 4 * nnz + 8 * (n + 1) + 4 * n * RP + 4 * n * RP + 4 * p * RP
    if kernel == "b_csc_f32":
        return 4 * nnz + 8 * (p + 1) + 4 * n * RP + 3 * 8 * p * RP
    if kernel == "b_ru_csr_f64":
        return 4 * nnz + 8 * (n + 1) + 8 * n * RP + 8 * n * RP + 8 * p * RP
    if kernel == "b_ru_true_resid":
        return 4 * nnz + 8 * (p + 1) + 8 * n * RP + 5 * 8 * p * RP
    if kernel == "b_update":
        return 6 * 8 * p * RP
    if kernel == "b_sdir":
        return 3 * 8 * p * RP + 4 * p * RP
    return None


def tuned_group_width(tune_file):
    """RHS group width the library's autotuner chose (its cache file holds
    lines `batch_rg:<n>:<p>:<nnz>:<RP>:<precision> <RG>`); 0 = untiled."""
    rg = 1
    try:
        with open(tune_file) as fh:
            for line in fh:
                if line.startswith("batch_rg:"):
                    rg = int(line.split()[1])
    except (OSError, ValueError, IndexError):
        pass
    return rg


def kernel_source_sha():
    """Hash of the sources that define the tiled product kernels (their launch
    shapes included): the traffic figures hold while it is unchanged."""
    h = hashlib.sha256()
    for f in ("tiled.cu", "tiled.h", "df.cuh"):
        with open(os.path.join(ROOT, "paper_1810_12437_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def captured_entry(kernel, rg=None):
    """The profiles/traffic.json entry of `kernel` if it was taken on the
    current kernel source and, when the entry names its RHS group width, at
    group width `rg`; else None."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            e = json.load(f).get(kernel)
    except Exception:
        return None
    if not e or e.get("source_sha") != kernel_source_sha():
        return None
    if rg is not None and "rhs_group" in e and e["rhs_group"] != rg:
        return None
    return e


def smem_wavefronts_for(kernel, chains_per_launch, rg=None):
    """ncu shared-memory wavefronts (l1tex__data_pipe_lsu_wavefronts_mem_shared.sum)
    per launch: the captured launch's count, which covered `live_chains`
    chains, scaled to `chains_per_launch` (every live chain gathers every
    entry once); None when absent or stale."""
    e = captured_entry(kernel, rg)
    if e and "smem_wavefronts_per_launch" in e:
        return e["smem_wavefronts_per_launch"] * chains_per_launch / e["live_chains"]
    return None


def traffic_for(kernel, alg_bytes_per_launch, n, p, nnz, rg=None):
    """ncu DRAM bytes (read + write) per launch, from profiles/traffic.json,
    if they were taken on the current kernel source and group width.  The
    capture is one launch with `live_chains` chains live; a timed launch with
    fewer moves less (the index stream is read once per launch for all
    groups, the vectors once per chain), so the captured bytes are scaled by
    the ratio of the two launches' algorithmic bytes (scope_table_bytes)."""
    e = captured_entry(kernel, rg)
    if not e:
        return None
    return e["dram_bytes_per_launch"] * alg_bytes_per_launch / scope_table_bytes(kernel, n, p, nnz, e["live_chains"])


def product_accounting(chain_iters, RG, tail, RP=16):
    """Work of the tiled products in one batched draw.  In iteration k the
    live chains are those with more than k iterations (live_k); finished
    chains are compacted away, so the main plan's launch covers ceil(live_k /
    RG) RHS groups.  With a tail plan (RG >= 2), iterations with one live
    chain run the group-width-1 plan instead, and the main plan's kernels of
    those iterations exit at their gate (in the profiled plain-launch mode
    they still appear as launches).  Returns per-plan iteration counts, group
    units, chain units (the sum of live_k) and the finalize kernel's slot
    units (the slots it covers, summed over the main plan's iterations)."""
    K = max(chain_iters) if chain_iters else 0
    live = [sum(1 for c in chain_iters if c > k) for k in range(K)]
    main = [L for L in live if not (tail and L == 1)]
    tl = [L for L in live if tail and L == 1]

    def slots(L):
        # the finalize kernel's slots: the live groups' RG slots each, rounded
        # up to a power of two (all RP slots for the untiled products)
        act = min(RP, -(-L // RG) * RG) if RG else RP
        a2 = 1
        while a2 < act:
            a2 *= 2
        return a2

    return {"iterations": K, "main_iterations": len(main), "tail_iterations": len(tl),
            "main_group_units": sum(-(-L // RG) for L in main) if RG else 0,
            "main_chain_units": sum(main), "tail_chain_units": sum(tl),
            "main_slot_units": sum(slots(L) for L in main), "tail_slots": slots(1)}


def scope_table_bytes(kernel, n, p, nnz, L):
    """Algorithmic bytes of one product pass over L live chains by the
    hot-path scope table's measure (binary X as int32 indices read once for
    the whole RHS block, int64 pointers, float32 gathered vectors read once,
    float64 p-vectors): CSR pass 4 nnz + 8 (n+1) + L (4p + 8n) (s gathered,
    omega read, u written); CSC pass 4 nnz + 8 (p+1) + L (4n + 24p) (u
    gathered; s, d read and v written in float64)."""
    if "csr" in kernel:
        return 4 * nnz + 8 * (n + 1) + L * (4 * p + 8 * n)
    if "csc" in kernel:
        return 4 * nnz + 8 * (p + 1) + L * (4 * n + 24 * p)
    return None


def roofline(table, acct, n, p, nnz, RG, peak, peak_kind, sm_mhz=None):
    """Roofline entry of the dominant kernel and the per-kernel table.
    `achieved` uses the scope table's algorithmic bytes (scope_table_bytes) summed
    over the launches that did work, divided by the kernel's total CUDA-event
    time; `impl_*` gives the same with the kernel's own per-group bytes
    (bytes_per_launch: 16-bit tile offsets, staged slices, tile partials)."""
    RP = 16

    def units(k):
        if k.startswith("bt1_"):
            return acct["tail_iterations"], acct["tail_chain_units"], acct["tail_iterations"]
        if k.startswith(("bt_cs", "bt_u")):
            return acct["main_iterations"], acct["main_chain_units"], acct["main_group_units"]
        return None, None, None

    def fin_bytes():
        # k_b_fin: per column, every covered slot's strip partials (float pairs
        # or floats), s and d read and v written (float64); with the tail plan
        # the one chain's partials over the group-width-1 plan's strips
        pv = 8 if PRECISION in ("df32", "fx64") else 4
        T_main = tile_geometry(n, p, RG, pv)[1] if RG else 0
        T_tail = tile_geometry(n, p, 1, pv)[1]
        return p * (acct["main_slot_units"] * (pv * T_main + 24)
                    + acct["tail_iterations"] * (pv * T_tail + 24 * acct["tail_slots"]))

    def impl_bytes(k, launches):
        if k == "bt_fin":
            return fin_bytes() if "main_slot_units" in acct else None
        it, _, gu = units(k)
        kk = k.replace("bt1_", "bt_")
        bb = bytes_per_launch(kk, n, p, nnz, RP, 1 if k.startswith("bt1_") else RG)
        if bb is None:
            return None
        return bb * (gu if gu is not None else launches)

    def alg_bytes(k):
        it, cu, _ = units(k)
        if it is None or scope_table_bytes(k, n, p, nnz, 1) is None:
            return None
        return it * (4 * nnz + 8 * ((n if "csr" in k else p) + 1)) + (
            scope_table_bytes(k, n, p, nnz, 1) - scope_table_bytes(k, n, p, nnz, 0)) * cu

    total_ms = sum(v[0] for v in table.values())
    per_k = {}
    for k, (ms, nl) in sorted(table.items()):
        it, cu, gu = units(k)
        ab, ib = alg_bytes(k), impl_bytes(k, nl)
        per_k[k] = {"avg_us": round(ms / nl * 1e3, 2), "launches": nl,
                    "working_launches": it if it is not None else nl,
                    "GBps": round(ab / (ms / 1e3) / 1e9, 1) if ab else None,
                    "impl_GBps": round(ib / (ms / 1e3) / 1e9, 1) if ib else None}
    kname, (kms, kn) = max(table.items(), key=lambda kv: kv[1][0])
    it, cu, gu = units(kname)
    work_launches = it if it else kn
    avg_s = kms / work_launches / 1e3
    ab, ib = alg_bytes(kname), impl_bytes(kname, kn)
    achieved = ab / work_launches / avg_s / 1e9 if ab else None
    impl_achieved = ib / work_launches / avg_s / 1e9 if ib else None
    chains_per_launch = (cu / work_launches) if cu else 1.0
    rg_k = 1 if kname.startswith("bt1_") else RG
    wf = smem_wavefronts_for(kname, chains_per_launch, rg_k)
    smem = None
    if wf:
        # one shared-memory wavefront per clock per SM (152 SMs) at the sampled SM clock
        peak_wf = 152 * (sm_mhz or 2070.0) * 1e6
        smem = {"wavefronts_per_launch": wf, "achieved_per_s": wf / avg_s, "peak_per_s": peak_wf,
                "frac": wf / avg_s / peak_wf,
                "note": "ncu shared-memory wavefronts of an all-chains-live launch (profiles/traffic.json) "
                        "scaled by live chains per launch, over the launch time; peak 1 wavefront/clock/SM"}
    return {"bound": "hbm", "kernel": kname, "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": (achieved / peak) if achieved else None,
            "traffic": traffic_for(kname, ab / work_launches, n, p, nnz, rg_k) if ab else None,
            "traffic_note": "ncu DRAM bytes of an all-chains-live launch (profiles/traffic.json) scaled by "
                            "algorithmic bytes to the average working launch",
            "shared_memory": smem,
            "peak_source": f"hbm_gbs of {peak_kind}",
            "bytes": "scope-table algorithmic bytes: int32 indices once per launch for all live "
                     "chains, vectors once per chain (scope_table_bytes)",
            "avg_launch_us": avg_s * 1e6, "working_launches": work_launches,
            "launches_profiled": kn,
            "algorithmic_bytes_per_launch": ab / work_launches if ab else None,
            "impl_bytes_per_launch": ib / work_launches if ib else None,
            "impl_achieved": impl_achieved,
            "impl_frac": (impl_achieved / peak) if impl_achieved else None,
            "rhs_group": RG, "accounting": acct,
            "kernel_shares": {k: round(v[0] / total_ms, 4) for k, v in sorted(table.items())},
            "per_kernel": per_k}


def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_1810_12437_gb300 as pb

    world, rank, local = dist_env()
    if args.gpus != world and world > 1:
        raise SystemExit(f"--gpus {args.gpus} but WORLD_SIZE {world}")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    P = make_workload(rank, args.small)
    X = pb.DeviceDesign.from_host(P.X, dev)
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(dev)
    ins = dict(omega=T(P.omega), z=T(P.z), lam=T(P.lam), tau=T(P.tau), eta=T(P.eta), delta=T(P.delta))
    out = torch.empty((NRHS, P.X.p), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    # the autotuned launch shapes are shared (through the cache file) with the
    # profiled pass below, so that the roofline describes the timed layout
    import tempfile
    tune_file = os.path.join(tempfile.mkdtemp(prefix="pcg_tune_"), "autotune.txt")
    ctx = pb.Context(precision=PRECISION, reliable_k=RELIABLE_K, stream=stream, autotune_cache=tune_file)

    def step():
        return pb.pcg_draw_beta_batched(ctx, X, **ins, tol=TOL, max_iter=20_000, out=out)

    res = None
    for _ in range(args.warmup):
        res = step()
    # every step reads the 0.92 GB index streams of X, far larger than the
    # 129 MB L2, so no separate flush is needed between steps
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches = 0
    iters = []
    e0.record(stream)
    for _ in range(args.steps):
        res = step()
        launches += pb.pcg_last_kernel_launches(ctx)
        iters.append(list(res.iters))
    e1.record(stream)
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, world, dev)
    value = job_value(world, ms)
    statuses = list(res.status)

    extras = {}
    if not args.no_extras:
        # plain single-RHS PCG on the same GPU and accuracy: the 16 chains one by one
        sctx = pb.Context(precision=PRECISION, reliable_k=RELIABLE_K, stream=stream)
        s_iters = []
        ch = lambda a, r: a[r].contiguous()
        for r in range(NRHS):   # warm-up and graph capture on chain 0 first
            if r == 0:
                pb.pcg_draw_beta(sctx, X, ch(ins["omega"], 0), ch(ins["z"], 0), ch(ins["lam"], 0),
                                 float(P.tau[0]), ch(ins["eta"], 0), ch(ins["delta"], 0), tol=TOL,
                                 max_iter=20_000)
        torch.cuda.synchronize(dev)
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        for r in range(NRHS):
            rr = pb.pcg_draw_beta(sctx, X, ch(ins["omega"], r), ch(ins["z"], r), ch(ins["lam"], r),
                                  float(P.tau[r]), ch(ins["eta"], r), ch(ins["delta"], r), tol=TOL,
                                  max_iter=20_000)
            s_iters.append(rr.iters)
        s1.record(stream)
        torch.cuda.synchronize(dev)
        single_ms = s0.elapsed_time(s1)
        extras["single_rhs"] = {"value": NRHS / (single_ms / 1e3), "unit": UNIT,
                                "iters": s_iters, "note": "same 16 chains as 16 sequential "
                                "single-RHS draws (plain PCG), same precision and stop rule"}
        # end to end through the public API with host buffers (pinned)
        host = {k: v.cpu().pin_memory() for k, v in ins.items()}
        hout = torch.empty((NRHS, P.X.p), dtype=torch.float64).pin_memory()
        dins = {k: torch.empty_like(v) for k, v in ins.items()}
        h2d = sum(v.numel() * v.element_size() for v in host.values())
        d2h = hout.numel() * hout.element_size()

        def e2e_step():
            for k in host:
                dins[k].copy_(host[k], non_blocking=True)
            r_ = pb.pcg_draw_beta_batched(ctx, X, **dins, tol=TOL, max_iter=20_000, out=out)
            hout.copy_(out, non_blocking=True)
            return r_

        e2e_step()
        torch.cuda.synchronize(dev)
        ee0, ee1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ee0.record(stream)
        ne = max(1, min(args.steps, 3))
        for _ in range(ne):
            e2e_step()
        ee1.record(stream)
        torch.cuda.synchronize(dev)
        e2e_ms = max_over_ranks(ee0.elapsed_time(ee1) / ne, world, dev)
        extras["e2e"] = {"value": job_value(world, e2e_ms), "unit": UNIT,
                         "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                         "note": "X resident (fixed design); per-step chain inputs host->device"}

    # roofline of the dominant kernel: per-kernel CUDA events on the launching stream
    pctx = pb.Context(precision=PRECISION, reliable_k=RELIABLE_K, stream=stream, profile=True,
                      autotune_cache=tune_file)
    pres = pb.pcg_draw_beta_batched(pctx, X, **ins, tol=TOL, max_iter=20_000, out=out)
    table = pb.profile_table(pctx)
    RG = tuned_group_width(tune_file)
    acct = product_accounting(list(pres.iters), RG, tail=any(k.startswith("bt1_") for k in table))
    peak, peak_kind = peaks()
    roof = roofline(table, acct, P.X.n, P.X.p, P.X.nnz, RG, peak, peak_kind, clk.get("sm_mhz"))

    forms = None
    if rank == 0 and not args.no_forms:
        forms = other_forms(pb, dev, stream)
        forms.update(single_forms(pb, dev, stream, P, X, ins))

    cpu = None
    if rank == 0 and world == 1 and not args.no_extras:
        cpu = cpu_baseline(P, iters[-1])

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": DTYPES.get(PRECISION, "f32"), "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": P.X.n, "p": P.X.p, "nnz": P.X.nnz, "nrhs": NRHS,
                   "tol": TOL, "precision": PRECISION,
                   "parallelism": f"replicas x{world} (independent chains per GPU)",
                   "l2": "inputs larger than L2 (0.92 GB of index streams per iteration)",
                   "iters_per_chain": iters[-1], "status": statuses},
        "e2e": extras.get("e2e"), "gpu_launches": launches, "roofline": roof, "cpu_baseline": cpu,
        "single_rhs": extras.get("single_rhs"), "clocks": clk, "forms": forms,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def other_forms(pb, dev, stream):
    """The uneven batch (float32 refined, float64 and double-float products)
    and the adjoint (float32 refined and double-float), each against plain single-RHS PCG on the
    same GPU, precision and stop rule (RMS 1e-6)."""
    import torch
    from paper_1810_12437_gb300 import inputs
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(dev)
    out = {}
    # uneven batch: 64 problems, n ~ logU[5e3, 2e5], p ~ logU[1e3, 3e4]
    probs = inputs.config4()
    dp = [dict(X=pb.DeviceDesign.from_host(P.X, dev), omega=T(P.omega), z=T(P.z), lam=T(P.lam),
               tau=float(P.tau), eta=T(P.eta), delta=T(P.delta)) for P in probs]
    def uneven_vs_single(prec):
        ctx = pb.Context(precision=prec, stream=stream)
        pb.pcg_draw_beta_uneven(ctx, dp, tol=TOL, max_iter=20_000)      # tunes and builds the graph
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        res = pb.pcg_draw_beta_uneven(ctx, dp, tol=TOL, max_iter=20_000)
        torch.cuda.synchronize(dev)
        t_uneven = time.perf_counter() - t0
        sctx = pb.Context(precision=prec, stream=stream)
        for d in dp[:2]:
            pb.pcg_draw_beta(sctx, d["X"], d["omega"], d["z"], d["lam"], d["tau"], d["eta"], d["delta"], tol=TOL)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        s_iters = []
        for d in dp:
            r = pb.pcg_draw_beta(sctx, d["X"], d["omega"], d["z"], d["lam"], d["tau"], d["eta"], d["delta"],
                                 tol=TOL, max_iter=20_000)
            s_iters.append(r.iters)
        torch.cuda.synchronize(dev)
        t_single = time.perf_counter() - t0
        return {"persistent_kernel_draws_per_s": len(dp) / t_uneven,
                "single_rhs_draws_per_s": len(dp) / t_single,
                "iters_sum_uneven": int(sum(r.iters for r in res)), "iters_sum_single": int(sum(s_iters)),
                "status_ok": all(r.status == 0 for r in res)}

    out["uneven"] = {"workload": "64 problems, n~logU[5e3,2e5], p~logU[1e3,3e4], log10 r~U(-4,-1.5), tau=0.01",
                     "nnz_total": int(sum(P.X.nnz for P in probs)),
                     "fp32_refined": uneven_vs_single("fp32_refined"), "fp64": uneven_vs_single("fp64"),
                     "df32": uneven_vs_single("df32")}
    del dp
    # adjoint: gradient of c^T beta on n=2e5, p=2e4
    P = inputs.config5()
    X = pb.DeviceDesign.from_host(P.X, dev)
    a = dict(omega=T(P.omega), z=T(P.z), lam=T(P.lam), eta=T(P.eta), delta=T(P.delta))
    def adjoint_vs_forward(prec):
        actx = pb.Context(precision=prec, stream=stream)
        dr = pb.pcg_draw_beta(actx, X, a["omega"], a["z"], a["lam"], P.tau, a["eta"], a["delta"], tol=TOL)
        pb.pcg_adjoint(actx, X, a["omega"], a["z"], a["lam"], P.tau, a["eta"], a["delta"], dr.beta, T(P.c),
                       tol=TOL)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        dr = pb.pcg_draw_beta(actx, X, a["omega"], a["z"], a["lam"], P.tau, a["eta"], a["delta"], tol=TOL)
        torch.cuda.synchronize(dev)
        t_fwd = time.perf_counter() - t0
        t0 = time.perf_counter()
        g = pb.pcg_adjoint(actx, X, a["omega"], a["z"], a["lam"], P.tau, a["eta"], a["delta"], dr.beta,
                           T(P.c), tol=TOL)
        torch.cuda.synchronize(dev)
        t_adj = time.perf_counter() - t0
        return {"forward_draws_per_s": 1.0 / t_fwd, "adjoint_gradients_per_s": 1.0 / t_adj,
                "forward_iters": dr.iters, "adjoint_iters": g["iters"], "adjoint_over_forward_time": t_adj / t_fwd}

    out["adjoint"] = {"workload": "n=200000, p=20000, log10 r~U(-4,-1.8), tau=1e-3, L = c^T beta",
                      "fp32_refined": adjoint_vs_forward("fp32_refined"), "df32": adjoint_vs_forward("df32")}
    return out


def oracle_sample(P, chains, S, threads):
    """Times the oracle, as it stands, on the host: for each chain, the
    right-hand side (Eq. 2.3) plus S CG iterations, the chains spread over
    `threads` host threads running at once (the oracle's C routines release
    the GIL, so each thread keeps one core busy and the threads contend for
    memory bandwidth as whole draws would).  Returns per-chain (rhs seconds,
    seconds per iteration) and the wall time of the sample."""
    import concurrent.futures as cf
    from oracle import oracle as O

    def one(r):
        om, lam, tau = P.omega[r], P.lam[r], float(P.tau[r])
        t0 = time.perf_counter()
        b = O.build_b(P.X, om, P.z[r], lam, tau, P.eta[r], P.delta[r])
        t1 = time.perf_counter()
        O.pcg(P.X, om, lam, tau, b, fixed_iters=S)
        t2 = time.perf_counter()
        return r, t1 - t0, (t2 - t1) / S

    w0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        res = list(ex.map(one, chains))
    return res, time.perf_counter() - w0


def projected_rate(res, threads, P):
    """Draws/s of whole draws projected from a sample: each chain's draw is
    its right-hand side plus its oracle iteration count times its measured
    seconds per iteration; `threads` cores work through the chains' total
    time in parallel."""
    total = 0.0
    srcs = set()
    for r, t_rhs, t_it in res:
        k, src = oracle_iters(P, r)
        srcs.add(src)
        total += t_rhs + k * t_it
    return len(res) / (total / threads), "; ".join(sorted(srcs))


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def single_forms(pb, dev, stream, P, X, ins):
    """Chain 0 of the bench workload as single-RHS draws on the same GPU and
    stop rule: the Jacobi against the prior preconditioner (Sec. 2.4, Sec.
    3), a warm start from the previous draw against a cold start (Sec.
    S4.1), and LSQR on the least-squares form (Sec. S7.1) against CG, both
    in float64."""
    import torch
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(dev)
    ch = lambda k: ins[k][0].contiguous()
    args = (ch("omega"), ch("z"), ch("lam"), float(P.tau[0]), ch("eta"), ch("delta"))

    def timed(fn, reps=2):
        fn()                                   # graph capture, plans
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(reps):
            r = fn()
        torch.cuda.synchronize(dev)
        return r, reps / (time.perf_counter() - t0)

    out = {"workload": "chain 0 of the bench workload (n=500000, p=50000), single-RHS draws"}
    pre = {}
    for name in ("prior", "jacobi"):
        c = pb.Context(precision=PRECISION, reliable_k=RELIABLE_K, stream=stream, preconditioner=name)
        r, rate = timed(lambda: pb.pcg_draw_beta(c, X, *args, tol=TOL, max_iter=20_000))
        pre[name] = {"iters": r.iters, "draws_per_s": rate, "status": r.status}
    out["preconditioner"] = pre
    # warm start from the previous draw (the same omega, lambda, tau; fresh eta, delta)
    rng = np.random.default_rng(99)
    eta2, delta2 = T(rng.standard_normal(P.X.n)), T(rng.standard_normal(P.X.p))
    cold = pb.Context(precision=PRECISION, reliable_k=RELIABLE_K, stream=stream)
    first = pb.pcg_draw_beta(cold, X, *args, tol=TOL, max_iter=20_000).beta.clone()
    warm = pb.Context(precision=PRECISION, reliable_k=RELIABLE_K, stream=stream, warm_start=True)
    a2 = (args[0], args[1], args[2], args[3], eta2, delta2)
    buf = torch.empty_like(first)
    rc, rate_c = timed(lambda: pb.pcg_draw_beta(cold, X, *a2, tol=TOL, max_iter=20_000))

    def warm_draw():
        buf.copy_(first)
        return pb.pcg_draw_beta(warm, X, *a2, tol=TOL, max_iter=20_000, out=buf)

    rw, rate_w = timed(warm_draw)
    out["warm_start"] = {"cold_iters": rc.iters, "warm_iters": rw.iters, "cold_draws_per_s": rate_c,
                         "warm_draws_per_s": rate_w,
                         "beta_0": "the previous draw of the same conditional (fresh eta, delta)"}
    f64 = pb.Context(precision="fp64", stream=stream)
    rl, rate_l = timed(lambda: pb.pcg_draw_beta_lsqr(f64, X, *args, tol=TOL, max_iter=20_000), reps=1)
    rp, rate_p = timed(lambda: pb.pcg_draw_beta(f64, X, *args, tol=TOL, max_iter=20_000), reps=1)
    out["lsqr"] = {"lsqr_iters": rl.iters, "lsqr_draws_per_s": rate_l, "cg_iters": rp.iters,
                   "cg_draws_per_s": rate_p, "precision": "fp64 (LSQR: untiled float64 gathers; "
                   "CG: the tiled float64 products)"}
    # whole Gibbs cycles of Sec. S1 (horseshoe; tau, lambda, omega updates + the draw)
    y = T(P.y[0])
    gctx = pb.Context(precision=PRECISION, reliable_k=RELIABLE_K, stream=stream)
    beta_start = pb.pcg_draw_beta(gctx, X, *args, tol=TOL, max_iter=20_000).beta.clone()
    gst = pb.GibbsState(omega=ch("omega").clone(), lam=ch("lam").clone(),
                        nu=torch.ones(P.X.p, dtype=torch.float64, device=dev),
                        beta=beta_start, tau=float(P.tau[0]), xi=1.0)
    pb.pcg_gibbs_step(gctx, X, y, gst, seed=2018, step=0, tol=TOL, max_iter=20_000)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    g_iters = []
    for k in range(1, 4):
        g_iters.append(pb.pcg_gibbs_step(gctx, X, y, gst, seed=2018, step=k, tol=TOL, max_iter=20_000).iters)
    torch.cuda.synchronize(dev)
    rate_g = 3 / (time.perf_counter() - t0)
    pctx = pb.Context(precision=PRECISION, reliable_k=RELIABLE_K, stream=stream, profile=True)
    pb.pcg_gibbs_step(pctx, X, y, gst, seed=2018, step=4, tol=TOL, max_iter=20_000)
    tab = pb.profile_table(pctx)
    upd_ms = sum(v[0] for k, v in tab.items() if k.startswith("g_"))
    out["gibbs"] = {"steps_per_s": rate_g, "draw_iters": g_iters,
                    "updates_ms": upd_ms, "tau": gst.tau,
                    "note": "cycles 1-3 from the workload's omega, lambda, tau and a draw of beta given them "
                            "(y carries no signal, so the chain moves towards smaller tau and shorter "
                            "draws); updates_ms: tau, lambda, psi = X beta, omega, eta, delta kernels "
                            "of one cycle"}
    return out


def cpu_baseline(P, gpu_iters):
    """The oracle, as it stands, on the host cores: one thread on chain 0
    (right-hand side + 16 CG iterations), and every core at once (one chain
    per thread, right-hand side + 6 iterations each); both projected to whole
    draws with the oracle's own iteration counts.  The value is the all-core
    rate."""
    S1, S2 = 16, 6
    one, w1 = oracle_sample(P, [0], S1, 1)
    rate1, src = projected_rate(one, 1, P)
    cores = host_cores()
    nthr = min(cores, NRHS)
    allc, w2 = oracle_sample(P, list(range(NRHS)), S2, nthr)
    rate_all, _ = projected_rate(allc, nthr, P)
    return {"value": rate_all, "unit": UNIT, "cores": nthr, "host_cores": cores, "kind": "oracle",
            "projected": True,
            "sample": f"{NRHS} chains on {nthr} threads at once, each RHS (Eq. 2.3) + {S2} CG "
                      f"iterations ({w2:.1f} s wall), projected to whole draws with the oracle's "
                      f"iteration counts ({src})",
            "seconds_per_iteration_all_cores": statistics.median(x[2] for x in allc),
            "single_thread": {"value": rate1, "unit": UNIT, "cores": 1, "projected": True,
                              "sample": f"chain 0: RHS + {S1} CG iterations ({w1:.1f} s)",
                              "seconds_per_iteration": one[0][2]}}


def oracle_iters(P, r, gpu_iters=None):
    try:
        with open(GOLDEN3) as f:
            g = json.load(f)
        if g["nnz"] == P.X.nnz and g["n"] == P.X.n:
            return int(g["chains"][r]["iters"]), "oracle iteration counts, tests/golden/config3_oracle.json"
    except Exception:
        pass
    if gpu_iters is not None:
        return int(gpu_iters[r]), "GPU iteration count of the same chain"
    return 1000, "assumed"


def run_reference(args):
    """The reference arm: the CPU oracle on the host cores.  Each step is a
    bounded sample of the workload, all 16 chains at once on min(cores, 16)
    threads, each chain's right-hand side plus S CG iterations; the printed
    rate projects whole draws from it (see projected_rate), and
    `sample_seconds_per_step` is the wall time a step actually took."""
    world, rank, local = dist_env()
    if rank != 0:
        return
    P = make_workload(0, args.small)
    S = 3
    cores = host_cores()
    nthr = min(cores, NRHS)
    rates, walls = [], []
    src = ""
    for k in range(args.warmup + args.steps):
        res, wall = oracle_sample(P, list(range(NRHS)), S, nthr)
        if k >= args.warmup:
            rate, src = projected_rate(res, nthr, P)
            rates.append(rate)
            walls.append(wall)
    value = statistics.median(rates)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": NRHS / value * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "projected": True,
            "sample_seconds_per_step": statistics.mean(walls),
            "config": {"workload": WORKLOAD, "n": P.X.n, "p": P.X.p, "nnz": P.X.nnz, "nrhs": NRHS,
                       "tol": TOL},
            "cpu_baseline": {"kind": "oracle", "cores": nthr, "host_cores": cores, "value": value,
                             "unit": UNIT, "projected": True,
                             "sample": f"per step all {NRHS} chains on {nthr} threads at once, "
                                       f"each RHS + {S} CG iterations, projected to whole draws "
                                       f"with the oracle's iteration counts ({src})"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
