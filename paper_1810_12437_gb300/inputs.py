"""Seeded synthetic inputs for the conditional beta draw.

This module only draws random inputs; it holds none of the sampler's
arithmetic (no right-hand side, no precision matrix, no solve).  It is the
one module that both the CPU oracle (``oracle/``) and the CUDA path use, so
that both sides see identical bytes.

Workload shapes follow the paper's healthcare designs (Sec. 4.1 and Sec. S7:
sparse binary X with n ~ 1e5..1e6 rows and p ~ 1e4..1e5 columns, whose
real data are proprietary).  Each column j of the binary design X is a
Bernoulli(r_j) process over the rows with log10 r_j ~ U(a, b); the Polya-Gamma
weights omega_i ~ U(0.05, 0.25); y_i ~ Bernoulli(0.3) and
z_i = (y_i - 1/2) / omega_i is the augmented response of Eq. 1.1; the local
scales lambda_j are half-Cauchy (the horseshoe prior of Sec. S1), some of them
inflated by 100 to mimic the few unshrunk signals; eta ~ N(0, I_n) and
delta ~ N(0, I_p) are the two Gaussian vectors of Prop. 2.1.

The generator uses numpy's PCG64 stream only, so the same seed gives the same
bytes on x86 and Arm hosts.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

SEED_BASE = 20181012


@dataclasses.dataclass
class Design:
    """Binary sparse design X (n x p) held as indices only, in both layouts.

    CSR: ``row_ptr`` (int64, n+1) and ``col_idx`` (int32, nnz), columns sorted
    within each row.  CSC: ``col_ptr`` (int64, p+1) and ``row_idx`` (int32,
    nnz), rows sorted within each column.  Every stored entry equals 1.
    """

    n: int
    p: int
    row_ptr: np.ndarray
    col_idx: np.ndarray
    col_ptr: np.ndarray
    row_idx: np.ndarray

    @property
    def nnz(self) -> int:
        return int(self.col_idx.shape[0])

    def dense(self) -> np.ndarray:
        """Dense float64 copy (only for tiny designs)."""
        x = np.zeros((self.n, self.p))
        rows = np.repeat(np.arange(self.n), np.diff(self.row_ptr))
        x[rows, self.col_idx] = 1.0
        return x


@dataclasses.dataclass
class Problem:
    """Inputs of one conditional draw (or of R draws sharing X).

    With R chains, ``omega, z, eta`` have shape (R, n); ``lam, delta, c``
    have shape (R, p); ``tau`` has shape (R,).  With one chain they are 1-D
    and ``tau`` is a float.
    """

    X: Design
    omega: np.ndarray
    z: np.ndarray
    lam: np.ndarray
    tau: object
    eta: np.ndarray
    delta: np.ndarray
    c: Optional[np.ndarray] = None
    y: Optional[np.ndarray] = None


def column_rates(rng: np.random.Generator, p: int, a: float, b: float) -> np.ndarray:
    """r_j = 10**U(a, b), one Bernoulli rate per column."""
    return 10.0 ** rng.uniform(a, b, size=p)


def binary_design_from_rates(rng: np.random.Generator, n: int, rates: np.ndarray) -> Design:
    """Draw X with independent entries X_ij ~ Bernoulli(rates[j]).

    Each column is generated as a Bernoulli process: the gaps between
    successive nonzero rows are Geometric(r_j), so rows come out sorted and
    distinct and the column count is Binomial(n, r_j).
    """
    p = int(rates.shape[0])
    rates = np.clip(np.asarray(rates, dtype=np.float64), 1e-12, 1.0)
    mean = n * rates
    m = np.ceil(mean + 8.0 * np.sqrt(mean * (1.0 - rates)) + 16.0).astype(np.int64)
    starts = np.zeros(p + 1, dtype=np.int64)
    np.cumsum(m, out=starts[1:])
    gaps = rng.geometric(np.repeat(rates, m)).astype(np.int64)
    cs = np.cumsum(gaps)
    base = np.zeros(p, dtype=np.int64)
    base[1:] = cs[starts[1:-1] - 1]
    pos = cs - np.repeat(base, m) - 1          # 0-based row of each draw
    last = cs[starts[1:] - 1] - base - 1       # row reached by each column's last gap
    keep = pos < n
    counts = np.zeros(p, dtype=np.int64)
    if p:
        counts[:] = np.add.reduceat(keep.astype(np.int64), starts[:-1])
    row_idx = pos[keep]
    short = np.nonzero(last < n)[0]
    if short.size:
        # A column whose gap budget ran out before row n (probability below
        # 1e-15 per column at the 8-sigma budget) is continued to the end.
        off = np.zeros(p + 1, dtype=np.int64)
        np.cumsum(counts, out=off[1:])
        cols = [row_idx[off[j]:off[j + 1]] for j in range(p)]
        for j in short:
            cur = int(last[j])
            while cur < n:
                steps = cur + np.cumsum(rng.geometric(rates[j], size=64))
                cols[j] = np.concatenate([cols[j], steps[steps < n]])
                cur = int(steps[-1])
            counts[j] = cols[j].shape[0]
        row_idx = np.concatenate(cols)
    col_ptr = np.zeros(p + 1, dtype=np.int64)
    np.cumsum(counts, out=col_ptr[1:])
    row_idx = row_idx.astype(np.int32)
    return design_from_csc(n, p, col_ptr, row_idx)


def design_from_csc(n: int, p: int, col_ptr: np.ndarray, row_idx: np.ndarray) -> Design:
    """Complete a binary design given its CSC indices (builds the CSR copy)."""
    col_ptr = np.ascontiguousarray(col_ptr, dtype=np.int64)
    row_idx = np.ascontiguousarray(row_idx, dtype=np.int32)
    nnz = int(row_idx.shape[0])
    cols = np.repeat(np.arange(p, dtype=np.int64), np.diff(col_ptr))
    key = row_idx.astype(np.int64) * max(p, 1) + cols
    key.sort()
    col_idx = (key % max(p, 1)).astype(np.int32)
    rows_sorted = key // max(p, 1)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows_sorted, minlength=n)[:n], out=row_ptr[1:])
    assert row_ptr[-1] == nnz
    return Design(n=n, p=p, row_ptr=row_ptr, col_idx=col_idx, col_ptr=col_ptr, row_idx=row_idx)


def design_from_dense(x: np.ndarray) -> Design:
    """Binary design from a dense 0/1 matrix (tests and tiny cases)."""
    x = np.asarray(x)
    n, p = x.shape
    rows, cols = np.nonzero(x.T)          # column-major walk: (col, row) pairs
    col_ptr = np.zeros(p + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=p), out=col_ptr[1:])
    return design_from_csc(n, p, col_ptr, cols.astype(np.int32))


def perturb_ulps(x: np.ndarray, seed: int) -> np.ndarray:
    """x with every entry multiplied by 1 + k 2^-52, k drawn uniformly from
    {-1, 0, 1}: the same input up to about one unit in the last place.  Runs
    on such copies measure how much an iteration count depends on rounding."""
    rng = np.random.default_rng(seed)
    x = np.asarray(x, dtype=np.float64)
    return x * (1.0 + rng.integers(-1, 2, size=x.shape) * 2.0 ** -52)


def relabel(P: "Problem", seed: int):
    """The same single-chain problem with its rows and columns relabelled by
    seeded random permutations: X'[row_perm[i], col_perm[j]] = X[i, j] and the
    vectors moved with them.  Returns (P', row_perm, col_perm); a draw of P'
    at coefficient col_perm[j] corresponds to coefficient j of P.  Every sum
    of the method runs over the same terms in another order."""
    rng = np.random.default_rng(seed)
    X = P.X
    row_perm = rng.permutation(X.n)
    col_perm = rng.permutation(X.p)
    cols = np.repeat(np.arange(X.p, dtype=np.int64), np.diff(X.col_ptr))
    new_r = row_perm[X.row_idx.astype(np.int64)]
    new_c = col_perm[cols]
    order = np.lexsort((new_r, new_c))
    col_ptr = np.zeros(X.p + 1, dtype=np.int64)
    np.cumsum(np.bincount(new_c, minlength=X.p), out=col_ptr[1:])
    X2 = design_from_csc(X.n, X.p, col_ptr, new_r[order].astype(np.int32))

    def mv(v, perm):
        out = np.empty_like(v)
        out[perm] = v
        return out

    P2 = Problem(X=X2, omega=mv(P.omega, row_perm), z=mv(P.z, row_perm), lam=mv(P.lam, col_perm),
                 tau=P.tau, eta=mv(P.eta, row_perm), delta=mv(P.delta, col_perm),
                 c=None if P.c is None else mv(P.c, col_perm),
                 y=None if P.y is None else mv(P.y, row_perm))
    return P2, row_perm, col_perm


def _lambda_half_cauchy(rng, size, inflate_frac=0.0):
    lam = np.abs(rng.standard_cauchy(size=size))
    lam = np.maximum(lam, 1e-300)
    if inflate_frac > 0:
        p = size if np.isscalar(size) else size[-1]
        k = int(round(inflate_frac * p))
        if k:
            if np.isscalar(size):
                idx = rng.choice(p, size=k, replace=False)
                lam[idx] *= 100.0
            else:
                for r in range(size[0]):
                    idx = rng.choice(p, size=k, replace=False)
                    lam[r, idx] *= 100.0
    return lam


def _obs_inputs(rng, shape):
    omega = rng.uniform(0.05, 0.25, size=shape)
    y = (rng.uniform(size=shape) < 0.3).astype(np.float64)
    z = (y - 0.5) / omega
    return omega, y, z


def make_problem(n: int, p: int, rate_lo: float, rate_hi: float, *, seed: int,
                 tau=0.01, nrhs: int = 0, inflate_frac: float = 0.0,
                 tau_log10_range=None, with_c: bool = False) -> Problem:
    """One seeded problem in the recipe above.

    ``nrhs == 0`` gives a single chain with 1-D vectors; ``nrhs = R > 0``
    gives R chains sharing X.  ``tau_log10_range=(lo, hi)`` draws one tau per
    chain with log10 tau ~ U(lo, hi); otherwise ``tau`` is used for all.
    """
    rng = np.random.default_rng(seed)
    X = binary_design_from_rates(rng, n, column_rates(rng, p, rate_lo, rate_hi))
    shape_n = (nrhs, n) if nrhs else n
    shape_p = (nrhs, p) if nrhs else p
    omega, y, z = _obs_inputs(rng, shape_n)
    lam = _lambda_half_cauchy(rng, shape_p, inflate_frac)
    if tau_log10_range is not None:
        t = 10.0 ** rng.uniform(tau_log10_range[0], tau_log10_range[1], size=max(nrhs, 1))
        tau_v = t if nrhs else float(t[0])
    else:
        tau_v = np.full(nrhs, float(tau)) if nrhs else float(tau)
    eta = rng.standard_normal(size=shape_n)
    delta = rng.standard_normal(size=shape_p)
    c = rng.standard_normal(size=shape_p) if with_c else None
    return Problem(X=X, omega=omega, z=z, lam=lam, tau=tau_v, eta=eta, delta=delta, c=c, y=y)


# ---------------------------------------------------------------------------
# The five workloads.  Sizes and laws are those of the benchmark configurations;
# where a law is not stated the reading is given next to it.
# ---------------------------------------------------------------------------

def config1(seed_offset: int = 0) -> Problem:
    """FP64 single draw: n=2000, p=500, log10 r ~ U(-2.5,-1), tau=0.01."""
    return make_problem(2000, 500, -2.5, -1.0, seed=SEED_BASE + 1 + seed_offset, tau=0.01)


def config2(seed_offset: int = 0) -> Problem:
    """FP32 + FP64 reliable updates: n=1e5, p=1e4, log10 r ~ U(-4,-1.3),
    2% of lambda scaled by 100, tau=1e-3."""
    return make_problem(100_000, 10_000, -4.0, -1.3, seed=SEED_BASE + 2 + seed_offset,
                        tau=1e-3, inflate_frac=0.02)


def config3(nrhs: int = 16, n: int = 500_000, p: int = 50_000, seed_offset: int = 0) -> Problem:
    """16 chains sharing X: n=5e5, p=5e4, log10 r ~ U(-4.5,-1.5); lambda as in
    config2; per-chain log10 tau ~ U(-3.5,-2.5) (reading: the law is unstated,
    centred on config2's tau=1e-3)."""
    return make_problem(n, p, -4.5, -1.5, seed=SEED_BASE + 3 + seed_offset, nrhs=nrhs,
                        inflate_frac=0.02, tau_log10_range=(-3.5, -2.5))


def config4(nprob: int = 64, seed_offset: int = 0, n_range=(5_000, 200_000),
            p_range=(1_000, 30_000)) -> list:
    """Uneven batch: independent problems with n ~ logU(n_range),
    p ~ logU(p_range), log10 r ~ U(-4,-1.5), omega/lambda/tau as config1."""
    rng = np.random.default_rng(SEED_BASE + 4 + seed_offset)
    ns = np.exp(rng.uniform(math.log(n_range[0]), math.log(n_range[1]), nprob)).astype(np.int64)
    ps = np.exp(rng.uniform(math.log(p_range[0]), math.log(p_range[1]), nprob)).astype(np.int64)
    seeds = rng.integers(0, 2**31, nprob)
    return [make_problem(int(ns[q]), int(ps[q]), -4.0, -1.5, seed=int(seeds[q]), tau=0.01)
            for q in range(nprob)]


def config5(n: int = 200_000, p: int = 20_000, seed_offset: int = 0) -> Problem:
    """Adjoint: n=2e5, p=2e4, log10 r ~ U(-4,-1.8) (reading: mean density 0.31%),
    tau=1e-3, c ~ N(0, I_p)."""
    return make_problem(n, p, -4.0, -1.8, seed=SEED_BASE + 5 + seed_offset, tau=1e-3,
                        with_c=True)


def config5_small(seed_offset: int = 0) -> Problem:
    """The 2000 x 500 instance of the adjoint checks (config1's law, with c)."""
    return make_problem(2000, 500, -2.5, -1.0, seed=SEED_BASE + 15 + seed_offset, tau=0.01,
                        with_c=True)
