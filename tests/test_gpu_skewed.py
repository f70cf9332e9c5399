"""Tiled products on a design with strongly skewed segment lengths.

Rows and columns range from empty to thousands of entries, spread over
several column tiles and row strips at every group width.  This stresses
the parts of the plan that uniform designs leave quiet:
- rounds whose segments differ widely in length, so lanes read many pad chunks;
- the choice of lanes per segment, which then differs from warp to warp;
- the CSR pass's lane-major index copy, including its all-sentinel row;
- the last, narrower tile.

The products are compared with the oracle element by element (single RHS),
and the batched draw after a fixed number of CG iterations with the oracle's
fixed-iteration PCG per chain (group width 2)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1810_12437_gb300 import inputs
from tests.gpu_helpers import T, dev, need_gpu, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pb():
    need_gpu()
    import paper_1810_12437_gb300 as pb
    pb.load_library()
    return pb


def skewed_design(n=30_011, p=61_003, seed=7):
    """Row lengths from a heavy-tailed law (most rows short, 1 % of rows
    empty, a few rows with thousands of entries), and a few dense columns."""
    rng = np.random.default_rng(seed)
    lens = np.minimum(p, (rng.pareto(1.2, n) * 6).astype(np.int64))
    lens[rng.random(n) < 0.01] = 0
    rows = np.repeat(np.arange(n), lens)
    cols = np.concatenate([rng.choice(p, size=L, replace=False) if L else np.zeros(0, np.int64) for L in lens])
    dense = rng.choice(p, size=5, replace=False)   # five columns with a quarter of the rows each
    for j in dense:
        r = rng.choice(n, size=n // 4, replace=False)
        rows = np.concatenate([rows, r])
        cols = np.concatenate([cols, np.full(r.size, j)])
    key = np.unique(cols.astype(np.int64) * n + rows)   # dedupe; sorted by column, then row
    cols, rows = key // n, key % n
    col_ptr = np.zeros(p + 1, dtype=np.int64)
    np.cumsum(np.bincount(cols, minlength=p), out=col_ptr[1:])
    return inputs.design_from_csc(n, p, col_ptr, rows.astype(np.int32))


@pytest.fixture(scope="module")
def skewed():
    return skewed_design()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-13), ("df32", 1e-12), ("fx64", 1e-12), ("fp32", 3e-6)])
def test_phi_mul_on_skewed_segments(pb, skewed, prec, tol):
    Xh = skewed
    rng = np.random.default_rng(3)
    omega = rng.uniform(0.05, 0.25, Xh.n)
    lam = np.abs(rng.standard_cauchy(Xh.p)) + 1e-3
    tau, v = 0.01, rng.standard_normal(Xh.p)
    X = __import__("paper_1810_12437_gb300").DeviceDesign.from_host(Xh, dev())
    ctx = pb.Context(precision=prec)
    out = pb.pcg_phi_mul(ctx, X, T(omega), T(lam), tau, T(v)).cpu().numpy()
    ref = O.phi_mul(Xh, omega, lam, tau, v)
    mag = O.xt_mul(Xh, omega * O.x_mul(Xh, np.abs(v))) + np.abs(v) / (tau * lam) ** 2
    assert np.all(np.abs(out - ref) <= tol * mag)


@pytest.mark.parametrize("prec", ["df32", "fx64"])
def test_batched_fixed_iterations_on_skewed_segments(pb, skewed, prec, monkeypatch):
    """Four chains in groups of two (several column tiles at this p), three
    CG iterations: every chain's beta equals the oracle's three-iteration
    PCG iterate."""
    monkeypatch.setenv("PCG_BETA_BATCH_RG", "2")
    Xh = skewed
    rng = np.random.default_rng(11)
    R = 4
    omega = rng.uniform(0.05, 0.25, (R, Xh.n))
    z = rng.standard_normal((R, Xh.n))
    eta = rng.standard_normal((R, Xh.n))
    lam = rng.uniform(0.5, 2.0, (R, Xh.p))
    delta = rng.standard_normal((R, Xh.p))
    tau = np.full(R, 0.05)
    X = __import__("paper_1810_12437_gb300").DeviceDesign.from_host(Xh, dev())
    ctx = pb.Context(precision=prec, stop_rule="relative")
    res = pb.pcg_draw_beta_batched(ctx, X, T(omega), T(z), T(lam), T(tau), T(eta), T(delta), tol=0.0, max_iter=3)
    beta = res.beta.cpu().numpy()
    for r in range(R):
        ref = O.draw_beta_cg(Xh, omega[r], z[r], lam[r], float(tau[r]), eta[r], delta[r], fixed_iters=3)[0]
        assert res.iters[r] == 3
        assert rel(beta[r], ref) < 1e-9, r
