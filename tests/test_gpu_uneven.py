"""Parity of the uneven batch (independent problems of different n and p in
one persistent kernel) with the oracle run problem by problem."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_1810_12437_gb300 import inputs
from tests.gpu_helpers import T, dev, need_gpu, rel
from tests.iteration_band import problem_window

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pb():
    need_gpu()
    import paper_1810_12437_gb300 as pb
    pb.load_library()
    return pb


def as_device(pb, P):
    X = pb.DeviceDesign.from_host(P.X, dev())
    return dict(X=X, omega=T(P.omega), z=T(P.z), lam=T(P.lam), tau=float(P.tau), eta=T(P.eta),
                delta=T(P.delta))


def small_batch(seed=0):
    """The uneven recipe (log10 r ~ U(-4,-1.5), tau = 0.01) at sizes the oracle
    finishes in seconds, plus degenerate members."""
    probs = inputs.config4(nprob=10, seed_offset=seed, n_range=(400, 12_000), p_range=(60, 2_000))
    # a member without nonzeros and a member with a single row
    e = inputs.make_problem(300, 70, -2.0, -1.0, seed=77, tau=0.01)
    e.X = inputs.design_from_dense(np.zeros((300, 70)))
    one = inputs.make_problem(1, 50, -0.5, -0.2, seed=78, tau=0.01)
    return probs + [e, one]


# fx64 runs as double-float in the persistent kernel (float pairs, TwoSum)
@pytest.mark.parametrize("prec,bound", [("fp64", 1e-6), ("fp32_refined", 1e-5), ("df32", 1e-6), ("fx64", 1e-6),
                                        ("fp32", 1e-3)])
def test_uneven_matches_oracle(pb, prec, bound):
    probs = small_batch()
    ctx = pb.Context(precision=prec)
    res = pb.pcg_draw_beta_uneven(ctx, [as_device(pb, P) for P in probs], tol=1e-6, max_iter=20_000)
    mode = "df32" if prec == "fx64" else prec
    for q, (P, r) in enumerate(zip(probs, res)):
        ref, k, _, st = O.draw_beta_cg(P.X, P.omega, P.z, P.lam, P.tau, P.eta, P.delta, tol=1e-6)
        assert r.status == pb.PCG_OK and st == O.OK, q
        beta = r.beta.cpu().numpy()
        # counts within the window of the oracle's band at the same storage
        # precision; draws against the oracle stopped by the same rule
        w = problem_window(mode, P)
        assert w.holds(r.iters), (q, r.iters, str(w))
        assert rel(beta, ref) < bound, q


def test_uneven_matches_single_path(pb):
    probs = small_batch(seed=3)
    ctx = pb.Context(precision="fp32_refined")
    res = pb.pcg_draw_beta_uneven(ctx, [as_device(pb, P) for P in probs], tol=1e-6, max_iter=20_000)
    for P, r in zip(probs, res):
        d = as_device(pb, P)
        s = pb.pcg_draw_beta(ctx, d["X"], d["omega"], d["z"], d["lam"], d["tau"], d["eta"], d["delta"],
                             tol=1e-6, max_iter=20_000)
        assert abs(s.iters - r.iters) <= max(3, 0.3 * s.iters)
        assert rel(r.beta.cpu().numpy(), s.beta.cpu().numpy()) < 1e-5


def test_uneven_repeatable_and_cached_shape(pb, tmp_path):
    """The autotuned tile shape is cached (in memory and in the cache file)
    and results do not depend on scheduling: two runs agree bit for bit."""
    probs = small_batch(seed=5)
    cache = str(tmp_path / "tune.txt")
    ctx = pb.Context(precision="fp32_refined", autotune_cache=cache)
    d = [as_device(pb, P) for P in probs]
    r1 = pb.pcg_draw_beta_uneven(ctx, d, tol=1e-6, max_iter=20_000)
    b1 = [r.beta.clone() for r in r1]
    r2 = pb.pcg_draw_beta_uneven(ctx, d, tol=1e-6, max_iter=20_000)
    assert pb.pcg_last_kernel_launches(ctx) == 1
    for a, b, x, y in zip(b1, [r.beta for r in r2], r1, r2):
        assert x.iters == y.iters and torch.equal(a, b)
    lines = open(cache).read().split("\n")
    assert any(l.startswith("uneven:") for l in lines)
    ctx2 = pb.Context(precision="fp32_refined", autotune_cache=cache)
    r3 = pb.pcg_draw_beta_uneven(ctx2, d, tol=1e-6, max_iter=20_000)
    assert pb.pcg_last_kernel_launches(ctx2) == 1    # shape read from the file: no tuning runs
    for a, y in zip(b1, r3):
        assert torch.equal(a, y.beta)


def test_uneven_with_empty_member(pb):
    P = inputs.make_problem(500, 80, -2.0, -1.0, seed=9, tau=0.01)
    d = as_device(pb, P)
    e0 = torch.zeros(0, dtype=torch.float64, device=dev())
    X0 = pb.DeviceDesign(7, 0, torch.zeros(8, dtype=torch.int64, device=dev()),
                         torch.zeros(0, dtype=torch.int32, device=dev()),
                         torch.zeros(1, dtype=torch.int64, device=dev()),
                         torch.zeros(0, dtype=torch.int32, device=dev()))
    z7 = torch.zeros(7, dtype=torch.float64, device=dev())
    empty = dict(X=X0, omega=z7 + 0.1, z=z7, lam=e0, tau=0.01, eta=z7, delta=e0)
    ctx = pb.Context(precision="fp64")
    res = pb.pcg_draw_beta_uneven(ctx, [empty, d], tol=1e-6, max_iter=5000)
    assert res[0].status == pb.PCG_OK and res[0].iters == 0
    ref = O.draw_beta_cg(P.X, P.omega, P.z, P.lam, P.tau, P.eta, P.delta, tol=1e-6)[0]
    assert rel(res[1].beta.cpu().numpy(), ref) < 1e-9


@pytest.mark.slow
def test_uneven_config4_full(pb):
    """64 problems, n ~ logU[5e3, 2e5], p ~ logU[1e3, 3e4]: every problem
    meets the stop rule for its true residual (oracle, float64), and six of
    them (largest, smallest, spread) match the oracle's full draw."""
    probs = inputs.config4()
    ctx = pb.Context(precision="fp32_refined")
    res = pb.pcg_draw_beta_uneven(ctx, [as_device(pb, P) for P in probs], tol=1e-6, max_iter=20_000)
    sizes = np.array([P.X.nnz for P in probs])
    pick = set(np.argsort(sizes)[[0, 1, 20, 40, 62, 63]].tolist())
    for q, (P, r) in enumerate(zip(probs, res)):
        assert r.status == pb.PCG_OK, q
        beta = r.beta.cpu().numpy()
        b = O.build_b(P.X, P.omega, P.z, P.lam, P.tau, P.eta, P.delta)
        rt = P.tau * P.lam * (b - O.phi_mul(P.X, P.omega, P.lam, P.tau, beta))
        assert np.sqrt(np.mean(rt ** 2)) <= 1.5e-6, q
        if q in pick:
            ref, k, _, _ = O.draw_beta_cg(P.X, P.omega, P.z, P.lam, P.tau, P.eta, P.delta, tol=1e-6)
            w = problem_window("fp32_refined", P)
            assert w.holds(r.iters) and rel(beta, ref) < 1e-5, (q, r.iters, str(w))
