"""Parity of the single-RHS CUDA path with the CPU oracle (element by element
on the same seeded inputs), step by step: right-hand side (Eq. 2.3), the
matrix-free product (Sec. 1), CG at a fixed iteration count (Algorithm S1),
the stopped draw (Eq. S2), the refined and float32 modes, and edge cases.

Tolerances: float64 products are compared to a few ulps times the summation
length; draws to relative L2 1e-5 (refined) and 1e-3 (pure float32).
Iteration counts: within the window of tests/iteration_band.py, i.e. within 2
of the oracle's band at the same storage precision (compensated sums; the
inputs and one-ulp perturbations of them), the float32 modes within the
bracket described there."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_1810_12437_gb300 import inputs
from tests.gpu_helpers import T, dev, device_problem, need_gpu, rel
from tests.iteration_band import problem_window

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pb():
    need_gpu()
    import paper_1810_12437_gb300 as pb
    pb.load_library()
    return pb


@pytest.fixture(scope="module")
def cfg1():
    return inputs.config1()


@pytest.fixture(scope="module")
def cfg2():
    return inputs.config2()


def ragged():
    """Spans several tiles with a ragged tail: odd n, p, short and long rows."""
    return inputs.make_problem(3001, 777, -3.0, -0.7, seed=inputs.SEED_BASE + 50, tau=0.02)


# ------------------------------------------------------------------ a1: RHS
@pytest.mark.parametrize("which", ["cfg1", "ragged", "cfg2"])
def test_build_rhs_matches_oracle(pb, which, cfg1, cfg2):
    P = {"cfg1": cfg1, "cfg2": cfg2, "ragged": ragged()}[which]
    X, a = device_problem(P)
    ctx = pb.Context(precision="fp64")
    b = pb.pcg_build_rhs(ctx, X, a["omega"], a["z"], a["lam"], P.tau, a["eta"], a["delta"]).cpu().numpy()
    ref = O.build_b(P.X, P.omega, P.z, P.lam, P.tau, P.eta, P.delta)
    scale = O.xt_mul(P.X, np.abs(P.omega * P.z) + np.sqrt(P.omega) * np.abs(P.eta)) + np.abs(P.delta / (P.tau * P.lam))
    assert np.all(np.abs(b - ref) <= 1e-13 * scale + 1e-300)


# ------------------------------------------------------------------ a3 + a4: Phi v
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-13), ("df32", 1e-12), ("fx64", 1e-12),
                                      ("fp32_refined", 3e-6), ("fp32", 3e-6)])
def test_phi_mul_matches_oracle(pb, cfg2, prec, tol):
    P = cfg2
    X, a = device_problem(P)
    v = np.random.default_rng(2).standard_normal(P.X.p)
    ctx = pb.Context(precision=prec)
    out = pb.pcg_phi_mul(ctx, X, a["omega"], a["lam"], P.tau, T(v)).cpu().numpy()
    ref = O.phi_mul(P.X, P.omega, P.lam, P.tau, v)
    # elementwise against the magnitude of the summed terms
    mag = O.xt_mul(P.X, P.omega * O.x_mul(P.X, np.abs(v))) + np.abs(v) / (P.tau * P.lam) ** 2
    assert np.all(np.abs(out - ref) <= tol * mag)


def well_conditioned():
    """The config-1 design with moderate scales lambda ~ U(0.5, 2): CG
    iterates at a fixed k are then insensitive to rounding order, so the
    same-k comparison isolates the arithmetic."""
    P = inputs.config1()
    P.lam = np.random.default_rng(1).uniform(0.5, 2.0, P.X.p)
    P.tau = 0.05
    return P


# ------------------------------------------------------------------ a2, a5-a7: same-k CG
@pytest.mark.parametrize("prec", ["fp64", "df32", "fx64"])
@pytest.mark.parametrize("k", [1, 2, 5, 13, 30])
def test_fixed_iterations_fp64(pb, k, prec):
    P = well_conditioned()
    X, a = device_problem(P)
    ctx = pb.Context(precision=prec, stop_rule="relative")
    res = pb.pcg_draw_beta(ctx, X, a["omega"], a["z"], a["lam"], P.tau, a["eta"], a["delta"],
                           tol=0.0, max_iter=k)
    assert res.status == pb.PCG_MAXITER and res.iters == k
    ref = O.draw_beta_cg(P.X, P.omega, P.z, P.lam, P.tau, P.eta, P.delta, fixed_iters=k)[0]
    assert rel(res.beta.cpu().numpy(), ref) < 1e-11


@pytest.mark.parametrize("use_graph", [True, False])
def test_draw_fp64_config1(pb, cfg1, use_graph):
    """config 1: FP64, stop at relative preconditioned residual 1e-10."""
    P = cfg1
    X, a = device_problem(P)
    ctx = pb.Context(precision="fp64", stop_rule="relative", use_graph=use_graph)
    res = pb.pcg_draw_beta(ctx, X, a["omega"], a["z"], a["lam"], P.tau, a["eta"], a["delta"],
                           tol=1e-10, max_iter=2000)
    ref, k, r, st = O.draw_beta_cg(P.X, P.omega, P.z, P.lam, P.tau, P.eta, P.delta, tol=1e-10,
                                   stop_rule=O.STOP_RELATIVE)
    chol = O.draw_beta_chol(P.X, P.omega, P.z, P.lam, P.tau, P.eta, P.delta)
    assert res.status == pb.PCG_OK and st == O.OK
    assert abs(res.iters - k) <= 2
    assert res.resid <= 1e-10
    beta = res.beta.cpu().numpy()
    assert rel(beta, ref) < 1e-9
    assert rel(beta, chol) < 1e-8


def test_graph_and_plain_launches_agree_bitwise(pb, cfg2):
    P = cfg2
    X, a = device_problem(P)
    outs = []
    for g in (True, False, True):
        ctx = pb.Context(precision="fp32_refined", use_graph=g)
        res = pb.pcg_draw_beta(ctx, X, a["omega"], a["z"], a["lam"], P.tau, a["eta"], a["delta"],
                               tol=1e-6, max_iter=2000)
        outs.append((res.iters, res.beta.cpu().numpy()))
    assert outs[0][0] == outs[1][0] == outs[2][0]
    assert np.array_equal(outs[0][1], outs[1][1]) and np.array_equal(outs[0][1], outs[2][1])


@pytest.mark.parametrize("prec,bound", [("fp32_refined", 1e-5), ("fp32", 1e-3)])
def test_draw_config2(pb, cfg2, prec, bound):
    """config 2: float32 products with float64 scalars (and float64 reliable
    updates in the refined mode), paper RMS stop 1e-6."""
    P = cfg2
    X, a = device_problem(P)
    ctx = pb.Context(precision=prec, reliable_k=50)
    res = pb.pcg_draw_beta(ctx, X, a["omega"], a["z"], a["lam"], P.tau, a["eta"], a["delta"],
                           tol=1e-6, max_iter=5000)
    ref, k, r, st = O.draw_beta_cg(P.X, P.omega, P.z, P.lam, P.tau, P.eta, P.delta, tol=1e-6)
    assert res.status == pb.PCG_OK and st == O.OK
    w = problem_window(prec, P)
    assert w.holds(res.iters), (res.iters, str(w))
    beta = res.beta.cpu().numpy()
    # against the oracle stopped by the same rule
    assert rel(beta, ref) < bound
    # the reported stop quantity holds for the true residual in the refined mode
    if prec == "fp32_refined":
        b = O.build_b(P.X, P.omega, P.z, P.lam, P.tau, P.eta, P.delta)
        rt = P.tau * P.lam * (b - O.phi_mul(P.X, P.omega, P.lam, P.tau, beta))
        assert np.sqrt(np.mean(rt ** 2)) <= 1.5e-6


@pytest.mark.parametrize("prec", ["fp64", "df32", "fx64"])
def test_draw_config2_fp64(pb, cfg2, prec):
    """float64, double-float and fixed-point products: iteration counts within
    2 of the oracle's band at the same storage precision (config 2: float64
    [130, 135], float pairs [133, 138]; the plain oracle takes 143)."""
    P = cfg2
    X, a = device_problem(P)
    ctx = pb.Context(precision=prec)
    res = pb.pcg_draw_beta(ctx, X, a["omega"], a["z"], a["lam"], P.tau, a["eta"], a["delta"],
                           tol=1e-6, max_iter=5000)
    ref, k, r, st = O.draw_beta_cg(P.X, P.omega, P.z, P.lam, P.tau, P.eta, P.delta, tol=1e-6)
    w = problem_window(prec, P)
    assert res.status == pb.PCG_OK and w.holds(res.iters), (res.iters, str(w))
    assert rel(res.beta.cpu().numpy(), ref) < 1e-6


# ------------------------------------------------------------------ edge cases
def test_design_without_nonzeros(pb):
    P = inputs.make_problem(40, 30, -1, -0.5, seed=5, tau=0.1)
    P.X = inputs.design_from_dense(np.zeros((40, 30)))
    X, a = device_problem(P)
    for prec in ("fp64", "fp32_refined", "fp32"):
        ctx = pb.Context(precision=prec)
        res = pb.pcg_draw_beta(ctx, X, a["omega"], a["z"], a["lam"], P.tau, a["eta"], a["delta"],
                               tol=1e-12, max_iter=10)
        assert res.status == pb.PCG_OK and res.iters == 1
        assert rel(res.beta.cpu().numpy(), P.tau * P.lam * P.delta) < 1e-14


@pytest.mark.parametrize("k", [1, 4])
def test_thm22_low_rank(pb, k):
    """Theorem 2.2: n = k rows gives at most k + 1 iterations (k + 2 allowed
    in float32)."""
    rng = np.random.default_rng(300 + k)
    x = (rng.uniform(size=(k, 400)) < 0.3).astype(float)
    P = inputs.Problem(inputs.design_from_dense(x), rng.uniform(0.05, 0.25, k), rng.standard_normal(k),
                       rng.uniform(0.5, 2.0, 400), 0.3, rng.standard_normal(k), rng.standard_normal(400))
    X, a = device_problem(P)
    for prec, extra in (("fp64", 0), ("fp32_refined", 1)):
        ctx = pb.Context(precision=prec, stop_rule="relative")
        res = pb.pcg_draw_beta(ctx, X, a["omega"], a["z"], a["lam"], P.tau, a["eta"], a["delta"],
                               tol=1e-9 if prec == "fp64" else 1e-6, max_iter=50)
        assert res.status == pb.PCG_OK and res.iters <= k + 1 + extra


def test_empty_and_tiny_shapes(pb):
    # p = 0: nothing to draw
    X0 = pb.DeviceDesign(5, 0, torch.zeros(6, dtype=torch.int64, device=dev()),
                         torch.zeros(0, dtype=torch.int32, device=dev()),
                         torch.zeros(1, dtype=torch.int64, device=dev()),
                         torch.zeros(0, dtype=torch.int32, device=dev()))
    ctx = pb.Context(precision="fp64")
    e = torch.zeros(5, dtype=torch.float64, device=dev())
    e0 = torch.zeros(0, dtype=torch.float64, device=dev())
    res = pb.pcg_draw_beta(ctx, X0, e + 0.1, e, e0, 1.0, e, e0)
    assert res.status == pb.PCG_OK and res.iters == 0
    # n = 1, p = 1, single entry: Phi = omega + 1/(tau lambda)^2 exactly
    P = inputs.Problem(inputs.design_from_dense(np.ones((1, 1))), np.array([0.2]), np.array([1.5]),
                       np.array([2.0]), 0.5, np.array([0.3]), np.array([-0.7]))
    X, a = device_problem(P)
    res = pb.pcg_draw_beta(ctx, X, a["omega"], a["z"], a["lam"], P.tau, a["eta"], a["delta"],
                           tol=1e-14, max_iter=5)
    want = (0.2 * 1.5 + np.sqrt(0.2) * 0.3 - 0.7 / (0.5 * 2.0)) / (0.2 + 1.0)
    assert res.iters == 1 and abs(res.beta.item() - want) < 1e-15 * 4


def test_zero_max_iter_and_loose_tol(pb, cfg1):
    P = cfg1
    X, a = device_problem(P)
    ctx = pb.Context(precision="fp64")
    res = pb.pcg_draw_beta(ctx, X, a["omega"], a["z"], a["lam"], P.tau, a["eta"], a["delta"],
                           tol=1e-6, max_iter=0)
    assert res.status == pb.PCG_MAXITER and res.iters == 0 and float(res.beta.abs().max()) == 0.0
    res = pb.pcg_draw_beta(ctx, X, a["omega"], a["z"], a["lam"], P.tau, a["eta"], a["delta"],
                           tol=1e30, max_iter=10)
    assert res.status == pb.PCG_OK and res.iters == 0


def test_bad_arguments_rejected(pb, cfg1):
    P = cfg1
    X, a = device_problem(P)
    ctx = pb.Context(precision="fp64")
    with pytest.raises(pb.PcgError):
        pb.pcg_draw_beta(ctx, X, a["omega"], a["z"], a["lam"], -1.0, a["eta"], a["delta"])
    with pytest.raises(ValueError):
        pb.pcg_draw_beta(ctx, X, a["omega"][:-1], a["z"], a["lam"], P.tau, a["eta"], a["delta"])


def test_check_design(pb, cfg1):
    P = cfg1
    X, _ = device_problem(P)
    ctx = pb.Context(precision="fp64")
    assert pb.pcg_check_design(ctx, X) == pb.PCG_OK
    # a CSC that holds a different entry set: the first row of a column with
    # a free row below it moves down by one (the column stays sorted)
    ri = P.X.row_idx.copy()
    j = next(j for j in range(P.X.p) if P.X.col_ptr[j + 1] > P.X.col_ptr[j] and ri[P.X.col_ptr[j]] > 0)
    ri[P.X.col_ptr[j]] -= 1
    Xb = pb.DeviceDesign(X.n, X.p, X.row_ptr, X.col_idx, X.col_ptr,
                         torch.from_numpy(ri).to(dev()))
    assert pb.pcg_check_design(ctx, Xb) == pb.PCG_BADARG
    # out-of-range and unsorted indices
    oor = X.row_idx.clone()
    oor[-1] = X.n + 5
    assert pb.pcg_check_design(ctx, pb.DeviceDesign(X.n, X.p, X.row_ptr, X.col_idx, X.col_ptr, oor)) == pb.PCG_BADARG
    uns = X.col_idx.clone()
    r = int(np.argmax(np.diff(P.X.row_ptr) > 2))
    s = int(P.X.row_ptr[r])
    uns[s], uns[s + 1] = X.col_idx[s + 1], X.col_idx[s]
    assert pb.pcg_check_design(ctx, pb.DeviceDesign(X.n, X.p, X.row_ptr, uns, X.col_ptr, X.row_idx)) == pb.PCG_BADARG


def test_solve_is_draw_with_given_rhs(pb, cfg1):
    P = cfg1
    X, a = device_problem(P)
    ctx = pb.Context(precision="fp64", stop_rule="relative")
    b = O.build_b(P.X, P.omega, P.z, P.lam, P.tau, P.eta, P.delta)
    res = pb.pcg_solve(ctx, X, a["omega"], a["lam"], P.tau, T(b), tol=1e-12, max_iter=2000)
    assert res.status == pb.PCG_OK
    chol = O.draw_beta_chol(P.X, P.omega, P.z, P.lam, P.tau, P.eta, P.delta)
    assert rel(res.beta.cpu().numpy(), chol) < 1e-9


def test_repeat_calls_deterministic(pb, cfg2):
    P = cfg2
    X, a = device_problem(P)
    ctx = pb.Context(precision="fp32_refined")
    r1 = pb.pcg_draw_beta(ctx, X, a["omega"], a["z"], a["lam"], P.tau, a["eta"], a["delta"])
    b1 = r1.beta.clone()
    r2 = pb.pcg_draw_beta(ctx, X, a["omega"], a["z"], a["lam"], P.tau, a["eta"], a["delta"])
    assert r1.iters == r2.iters and torch.equal(b1, r2.beta)


def test_bank_order_changes_only_rounding(pb, monkeypatch):
    """The plan's bank-aware entry order permutes entries inside segments:
    at a fixed iteration count on a well-conditioned instance, draws with and
    without it agree to rounding (double-float and float32 products), and
    exactly with fixed-point products (integer sums do not depend on order)."""
    P = well_conditioned()
    X, a = device_problem(P)
    for prec, tol in (("df32", 1e-11), ("fp32", 1e-5), ("fx64", 0.0)):
        outs = []
        for flag in ("1", "0"):
            monkeypatch.setenv("PCG_BETA_BANK_PERMUTE", flag)
            ctx = pb.Context(precision=prec, reliable_k=0)
            r = pb.pcg_draw_beta(ctx, X, a["omega"], a["z"], a["lam"], P.tau, a["eta"], a["delta"],
                                 tol=0.0, max_iter=20)
            outs.append(r.beta.cpu().numpy())
        if tol == 0.0:
            assert np.array_equal(outs[0], outs[1]), prec
        else:
            assert rel(outs[0], outs[1]) < tol, prec


def test_plan_cache_follows_the_design_content(pb):
    """The tiled plan is built once per design and reused by later calls;
    writing a different design (the rows permuted: same sizes and nonzero
    count) into the same device buffers is seen by the plan's content hash,
    the plan is rebuilt, and the draw matches the oracle for the new design."""
    P = inputs.make_problem(4000, 500, -2.0, -1.0, seed=31, tau=0.05)
    P.lam = np.random.default_rng(4).uniform(0.5, 2.0, P.X.p)
    X, a = device_problem(P)
    ctx = pb.Context(precision="fp64", profile=True)
    args = (a["omega"], a["z"], a["lam"], P.tau, a["eta"], a["delta"])
    r1 = pb.pcg_draw_beta(ctx, X, *args, tol=1e-10, max_iter=3000)
    b1 = r1.beta.cpu().numpy()
    r2 = pb.pcg_draw_beta(ctx, X, *args, tol=1e-10, max_iter=3000)
    assert np.array_equal(b1, r2.beta.cpu().numpy())
    assert pb.profile_table(ctx)["plan_bounds"][1] == 2   # one plan (two sides) for both calls
    dense = np.zeros((P.X.n, P.X.p))
    for j in range(P.X.p):
        dense[P.X.row_idx[P.X.col_ptr[j]:P.X.col_ptr[j + 1]], j] = 1.0
    X2 = inputs.design_from_dense(dense[np.random.default_rng(5).permutation(P.X.n)])
    assert X2.nnz == P.X.nnz
    X.row_ptr.copy_(torch.from_numpy(X2.row_ptr))
    X.col_idx.copy_(torch.from_numpy(X2.col_idx))
    X.col_ptr.copy_(torch.from_numpy(X2.col_ptr))
    X.row_idx.copy_(torch.from_numpy(X2.row_idx))
    r3 = pb.pcg_draw_beta(ctx, X, *args, tol=1e-10, max_iter=3000)
    assert pb.profile_table(ctx)["plan_bounds"][1] == 4   # rebuilt for the new content
    ref = O.draw_beta_cg(X2, P.omega, P.z, P.lam, P.tau, P.eta, P.delta, tol=1e-10)[0]
    b3 = r3.beta.cpu().numpy()
    assert rel(b3, ref) < 1e-9
    assert rel(b3, b1) > 1e-3
