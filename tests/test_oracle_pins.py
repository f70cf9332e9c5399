"""Pins for the CPU oracle: checks against what the paper and the mathematics
fix, never against the oracle's own formulas retyped.

Each test names the passage it rests on.  Together they are chosen so that a
dropped term, a wrong sign or index, or a transposed operand anywhere in
``oracle/pcg_oracle.c`` fails at least one of them (``test_oracle_mutations``
plants such mistakes and checks exactly that).
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import oracle as O
from paper_1810_12437_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def golden_constants():
    vals = {}
    with open(os.path.join(GOLDEN, "paper_constants.txt")) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                k, v = line.split()[:2]
                vals[k] = float(v)
    return vals


def small_problem(n=60, p=20, lo=-1.0, hi=-0.3, seed=7, tau=0.05):
    """A tiny, well-conditioned instance of the input recipe."""
    return inputs.make_problem(n, p, lo, hi, seed=seed, tau=tau)


def dense_phi_numpy(P):
    """Phi from a dense copy of X (independent of the oracle's index loops)."""
    x = P.X.dense()
    return x.T @ (P.omega[:, None] * x) + np.diag(1.0 / (P.tau * P.lam) ** 2)


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300)


# --------------------------------------------------------------------------
# right-hand side (Prop. 2.1, Eq. 2.3)
# --------------------------------------------------------------------------

def test_b_design_without_nonzeros_is_prior_term():
    """X = 0 leaves only the third term of Eq. 2.3: b = delta / (tau lambda)."""
    P = small_problem()
    X0 = inputs.design_from_dense(np.zeros((P.X.n, P.X.p)))
    b = O.build_b(X0, P.omega, P.z, P.lam, P.tau, P.eta, P.delta)
    assert np.array_equal(b, P.delta / (P.tau * P.lam))


def test_b_single_row_by_hand():
    """n = 1, X = [1, 0, 1]: Eq. 2.3 evaluated by hand."""
    X = inputs.design_from_dense(np.array([[1.0, 0.0, 1.0]]))
    omega, z, eta = np.array([0.25]), np.array([2.0]), np.array([-1.0])
    lam, delta, tau = np.array([1.0, 2.0, 4.0]), np.array([0.5, 1.0, -2.0]), 0.5
    b = O.build_b(X, omega, z, lam, tau, eta, delta)
    # omega z = 0.5 ; sqrt(omega) eta = -0.5 ; delta/(tau lambda) = 1, 1, -1
    assert np.allclose(b, [0.5 - 0.5 + 1.0, 1.0, 0.5 - 0.5 - 1.0], rtol=0, atol=1e-15)


def test_b_moments_match_prop21():
    """Prop. 2.1: E[b] = X^T Omega z and Var(b) = Phi over fresh (eta, delta)."""
    P = inputs.make_problem(12, 5, -0.6, -0.2, seed=11, tau=0.7)
    phi = dense_phi_numpy(P)
    mean = P.X.dense().T @ (P.omega * P.z)
    rng = np.random.default_rng(5)
    N = 40_000
    bs = np.empty((N, P.X.p))
    for k in range(N):
        bs[k] = O.build_b(P.X, P.omega, P.z, P.lam, P.tau, rng.standard_normal(P.X.n),
                          rng.standard_normal(P.X.p))
    se_mean = np.sqrt(np.diag(phi) / N)
    assert np.all(np.abs(bs.mean(0) - mean) <= 5 * se_mean)
    cov = np.cov(bs.T)
    se_cov = np.sqrt((np.outer(np.diag(phi), np.diag(phi)) + phi ** 2) / N)
    assert np.all(np.abs(cov - phi) <= 6 * se_cov)


# --------------------------------------------------------------------------
# operator and direct path
# --------------------------------------------------------------------------

def test_phi_mul_equals_dense_phi_times_v():
    """Sec. 1: X^T (Omega (X v)) + tau^-2 Lambda^-2 v equals the formed Phi times v."""
    P = inputs.config1()
    phi = dense_phi_numpy(P)
    v = np.random.default_rng(3).standard_normal(P.X.p)
    assert rel(O.phi_mul(P.X, P.omega, P.lam, P.tau, v), phi @ v) < 1e-13


def test_xt_mul_is_transpose_of_x_mul():
    """<X v, w> = <v, X^T w> for the CSR and CSC walks of the same X."""
    P = inputs.config1()
    rng = np.random.default_rng(4)
    v, w = rng.standard_normal(P.X.p), rng.standard_normal(P.X.n)
    lhs = O.x_mul(P.X, v) @ w
    rhs = v @ O.xt_mul(P.X, w)
    assert abs(lhs - rhs) <= 1e-11 * (abs(lhs) + 1)
    x = P.X.dense()
    assert rel(O.x_mul(P.X, v), x @ v) < 1e-14
    assert rel(O.xt_mul(P.X, w), x.T @ w) < 1e-14


def test_dense_phi_matches_numpy():
    """Eq. 1.2 formed from index loops equals the dense-matrix product."""
    P = inputs.config1()
    assert rel(O.dense_phi(P.X, P.omega, P.lam, P.tau), dense_phi_numpy(P)) < 1e-14


def test_cholesky_and_solve_match_lapack():
    """The hand-written factorisation agrees with LAPACK's (numpy)."""
    P = inputs.config1()
    phi = dense_phi_numpy(P)
    l = O.cholesky(phi)
    assert rel(l, np.linalg.cholesky(phi)) < 1e-12
    b = np.random.default_rng(8).standard_normal(P.X.p)
    assert rel(O.chol_solve(l, b), np.linalg.solve(phi, b)) < 1e-9


@pytest.mark.parametrize("cfg", ["small", "config1"])
def test_direct_draw_equals_least_squares(cfg):
    """Sec. S7.1, Eq. S6: beta solves min || X~ beta - b~ || with
    X~ = [Omega^1/2 X ; tau^-1 Lambda^-1] and b~ = [Omega^1/2 z + eta ; delta].
    numpy's SVD least squares never forms Phi or b, so this pins the right-hand
    side, the formed Phi and the Cholesky solve together."""
    P = small_problem() if cfg == "small" else inputs.config1()
    x = P.X.dense()
    sw = np.sqrt(P.omega)
    xt = np.vstack([sw[:, None] * x, np.diag(1.0 / (P.tau * P.lam))])
    bt = np.concatenate([sw * P.z + P.eta, P.delta])
    ref = np.linalg.lstsq(xt, bt, rcond=None)[0]
    beta = O.draw_beta_chol(P.X, P.omega, P.z, P.lam, P.tau, P.eta, P.delta)
    assert rel(beta, ref) < 1e-8


def test_tiny_exact_rational_draw():
    """Brute force in exact rational arithmetic on a 3 x 2 design."""
    xs = [[1, 0], [1, 1], [0, 1]]
    om = [Fraction(1, 4), Fraction(1, 9), Fraction(1, 16)]
    sq = [Fraction(1, 2), Fraction(1, 3), Fraction(1, 4)]
    z = [Fraction(2), Fraction(-3), Fraction(5)]
    eta = [Fraction(1), Fraction(-2), Fraction(3)]
    tau, lam = Fraction(1, 2), [Fraction(1), Fraction(2)]
    delta = [Fraction(3), Fraction(-1)]
    phi = [[sum(xs[i][a] * om[i] * xs[i][c] for i in range(3)) + (1 / (tau * lam[a]) ** 2 if a == c else 0)
            for c in range(2)] for a in range(2)]
    b = [sum(xs[i][a] * (om[i] * z[i] + sq[i] * eta[i]) for i in range(3)) + delta[a] / (tau * lam[a])
         for a in range(2)]
    det = phi[0][0] * phi[1][1] - phi[0][1] * phi[1][0]
    exact = [(phi[1][1] * b[0] - phi[0][1] * b[1]) / det, (phi[0][0] * b[1] - phi[1][0] * b[0]) / det]
    X = inputs.design_from_dense(np.array(xs, dtype=float))
    args = (X, np.array([float(v) for v in om]), np.array([float(v) for v in z]),
            np.array([float(v) for v in lam]), float(tau), np.array([float(v) for v in eta]),
            np.array([float(v) for v in delta]))
    want = np.array([float(v) for v in exact])
    assert rel(O.draw_beta_chol(*args), want) < 1e-15
    beta_cg, k, _, st = O.draw_beta_cg(*args, tol=1e-14, stop_rule=O.STOP_RELATIVE)
    assert st == O.OK and k <= 2 and rel(beta_cg, want) < 1e-14


# --------------------------------------------------------------------------
# conjugate gradient (Sec. 2.2-2.5, Algorithm S1, Eq. S2)
# --------------------------------------------------------------------------

def test_cg_matches_cholesky_config1():
    """CG at relative 1e-10 reproduces the direct solution (Sec. 2.2)."""
    P = inputs.config1()
    ref = O.draw_beta_chol(P.X, P.omega, P.z, P.lam, P.tau, P.eta, P.delta)
    beta, k, res, st = O.draw_beta_cg(P.X, P.omega, P.z, P.lam, P.tau, P.eta, P.delta,
                                      tol=1e-10, stop_rule=O.STOP_RELATIVE)
    assert st == O.OK and res <= 1e-10 and 0 < k < P.X.p
    assert rel(beta, ref) < 1e-8


def test_cg_exact_after_p_iterations():
    """Sec. 2.2: CG is exact after p iterations (p = 20)."""
    P = small_problem(n=60, p=20)
    ref = O.draw_beta_chol(P.X, P.omega, P.z, P.lam, P.tau, P.eta, P.delta)
    beta = O.draw_beta_cg(P.X, P.omega, P.z, P.lam, P.tau, P.eta, P.delta, fixed_iters=20)[0]
    assert rel(beta, ref) < 1e-10


@pytest.mark.parametrize("k", [1, 3, 7])
def test_thm22_low_rank_converges_in_k_plus_1(k):
    """Theorem 2.2: with n = k rows, Phi~ = I + (rank k), so it has at most
    k + 1 distinct eigenvalues and PCG is exact within k + 1 iterations."""
    rng = np.random.default_rng(100 + k)
    x = (rng.uniform(size=(k, 300)) < 0.3).astype(float)
    X = inputs.design_from_dense(x)
    omega = rng.uniform(0.05, 0.25, k)
    # moderate scales keep rounding far below the exact-termination drop
    lam = rng.uniform(0.5, 2.0, 300)
    tau = 0.3
    z, eta, delta = rng.standard_normal(k), rng.standard_normal(k), rng.standard_normal(300)
    ref = O.draw_beta_chol(X, omega, z, lam, tau, eta, delta)
    beta, iters, res, st = O.draw_beta_cg(X, omega, z, lam, tau, eta, delta, tol=1e-9,
                                          stop_rule=O.STOP_RELATIVE)
    # a generic b touches every eigenvector, so the count is exactly k + 1
    assert st == O.OK and iters == k + 1
    assert rel(beta, ref) < 1e-9


def test_design_without_nonzeros_one_iteration():
    """X = 0 gives Phi = M, Phi~ = I: one iteration, beta = M^-1 b = tau lambda delta."""
    P = small_problem(n=40, p=30)
    X0 = inputs.design_from_dense(np.zeros((40, 30)))
    beta, k, res, st = O.draw_beta_cg(X0, P.omega, P.z, P.lam, P.tau, P.eta, P.delta, tol=1e-12)
    assert st == O.OK and k == 1
    assert rel(beta, P.tau * P.lam * P.delta) < 1e-14


def test_rho_is_true_preconditioned_residual():
    """Sec. S4.2: rho_k = ||tau lambda (.) (b - Phi beta_k)||^2, with the
    residual recomputed from the formed Phi at every k."""
    P = inputs.config1()
    phi = dense_phi_numpy(P)
    b = O.build_b(P.X, P.omega, P.z, P.lam, P.tau, P.eta, P.delta)
    _, K, _, _, hist = O.pcg(P.X, P.omega, P.lam, P.tau, b, tol=1e-10,
                             stop_rule=O.STOP_RELATIVE, want_hist=True)
    for k in range(0, K + 1, max(1, K // 6)):
        bk = O.pcg(P.X, P.omega, P.lam, P.tau, b, fixed_iters=k)[0] if k else np.zeros(P.X.p)
        true = np.sum((P.tau * P.lam * (b - phi @ bk)) ** 2)
        assert abs(hist[k] - true) <= 1e-6 * true + 1e-22 * hist[0]


def test_stop_rule_rms_is_first_crossing():
    """Eq. S2: stop at the first k with p^-1/2 ||r~_k|| <= tol."""
    P = inputs.config1()
    b = O.build_b(P.X, P.omega, P.z, P.lam, P.tau, P.eta, P.delta)
    tol = 1e-6
    beta, k, res, st, hist = O.pcg(P.X, P.omega, P.lam, P.tau, b, tol=tol, want_hist=True)
    rms = np.sqrt(hist / P.X.p)
    assert st == O.OK and rms[k] <= tol and np.all(rms[:k] > tol)
    assert res == pytest.approx(rms[k], rel=1e-15)


def test_maxiter_status():
    P = inputs.config1()
    _, k, _, st = O.draw_beta_cg(P.X, P.omega, P.z, P.lam, P.tau, P.eta, P.delta,
                                 tol=1e-14, max_iter=3)
    assert st == O.MAXITER and k == 3


def test_thm23_eigenvalue_bounds():
    """Theorem 2.3: 1 <= nu_k(Phi~) <= 1 + tau^2 lambda_(k)^2 nu_1(X^T Omega X)."""
    P = inputs.config1()
    phi = O.dense_phi(P.X, P.omega, P.lam, P.tau)
    t = P.tau * P.lam
    phit = t[:, None] * phi * t[None, :]
    nu = np.sort(np.linalg.eigvalsh(phit))[::-1]
    x = P.X.dense()
    nu1 = np.linalg.eigvalsh(x.T @ (P.omega[:, None] * x)).max()
    lam_sorted = np.sort(P.lam)[::-1]
    upper = 1 + P.tau ** 2 * lam_sorted ** 2 * nu1
    assert np.all(nu >= 1 - 1e-9)
    assert np.all(nu <= upper * (1 + 1e-9))


def test_thm21_error_bound_and_monotone_phi_norm_error():
    """Theorem 2.1 applied to the preconditioned system (Sec. 2.4) and the
    optimality property of Sec. 2.2: ||beta_k - beta||_Phi decreases
    monotonically and stays below 2 ((sqrt k~ - 1)/(sqrt k~ + 1))^k."""
    P = small_problem(n=80, p=40, seed=21)
    phi = dense_phi_numpy(P)
    t = P.tau * P.lam
    ev = np.linalg.eigvalsh(t[:, None] * phi * t[None, :])
    kap = ev.max() / ev.min()
    q = (math.sqrt(kap) - 1) / (math.sqrt(kap) + 1)
    b = O.build_b(P.X, P.omega, P.z, P.lam, P.tau, P.eta, P.delta)
    star = np.linalg.solve(phi, b)

    def phinorm(e):
        return math.sqrt(e @ phi @ e)

    e0 = phinorm(star)
    prev = e0
    for k in range(1, 25):
        bk = O.pcg(P.X, P.omega, P.lam, P.tau, b, fixed_iters=k)[0]
        ek = phinorm(bk - star)
        assert ek <= 2 * q ** k * e0 * (1 + 1e-9) + 1e-12 * e0
        assert ek <= prev * (1 + 1e-9) + 1e-13 * e0
        prev = ek


def test_thm24_printed_constant():
    """Sec. 2.5: kappa~ = 1 + 100 gives log10 factor about -0.0867 <= -0.086,
    and 100 further iterations reduce the error by 2 * 10^-8.67 ~ 10^-8.3."""
    g = golden_constants()
    kap = 101.0
    f = math.log10((math.sqrt(kap) - 1) / (math.sqrt(kap) + 1))
    assert f <= g["thm24_log10_factor_bound"]
    assert abs(f - (-0.0867)) < 5e-4
    assert abs(math.log10(2) + 100 * g["thm24_log10_factor_bound"] - g["thm24_reduction_after_100_log10"]) < 0.05


def test_sampler_distribution():
    """Prop. 2.1 end to end: beta ~ N(Phi^-1 X^T Omega z, Phi^-1).  With
    Phi = L L^T, xi = L^T (beta - mu) must be N(0, I)."""
    P = inputs.make_problem(200, 20, -1.3, -0.5, seed=31, tau=0.2)
    phi = dense_phi_numpy(P)
    L = np.linalg.cholesky(phi)
    mu = np.linalg.solve(phi, P.X.dense().T @ (P.omega * P.z))
    rng = np.random.default_rng(9)
    N = 40_000
    xi = np.empty((N, P.X.p))
    for k in range(N):
        beta = O.draw_beta_cg(P.X, P.omega, P.z, P.lam, P.tau, rng.standard_normal(P.X.n),
                              rng.standard_normal(P.X.p), tol=1e-12,
                              stop_rule=O.STOP_RELATIVE)[0]
        xi[k] = L.T @ (beta - mu)
    assert np.all(np.abs(xi.mean(0)) <= 5 / math.sqrt(N))
    assert np.all(np.abs(xi.var(0) - 1) <= 5 * math.sqrt(2 / N))
    c = np.cov(xi.T) - np.eye(P.X.p)
    assert np.abs(c).max() <= 6 / math.sqrt(N)


# --------------------------------------------------------------------------
# adjoint (not in the paper: implicit differentiation of beta = Phi^-1 b)
# --------------------------------------------------------------------------

def _loss_chol(X, omega, z, lam, tau, eta, delta, c):
    return c @ O.draw_beta_chol(X, omega, z, lam, tau, eta, delta)


@pytest.mark.parametrize("mode", ["draw", "solve"])
def test_adjoint_matches_central_differences(mode):
    """Gradient of L = c^T beta against central differences (h = 1e-6, FP64)."""
    P = inputs.make_problem(120, 40, -1.3, -0.5, seed=41, tau=0.1, with_c=True)
    X = P.X
    beta, g = O.adjoint_chol(X, P.omega, P.z, P.lam, P.tau, P.eta, P.delta, P.c, mode=mode)
    b0 = O.build_b(X, P.omega, P.z, P.lam, P.tau, P.eta, P.delta)
    h = 1e-6

    def loss(omega=P.omega, lam=P.lam, tau=P.tau, b=None):
        if mode == "draw":
            return _loss_chol(X, omega, P.z, lam, tau, P.eta, P.delta, P.c)
        # solve mode: b held fixed while Phi moves
        l = O.cholesky(dense_phi_numpy(inputs.Problem(X, omega, P.z, lam, tau, P.eta, P.delta)))
        return P.c @ O.chol_solve(l, b0 if b is None else b)

    for j in [0, 7, 23, 39]:
        e = np.zeros(X.p)
        e[j] = h
        fd = (loss(lam=P.lam * np.exp(e)) - loss(lam=P.lam * np.exp(-e))) / (2 * h)
        assert fd == pytest.approx(g["log_lambda"][j], rel=1e-5, abs=1e-7 * (abs(fd) + 1))
    fd = (loss(tau=P.tau * math.exp(h)) - loss(tau=P.tau * math.exp(-h))) / (2 * h)
    assert fd == pytest.approx(g["log_tau"], rel=1e-5, abs=1e-8)
    for i in [0, 33, 119]:
        e = np.zeros(X.n)
        e[i] = h
        fd = (loss(omega=P.omega + e) - loss(omega=P.omega - e)) / (2 * h)
        assert fd == pytest.approx(g["omega"][i], rel=1e-5, abs=1e-7 * (abs(fd) + 1))
    if mode == "solve":
        for j in [3, 17]:
            # L is linear in b: a unit step is exact and free of cancellation
            e = np.zeros(X.p)
            e[j] = 1.0
            fd = (loss(b=b0 + e) - loss(b=b0 - e)) / 2.0
            assert fd == pytest.approx(g["b"][j], rel=1e-6)


def test_adjoint_symmetry_and_cg_agree_with_cholesky():
    """dL/db = Phi^-1 c is the draw with b := c (Phi symmetric); the CG and
    Cholesky gradients agree on the 2000 x 500 instance."""
    P = inputs.config5_small()
    X = P.X
    beta_c, gc = O.adjoint_chol(X, P.omega, P.z, P.lam, P.tau, P.eta, P.delta, P.c)
    beta_g, gg = O.adjoint_cg(X, P.omega, P.z, P.lam, P.tau, P.eta, P.delta, P.c, tol=1e-13,
                              stop_rule=O.STOP_RELATIVE)
    sol_c = O.pcg(X, P.omega, P.lam, P.tau, P.c, tol=1e-13, stop_rule=O.STOP_RELATIVE)[0]
    assert rel(gc["b"], sol_c) < 1e-9
    for key in ("b", "omega", "log_lambda"):
        assert rel(gg[key], gc[key]) < 1e-8, key
    assert gg["log_tau"] == pytest.approx(gc["log_tau"], rel=1e-8)


# --------------------------------------------------------------------------
# unshrunk coefficients (Sec. S4.3)
# --------------------------------------------------------------------------
def test_unshrunk_reduces_to_shrunk_when_scales_match():
    """Sec. S4.3 with sigma_j^-2 = tau^-2 lambda_j^-2 and gamma_j = tau lambda_j
    is the shrinkage model: the draw, the right-hand side and the CG path (its
    iteration count) equal the C oracle's."""
    P = small_problem(n=80, p=24, seed=11)
    q1 = 5
    prec = 1.0 / (P.tau * P.lam[:q1]) ** 2
    gam = P.tau * P.lam[:q1]
    b = O.build_b_unshrunk(P.X, P.omega, P.z, P.lam, P.tau, P.eta, P.delta, prec)
    assert rel(b, O.build_b(P.X, P.omega, P.z, P.lam, P.tau, P.eta, P.delta)) < 1e-13
    beta = O.draw_beta_chol_unshrunk(P.X, P.omega, P.z, P.lam, P.tau, P.eta, P.delta, prec)
    assert rel(beta, O.draw_beta_chol(P.X, P.omega, P.z, P.lam, P.tau, P.eta, P.delta)) < 1e-11
    ref, k, _, _ = O.pcg(P.X, P.omega, P.lam, P.tau, b, tol=1e-10)
    got, k2, _, st = O.pcg_unshrunk(P.X, P.omega, P.lam, P.tau, b, prec, gam, tol=1e-10)
    assert st == O.OK and k2 == k and rel(got, ref) < 1e-10


def test_unshrunk_flat_prior_intercept_closed_form():
    """An intercept-only model (X a column of ones) under the flat prior of
    Sec. S4.3 (sigma = infinity): Phi = sum_i omega_i and
    b = sum_i (omega_i z_i + omega_i^1/2 eta_i), so beta = b / Phi."""
    rng = np.random.default_rng(3)
    n = 500
    X = inputs.design_from_dense(np.ones((n, 1)))
    om = rng.uniform(0.05, 0.25, n)
    z = rng.standard_normal(n) / om
    eta = rng.standard_normal(n)
    want = (om @ z + np.sqrt(om) @ eta) / om.sum()
    lam, delta = np.ones(1), rng.standard_normal(1)   # lambda, delta unused for an unshrunk flat coefficient
    got = O.draw_beta_chol_unshrunk(X, om, z, lam, 0.1, eta, delta, [0.0])
    assert abs(got[0] - want) <= 1e-12 * abs(want)
    b = O.build_b_unshrunk(X, om, z, lam, 0.1, eta, delta, [0.0])
    beta, k, _, st = O.pcg_unshrunk(X, om, lam, 0.1, b, [0.0], [1.0], tol=1e-12)
    assert st == O.OK and k == 1 and abs(beta[0] - want) <= 1e-12 * abs(want)


def test_unshrunk_cg_matches_cholesky_and_ignores_gamma():
    """With an intercept column, a flat and two proper unshrunk priors: the
    PCG solution equals the Cholesky draw, and the preconditioner scales gamma
    (Sec. S4.3) change the path but not the solution."""
    P = small_problem(n=120, p=30, seed=5)
    dense = P.X.dense()
    dense[:, 0] = 1.0
    P.X = inputs.design_from_dense(dense)
    prec = np.array([0.0, 0.01, 4.0])
    ref = O.draw_beta_chol_unshrunk(P.X, P.omega, P.z, P.lam, P.tau, P.eta, P.delta, prec)
    b = O.build_b_unshrunk(P.X, P.omega, P.z, P.lam, P.tau, P.eta, P.delta, prec)
    for gam in ([1.0, 1.0, 1.0], [100.0, 0.01, 3.0]):
        beta, k, _, st = O.pcg_unshrunk(P.X, P.omega, P.lam, P.tau, b, prec, gam, tol=1e-12,
                                        stop_rule=O.STOP_RELATIVE)
        assert st == O.OK
        assert rel(beta, ref) < 1e-9


# --------------------------------------------------------------------------
# compensated sums: the same sums, accumulated more accurately
# --------------------------------------------------------------------------

def test_compensated_sums_match_correctly_rounded_sums():
    """Neumaier's compensated summation returns the exactly rounded sum
    (math.fsum) on sums whose plain left-to-right value is wrong by whole
    units: one row / column holding 1e16, 1, -1e16, 1, ... and random rows of
    config 1 (within one unit in the last place of the exact sum)."""
    big = np.array([1e16, 1.0, -1e16, 1.0, 3.0, 1e16, -1e16, 0.5])
    X = inputs.design_from_dense(np.ones((1, big.size)))
    want = math.fsum(big)
    assert O.x_mul(X, big)[0] != want                     # plain sums lose the small terms
    assert O.x_mul_comp(X, big)[0] == want
    assert O.xt_mul_comp(inputs.design_from_dense(np.ones((big.size, 1))), big)[0] == want
    assert O.dot_comp(big, np.ones_like(big)) == want
    P = inputs.config1()
    rng = np.random.default_rng(8)
    v = rng.standard_normal(P.X.p) * 10.0 ** rng.uniform(-8, 8, P.X.p)
    w = rng.standard_normal(P.X.n) * 10.0 ** rng.uniform(-8, 8, P.X.n)
    x = P.X.dense()
    exact_r = np.array([math.fsum(v[x[i] > 0]) for i in range(P.X.n)])
    exact_c = np.array([math.fsum(w[x[:, j] > 0]) for j in range(P.X.p)])
    assert np.all(np.abs(O.x_mul_comp(P.X, v) - exact_r) <= np.spacing(np.abs(exact_r)))
    assert np.all(np.abs(O.xt_mul_comp(P.X, w) - exact_c) <= np.spacing(np.abs(exact_c)))
    prods = v * v[::-1]
    assert abs(O.dot_comp(v, v[::-1]) - math.fsum(prods)) <= np.spacing(abs(math.fsum(prods)))


def test_compensated_cg_is_the_same_algorithm():
    """The compensated mode changes only rounding: on config 1 (well enough
    conditioned that iterates do not amplify rounding) it takes the plain
    mode's iteration count and reaches the same beta, equal to Cholesky's."""
    P = inputs.config1()
    b = O.build_b(P.X, P.omega, P.z, P.lam, P.tau, P.eta, P.delta)
    plain = O.pcg(P.X, P.omega, P.lam, P.tau, b, tol=1e-10, stop_rule=O.STOP_RELATIVE)
    comp = O.pcg(P.X, P.omega, P.lam, P.tau, b, tol=1e-10, stop_rule=O.STOP_RELATIVE,
                 sums="compensated")
    chol = O.draw_beta_chol(P.X, P.omega, P.z, P.lam, P.tau, P.eta, P.delta)
    assert comp[3] == O.OK and comp[1] == plain[1]
    assert rel(comp[0], plain[0]) < 1e-11 and rel(comp[0], chol) < 1e-8


# --------------------------------------------------------------------------
# status branches (Sec. 2.4: Phi is SPD in exact arithmetic, so a
# non-positive curvature or a non-finite scalar is a reported failure)
# --------------------------------------------------------------------------

def _one_row_problem(omega0):
    """X = one row of ones (p = 6): Phi = omega_0 1 1^T + diag(d), which is
    indefinite once omega_0 < -min(d) / p."""
    p = 6
    X = inputs.design_from_dense(np.ones((1, p)))
    lam = np.linspace(0.5, 1.5, p)
    return X, np.array([omega0]), lam, 1.0


def test_breakdown_on_indefinite_phi():
    """omega_0 = -1e6 makes s . Phi s < 0 for the first direction s = M^-1 b
    with b = 1: the oracle stops before any product is applied to beta."""
    X, omega, lam, tau = _one_row_problem(-1e6)
    b = np.ones(X.p)
    s = (tau * lam) ** 2 * b
    phi = omega[0] * np.ones((X.p, X.p)) + np.diag(1.0 / (tau * lam) ** 2)
    assert s @ phi @ s < 0
    for sums in ("plain", "compensated"):
        beta, k, _, st = O.pcg(X, omega, lam, tau, b, tol=1e-12, sums=sums)
        assert st == O.BREAKDOWN and k == 0 and np.all(beta == 0.0)
    # the same matrix with omega_0 > 0 is SPD: no breakdown, solution by numpy
    X, omega, lam, tau = _one_row_problem(0.2)
    beta, k, _, st = O.pcg(X, omega, lam, tau, b, tol=1e-13, stop_rule=O.STOP_RELATIVE)
    phi = 0.2 * np.ones((X.p, X.p)) + np.diag(1.0 / (tau * lam) ** 2)
    assert st == O.OK and rel(beta, np.linalg.solve(phi, b)) < 1e-12


def test_nonfinite_inputs_reported():
    """A NaN in delta makes b, and so rho_0, NaN: NONFINITE before the first
    product.  An infinite omega makes the first curvature s . Phi s infinite:
    NONFINITE at the first product, beta still beta_0 = 0."""
    P = small_problem()
    delta = P.delta.copy()
    delta[3] = np.nan
    b = O.build_b(P.X, P.omega, P.z, P.lam, P.tau, P.eta, delta)
    assert np.isnan(b[3])
    beta, k, _, st = O.pcg(P.X, P.omega, P.lam, P.tau, b)
    assert st == O.NONFINITE and k == 0
    omega = P.omega.copy()
    omega[int(np.argmax(np.diff(P.X.row_ptr)))] = np.inf
    b = O.build_b(P.X, P.omega, P.z, P.lam, P.tau, P.eta, P.delta)
    for sums in ("plain", "compensated"):
        beta, k, _, st = O.pcg(P.X, omega, P.lam, P.tau, b, sums=sums)
        assert st == O.NONFINITE and k == 0 and np.all(beta == 0.0)


# --------------------------------------------------------------------------
# Jacobi preconditioner (Sec. 2.4, Sec. 3) and initial vectors (Sec. S4.1)
# --------------------------------------------------------------------------

def test_phi_diag_is_diagonal_of_dense_phi():
    """Sec. 2.4's Jacobi M = diag(Phi_11 .. Phi_pp) equals the formed Phi's diagonal."""
    for P in (inputs.config1(), small_problem()):
        assert rel(O.phi_diag(P.X, P.omega, P.lam, P.tau), np.diag(dense_phi_numpy(P))) < 1e-15


def test_jacobi_pcg_reaches_the_cholesky_solution():
    """PCG with M^-1 = 1 / diag(Phi) solves the same system (config 1, relative
    stop 1e-12 on the prior-preconditioned residual of Eq. S2)."""
    P = inputs.config1()
    b = O.build_b(P.X, P.omega, P.z, P.lam, P.tau, P.eta, P.delta)
    minv = 1.0 / O.phi_diag(P.X, P.omega, P.lam, P.tau)
    chol = O.draw_beta_chol(P.X, P.omega, P.z, P.lam, P.tau, P.eta, P.delta)
    beta, k, res, st = O.pcg(P.X, P.omega, P.lam, P.tau, b, tol=1e-12,
                             stop_rule=O.STOP_RELATIVE, minv=minv)
    assert st == O.OK and 0 < k < P.X.p and res <= 1e-12
    assert rel(beta, chol) < 1e-9
    # the reported stop quantity is the prior-preconditioned norm of the true residual
    rt = P.tau * P.lam * (b - O.phi_mul(P.X, P.omega, P.lam, P.tau, beta))
    rb = P.tau * P.lam * b
    assert abs(np.linalg.norm(rt) / np.linalg.norm(rb) - res) <= 1e-3 * res + 1e-15


def test_jacobi_is_prior_preconditioner_without_data():
    """With X = 0, diag(Phi) = tau^-2 lambda^-2 = M: the Jacobi and prior
    preconditioners coincide, and both solve in one iteration (Thm 2.2, k = 0)."""
    P = small_problem()
    X0 = inputs.design_from_dense(np.zeros((P.X.n, P.X.p)))
    b = O.build_b(X0, P.omega, P.z, P.lam, P.tau, P.eta, P.delta)
    minv = 1.0 / O.phi_diag(X0, P.omega, P.lam, P.tau)
    prior = O.pcg(X0, P.omega, P.lam, P.tau, b, tol=1e-14)
    jac = O.pcg(X0, P.omega, P.lam, P.tau, b, tol=1e-14, minv=minv)
    assert prior[1] == jac[1] == 1
    assert rel(jac[0], (P.tau * P.lam) ** 2 * b) < 1e-15 and rel(jac[0], prior[0]) < 1e-15


def test_warm_start():
    """Sec. S4.1: an initial vector beta_0 gives r_0 = b - Phi beta_0.
    beta_0 = 0 is the default exactly; beta_0 at the solution stops before any
    product; beta_0 = an early iterate is refined to the Cholesky solution, and
    its first stop quantity is the norm of b - Phi beta_0."""
    P = inputs.config1()
    b = O.build_b(P.X, P.omega, P.z, P.lam, P.tau, P.eta, P.delta)
    base = O.pcg(P.X, P.omega, P.lam, P.tau, b, tol=1e-10, stop_rule=O.STOP_RELATIVE)
    zero = O.pcg(P.X, P.omega, P.lam, P.tau, b, tol=1e-10, stop_rule=O.STOP_RELATIVE,
                 beta0=np.zeros(P.X.p))
    assert zero[1] == base[1] and np.array_equal(zero[0], base[0])
    chol = O.draw_beta_chol(P.X, P.omega, P.z, P.lam, P.tau, P.eta, P.delta)
    at = O.pcg(P.X, P.omega, P.lam, P.tau, b, tol=1e-8, stop_rule=O.STOP_RELATIVE, beta0=chol)
    assert at[1] == 0 and at[3] == O.OK and np.array_equal(at[0], chol)
    early = O.pcg(P.X, P.omega, P.lam, P.tau, b, fixed_iters=4)[0]
    beta, k, res, st, hist = O.pcg(P.X, P.omega, P.lam, P.tau, b, tol=1e-10,
                                   stop_rule=O.STOP_RELATIVE, beta0=early, want_hist=True)
    r0 = P.tau * P.lam * (b - P.X.dense().T @ (P.omega * (P.X.dense() @ early))
                          - early / (P.tau * P.lam) ** 2)
    assert abs(hist[0] - r0 @ r0) <= 1e-10 * (r0 @ r0)
    assert st == O.OK and 0 < k < base[1] + 5 and rel(beta, chol) < 1e-8


# --------------------------------------------------------------------------
# LSQR on the least-squares form (Sec. S7.1, Eq. S6)
# --------------------------------------------------------------------------

def test_lsqr_solves_the_normal_equations():
    """Eq. S6: the minimiser of ||Xt beta - bt|| solves Phi beta = b.  On
    config 1 LSQR reaches the Cholesky draw and takes CG's iteration count
    (the two are the same Krylov method on this system)."""
    P = inputs.config1()
    chol = O.draw_beta_chol(P.X, P.omega, P.z, P.lam, P.tau, P.eta, P.delta)
    beta, k, res, st = O.draw_beta_lsqr(P.X, P.omega, P.z, P.lam, P.tau, P.eta, P.delta, tol=1e-10,
                                        stop_rule=O.STOP_RELATIVE)
    k_cg = O.draw_beta_cg(P.X, P.omega, P.z, P.lam, P.tau, P.eta, P.delta, tol=1e-10,
                          stop_rule=O.STOP_RELATIVE)[1]
    assert st == O.OK and res <= 1e-10 and k == k_cg
    assert rel(beta, chol) < 1e-8


def test_lsqr_iterates_equal_pcg_iterates():
    """LSQR with A = Xt diag(tau lambda) and PCG with M^-1 = tau^2 lambda^2
    build the same iterates in exact arithmetic: at a fixed k on a
    well-conditioned instance they agree to rounding (measured 3e-16 at k =
    1 growing to 5e-10 at k = 9 as the residual shrinks)."""
    P = small_problem(n=200, p=40, tau=0.3)
    P.lam = np.random.default_rng(2).uniform(0.5, 2.0, P.X.p)
    b = O.build_b(P.X, P.omega, P.z, P.lam, P.tau, P.eta, P.delta)
    for k, bound in ((1, 1e-14), (2, 1e-13), (5, 1e-11), (9, 5e-9)):
        ls, kk, _, st = O.draw_beta_lsqr(P.X, P.omega, P.z, P.lam, P.tau, P.eta, P.delta, tol=0.0,
                                         max_iter=k)
        cg = O.pcg(P.X, P.omega, P.lam, P.tau, b, fixed_iters=k)[0]
        assert st == O.MAXITER and kk == k and rel(ls, cg) < bound, k


def test_lsqr_residual_estimate_is_eq_s2():
    """LSQR's ||A^T r|| = phibar alpha |c| is the prior-preconditioned
    residual of Eq. S2, recomputed here from b - Phi beta."""
    P = inputs.make_problem(4000, 600, -3.0, -1.0, seed=44, tau=1e-2, inflate_frac=0.02)
    beta, k, res, st = O.draw_beta_lsqr(P.X, P.omega, P.z, P.lam, P.tau, P.eta, P.delta, tol=1e-7)
    b = O.build_b(P.X, P.omega, P.z, P.lam, P.tau, P.eta, P.delta)
    rt = P.tau * P.lam * (b - dense_phi_numpy(P) @ beta)
    assert st == O.OK and k > 5 and res <= 1e-7
    assert abs(np.sqrt(np.mean(rt ** 2)) - res) <= 1e-3 * res


@pytest.mark.parametrize("k", [1, 3])
def test_lsqr_low_rank_and_empty_design(k):
    """Thm 2.2 (n = k rows: at most k + 1 iterations) and X = 0 (one
    iteration, beta = tau^2 lambda^2 b)."""
    rng = np.random.default_rng(500 + k)
    x = (rng.uniform(size=(k, 60)) < 0.3).astype(float)
    P = inputs.Problem(inputs.design_from_dense(x), rng.uniform(0.05, 0.25, k), rng.standard_normal(k),
                       rng.uniform(0.5, 2.0, 60), 0.3, rng.standard_normal(k), rng.standard_normal(60))
    _, kk, _, st = O.draw_beta_lsqr(P.X, P.omega, P.z, P.lam, P.tau, P.eta, P.delta, tol=1e-10,
                                    stop_rule=O.STOP_RELATIVE)
    assert st == O.OK and kk <= k + 1
    Q = small_problem()
    Q.X = inputs.design_from_dense(np.zeros((Q.X.n, Q.X.p)))
    beta, kk, _, st = O.draw_beta_lsqr(Q.X, Q.omega, Q.z, Q.lam, Q.tau, Q.eta, Q.delta, tol=1e-12)
    assert st == O.OK and kk == 1 and rel(beta, Q.tau * Q.lam * Q.delta) < 1e-14


def test_lsqr_nonfinite_input_reported():
    """A NaN in delta makes bt, and so beta_1, NaN: NONFINITE under both stop
    rules, before any x update."""
    P = small_problem()
    P.delta = P.delta.copy()
    P.delta[2] = np.nan
    for rule in (O.STOP_RMS, O.STOP_RELATIVE):
        _, k, _, st = O.draw_beta_lsqr(P.X, P.omega, P.z, P.lam, P.tau, P.eta, P.delta, stop_rule=rule)
        assert st == O.NONFINITE and k == 0
