"""CPU pins for the oracle's Gibbs pieces (row f3, Sec. S1): the counter-based
generator, the Polya-Gamma sampler and the horseshoe scale updates.

Each piece is fixed by something other than itself: the generator by the
published known-answer vectors; the uniform, exponential, normal and Gamma
draws by their moments; PolyaGamma(1, c) by its closed-form mean tanh(c/2) /
(2c) and variance (sinh c - c) / (4 c^3 cosh^2(c/2)) (1/4 and 1/24 at c = 0);
every scale update by the probability integral transform of the exact
conditional it draws from (inverse gamma: P(X <= x) = Q(a, b/x)), which
makes exp(-b/x) (shape 1) or Q(a, b/x) uniform over independent counters."""
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_1810_12437_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def kat():
    rows = []
    for line in open(os.path.join(GOLDEN, "philox_kat.txt")):
        if line.strip() and not line.startswith("#"):
            w = [int(x, 16) for x in line.split()]
            rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


def test_philox_known_answers():
    for ctr, key, want in kat():
        assert [int(x) for x in O.philox(ctr, key)] == want


def test_uniform_mapping_from_the_generator_words():
    """The first two uniforms of counter (index 0, stream 0, step 0, block 0)
    under key 0 are ((w0 >> 5) 2^26 + (w1 >> 6) + 1/2) / 2^53 and the same from
    (w2, w3), with w the first known-answer output."""
    w = kat()[0][2]
    want = [((w[0] >> 5) * 2 ** 26 + (w[1] >> 6) + 0.5) / 2 ** 53,
            ((w[2] >> 5) * 2 ** 26 + (w[3] >> 6) + 0.5) / 2 ** 53]
    got = O.rng_draws("uniform", 2, 0, 0, 0, 0)
    assert list(got) == want


def test_draw_moments():
    N = 200_000
    u = O.rng_draws("uniform", N, 7, 3, 1, 0)
    assert abs(u.mean() - 0.5) < 5 * math.sqrt(1 / 12 / N) and u.min() > 0 and u.max() < 1
    e = O.rng_draws("exp", N, 7, 4, 1, 0)
    assert abs(e.mean() - 1) < 5 / math.sqrt(N) and abs(e.var() - 1) < 0.03
    z = O.rng_draws("normal", N, 7, 5, 1, 0)
    assert abs(z.mean()) < 5 / math.sqrt(N) and abs(z.var() - 1) < 0.02
    for a in (1.0, 2.5, 25_000.5):
        g = O.rng_draws("gamma", 40_000, 7, 6, 1, 0, a)
        assert abs(g.mean() - a) < 5 * math.sqrt(a / 40_000) and abs(g.var() / a - 1) < 0.05, a


@pytest.mark.parametrize("c", [0.0, 0.4, 2.0, 8.0, 30.0, -3.0])
def test_polya_gamma_moments(c):
    N = 200_000
    w = O.pg1(np.full(N, c), seed=123, step=1)
    a = abs(c)
    mean = 0.25 if a == 0 else math.tanh(a / 2) / (2 * a)
    var = 1 / 24 if a == 0 else (math.sinh(a) - a) / (4 * a ** 3 * math.cosh(a / 2) ** 2)
    assert w.min() > 0
    assert abs(w.mean() - mean) < 5 * math.sqrt(var / N)
    # the variance of a sample variance: (mu4 - var^2) / N, bounded here by 3 var^2 / N x 4
    assert abs(w.var() - var) < 0.03 * var


def test_polya_gamma_series_forms_agree():
    """The sampler's two coefficient forms of the J*(1, 0) density (small x
    and large x) are the same function; the density integrates to 1 with mean
    1 (PG(1, 0) = J*(1, 0) / 4 has mean 1/4)."""
    for x in (0.2, 0.45, 0.64, 0.9, 1.6):
        small = O.pg_series(x, t=1e9)
        large = O.pg_series(x, t=0.0)
        assert abs(small - large) <= 1e-12 * max(abs(large), 1e-300), x
    xs = np.linspace(1e-4, 12.0, 120_001)
    f = np.array([O.pg_series(x, t=0.64) for x in xs])
    dx = xs[1] - xs[0]
    assert abs(np.sum(f) * dx - 1.0) < 1e-4
    assert abs(np.sum(xs * f) * dx - 1.0) < 1e-3


def _uniform_ks(u):
    """Kolmogorov-Smirnov distance of a sample from U(0, 1)."""
    u = np.sort(np.asarray(u))
    n = u.size
    return max(np.max(np.arange(1, n + 1) / n - u), np.max(u - np.arange(n) / n))


def test_scale_updates_draw_their_conditionals():
    """For fixed inputs, over many Gibbs steps (independent counters):
    xi ~ IG(1, 1 + 1/tau^2), tau^2 ~ IG((p+1)/2, 1/xi + sum beta^2/(2 lambda^2)),
    nu_j ~ IG(1, 1 + 1/lambda_j^2), lambda_j^2 ~ IG(1, 1/nu_j + beta_j^2/(2 tau^2)),
    each with the values drawn before it in the same step."""
    from scipy.special import gammaincc
    p = 50
    rng = np.random.default_rng(3)
    beta = rng.standard_normal(p) * 0.3
    lam = rng.uniform(0.2, 3.0, p)
    nu = rng.uniform(0.5, 2.0, p)
    tau, xi = 0.4, 1.3
    u_xi, u_tau, u_nu, u_lam = [], [], [], []
    for step in range(3000):
        lam2, nu2, tau2, xi2 = O.gibbs_scales(beta, lam, nu, tau, xi, seed=11, step=step)
        u_xi.append(math.exp(-(1 + 1 / tau ** 2) / xi2))
        a = (p + 1) / 2
        b = 1 / xi2 + np.sum(beta ** 2 / (2 * lam ** 2))
        u_tau.append(gammaincc(a, b / tau2 ** 2))
        u_nu.extend(np.exp(-(1 + 1 / lam ** 2) / nu2))
        u_lam.extend(np.exp(-(1 / nu2 + beta ** 2 / (2 * tau2 ** 2)) / lam2 ** 2))
    for name, u in (("xi", u_xi), ("tau", u_tau), ("nu", u_nu), ("lambda", u_lam)):
        n = len(u)
        assert _uniform_ks(u) < 1.63 / math.sqrt(n), name       # 1% level


def test_gibbs_step_composes_the_cycle():
    """One cycle: the scale and omega updates of the same seed and step, then
    the beta draw; the CG and Cholesky versions of step 4 agree."""
    P = inputs.make_problem(600, 40, -1.5, -0.7, seed=21, tau=0.3)
    y = P.y
    beta0 = np.random.default_rng(4).standard_normal(P.X.p) * 0.2
    lam0, nu0 = np.ones(P.X.p), np.ones(P.X.p)
    chol = O.gibbs_step(P.X, y, beta0, lam0, nu0, 0.3, 1.0, seed=5, step=2)
    cg = O.gibbs_step(P.X, y, beta0, lam0, nu0, 0.3, 1.0, seed=5, step=2, draw="cg", tol=1e-12,
                      stop_rule=O.STOP_RELATIVE)
    lam, nu, tau, xi = O.gibbs_scales(beta0, lam0, nu0, 0.3, 1.0, seed=5, step=2)
    omega, z, eta, delta = O.gibbs_omega(P.X, y, beta0, seed=5, step=2)
    assert np.array_equal(chol["lam"], lam) and chol["tau"] == tau and np.array_equal(chol["omega"], omega)
    assert np.allclose(omega * z, y - 0.5, rtol=1e-15, atol=0)
    # omega is PG(1, x_i^T beta): the same counters applied to psi = X beta (dense)
    psi = P.X.dense() @ beta0
    assert np.allclose(O.pg1(psi, seed=5, stream=O.STREAM_OMEGA, step=2), omega, rtol=1e-13, atol=0)
    assert np.all(omega > 0)
    assert np.linalg.norm(cg["beta"] - chol["beta"]) < 1e-9 * np.linalg.norm(chol["beta"])
    # eta and delta are standard normals of their own streams
    assert np.array_equal(eta[:3], [O.rng_draws("normal", 1, 5, i, O.STREAM_ETA, 2)[0] for i in range(3)])
    assert np.array_equal(delta[:3], [O.rng_draws("normal", 1, 5, j, O.STREAM_DELTA, 2)[0] for j in range(3)])
