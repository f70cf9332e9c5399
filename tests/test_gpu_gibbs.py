"""The Gibbs cycle of Sec. S1 on the GPU (pcg_gibbs_step, row f3) against the
oracle's cycle (oracle/pcg_oracle.c: the same Philox4x32-10 counters, the
same samplers written independently).

The scale updates and the Polya-Gamma draws consume the same random numbers
on both sides, so they agree element by element to the rounding of exp, log,
pow and erfc.  A rejection decision could in principle flip where a variate
lands within rounding of its threshold; the tests allow that for a tiny
fraction of elements and check the distribution as well.  The beta draw is
the library's PCG, compared with the oracle's PCG on the same inputs."""
import math

import numpy as np
import pytest
import torch

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


def problem(seed=81):
    P = inputs.make_problem(3000, 300, -2.0, -1.0, seed=seed, tau=0.1)
    rng = np.random.default_rng(seed)
    beta0 = rng.standard_normal(P.X.p) * 0.3
    return P, beta0


def state(pb, P, beta0, tau=0.1, xi=1.0):
    return pb.GibbsState(omega=torch.zeros(P.X.n, dtype=torch.float64, device=dev()),
                         lam=T(np.ones(P.X.p)), nu=T(np.ones(P.X.p)), beta=T(beta0), tau=tau, xi=xi)


def test_one_cycle_matches_oracle(pb):
    P, beta0 = problem()
    X = pb.DeviceDesign.from_host(P.X, dev())
    st = state(pb, P, beta0)
    ctx = pb.Context(precision="fp64", stop_rule="relative")
    res = pb.pcg_gibbs_step(ctx, X, T(P.y), st, seed=2024, step=3, tol=1e-12, max_iter=3000)
    assert res.status == pb.PCG_OK
    lam, nu, tau, xi = O.gibbs_scales(beta0, np.ones(P.X.p), np.ones(P.X.p), 0.1, 1.0, seed=2024, step=3)
    assert abs(st.tau - tau) <= 1e-13 * tau and abs(st.xi - xi) <= 1e-13 * xi
    assert np.all(np.abs(st.lam.cpu().numpy() - lam) <= 1e-13 * lam)
    assert np.all(np.abs(st.nu.cpu().numpy() - nu) <= 1e-13 * nu)
    omega, z, eta, delta = O.gibbs_omega(P.X, P.y, beta0, seed=2024, step=3)
    got = st.omega.cpu().numpy()
    close = np.abs(got - omega) <= 1e-12 * omega
    assert close.mean() >= 0.999, close.mean()
    if close.all():
        # the same inputs to step 4: the oracle's PCG draw to the same rule
        ref = O.draw_beta_cg(P.X, omega, z, lam, tau, eta, delta, tol=1e-12, stop_rule=O.STOP_RELATIVE)[0]
        assert rel(st.beta.cpu().numpy(), ref) < 1e-8


def test_chain_tracks_the_oracle_chain(pb):
    """Five cycles from the same state and seed: the GPU chain and the
    oracle's chain stay together (same random numbers, rounding only)."""
    P, beta0 = problem(82)
    X = pb.DeviceDesign.from_host(P.X, dev())
    st = state(pb, P, beta0)
    ctx = pb.Context(precision="fp64", stop_rule="relative")
    ref = dict(beta=beta0, lam=np.ones(P.X.p), nu=np.ones(P.X.p), tau=0.1, xi=1.0)
    for step in range(5):
        res = pb.pcg_gibbs_step(ctx, X, T(P.y), st, seed=77, step=step, tol=1e-12, max_iter=3000)
        assert res.status == pb.PCG_OK
        ref = O.gibbs_step(P.X, P.y, ref["beta"], ref["lam"], ref["nu"], ref["tau"], ref["xi"], seed=77,
                           step=step, draw="cg", tol=1e-12, stop_rule=O.STOP_RELATIVE)
    assert rel(st.beta.cpu().numpy(), ref["beta"]) < 1e-6
    assert abs(st.tau - ref["tau"]) < 1e-6 * ref["tau"]
    assert rel(st.lam.cpu().numpy(), ref["lam"]) < 1e-6


def test_polya_gamma_draws_on_the_gpu(pb):
    """Rows with one nonzero each in column i mod 3 and beta* = (0, 1, 4):
    the omega draws of the three row classes have PolyaGamma(1, c) means and
    variances for c = 0, 1 and 4."""
    n, p = 150_000, 3
    dense_cols = np.arange(n) % 3
    col_ptr = np.zeros(p + 1, dtype=np.int64)
    np.cumsum(np.bincount(dense_cols, minlength=p), out=col_ptr[1:])
    row_idx = np.concatenate([np.nonzero(dense_cols == j)[0] for j in range(p)]).astype(np.int32)
    Xh = inputs.design_from_csc(n, p, col_ptr, row_idx)
    X = pb.DeviceDesign.from_host(Xh, dev())
    y = np.zeros(n)
    st = pb.GibbsState(omega=torch.zeros(n, dtype=torch.float64, device=dev()), lam=T(np.ones(p)),
                       nu=T(np.ones(p)), beta=T(np.array([0.0, 1.0, 4.0])), tau=1.0, xi=1.0)
    ctx = pb.Context(precision="fp64")
    pb.pcg_gibbs_step(ctx, X, T(y), st, seed=5, step=0, tol=1e-8, max_iter=100)
    w = st.omega.cpu().numpy()
    for j, c in enumerate((0.0, 1.0, 4.0)):
        s = w[dense_cols == j]
        mean = 0.25 if c == 0 else math.tanh(c / 2) / (2 * c)
        var = 1 / 24 if c == 0 else (math.sinh(c) - c) / (4 * c ** 3 * math.cosh(c / 2) ** 2)
        assert abs(s.mean() - mean) < 5 * math.sqrt(var / s.size), c
        assert abs(s.var() - var) < 0.05 * var, c
    # and element by element against the oracle's draws of the same counters
    psi = np.array([0.0, 1.0, 4.0])[dense_cols]
    ref = O.pg1(psi, seed=5, stream=O.STREAM_OMEGA, step=0)
    assert (np.abs(w - ref) <= 1e-12 * ref).mean() >= 0.9999


def test_gibbs_arguments(pb):
    P, beta0 = problem()
    X = pb.DeviceDesign.from_host(P.X, dev())
    ctx = pb.Context(precision="fp64")
    with pytest.raises(pb.PcgError):
        pb.pcg_gibbs_step(ctx, X, T(P.y), state(pb, P, beta0, tau=-1.0), seed=1, step=0)
    pb.pcg_set_unshrunk(ctx, T(np.array([0.0])), T(np.array([1.0])))
    with pytest.raises(pb.PcgError) as ei:
        pb.pcg_gibbs_step(ctx, X, T(P.y), state(pb, P, beta0), seed=1, step=0)
    assert ei.value.status == pb.PCG_BADARG
