"""pcg_draw_beta_lsqr: the draw by LSQR on the least-squares form of Sec. S7.1
(Eq. S6), against the oracle's LSQR (oracle_lsqr) and the direct draw.  Same-k
comparisons isolate the arithmetic (and check LSQR's iterates against PCG's,
which they equal in exact arithmetic); stopped draws check the iteration count
against the oracle LSQR's band (compensated sums, the inputs and one-ulp
perturbations of them, tests/iteration_band.py) and the true residual."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_1810_12437_gb300 import inputs
from tests.gpu_helpers import T, dev, device_problem, need_gpu, rel
from tests.iteration_band import band_of

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pb():
    need_gpu()
    import paper_1810_12437_gb300 as pb
    pb.load_library()
    return pb


def lsqr(pb, ctx, P, X, a, **kw):
    return pb.pcg_draw_beta_lsqr(ctx, X, a["omega"], a["z"], a["lam"], P.tau, a["eta"], a["delta"], **kw)


def well_conditioned():
    P = inputs.config1()
    P.lam = np.random.default_rng(1).uniform(0.5, 2.0, P.X.p)
    P.tau = 0.05
    return P


@pytest.mark.parametrize("k", [1, 3, 8])
def test_lsqr_same_k(pb, k):
    P = well_conditioned()
    X, a = device_problem(P)
    ctx = pb.Context(precision="fp64", stop_rule="relative")
    res = lsqr(pb, ctx, P, X, a, tol=0.0, max_iter=k)
    assert res.status == pb.PCG_MAXITER and res.iters == k
    ref = O.draw_beta_lsqr(P.X, P.omega, P.z, P.lam, P.tau, P.eta, P.delta, tol=0.0, max_iter=k)[0]
    cg = O.draw_beta_cg(P.X, P.omega, P.z, P.lam, P.tau, P.eta, P.delta, fixed_iters=k)[0]
    got = res.beta.cpu().numpy()
    assert rel(got, ref) < 1e-11
    assert rel(got, cg) < 1e-9


@pytest.mark.parametrize("use_graph", [True, False])
def test_lsqr_config1_matches_cholesky(pb, use_graph):
    P = inputs.config1()
    X, a = device_problem(P)
    ctx = pb.Context(precision="fp64", stop_rule="relative", use_graph=use_graph)
    res = lsqr(pb, ctx, P, X, a, tol=1e-10, max_iter=2000)
    ref, k, _, st = O.draw_beta_lsqr(P.X, P.omega, P.z, P.lam, P.tau, P.eta, P.delta, tol=1e-10,
                                     stop_rule=O.STOP_RELATIVE)
    chol = O.draw_beta_chol(P.X, P.omega, P.z, P.lam, P.tau, P.eta, P.delta)
    assert res.status == pb.PCG_OK and st == O.OK and abs(res.iters - k) <= 2
    assert res.resid <= 1e-10
    assert rel(res.beta.cpu().numpy(), ref) < 1e-9 and rel(res.beta.cpu().numpy(), chol) < 1e-8


def test_lsqr_config2_band_and_true_residual(pb):
    P = inputs.config2()
    X, a = device_problem(P)
    ctx = pb.Context(precision="fp64")
    res = lsqr(pb, ctx, P, X, a, tol=1e-6, max_iter=5000)
    ref = O.draw_beta_lsqr(P.X, P.omega, P.z, P.lam, P.tau, P.eta, P.delta, tol=1e-6)[0]

    def run(om, lm):
        return O.draw_beta_lsqr(P.X, om, P.z, lm, P.tau, P.eta, P.delta, tol=1e-6, sums="compensated")[1]

    band = band_of(run, P.omega, P.lam)
    assert res.status == pb.PCG_OK and band.holds(res.iters), (res.iters, str(band))
    beta = res.beta.cpu().numpy()
    assert rel(beta, ref) < 1e-6
    b = O.build_b(P.X, P.omega, P.z, P.lam, P.tau, P.eta, P.delta)
    rt = P.tau * P.lam * (b - O.phi_mul(P.X, P.omega, P.lam, P.tau, beta))
    true_rms = np.sqrt(np.mean(rt ** 2))
    assert true_rms <= 1.5e-6 and abs(true_rms - res.resid) <= 0.05 * res.resid


def test_lsqr_graph_and_plain_agree_bitwise(pb):
    P = inputs.config2()
    X, a = device_problem(P)
    outs = []
    for g in (True, False):
        r = lsqr(pb, pb.Context(precision="fp64", use_graph=g), P, X, a, tol=1e-6, max_iter=5000)
        outs.append((r.iters, r.beta.cpu().numpy()))
    assert outs[0][0] == outs[1][0] and np.array_equal(outs[0][1], outs[1][1])


def test_lsqr_edge_cases_and_arguments(pb):
    # X without nonzeros: one iteration, beta = tau^2 lambda^2 b = tau lambda delta
    P = inputs.make_problem(40, 30, -1, -0.5, seed=5, tau=0.1)
    P.X = inputs.design_from_dense(np.zeros((40, 30)))
    X, a = device_problem(P)
    ctx = pb.Context(precision="fp64")
    res = lsqr(pb, ctx, P, X, a, tol=1e-12, max_iter=10)
    assert res.status == pb.PCG_OK and res.iters == 1
    assert rel(res.beta.cpu().numpy(), P.tau * P.lam * P.delta) < 1e-14
    # loose tolerance: no iteration, beta = 0; NaN delta: PCG_NONFINITE
    P = well_conditioned()
    X, a = device_problem(P)
    res = lsqr(pb, ctx, P, X, a, tol=1e30, max_iter=10)
    assert res.status == pb.PCG_OK and res.iters == 0 and float(res.beta.abs().max()) == 0.0
    bad = a["delta"].clone()
    bad[3] = float("nan")
    res = pb.pcg_draw_beta_lsqr(ctx, X, a["omega"], a["z"], a["lam"], P.tau, a["eta"], bad)
    assert res.status == pb.PCG_NONFINITE
    for opts in (dict(preconditioner="jacobi"), dict(warm_start=True)):
        with pytest.raises(pb.PcgError) as ei:
            lsqr(pb, pb.Context(precision="fp64", **opts), P, X, a, out=torch.zeros(P.X.p, dtype=torch.float64,
                                                                                     device=dev()))
        assert ei.value.status == pb.PCG_BADARG
    with pytest.raises(pb.PcgError):
        pb.pcg_draw_beta_lsqr(ctx, X, a["omega"], a["z"], a["lam"], -1.0, a["eta"], a["delta"])
    # a NaN under the relative rule too
    rctx = pb.Context(precision="fp64", stop_rule="relative")
    res = pb.pcg_draw_beta_lsqr(rctx, X, a["omega"], a["z"], a["lam"], P.tau, a["eta"], bad)
    assert res.status == pb.PCG_NONFINITE
