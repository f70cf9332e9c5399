"""Unshrunk coefficients (Sec. S4.3) on the GPU: coefficients 0 .. q1-1 with
their own prior precisions (a flat prior included) and preconditioner scales,
against the oracle's plain definition of that model."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_1810_12437_gb300 import inputs
from tests.iteration_band import band_of
from tests.gpu_helpers import T, dev, device_problem, need_gpu, rel

pytestmark = pytest.mark.gpu

PREC = np.array([0.0, 0.01, 4.0])     # flat prior (intercept), weak, moderate
GAMMA = np.array([2.0, 1.0, 0.5])     # preconditioner scales (any positive values)


@pytest.fixture(scope="module")
def pb():
    need_gpu()
    import paper_1810_12437_gb300 as pb
    pb.load_library()
    return pb


def with_intercept(P):
    """Column 0 of X becomes an all-ones intercept column."""
    dense = P.X.dense()
    dense[:, 0] = 1.0
    P.X = inputs.design_from_dense(dense)
    return P


def single_problem():
    P = inputs.make_problem(3000, 400, -2.0, -1.0, seed=41, tau=0.05)
    return with_intercept(P)


@pytest.mark.parametrize("prec,bound", [("fp64", 1e-8), ("df32", 1e-6), ("fx64", 1e-6)])
def test_unshrunk_draw_matches_oracle(pb, prec, bound):
    P = single_problem()
    X, a = device_problem(P)
    ctx = pb.Context(precision=prec)
    pb.pcg_set_unshrunk(ctx, T(PREC), T(GAMMA))
    res = pb.pcg_draw_beta(ctx, X, a["omega"], a["z"], a["lam"], P.tau, a["eta"], a["delta"],
                           tol=1e-10, max_iter=5000)
    assert res.status == pb.PCG_OK
    ref = O.draw_beta_chol_unshrunk(P.X, P.omega, P.z, P.lam, P.tau, P.eta, P.delta, PREC)
    assert rel(res.beta.cpu().numpy(), ref) < bound
    b = O.build_b_unshrunk(P.X, P.omega, P.z, P.lam, P.tau, P.eta, P.delta, PREC)
    _, k, _, st = O.pcg_unshrunk(P.X, P.omega, P.lam, P.tau, b, PREC, GAMMA, tol=1e-10)
    assert st == O.OK
    # iteration count within 2 of the oracle's band at the same storage
    # precision (compensated sums; the inputs and one-ulp perturbations)
    vec = "f64" if prec == "fp64" else "f32x2"

    def run(om, lm):
        bb = O.build_b_unshrunk(P.X, om, P.z, lm, P.tau, P.eta, P.delta, PREC)
        return O.pcg_unshrunk(P.X, om, lm, P.tau, bb, PREC, GAMMA, tol=1e-10, sums="compensated",
                              vec=vec)[1]

    band = band_of(run, P.omega, P.lam)
    assert band.holds(res.iters), (res.iters, str(band))


def test_unshrunk_differs_from_shrinkage_and_clears(pb):
    """The setting changes the draw, and q1 = 0 restores the shrinkage model."""
    P = single_problem()
    X, a = device_problem(P)
    ctx = pb.Context(precision="fp64")
    args = (a["omega"], a["z"], a["lam"], P.tau, a["eta"], a["delta"])
    pb.pcg_set_unshrunk(ctx, T(PREC), T(GAMMA))
    b_un = pb.pcg_draw_beta(ctx, X, *args, tol=1e-10, max_iter=5000).beta.cpu().numpy()
    pb.pcg_set_unshrunk(ctx)
    b_sh = pb.pcg_draw_beta(ctx, X, *args, tol=1e-10, max_iter=5000).beta.cpu().numpy()
    ref = O.draw_beta_chol(P.X, P.omega, P.z, P.lam, P.tau, P.eta, P.delta)
    assert rel(b_sh, ref) < 1e-8
    assert rel(b_un, b_sh) > 1e-3


def test_unshrunk_rhs_and_phi_mul(pb):
    P = single_problem()
    X, a = device_problem(P)
    ctx = pb.Context(precision="fp64")
    pb.pcg_set_unshrunk(ctx, T(PREC), T(GAMMA))
    b = pb.pcg_build_rhs(ctx, X, a["omega"], a["z"], a["lam"], P.tau, a["eta"], a["delta"]).cpu().numpy()
    ref_b = O.build_b_unshrunk(P.X, P.omega, P.z, P.lam, P.tau, P.eta, P.delta, PREC)
    assert rel(b, ref_b) < 1e-13
    v = np.random.default_rng(8).standard_normal(P.X.p)
    out = pb.pcg_phi_mul(ctx, X, a["omega"], a["lam"], P.tau, T(v)).cpu().numpy()
    ref = O.dense_phi_unshrunk(P.X, P.omega, P.lam, P.tau, PREC) @ v
    assert rel(out, ref) < 1e-13


@pytest.mark.parametrize("prec", ["df32", "fp32_refined"])
def test_unshrunk_batched_matches_oracle(pb, prec):
    """Four chains sharing X with their own omega, lambda and tau: every chain
    takes the same unshrunk coefficients."""
    P = inputs.make_problem(3000, 400, -2.0, -1.0, seed=42, nrhs=4, tau_log10_range=(-1.6, -1.0))
    P = with_intercept(P)
    X = pb.DeviceDesign.from_host(P.X, dev())
    ctx = pb.Context(precision=prec)
    pb.pcg_set_unshrunk(ctx, T(PREC), T(GAMMA))
    res = pb.pcg_draw_beta_batched(ctx, X, omega=T(P.omega), z=T(P.z), lam=T(P.lam), tau=T(P.tau),
                                   eta=T(P.eta), delta=T(P.delta), tol=1e-8, max_iter=5000)
    beta = res.beta.cpu().numpy()
    for r in range(4):
        ref = O.draw_beta_chol_unshrunk(P.X, P.omega[r], P.z[r], P.lam[r], float(P.tau[r]), P.eta[r],
                                        P.delta[r], PREC)
        assert res.status[r] == pb.PCG_OK
        assert rel(beta[r], ref) < 1e-5, r


def test_unshrunk_bad_arguments(pb):
    P = single_problem()
    X, a = device_problem(P)
    ctx = pb.Context(precision="fp64")
    with pytest.raises(pb.PcgError):
        pb.pcg_set_unshrunk(ctx, T([1.0, -1.0]), T([1.0, 1.0]))        # negative precision
    with pytest.raises(pb.PcgError):
        pb.pcg_set_unshrunk(ctx, T([1.0]), T([0.0]))                   # gamma must be positive
    # more unshrunk coefficients than columns of X
    pb.pcg_set_unshrunk(ctx, T(np.ones(P.X.p + 1)), T(np.ones(P.X.p + 1)))
    with pytest.raises(pb.PcgError):
        pb.pcg_draw_beta(ctx, X, a["omega"], a["z"], a["lam"], P.tau, a["eta"], a["delta"])
    # the uneven batch and the adjoint assume the shrinkage prior throughout
    pb.pcg_set_unshrunk(ctx, T(PREC), T(GAMMA))
    with pytest.raises(pb.PcgError):
        pb.pcg_draw_beta_uneven(ctx, [dict(X=X, tau=P.tau, **a)], tol=1e-6, max_iter=100)
    pb.pcg_set_unshrunk(ctx)
    res = pb.pcg_draw_beta(ctx, X, a["omega"], a["z"], a["lam"], P.tau, a["eta"], a["delta"])
    assert res.status == pb.PCG_OK
