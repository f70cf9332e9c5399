"""The Jacobi preconditioner (Sec. 2.4, compared in Sec. 3) and warm starts
(Sec. S4.1) of the single-RHS path, against the oracle's general PCG
(oracle_pcg_ex: the same recursion with M^-1 = 1 / diag(Phi), or r_0 = b -
Phi beta_0).  The stop rule tests ||tau lambda (.) r|| (Eq. S2) whatever the
preconditioner.  Same-k comparisons on a well-conditioned instance isolate
the arithmetic; stopped draws on the paper-shaped configs check iteration
counts against the oracle's band at the same storage precision
(tests/iteration_band.py) and the draw itself."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_1810_12437_gb300 import inputs
from tests.gpu_helpers import T, dev, device_problem, need_gpu, rel
from tests.iteration_band import SLACK, problem_band

pytestmark = pytest.mark.gpu

VEC = {"fp64": "f64", "df32": "f32x2", "fx64": "f32x2"}


@pytest.fixture(scope="module")
def pb():
    need_gpu()
    import paper_1810_12437_gb300 as pb
    pb.load_library()
    return pb


def well_conditioned():
    P = inputs.config1()
    P.lam = np.random.default_rng(1).uniform(0.5, 2.0, P.X.p)
    P.tau = 0.05
    return P


def draw(pb, ctx, P, X, a, **kw):
    return pb.pcg_draw_beta(ctx, X, a["omega"], a["z"], a["lam"], P.tau, a["eta"], a["delta"], **kw)


@pytest.mark.parametrize("prec", ["fp64", "df32", "fx64"])
@pytest.mark.parametrize("k", [1, 3, 8])
def test_jacobi_same_k(pb, prec, k):
    P = well_conditioned()
    X, a = device_problem(P)
    ctx = pb.Context(precision=prec, stop_rule="relative", preconditioner="jacobi")
    res = draw(pb, ctx, P, X, a, tol=0.0, max_iter=k)
    assert res.status == pb.PCG_MAXITER and res.iters == k
    minv = 1.0 / O.phi_diag(P.X, P.omega, P.lam, P.tau)
    ref = O.draw_beta_cg(P.X, P.omega, P.z, P.lam, P.tau, P.eta, P.delta, fixed_iters=k, minv=minv)[0]
    assert rel(res.beta.cpu().numpy(), ref) < 1e-11


@pytest.mark.parametrize("prec,cfg", [("fp64", "config1"), ("df32", "config1"), ("fp64", "config2"),
                                      ("df32", "config2"), ("fx64", "config2"), ("fp32_refined", "config2")])
def test_jacobi_stopped_draw(pb, prec, cfg):
    """The stopped Jacobi draw: within the oracle's Jacobi band (float32
    refined: within 3x its top, the mode's restarts) and the oracle's stopped
    Jacobi draw; the reported stop quantity is that of the true residual."""
    P = getattr(inputs, cfg)()
    kw = dict(tol=1e-10, stop_rule=O.STOP_RELATIVE) if cfg == "config1" else dict(tol=1e-6)
    X, a = device_problem(P)
    ctx = pb.Context(precision=prec, preconditioner="jacobi",
                     stop_rule="relative" if cfg == "config1" else "rms")
    res = draw(pb, ctx, P, X, a, tol=kw["tol"], max_iter=2000)
    minv = 1.0 / O.phi_diag(P.X, P.omega, P.lam, P.tau)
    ref, k, r, st = O.draw_beta_cg(P.X, P.omega, P.z, P.lam, P.tau, P.eta, P.delta, minv=minv, **kw)
    assert res.status == pb.PCG_OK and st == O.OK
    if prec in VEC:
        band = problem_band(P, precond="jacobi", vec=VEC[prec], **kw)
        assert band.holds(res.iters), (res.iters, str(band))
        assert rel(res.beta.cpu().numpy(), ref) < 1e-6
    else:
        band = problem_band(P, precond="jacobi", vec="f32", **kw)
        assert band.lo - SLACK <= res.iters <= 3 * band.hi + SLACK, (res.iters, str(band))
        assert rel(res.beta.cpu().numpy(), ref) < 1e-5
    b = O.build_b(P.X, P.omega, P.z, P.lam, P.tau, P.eta, P.delta)
    rt = P.tau * P.lam * (b - O.phi_mul(P.X, P.omega, P.lam, P.tau, res.beta.cpu().numpy()))
    if cfg == "config2":
        assert np.sqrt(np.mean(rt ** 2)) <= 1.5e-6


def test_jacobi_is_prior_without_data(pb):
    """X with no nonzeros: diag(Phi) = tau^-2 lambda^-2, so Jacobi is the
    prior preconditioner and one iteration gives beta = tau^2 lambda^2 b."""
    P = inputs.make_problem(40, 30, -1, -0.5, seed=5, tau=0.1)
    P.X = inputs.design_from_dense(np.zeros((40, 30)))
    X, a = device_problem(P)
    for prec in ("fp64", "df32"):
        ctx = pb.Context(precision=prec, preconditioner="jacobi")
        res = draw(pb, ctx, P, X, a, tol=1e-12, max_iter=10)
        assert res.status == pb.PCG_OK and res.iters == 1
        assert rel(res.beta.cpu().numpy(), P.tau * P.lam * P.delta) < 1e-14


@pytest.mark.parametrize("precond", ["prior", "jacobi"])
@pytest.mark.parametrize("prec", ["fp64", "df32"])
def test_warm_start(pb, prec, precond):
    """Sec. S4.1: beta_0 in the output buffer.  beta_0 = 0 gives the cold
    draw bit for bit; beta_0 = the solution stops before any product;
    beta_0 = an early iterate is refined to the oracle's warm-started draw,
    taking its iteration count (same k on this well-conditioned instance)."""
    P = well_conditioned()
    X, a = device_problem(P)
    kw = dict(tol=1e-10, max_iter=2000)
    cold = draw(pb, pb.Context(precision=prec, stop_rule="relative", preconditioner=precond), P, X, a, **kw)
    ctx = pb.Context(precision=prec, stop_rule="relative", preconditioner=precond, warm_start=True)
    zero = torch.zeros(P.X.p, dtype=torch.float64, device=dev())
    res0 = draw(pb, ctx, P, X, a, out=zero, **kw)
    assert res0.iters == cold.iters and torch.equal(res0.beta, cold.beta)
    b = O.build_b(P.X, P.omega, P.z, P.lam, P.tau, P.eta, P.delta)
    minv = 1.0 / O.phi_diag(P.X, P.omega, P.lam, P.tau) if precond == "jacobi" else None
    chol = O.draw_beta_chol(P.X, P.omega, P.z, P.lam, P.tau, P.eta, P.delta)
    at = draw(pb, ctx, P, X, a, out=T(chol), tol=1e-8, max_iter=100)
    assert at.status == pb.PCG_OK and at.iters == 0 and np.array_equal(at.beta.cpu().numpy(), chol)
    early = O.pcg(P.X, P.omega, P.lam, P.tau, b, fixed_iters=3, minv=minv)[0]
    ref, k, _, st = O.pcg(P.X, P.omega, P.lam, P.tau, b, tol=1e-10, stop_rule=O.STOP_RELATIVE,
                          beta0=early, minv=minv)
    res = draw(pb, ctx, P, X, a, out=T(early), **kw)
    assert res.status == pb.PCG_OK and abs(res.iters - k) <= SLACK and 0 < k < cold.iters, (res.iters, k)
    assert rel(res.beta.cpu().numpy(), ref) < 1e-8 and rel(res.beta.cpu().numpy(), chol) < 1e-8


def test_warm_start_solve_and_argument_checks(pb):
    P = well_conditioned()
    X, a = device_problem(P)
    b = O.build_b(P.X, P.omega, P.z, P.lam, P.tau, P.eta, P.delta)
    chol = O.draw_beta_chol(P.X, P.omega, P.z, P.lam, P.tau, P.eta, P.delta)
    ctx = pb.Context(precision="fp64", stop_rule="relative", warm_start=True)
    x0 = T(0.5 * chol)
    res = pb.pcg_solve(ctx, X, a["omega"], a["lam"], P.tau, T(b), tol=1e-12, max_iter=1000, out=x0)
    assert res.status == pb.PCG_OK and rel(res.beta.cpu().numpy(), chol) < 1e-9
    with pytest.raises(ValueError):
        pb.pcg_draw_beta(ctx, X, a["omega"], a["z"], a["lam"], P.tau, a["eta"], a["delta"])
    # the batched and uneven paths and the adjoint refuse the options they do not run
    Q = inputs.make_problem(500, 60, -2.0, -1.0, seed=3, nrhs=2, tau=0.05)
    XQ = pb.DeviceDesign.from_host(Q.X, dev())
    for opts in (dict(preconditioner="jacobi"), dict(warm_start=True)):
        c = pb.Context(precision="df32", **opts)
        with pytest.raises(pb.PcgError) as ei:
            pb.pcg_draw_beta_batched(c, XQ, T(Q.omega), T(Q.z), T(Q.lam), T(Q.tau), T(Q.eta), T(Q.delta),
                                     out=torch.zeros((2, Q.X.p), dtype=torch.float64, device=dev()))
        assert ei.value.status == pb.PCG_BADARG
    c = pb.Context(precision="fp64", warm_start=True)
    with pytest.raises(pb.PcgError) as ei:
        pb.pcg_adjoint(c, X, a["omega"], a["z"], a["lam"], P.tau, a["eta"], a["delta"], T(chol), T(b))
    assert ei.value.status == pb.PCG_BADARG
    with pytest.raises(pb.PcgError):
        pb.Context(precision="fp64", preconditioner=7)


def test_adaptive_choice_picks_the_faster_preconditioner(pb):
    """Sec. 3's adaptive choice with library contexts: on config 2, whose Phi
    is strongly diagonally dominant, the Jacobi draw (6 iterations) beats the
    prior one (about 130); every returned draw meets the stop rule for its
    true residual."""
    from paper_1810_12437_gb300.adaptive import AdaptivePreconditioner
    P = inputs.config2()
    X, a = device_problem(P)
    ad = AdaptivePreconditioner(lambda name: pb.Context(precision="df32", preconditioner=name), period=2)
    b = O.build_b(P.X, P.omega, P.z, P.lam, P.tau, P.eta, P.delta)
    for step in range(3):
        res = ad.run(step, lambda ctx: draw(pb, ctx, P, X, a, tol=1e-6, max_iter=5000))
        assert res.status == pb.PCG_OK
        rt = P.tau * P.lam * (b - O.phi_mul(P.X, P.omega, P.lam, P.tau, res.beta.cpu().numpy()))
        assert np.sqrt(np.mean(rt ** 2)) <= 1.5e-6
    assert ad.current == "jacobi" and len(ad.history) == 2
