"""Failure statuses on the GPU, for every entry point that solves.

Each failure is made by an input value or a short wait, never by a device
fault: a NaN in delta makes b, and so the first CG scalar rho_0, NaN
(PCG_NONFINITE before any product); omega_i = -1e12 on every row makes Phi =
X^T Omega X + tau^-2 Lambda^-2 indefinite, so that the first curvature s.Phi s
is negative (PCG_BREAKDOWN at the first product, as Sec. 2.4's SPD argument
no longer holds) -- reachable through pcg_solve, which takes b as given: in a
draw, Eq. 2.3's Omega^1/2 turns a negative omega into a NaN right-hand side
(PCG_NONFINITE, as the draws below show); an idle limit of one microsecond
makes the uneven batch's idle CTAs give up (PCG_TIMEOUT) while another CTA is
still working.  The oracle reports the same status at the same iteration on
the same inputs, and the context stays usable afterwards."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_1810_12437_gb300 import inputs
from tests.gpu_helpers import T, dev, device_problem, need_gpu, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pb():
    need_gpu()
    import paper_1810_12437_gb300 as pb
    pb.load_library()
    return pb


def base_problem(seed=61):
    P = inputs.make_problem(3000, 400, -2.0, -1.0, seed=seed, tau=0.05)
    P.lam = np.random.default_rng(seed).uniform(0.5, 2.0, P.X.p)
    return P


def with_nan_delta(P):
    P.delta = P.delta.copy()
    P.delta[3] = np.nan
    return P


def with_indefinite_omega(P):
    P.omega = np.full_like(P.omega, -1e12)
    return P


def oracle_status(P):
    _, k, _, st = O.draw_beta_cg(P.X, P.omega, P.z, P.lam, P.tau, P.eta, P.delta, tol=1e-8,
                                 max_iter=1000)
    return st, k


STATUS = {O.NONFINITE: "PCG_NONFINITE", O.BREAKDOWN: "PCG_BREAKDOWN", O.OK: "PCG_OK"}


@pytest.mark.parametrize("prec", ["fp64", "df32", "fx64", "fp32_refined"])
def test_single_draw_statuses(pb, prec):
    ctx = pb.Context(precision=prec)
    for make, want in ((with_nan_delta, O.NONFINITE), (with_indefinite_omega, O.NONFINITE)):
        P = make(base_problem())
        st_ref, k_ref = oracle_status(P)
        assert st_ref == want and k_ref == 0
        X, a = device_problem(P)
        res = pb.pcg_draw_beta(ctx, X, a["omega"], a["z"], a["lam"], P.tau, a["eta"], a["delta"],
                               tol=1e-8, max_iter=1000)
        assert res.status == getattr(pb, STATUS[want]) and res.iters == k_ref, (prec, make, res.status)
    # breakdown: the indefinite Phi with a finite right-hand side (pcg_solve)
    P = base_problem()
    b = O.build_b(P.X, P.omega, P.z, P.lam, P.tau, P.eta, P.delta)
    Q = with_indefinite_omega(base_problem())
    _, k_ref, _, st_ref = O.pcg(Q.X, Q.omega, Q.lam, Q.tau, b, tol=1e-8, max_iter=1000)
    assert st_ref == O.BREAKDOWN and k_ref == 0
    X, a = device_problem(Q)
    res = pb.pcg_solve(ctx, X, a["omega"], a["lam"], Q.tau, T(b), tol=1e-8, max_iter=1000)
    assert res.status == pb.PCG_BREAKDOWN and res.iters == 0, (prec, res.status)
    # the same context then draws a valid problem correctly
    P = base_problem()
    X, a = device_problem(P)
    res = pb.pcg_draw_beta(ctx, X, a["omega"], a["z"], a["lam"], P.tau, a["eta"], a["delta"],
                           tol=1e-8, max_iter=1000)
    ref = O.draw_beta_cg(P.X, P.omega, P.z, P.lam, P.tau, P.eta, P.delta, tol=1e-8)[0]
    assert res.status == pb.PCG_OK and rel(res.beta.cpu().numpy(), ref) < 1e-6


@pytest.mark.parametrize("prec", ["df32", "fx64", "fp32_refined"])
def test_batched_per_chain_statuses(pb, prec):
    """Four chains on one X: a NaN delta in chain 1 and a negative omega in
    chain 2 (a NaN right-hand side through Eq. 2.3's Omega^1/2) stop those
    chains as non-finite; chains 0 and 3 converge and match the oracle."""
    Q = inputs.make_problem(3000, 400, -2.0, -1.0, seed=62, nrhs=4, tau_log10_range=(-1.6, -1.0))
    Q.lam = np.random.default_rng(62).uniform(0.5, 2.0, Q.lam.shape)
    Q.delta[1, 3] = np.nan
    Q.omega[2] = -1e12
    X = pb.DeviceDesign.from_host(Q.X, dev())
    ctx = pb.Context(precision=prec)
    res = pb.pcg_draw_beta_batched(ctx, X, omega=T(Q.omega), z=T(Q.z), lam=T(Q.lam), tau=T(Q.tau),
                                   eta=T(Q.eta), delta=T(Q.delta), tol=1e-8, max_iter=2000)
    assert list(res.status) == [pb.PCG_OK, pb.PCG_NONFINITE, pb.PCG_NONFINITE, pb.PCG_OK], list(res.status)
    assert res.iters[1] == 0 and res.iters[2] == 0
    beta = res.beta.cpu().numpy()
    for r in (0, 3):
        ref = O.draw_beta_cg(Q.X, Q.omega[r], Q.z[r], Q.lam[r], float(Q.tau[r]), Q.eta[r], Q.delta[r],
                             tol=1e-8)[0]
        assert rel(beta[r], ref) < 1e-5, r


def as_device(pb, P):
    X = pb.DeviceDesign.from_host(P.X, dev())
    return dict(X=X, omega=T(P.omega), z=T(P.z), lam=T(P.lam), tau=float(P.tau), eta=T(P.eta),
                delta=T(P.delta))


@pytest.mark.parametrize("prec", ["fp64", "fp32_refined"])
def test_uneven_per_problem_statuses(pb, prec):
    probs = [base_problem(63), with_nan_delta(base_problem(64)), with_indefinite_omega(base_problem(65)),
             inputs.make_problem(900, 150, -2.0, -1.0, seed=66, tau=0.05)]
    want = [oracle_status(P)[0] for P in probs]
    assert want == [O.OK, O.NONFINITE, O.NONFINITE, O.OK]
    ctx = pb.Context(precision=prec)
    res = pb.pcg_draw_beta_uneven(ctx, [as_device(pb, P) for P in probs], tol=1e-8, max_iter=2000)
    assert [r.status for r in res] == [getattr(pb, STATUS[w]) for w in want]
    assert res[1].iters == 0 and res[2].iters == 0
    for q in (0, 3):
        P = probs[q]
        ref = O.draw_beta_cg(P.X, P.omega, P.z, P.lam, P.tau, P.eta, P.delta, tol=1e-8)[0]
        assert rel(res[q].beta.cpu().numpy(), ref) < 1e-5, q


def test_uneven_idle_limit_gives_timeout(pb):
    """The uneven kernel's only wait is that of a CTA which finds no work: it
    gives up once no tile anywhere has completed for the idle limit.  With a
    limit of one microsecond, idle CTAs give up while the large member's
    tiles are still running; every CTA then leaves at its next claim (none
    waits for another), the call returns PCG_TIMEOUT, and a context with the
    default limit then draws the same batch correctly on the same device."""
    probs = [inputs.make_problem(120_000, 12_000, -4.0, -1.5, seed=67, tau=0.01),
             inputs.make_problem(2000, 300, -2.0, -1.0, seed=68, tau=0.01)]
    d = [as_device(pb, P) for P in probs]
    ctx = pb.Context(precision="fp64", idle_limit_s=1e-6)
    with pytest.raises(pb.PcgError) as ei:
        pb.pcg_draw_beta_uneven(ctx, d, tol=1e-6, max_iter=20_000)
    assert ei.value.status == pb.PCG_TIMEOUT
    torch.cuda.synchronize()
    ok = pb.Context(precision="fp64")
    res = pb.pcg_draw_beta_uneven(ok, d, tol=1e-6, max_iter=20_000)
    for P, r in zip(probs, res):
        ref = O.draw_beta_cg(P.X, P.omega, P.z, P.lam, P.tau, P.eta, P.delta, tol=1e-6)[0]
        assert r.status == pb.PCG_OK and rel(r.beta.cpu().numpy(), ref) < 1e-6


@pytest.mark.parametrize("bad", [0.0, -1.0, float("nan"), 1e9])
def test_idle_limit_option_checked(pb, bad):
    with pytest.raises(pb.PcgError) as ei:
        pb.Context(precision="fp64", idle_limit_s=bad)
    assert ei.value.status == pb.PCG_BADARG
