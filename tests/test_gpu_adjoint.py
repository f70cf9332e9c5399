"""Parity of the adjoint (gradient of L = c^T beta through one more
prior-preconditioned CG solve) with the oracle's dense-Cholesky gradient, and
of the autograd wrapper with central finite differences of the CUDA draw."""
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


@pytest.mark.parametrize("mode", ["draw", "solve"])
@pytest.mark.parametrize("prec,bound,tol", [("fp64", 1e-8, 1e-12), ("fp32_refined", 1e-5, 1e-9)])
def test_adjoint_matches_cholesky_gradient(pb, mode, prec, bound, tol):
    P = inputs.config5_small()
    X, a = device_problem(P)
    ctx = pb.Context(precision=prec, stop_rule="relative")
    dr = pb.pcg_draw_beta(ctx, X, a["omega"], a["z"], a["lam"], P.tau, a["eta"], a["delta"],
                          tol=tol, max_iter=5000)
    g = pb.pcg_adjoint(ctx, X, a["omega"], a["z"], a["lam"], P.tau, a["eta"], a["delta"], dr.beta,
                       T(P.c), mode=mode, tol=tol, max_iter=5000)
    assert dr.status == pb.PCG_OK and g["status"] == pb.PCG_OK
    beta_c, gc = O.adjoint_chol(P.X, P.omega, P.z, P.lam, P.tau, P.eta, P.delta, P.c, mode=mode)
    assert rel(dr.beta.cpu().numpy(), beta_c) < bound
    for key in ("b", "omega", "log_lambda"):
        assert rel(g[key].cpu().numpy(), gc[key]) < bound, key
    assert abs(g["log_tau"] - gc["log_tau"]) <= bound * (abs(gc["log_tau"]) + np.abs(gc["log_lambda"]).sum())


@pytest.mark.slow
def test_adjoint_config5_against_oracle_cg(pb):
    """n = 2e5, p = 2e4: refined-mode gradient against the oracle's CG gradient."""
    P = inputs.config5()
    X, a = device_problem(P)
    ctx = pb.Context(precision="fp32_refined")
    dr = pb.pcg_draw_beta(ctx, X, a["omega"], a["z"], a["lam"], P.tau, a["eta"], a["delta"],
                          tol=1e-8, max_iter=5000)
    g = pb.pcg_adjoint(ctx, X, a["omega"], a["z"], a["lam"], P.tau, a["eta"], a["delta"], dr.beta,
                       T(P.c), mode="draw", tol=1e-8, max_iter=5000)
    beta_o, go = O.adjoint_cg(P.X, P.omega, P.z, P.lam, P.tau, P.eta, P.delta, P.c, tol=1e-8)
    assert rel(dr.beta.cpu().numpy(), beta_o) < 1e-5
    for key in ("b", "omega", "log_lambda"):
        assert rel(g[key].cpu().numpy(), go[key]) < 1e-5, key


@pytest.mark.parametrize("mode", ["draw", "solve"])
def test_autograd_against_central_differences(pb, mode):
    """torch.autograd through the CUDA draw (float64 mode, tight tolerance)
    against central differences h = 1e-6 of the CUDA forward itself."""
    from paper_1810_12437_gb300.autograd import PcgBetaFn, PcgSolveFn
    P = inputs.make_problem(300, 60, -1.5, -0.6, seed=61, tau=0.1, with_c=True)
    X, a = device_problem(P)
    ctx = pb.Context(precision="fp64", stop_rule="relative")
    c = T(P.c)
    b0 = T(O.build_b(P.X, P.omega, P.z, P.lam, P.tau, P.eta, P.delta))

    def loss(om, ll, lt, b=None):
        if mode == "draw":
            beta = PcgBetaFn.apply(om, ll, lt, a["z"], a["eta"], a["delta"], X, ctx, 1e-14, 5000)
        else:
            beta = PcgSolveFn.apply(om, ll, lt, b0 if b is None else b, X, ctx, 1e-14, 5000)
        return (c * beta).sum()

    om = a["omega"].clone().requires_grad_(True)
    ll = torch.log(a["lam"]).clone().requires_grad_(True)
    lt = torch.tensor(np.log(P.tau), dtype=torch.float64, device=dev(), requires_grad=True)
    bb = b0.clone().requires_grad_(True)
    L = loss(om, ll, lt, bb if mode == "solve" else None)
    L.backward()
    h = 1e-6
    with torch.no_grad():
        for j in (0, 17, 59):
            e = torch.zeros_like(ll)
            e[j] = h
            fd = (loss(om, ll + e, lt) - loss(om, ll - e, lt)).item() / (2 * h)
            assert fd == pytest.approx(ll.grad[j].item(), rel=1e-5, abs=1e-7 * (abs(fd) + 1))
        fd = (loss(om, ll, lt + h) - loss(om, ll, lt - h)).item() / (2 * h)
        assert fd == pytest.approx(lt.grad.item(), rel=1e-5, abs=1e-8)
        for i in (0, 150, 299):
            e = torch.zeros_like(om)
            e[i] = h
            fd = (loss(om + e, ll, lt) - loss(om - e, ll, lt)).item() / (2 * h)
            assert fd == pytest.approx(om.grad[i].item(), rel=1e-5, abs=1e-7 * (abs(fd) + 1))
        if mode == "solve":
            for j in (3, 40):
                e = torch.zeros_like(bb)
                e[j] = 1.0
                fd = (loss(om, ll, lt, bb + e) - loss(om, ll, lt, bb - e)).item() / 2.0
                assert fd == pytest.approx(bb.grad[j].item(), rel=1e-7, abs=1e-12)
