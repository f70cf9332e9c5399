"""Autograd wrappers of the CUDA draw (argument marshalling only).

``PcgBetaFn.apply(omega, log_lambda, log_tau, z, eta, delta, X, ctx, tol, max_iter)``
returns the draw beta of Prop. 2.1 with lambda = exp(log_lambda), tau =
exp(log_tau); its backward calls ``pcg_adjoint`` in DRAW mode, i.e. one more
prior-preconditioned CG solve Phi g = dL/dbeta and fused products, giving
gradients for omega, log_lambda and log_tau with (z, eta, delta) held fixed.

``PcgSolveFn.apply(omega, log_lambda, log_tau, b, X, ctx, tol, max_iter)``
returns beta = Phi^-1 b and differentiates in SOLVE mode (b is an input).

Both are implicit differentiation of beta = Phi^-1 b with
Phi = X^T Omega X + tau^-2 Lambda^-2; the paper has no counterpart.
"""
from __future__ import annotations

import math

import torch

from . import _native as nat


def _f64(t):
    return t.detach().to(torch.float64).contiguous()


class PcgBetaFn(torch.autograd.Function):
    @staticmethod
    def forward(fctx, omega, log_lambda, log_tau, z, eta, delta, X, pctx, tol=1e-10, max_iter=10_000):
        lam = torch.exp(_f64(log_lambda))
        tau = math.exp(float(log_tau))
        om, zz, et, de = _f64(omega), _f64(z), _f64(eta), _f64(delta)
        res = nat.pcg_draw_beta(pctx, X, om, zz, lam, tau, et, de, tol=tol, max_iter=max_iter)
        if res.status != nat.PCG_OK:
            raise nat.PcgError(res.status, pctx.last_error())
        fctx.save_for_backward(om, lam, zz, et, de, res.beta)
        fctx.tau, fctx.X, fctx.pctx, fctx.tol, fctx.max_iter = tau, X, pctx, tol, max_iter
        return res.beta.clone()

    @staticmethod
    def backward(fctx, grad_beta):
        om, lam, zz, et, de, beta = fctx.saved_tensors
        g = nat.pcg_adjoint(fctx.pctx, fctx.X, om, zz, lam, fctx.tau, et, de, beta, _f64(grad_beta),
                            mode="draw", tol=fctx.tol, max_iter=fctx.max_iter)
        if g["status"] != nat.PCG_OK:
            raise nat.PcgError(g["status"], fctx.pctx.last_error())
        g_tau = torch.tensor(g["log_tau"], dtype=torch.float64, device=beta.device)
        return g["omega"], g["log_lambda"], g_tau, None, None, None, None, None, None, None


class PcgSolveFn(torch.autograd.Function):
    @staticmethod
    def forward(fctx, omega, log_lambda, log_tau, b, X, pctx, tol=1e-10, max_iter=10_000):
        lam = torch.exp(_f64(log_lambda))
        tau = math.exp(float(log_tau))
        om, bb = _f64(omega), _f64(b)
        res = nat.pcg_solve(pctx, X, om, lam, tau, bb, tol=tol, max_iter=max_iter)
        if res.status != nat.PCG_OK:
            raise nat.PcgError(res.status, pctx.last_error())
        fctx.save_for_backward(om, lam, res.beta)
        fctx.tau, fctx.X, fctx.pctx, fctx.tol, fctx.max_iter = tau, X, pctx, tol, max_iter
        return res.beta.clone()

    @staticmethod
    def backward(fctx, grad_beta):
        om, lam, beta = fctx.saved_tensors
        g = nat.pcg_adjoint(fctx.pctx, fctx.X, om, None, lam, fctx.tau, None, None, beta,
                            _f64(grad_beta), mode="solve", tol=fctx.tol, max_iter=fctx.max_iter)
        if g["status"] != nat.PCG_OK:
            raise nat.PcgError(g["status"], fctx.pctx.last_error())
        g_tau = torch.tensor(g["log_tau"], dtype=torch.float64, device=beta.device)
        return g["omega"], g["log_lambda"], g_tau, g["b"], None, None, None, None
