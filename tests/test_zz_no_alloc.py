"""The allocation-free product pcg_phi_mul_noalloc, called through the C ABI.

Callers that cannot allocate device memory (inside a stream capture, under a
host allocator that owns the device, in latency-critical loops) use this
entry point; its intermediate lives in a fixed 8 MiB device array instead of
a context workspace.  The tests compare it, on two calls in a row, with the
oracle's Phi v and with pcg_phi_mul (float64 mode), within the float64
product tolerance the other parity tests use; they cover the largest n the
fixed array accepts, n = 0 (no rows: Phi v = tau^-2 lambda^-2 v), and check
that an oversized n is rejected before any GPU work.  The file is collected
last so that a stopped run has run the rest.
"""
import ctypes

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_1810_12437_gb300 import inputs
from tests.gpu_helpers import T, dev, need_gpu

pytestmark = pytest.mark.gpu


def _lib():
    need_gpu()
    import paper_1810_12437_gb300 as pb
    return pb, pb.load_library()


def _call(lib, X, om, lam, tau, vt, out, stream):
    csr, csc = X.csr(), X.csc()
    return lib.pcg_phi_mul_noalloc(ctypes.byref(csr), ctypes.byref(csc),
                                   ctypes.c_void_p(om.data_ptr() if om.numel() else 0),
                                   ctypes.c_void_p(lam.data_ptr()), float(tau),
                                   ctypes.c_void_p(vt.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                   ctypes.c_void_p(stream.cuda_stream))


def _magnitude(P, v):
    """Sum of the absolute terms of Phi v (the scale of its rounding error)."""
    return O.xt_mul(P.X, P.omega * O.x_mul(P.X, np.abs(v))) + np.abs(v) / (P.tau * P.lam) ** 2


def _check(P, calls=2, against_context=True):
    pb, lib = _lib()
    X = pb.DeviceDesign.from_host(P.X, dev())
    om, lam = T(P.omega), T(P.lam)
    ctx = pb.Context(precision="fp64") if against_context else None
    stream = torch.cuda.current_stream(dev())
    rng = np.random.default_rng(11)
    for call in range(calls):
        v = rng.standard_normal(P.X.p)
        vt = T(v)
        out = torch.full((P.X.p,), float("nan"), dtype=torch.float64, device=dev())
        assert _call(lib, X, om, lam, P.tau, vt, out, stream) == pb.PCG_OK
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got)), call
        tol = 1e-13 * _magnitude(P, v)
        assert np.all(np.abs(got - O.phi_mul(P.X, P.omega, P.lam, P.tau, v)) <= tol), call
        if ctx is not None:
            ref = pb.pcg_phi_mul(ctx, X, om, lam, P.tau, vt).cpu().numpy()
            assert np.all(np.abs(got - ref) <= tol), call


def test_noalloc_phi_mul_matches_oracle_and_context_entry_point():
    _check(inputs.config2())


def test_noalloc_phi_mul_at_the_largest_n():
    """n equal to the fixed array's size (2^20 rows), a sparse design."""
    pb, _ = _lib()
    P = inputs.make_problem(pb.NOALLOC_MAX_N, 1500, -4.0, -2.0, seed=inputs.SEED_BASE + 70, tau=0.05)
    assert P.X.n == pb.NOALLOC_MAX_N
    _check(P, calls=2, against_context=False)


def test_noalloc_phi_mul_without_rows():
    """n = 0: X^T Omega X vanishes and Phi v = tau^-2 lambda^-2 v."""
    pb, lib = _lib()
    p = 37
    rng = np.random.default_rng(12)
    lam, v, tau = rng.uniform(0.5, 2.0, p), rng.standard_normal(p), 0.3
    X = pb.DeviceDesign(0, p, torch.zeros(1, dtype=torch.int64, device=dev()),
                        torch.zeros(0, dtype=torch.int32, device=dev()),
                        torch.zeros(p + 1, dtype=torch.int64, device=dev()),
                        torch.zeros(0, dtype=torch.int32, device=dev()))
    om = torch.zeros(0, dtype=torch.float64, device=dev())
    out = torch.full((p,), float("nan"), dtype=torch.float64, device=dev())
    assert _call(lib, X, om, T(lam), tau, T(v), out, torch.cuda.current_stream(dev())) == pb.PCG_OK
    torch.cuda.synchronize()
    want = v / (tau * lam) ** 2
    assert np.all(np.abs(out.cpu().numpy() - want) <= 1e-15 * np.abs(want))


def test_noalloc_rejects_oversized_n():
    pb, lib = _lib()
    n = pb.NOALLOC_MAX_N + 1
    p = 4
    # real, correctly sized buffers: a rejected call must not touch them anyway
    X = pb.DeviceDesign(n, p, torch.zeros(n + 1, dtype=torch.int64, device=dev()),
                        torch.zeros(0, dtype=torch.int32, device=dev()),
                        torch.zeros(p + 1, dtype=torch.int64, device=dev()),
                        torch.zeros(0, dtype=torch.int32, device=dev()))
    om = torch.full((n,), 0.1, dtype=torch.float64, device=dev())
    lam = torch.ones(p, dtype=torch.float64, device=dev())
    v = torch.ones(p, dtype=torch.float64, device=dev())
    out = torch.zeros(p, dtype=torch.float64, device=dev())
    csr, csc = X.csr(), X.csc()
    st = lib.pcg_phi_mul_noalloc(ctypes.byref(csr), ctypes.byref(csc), ctypes.c_void_p(om.data_ptr()),
                                 ctypes.c_void_p(lam.data_ptr()), 1.0, ctypes.c_void_p(v.data_ptr()),
                                 ctypes.c_void_p(out.data_ptr()), None)
    assert st == pb.PCG_BADARG
    torch.cuda.synchronize()
    assert float(out.abs().max()) == 0.0
