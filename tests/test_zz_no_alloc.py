"""The allocation-free product pcg_phi_mul_noalloc, called through the C ABI.

Callers that cannot allocate device memory (inside a stream capture, under a
host allocator that owns the device, in latency-critical loops) use this
entry point; its intermediate lives in a fixed 8 MiB device array instead of
a context workspace.  The test compares it with pcg_phi_mul (float64 mode) on
two calls in a row, within the float64 product tolerance the other parity
tests use, and checks that an oversized n is rejected before any GPU work.
It sits in a file collected last so that a stopped run has run the rest.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_1810_12437_gb300 import inputs
from tests.gpu_helpers import T, dev, need_gpu

pytestmark = pytest.mark.gpu


def test_noalloc_phi_mul_matches_context_entry_point():
    need_gpu()
    import paper_1810_12437_gb300 as pb
    from paper_1810_12437_gb300._native import _Csc, _Csr
    lib = pb.load_library()
    P = inputs.config2()
    X = pb.DeviceDesign.from_host(P.X, dev())
    om, lam = T(P.omega), T(P.lam)
    ctx = pb.Context(precision="fp64")
    csr, csc = X.csr(), X.csc()
    stream = torch.cuda.current_stream(dev())
    rng = np.random.default_rng(11)
    x_abs = lambda v: np.abs(v)
    for call in range(2):
        v = rng.standard_normal(P.X.p)
        vt = T(v)
        out = torch.full((P.X.p,), float("nan"), dtype=torch.float64, device=dev())
        st = lib.pcg_phi_mul_noalloc(ctypes.byref(csr), ctypes.byref(csc),
                                     ctypes.c_void_p(om.data_ptr()), ctypes.c_void_p(lam.data_ptr()),
                                     float(P.tau), ctypes.c_void_p(vt.data_ptr()),
                                     ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
        assert st == pb.PCG_OK
        torch.cuda.synchronize()
        ref = pb.pcg_phi_mul(ctx, X, om, lam, P.tau, vt).cpu().numpy()
        got = out.cpu().numpy()
        # the float64 product tolerance of the pcg_phi_mul parity test
        from oracle import oracle as O
        mag = O.xt_mul(P.X, P.omega * O.x_mul(P.X, x_abs(v))) + x_abs(v) / (P.tau * P.lam) ** 2
        assert np.all(np.isfinite(got)), call
        assert np.all(np.abs(got - ref) <= 1e-13 * mag), call


def test_noalloc_rejects_oversized_n():
    need_gpu()
    import paper_1810_12437_gb300 as pb
    lib = pb.load_library()
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
