"""Thin ctypes binding of the C ABI in ``include/pcg_beta.h``.

Only argument marshalling lives here: torch CUDA tensors are checked for
device, dtype, contiguity and length, and their device pointers are handed to
the library, which runs every step of the draw in its own CUDA kernels.
There is no CPU path: if the library is missing the first call raises.
The function names are those of the C entry points.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import threading
from typing import Optional, Sequence

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_pcg_beta.so")

PCG_OK, PCG_MAXITER, PCG_BREAKDOWN, PCG_NONFINITE, PCG_BADARG, PCG_TIMEOUT, PCG_CUDA = range(7)
STATUS_NAMES = {0: "OK", 1: "MAXITER", 2: "BREAKDOWN", 3: "NONFINITE", 4: "BADARG",
                5: "TIMEOUT", 6: "CUDA"}
PREC = {"fp64": 0, "fp32_refined": 1, "fp32": 2, "df32": 3, "fx64": 4}
STOP = {"rms": 0, "paper_rms": 0, "relative": 1}
ADJ = {"solve": 0, "draw": 1}
PRECOND = {"prior": 0, "jacobi": 1}


class PcgError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class _Csr(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("p", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("row_ptr", ctypes.c_void_p), ("col_idx", ctypes.c_void_p)]


class _Csc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("p", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("col_ptr", ctypes.c_void_p), ("row_idx", ctypes.c_void_p)]


class _Options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("reliable_k", ctypes.c_int),
                ("stop_rule", ctypes.c_int), ("use_graph", ctypes.c_int),
                ("autotune_cache", ctypes.c_char_p), ("profile", ctypes.c_int),
                ("idle_limit_s", ctypes.c_double), ("preconditioner", ctypes.c_int),
                ("warm_start", ctypes.c_int)]


class _Problem(ctypes.Structure):
    _fields_ = [("X_csr", _Csr), ("X_csc", _Csc), ("omega", ctypes.c_void_p),
                ("z", ctypes.c_void_p), ("lambda_", ctypes.c_void_p), ("eta", ctypes.c_void_p),
                ("delta", ctypes.c_void_p), ("tau", ctypes.c_double), ("beta", ctypes.c_void_p)]


_lib = None
_lock = threading.Lock()


def load_library(path: str = LIB_PATH):
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(
                f"the CUDA library {path} is missing: build it with "
                "`python -c 'import __graft_entry__ as g; g.build()'` (there is no CPU fallback)")
        lib = ctypes.CDLL(path)
        P, D, I, I64 = ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_int64
        pI, pD = ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)
        pCsr, pCsc = ctypes.POINTER(_Csr), ctypes.POINTER(_Csc)
        sig = {
            "pcg_options_default": ([ctypes.POINTER(_Options)], I),
            "pcg_ctx_create": ([ctypes.POINTER(P), ctypes.POINTER(_Options), P], I),
            "pcg_ctx_destroy": ([P], None),
            "pcg_last_error": ([P], ctypes.c_char_p),
            "pcg_check_design": ([P, pCsr, pCsc], I),
            "pcg_set_unshrunk": ([P, I, P, P], I),
            "pcg_build_rhs": ([P, pCsc, P, P, P, D, P, P, P], I),
            "pcg_phi_mul": ([P, pCsr, pCsc, P, P, D, P, P], I),
            "pcg_draw_beta": ([P, pCsr, pCsc, P, P, P, D, P, P, D, I, P, pI, pD], I),
            "pcg_solve": ([P, pCsr, pCsc, P, P, D, P, D, I, P, pI, pD], I),
            "pcg_draw_beta_batched": ([P, pCsr, pCsc, I, P, P, P, P, P, P, D, I, P, pI, pD, pI], I),
            "pcg_draw_beta_uneven": ([P, I, ctypes.POINTER(_Problem), D, I, pI, pD, pI], I),
            "pcg_adjoint": ([P, pCsr, pCsc, P, P, P, D, P, P, P, P, I, D, I, P, P, P, pD, pI, pD], I),
            "pcg_profile_count": ([P], I),
            "pcg_profile_entry": ([P, I, ctypes.POINTER(ctypes.c_char_p), pD,
                                   ctypes.POINTER(ctypes.c_int64)], I),
            "pcg_profile_reset": ([P], None),
            "pcg_last_kernel_launches": ([P], I64),
            "pcg_phi_mul_noalloc": ([pCsr, pCsc, P, P, D, P, P, P], I),
            "pcg_tiled_plan_applies": ([I64, I64, I64, I, I, pI, pI], I),
            "pcg_draw_beta_lsqr": ([P, pCsr, pCsc, P, P, P, D, P, P, D, I, P, pI, pD], I),
            "pcg_gibbs_step": ([P, pCsr, pCsc, P, ctypes.c_uint64, ctypes.c_uint32, P, P, P, pD, pD, P, D, I,
                                pI, pD], I),
        }
        for name, (args, res) in sig.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = res
        _lib = lib
        return lib


def exported_symbols() -> Sequence[str]:
    return ["pcg_options_default", "pcg_ctx_create", "pcg_ctx_destroy", "pcg_last_error",
            "pcg_check_design", "pcg_build_rhs", "pcg_phi_mul", "pcg_draw_beta", "pcg_solve",
            "pcg_draw_beta_batched", "pcg_draw_beta_uneven", "pcg_adjoint", "pcg_profile_count",
            "pcg_profile_entry", "pcg_profile_reset", "pcg_last_kernel_launches",
            "pcg_phi_mul_noalloc", "pcg_set_unshrunk", "pcg_tiled_plan_applies", "pcg_draw_beta_lsqr",
            "pcg_gibbs_step"]


# ---------------------------------------------------------------------------
# argument helpers
# ---------------------------------------------------------------------------

def _ptr(t: Optional[torch.Tensor]):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _dev(t, dtype, numel, name, device):
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch tensor")
    if t.device.type != "cuda":
        raise ValueError(f"{name} must be on a CUDA device")
    if device is not None and t.device != device:
        raise ValueError(f"{name} is on {t.device}, expected {device}")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} has {t.numel()} elements, expected {numel}")
    return t


@dataclasses.dataclass
class DeviceDesign:
    """Binary X held on the device as indices only, in CSR and CSC layouts."""

    n: int
    p: int
    row_ptr: torch.Tensor
    col_idx: torch.Tensor
    col_ptr: torch.Tensor
    row_idx: torch.Tensor

    @property
    def nnz(self) -> int:
        return int(self.col_idx.numel())

    @property
    def device(self):
        return self.row_ptr.device

    @classmethod
    def from_host(cls, X, device="cuda") -> "DeviceDesign":
        """Copy a host design (numpy arrays: row_ptr, col_idx, col_ptr, row_idx)."""
        t = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a)).to(device=device, dtype=dt)
        return cls(int(X.n), int(X.p), t(X.row_ptr, torch.int64), t(X.col_idx, torch.int32),
                   t(X.col_ptr, torch.int64), t(X.row_idx, torch.int32))

    def csr(self) -> _Csr:
        _dev(self.row_ptr, torch.int64, self.n + 1, "row_ptr", None)
        _dev(self.col_idx, torch.int32, None, "col_idx", None)
        return _Csr(self.n, self.p, self.nnz, self.row_ptr.data_ptr(),
                    self.col_idx.data_ptr() if self.nnz else 0)

    def csc(self) -> _Csc:
        _dev(self.col_ptr, torch.int64, self.p + 1, "col_ptr", None)
        _dev(self.row_idx, torch.int32, self.nnz, "row_idx", None)
        return _Csc(self.n, self.p, self.nnz, self.col_ptr.data_ptr(),
                    self.row_idx.data_ptr() if self.nnz else 0)


class Context:
    """Owns a ``pcg_ctx``: workspace, cached graphs, options and stream."""

    def __init__(self, precision="df32", reliable_k=50, stop_rule="rms", use_graph=True,
                 stream: Optional[torch.cuda.Stream] = None, autotune_cache: Optional[str] = None,
                 profile: bool = False, idle_limit_s: Optional[float] = None,
                 preconditioner: str = "prior", warm_start: bool = False):
        lib = load_library()
        opt = _Options()
        lib.pcg_options_default(ctypes.byref(opt))
        opt.precision = PREC[precision] if isinstance(precision, str) else int(precision)
        opt.reliable_k = int(reliable_k)
        opt.stop_rule = STOP[stop_rule] if isinstance(stop_rule, str) else int(stop_rule)
        opt.use_graph = 1 if use_graph else 0
        self._cache_path = autotune_cache.encode() if autotune_cache else None
        opt.autotune_cache = self._cache_path
        opt.profile = 1 if profile else 0
        if idle_limit_s is not None:
            opt.idle_limit_s = float(idle_limit_s)
        opt.preconditioner = PRECOND[preconditioner] if isinstance(preconditioner, str) else int(preconditioner)
        opt.warm_start = 1 if warm_start else 0
        self.warm_start = bool(warm_start)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.device = self.stream.device
        self.precision = precision
        self._h = ctypes.c_void_p(0)
        with torch.cuda.device(self.device):
            st = lib.pcg_ctx_create(ctypes.byref(self._h), ctypes.byref(opt),
                                    ctypes.c_void_p(self.stream.cuda_stream))
        if st != PCG_OK:
            raise PcgError(st, "pcg_ctx_create failed")
        self._lib = lib

    @property
    def handle(self):
        return self._h

    def last_error(self) -> str:
        return self._lib.pcg_last_error(self._h).decode()

    def close(self):
        if self._h:
            self._lib.pcg_ctx_destroy(self._h)
            self._h = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def check(self, st: int, fatal=(PCG_BADARG, PCG_TIMEOUT, PCG_CUDA)) -> int:
        if st in fatal:
            raise PcgError(st, self.last_error())
        return st


def pcg_ctx_create(**kw) -> Context:
    return Context(**kw)


def pcg_ctx_destroy(ctx: Context) -> None:
    ctx.close()


def pcg_last_error(ctx: Context) -> str:
    return ctx.last_error()


def pcg_check_design(ctx: Context, X: DeviceDesign) -> int:
    """PCG_OK or PCG_BADARG (not raised) for an invalid or inconsistent design."""
    csr, csc = X.csr(), X.csc()
    with torch.cuda.device(ctx.device):
        return ctx.check(ctx._lib.pcg_check_design(ctx.handle, ctypes.byref(csr), ctypes.byref(csc)),
                         fatal=(PCG_TIMEOUT, PCG_CUDA))


def pcg_set_unshrunk(ctx: Context, prior_prec=None, precond_scale=None) -> None:
    """Coefficients 0 .. q1-1 unshrunk (Sec. S4.3): prior precisions
    sigma_j^-2 (>= 0; 0 = flat prior) and preconditioner scales gamma_j (> 0),
    float64 device tensors of q1 entries each; None (or q1 = 0) clears."""
    f = torch.float64
    if prior_prec is None or prior_prec.numel() == 0:
        with torch.cuda.device(ctx.device):
            ctx.check(ctx._lib.pcg_set_unshrunk(ctx.handle, 0, None, None))
        return
    q1 = int(prior_prec.numel())
    dev = prior_prec.device
    _dev(prior_prec, f, q1, "prior_prec", dev)
    _dev(precond_scale, f, q1, "precond_scale", dev)
    with torch.cuda.device(ctx.device):
        ctx.check(ctx._lib.pcg_set_unshrunk(ctx.handle, q1, _ptr(prior_prec), _ptr(precond_scale)))


def pcg_build_rhs(ctx, X, omega, z, lam, tau, eta, delta, out=None):
    """b of Eq. 2.3 (float64, length p)."""
    f = torch.float64
    dev = X.device
    for name, t, m in (("omega", omega, X.n), ("z", z, X.n), ("eta", eta, X.n),
                       ("lambda", lam, X.p), ("delta", delta, X.p)):
        _dev(t, f, m, name, dev)
    out = torch.empty(X.p, dtype=f, device=dev) if out is None else _dev(out, f, X.p, "out", dev)
    csc = X.csc()
    with torch.cuda.device(ctx.device):
        ctx.check(ctx._lib.pcg_build_rhs(ctx.handle, ctypes.byref(csc), _ptr(omega), _ptr(z), _ptr(lam),
                                         float(tau), _ptr(eta), _ptr(delta), _ptr(out)))
    return out


def pcg_phi_mul(ctx, X, omega, lam, tau, v, out=None):
    """Phi v = X^T Omega X v + tau^-2 lambda^-2 v (float64 in and out)."""
    f = torch.float64
    dev = X.device
    _dev(omega, f, X.n, "omega", dev)
    _dev(lam, f, X.p, "lambda", dev)
    _dev(v, f, X.p, "v", dev)
    out = torch.empty(X.p, dtype=f, device=dev) if out is None else _dev(out, f, X.p, "out", dev)
    csr, csc = X.csr(), X.csc()
    with torch.cuda.device(ctx.device):
        ctx.check(ctx._lib.pcg_phi_mul(ctx.handle, ctypes.byref(csr), ctypes.byref(csc), _ptr(omega),
                                       _ptr(lam), float(tau), _ptr(v), _ptr(out)))
    return out


@dataclasses.dataclass
class DrawResult:
    beta: torch.Tensor
    iters: object
    resid: object
    status: object


def _warm_out(ctx, out, p, dev):
    """The output buffer; with the context's warm start it must be given and
    hold beta_0 (Sec. S4.1)."""
    f = torch.float64
    if out is None:
        if getattr(ctx, "warm_start", False):
            raise ValueError("warm_start: pass out= holding the initial vector beta_0")
        return torch.empty(p, dtype=f, device=dev)
    return _dev(out, f, p, "out", dev)


def pcg_draw_beta(ctx, X, omega, z, lam, tau, eta, delta, tol=1e-6, max_iter=10_000, out=None):
    """One draw of beta ~ N(Phi^-1 X^T Omega z, Phi^-1) (Prop. 2.1).  With a
    warm-start context, `out` holds beta_0 on entry and the draw on return."""
    f = torch.float64
    dev = X.device
    for name, t, m in (("omega", omega, X.n), ("z", z, X.n), ("eta", eta, X.n),
                       ("lambda", lam, X.p), ("delta", delta, X.p)):
        _dev(t, f, m, name, dev)
    out = _warm_out(ctx, out, X.p, dev)
    csr, csc = X.csr(), X.csc()
    it, rs = ctypes.c_int(0), ctypes.c_double(0.0)
    with torch.cuda.device(ctx.device):
        st = ctx.check(ctx._lib.pcg_draw_beta(ctx.handle, ctypes.byref(csr), ctypes.byref(csc),
                                              _ptr(omega), _ptr(z), _ptr(lam), float(tau), _ptr(eta),
                                              _ptr(delta), float(tol), int(max_iter), _ptr(out),
                                              ctypes.byref(it), ctypes.byref(rs)))
    return DrawResult(out, it.value, rs.value, st)


def pcg_draw_beta_lsqr(ctx, X, omega, z, lam, tau, eta, delta, tol=1e-6, max_iter=10_000, out=None):
    """The draw of Prop. 2.1 by LSQR on the least-squares form (Sec. S7.1),
    float64, under the context's stop rule."""
    f = torch.float64
    dev = X.device
    for name, t, m in (("omega", omega, X.n), ("z", z, X.n), ("eta", eta, X.n),
                       ("lambda", lam, X.p), ("delta", delta, X.p)):
        _dev(t, f, m, name, dev)
    out = torch.empty(X.p, dtype=f, device=dev) if out is None else _dev(out, f, X.p, "out", dev)
    csr, csc = X.csr(), X.csc()
    it, rs = ctypes.c_int(0), ctypes.c_double(0.0)
    with torch.cuda.device(ctx.device):
        st = ctx.check(ctx._lib.pcg_draw_beta_lsqr(ctx.handle, ctypes.byref(csr), ctypes.byref(csc),
                                                   _ptr(omega), _ptr(z), _ptr(lam), float(tau), _ptr(eta),
                                                   _ptr(delta), float(tol), int(max_iter), _ptr(out),
                                                   ctypes.byref(it), ctypes.byref(rs)))
    return DrawResult(out, it.value, rs.value, st)


@dataclasses.dataclass
class GibbsState:
    """State of the Gibbs sampler of Sec. S1 (horseshoe prior): device
    vectors omega (n), lam, nu, beta (p) and host scalars tau, xi."""
    omega: torch.Tensor
    lam: torch.Tensor
    nu: torch.Tensor
    beta: torch.Tensor
    tau: float
    xi: float


def pcg_gibbs_step(ctx, X, y, state: GibbsState, seed: int, step: int, tol=1e-6, max_iter=10_000):
    """One cycle tau -> lambda -> omega -> beta of Sec. S1, in place on
    `state`; returns the beta draw's DrawResult (beta is state.beta)."""
    f = torch.float64
    dev = X.device
    _dev(y, f, X.n, "y", dev)
    _dev(state.omega, f, X.n, "omega", dev)
    for name, t in (("lambda", state.lam), ("nu", state.nu), ("beta", state.beta)):
        _dev(t, f, X.p, name, dev)
    csr, csc = X.csr(), X.csc()
    it, rs = ctypes.c_int(0), ctypes.c_double(0.0)
    tau, xi = ctypes.c_double(state.tau), ctypes.c_double(state.xi)
    with torch.cuda.device(ctx.device):
        st = ctx.check(ctx._lib.pcg_gibbs_step(ctx.handle, ctypes.byref(csr), ctypes.byref(csc), _ptr(y),
                                               int(seed) & (2 ** 64 - 1), int(step) & 0xffffffff,
                                               _ptr(state.omega), _ptr(state.lam), _ptr(state.nu),
                                               ctypes.byref(tau), ctypes.byref(xi), _ptr(state.beta),
                                               float(tol), int(max_iter), ctypes.byref(it), ctypes.byref(rs)))
    state.tau, state.xi = tau.value, xi.value
    return DrawResult(state.beta, it.value, rs.value, st)


def pcg_solve(ctx, X, omega, lam, tau, rhs, tol=1e-6, max_iter=10_000, out=None):
    """Solve Phi x = rhs by the same preconditioned CG (warm start as in
    pcg_draw_beta)."""
    f = torch.float64
    dev = X.device
    _dev(omega, f, X.n, "omega", dev)
    _dev(lam, f, X.p, "lambda", dev)
    _dev(rhs, f, X.p, "rhs", dev)
    out = _warm_out(ctx, out, X.p, dev)
    csr, csc = X.csr(), X.csc()
    it, rs = ctypes.c_int(0), ctypes.c_double(0.0)
    with torch.cuda.device(ctx.device):
        st = ctx.check(ctx._lib.pcg_solve(ctx.handle, ctypes.byref(csr), ctypes.byref(csc), _ptr(omega),
                                          _ptr(lam), float(tau), _ptr(rhs), float(tol), int(max_iter),
                                          _ptr(out), ctypes.byref(it), ctypes.byref(rs)))
    return DrawResult(out, it.value, rs.value, st)


def pcg_draw_beta_batched(ctx, X, omega, z, lam, tau, eta, delta, tol=1e-6, max_iter=10_000, out=None):
    """R draws sharing X: omega, z, eta (R, n); lam, delta (R, p); tau (R,)."""
    f = torch.float64
    dev = X.device
    R = int(tau.numel())
    for name, t, m in (("omega", omega, R * X.n), ("z", z, R * X.n), ("eta", eta, R * X.n),
                       ("lambda", lam, R * X.p), ("delta", delta, R * X.p), ("tau", tau, R)):
        _dev(t, f, m, name, dev)
    out = torch.empty((R, X.p), dtype=f, device=dev) if out is None else _dev(out, f, R * X.p, "out", dev)
    csr, csc = X.csr(), X.csc()
    it = (ctypes.c_int * R)()
    rs = (ctypes.c_double * R)()
    ss = (ctypes.c_int * R)()
    with torch.cuda.device(ctx.device):
        st = ctx.check(ctx._lib.pcg_draw_beta_batched(
            ctx.handle, ctypes.byref(csr), ctypes.byref(csc), R, _ptr(omega), _ptr(z), _ptr(lam),
            _ptr(tau), _ptr(eta), _ptr(delta), float(tol), int(max_iter), _ptr(out), it, rs, ss))
    return DrawResult(out, list(it), list(rs), list(ss))


def pcg_draw_beta_uneven(ctx, problems, tol=1e-6, max_iter=10_000):
    """Independent problems of uneven size: a list of dicts with keys
    X (DeviceDesign), omega, z, lam, tau, eta, delta (device tensors) and
    optionally out.  Returns a list of DrawResult."""
    f = torch.float64
    Q = len(problems)
    arr = (_Problem * max(Q, 1))()
    outs = []
    keep = []
    for q, pr in enumerate(problems):
        X = pr["X"]
        dev = X.device
        for name, m in (("omega", X.n), ("z", X.n), ("eta", X.n), ("lam", X.p), ("delta", X.p)):
            _dev(pr[name], f, m, name, dev)
        out = pr.get("out")
        out = torch.empty(X.p, dtype=f, device=dev) if out is None else _dev(out, f, X.p, "out", dev)
        outs.append(out)
        csr, csc = X.csr(), X.csc()
        keep.append((csr, csc))
        arr[q] = _Problem(csr, csc, pr["omega"].data_ptr(), pr["z"].data_ptr(), pr["lam"].data_ptr(),
                          pr["eta"].data_ptr(), pr["delta"].data_ptr(), float(pr["tau"]), out.data_ptr())
    it = (ctypes.c_int * max(Q, 1))()
    rs = (ctypes.c_double * max(Q, 1))()
    ss = (ctypes.c_int * max(Q, 1))()
    with torch.cuda.device(ctx.device):
        ctx.check(ctx._lib.pcg_draw_beta_uneven(ctx.handle, Q, arr, float(tol), int(max_iter), it, rs, ss))
    return [DrawResult(outs[q], it[q], rs[q], ss[q]) for q in range(Q)]


def pcg_adjoint(ctx, X, omega, z, lam, tau, eta, delta, beta, grad_beta, mode="draw", tol=1e-10,
                max_iter=10_000):
    """Gradient of a loss with dL/dbeta = grad_beta.  Returns a dict with
    b, omega, log_lambda (device tensors), log_tau (float), iters, resid, status."""
    f = torch.float64
    dev = X.device
    _dev(omega, f, X.n, "omega", dev)
    _dev(lam, f, X.p, "lambda", dev)
    _dev(beta, f, X.p, "beta", dev)
    _dev(grad_beta, f, X.p, "grad_beta", dev)
    m = ADJ[mode] if isinstance(mode, str) else int(mode)
    if m == 1:
        _dev(z, f, X.n, "z", dev)
        _dev(eta, f, X.n, "eta", dev)
        _dev(delta, f, X.p, "delta", dev)
    g_b = torch.empty(X.p, dtype=f, device=dev)
    g_om = torch.empty(X.n, dtype=f, device=dev)
    g_ll = torch.empty(X.p, dtype=f, device=dev)
    g_lt = ctypes.c_double(0.0)
    it, rs = ctypes.c_int(0), ctypes.c_double(0.0)
    csr, csc = X.csr(), X.csc()
    with torch.cuda.device(ctx.device):
        st = ctx.check(ctx._lib.pcg_adjoint(
            ctx.handle, ctypes.byref(csr), ctypes.byref(csc), _ptr(omega), _ptr(z), _ptr(lam),
            float(tau), _ptr(eta), _ptr(delta), _ptr(beta), _ptr(grad_beta), m, float(tol),
            int(max_iter), _ptr(g_b), _ptr(g_om), _ptr(g_ll), ctypes.byref(g_lt), ctypes.byref(it),
            ctypes.byref(rs)))
    return dict(b=g_b, omega=g_om, log_lambda=g_ll, log_tau=g_lt.value, iters=it.value,
                resid=rs.value, status=st)


def pcg_profile_count(ctx: Context) -> int:
    return int(ctx._lib.pcg_profile_count(ctx.handle))


def pcg_profile_entry(ctx: Context, i: int):
    """(kernel name, total milliseconds, launches) of profiled kernel i."""
    name, ms, n = ctypes.c_char_p(), ctypes.c_double(), ctypes.c_int64()
    ctx.check(ctx._lib.pcg_profile_entry(ctx.handle, int(i), ctypes.byref(name), ctypes.byref(ms),
                                         ctypes.byref(n)))
    return name.value.decode(), ms.value, n.value


def pcg_profile_reset(ctx: Context) -> None:
    ctx._lib.pcg_profile_reset(ctx.handle)


def pcg_last_kernel_launches(ctx: Context) -> int:
    return int(ctx._lib.pcg_last_kernel_launches(ctx.handle))


def profile_table(ctx: Context) -> dict:
    """All profiled kernels: name -> (total ms, launches)."""
    out = {}
    for i in range(pcg_profile_count(ctx)):
        name, ms, n = pcg_profile_entry(ctx, i)
        out[name] = (ms, n)
    return out


NOALLOC_MAX_N = 1048576


def pcg_tiled_plan_applies(n, p, nnz, precision="df32", rhs_group=1):
    """(column tiles, row strips) of the shared-memory tiled products for a
    design of this shape, or None when the calls use the untiled products.
    Host arithmetic only."""
    lib = load_library()
    tc, tr = ctypes.c_int(0), ctypes.c_int(0)
    prec = PREC[precision] if isinstance(precision, str) else int(precision)
    ok = lib.pcg_tiled_plan_applies(int(n), int(p), int(nnz), prec, int(rhs_group), ctypes.byref(tc),
                                    ctypes.byref(tr))
    return (tc.value, tr.value) if ok else None


def pcg_phi_mul_noalloc(X, omega, lam, tau, v, out, stream=None):
    """Phi v into the caller's `out` with no device allocation (float64).
    Queues the work on `stream` (default: the current stream) and returns the
    status without waiting."""
    lib = load_library()
    f = torch.float64
    dev = X.device
    _dev(omega, f, X.n, "omega", dev)
    _dev(lam, f, X.p, "lambda", dev)
    _dev(v, f, X.p, "v", dev)
    _dev(out, f, X.p, "out", dev)
    s = stream if stream is not None else torch.cuda.current_stream(dev)
    csr, csc = X.csr(), X.csc()
    with torch.cuda.device(dev):
        return lib.pcg_phi_mul_noalloc(ctypes.byref(csr), ctypes.byref(csc), _ptr(omega), _ptr(lam),
                                       float(tau), _ptr(v), _ptr(out), ctypes.c_void_p(s.cuda_stream))
