"""CPU oracle for the conditional beta draw (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module.  The library never does.  It wraps the
plain C FP64 routines in ``pcg_oracle.c`` and composes them, step by step,
into the draw of Prop. 2.1 (right-hand side by Eq. 2.3, then Phi beta = b by
Eq. 2.4):

* ``draw_beta_cg``   -- prior-preconditioned CG (Sec. 2.4, Algorithm S1,
                        stop rule Eq. S2);
* ``draw_beta_chol`` -- the direct sampler: dense Phi, Cholesky, two
                        triangular solves (Sec. 1);
* ``adjoint``        -- gradient of L = c^T beta, by implicit differentiation
                        of beta = Phi^-1 b (not in the paper; derivation in
                        the docstring);
* ``*_unshrunk``     -- the same draw with unshrunk coefficients (Sec. S4.3):
                        their own prior precisions in Phi and Eq. 2.3 and
                        separate preconditioner scales (plain numpy, small
                        cases).

Every function takes the same numpy inputs as the CUDA path (see
``paper_1810_12437_gb300.inputs``).  Parity: each routine is pinned by the
``-m "not gpu"`` tests in ``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sysconfig
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pcg_oracle.c")
_LIB = os.path.join(_HERE, "_pcg_oracle.so")
_lock = threading.Lock()
_lib = None

STOP_RMS = 0
STOP_RELATIVE = 1
OK, MAXITER, BREAKDOWN, NONFINITE = 0, 1, 2, 3
SUM_PLAIN, SUM_COMPENSATED, SUM_FLOAT32 = 0, 1, 2
_SUMS = {"plain": SUM_PLAIN, "compensated": SUM_COMPENSATED, "float32": SUM_FLOAT32}
_VECS = {"f64": 0, "f32x2": 1, "f32": 2}


def build(force: bool = False) -> str:
    """Compile pcg_oracle.c into _pcg_oracle.so with gcc (plain -O2, no
    vector extensions, so that x86 and Arm builds round identically)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fno-fast-math", "-ffp-contract=off", "-fPIC",
                               "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _bind(lib):
    P = ctypes.c_void_p
    I64 = ctypes.c_int64
    D = ctypes.c_double
    I = ctypes.c_int
    lib.oracle_x_mul.argtypes = [I64, P, P, P, P]
    lib.oracle_xt_mul.argtypes = [I64, P, P, P, P]
    lib.oracle_phi_mul.argtypes = [I64, I64, P, P, P, P, P, P, D, P, P, P]
    lib.oracle_build_b.argtypes = [I64, I64, P, P, P, P, P, D, P, P, P, P]
    lib.oracle_pcg.argtypes = [I64, I64, P, P, P, P, P, P, D, P, D, I, I, I, P, P, P, P]
    lib.oracle_pcg.restype = I
    lib.oracle_pcg_ex.argtypes = [I64, I64, P, P, P, P, P, P, D, P, P, P, D, I, I, I, I, I, P, P, P, P]
    lib.oracle_pcg_ex.restype = I
    lib.oracle_x_mul_comp.argtypes = [I64, P, P, P, P]
    lib.oracle_xt_mul_comp.argtypes = [I64, P, P, P, P]
    lib.oracle_dot_comp.argtypes = [I64, P, P]
    lib.oracle_dot_comp.restype = D
    lib.oracle_phi_diag.argtypes = [I64, P, P, P, P, D, P]
    lib.oracle_lsqr.argtypes = [I64, I64, P, P, P, P, P, P, P, D, P, P, D, I, I, I, P, P, P]
    lib.oracle_lsqr.restype = I
    U32, U64 = ctypes.c_uint32, ctypes.c_uint64
    lib.oracle_philox.argtypes = [P, P, P]
    lib.oracle_pg_series.argtypes = [D, D, I]
    lib.oracle_pg_series.restype = D
    lib.oracle_pg1.argtypes = [I64, P, U64, U32, U32, P]
    lib.oracle_rng_draws.argtypes = [I, I64, U64, U32, U32, U32, D, P]
    lib.oracle_gibbs_scales.argtypes = [I64, P, P, P, P, P, U64, U32]
    lib.oracle_gibbs_omega.argtypes = [I64, I64, P, P, P, P, U64, U32, P, P, P, P]
    lib.oracle_dense_phi.argtypes = [I64, I64, P, P, P, P, D, P]
    lib.oracle_cholesky.argtypes = [I64, P]
    lib.oracle_cholesky.restype = I
    lib.oracle_chol_solve.argtypes = [I64, P, P, P]
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = _bind(ctypes.CDLL(_LIB))
    return _lib


def use_library(path):
    """Bind the oracle to another build of pcg_oracle.c (the mutation tests
    compile deliberately broken copies and check that the pins reject them).
    Returns the previously bound library so it can be restored."""
    global _lib
    _load()
    with _lock:
        prev = _lib
        _lib = _bind(ctypes.CDLL(path)) if isinstance(path, str) else path
    return prev


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def x_mul(X, v):
    """X v for binary CSR X."""
    lib = _load()
    v = _f64(v)
    out = np.empty(X.n)
    lib.oracle_x_mul(X.n, _p(X.row_ptr), _p(X.col_idx), _p(v), _p(out))
    return out


def xt_mul(X, w):
    """X^T w for binary CSC X."""
    lib = _load()
    w = _f64(w)
    out = np.empty(X.p)
    lib.oracle_xt_mul(X.p, _p(X.col_ptr), _p(X.row_idx), _p(w), _p(out))
    return out


def phi_mul(X, omega, lam, tau, v):
    """Phi v = X^T Omega X v + tau^-2 lambda^-2 v, matrix-free (Sec. 1)."""
    lib = _load()
    omega, lam, v = _f64(omega), _f64(lam), _f64(v)
    out = np.empty(X.p)
    work = np.empty(max(X.n, 1))
    lib.oracle_phi_mul(X.n, X.p, _p(X.row_ptr), _p(X.col_idx), _p(X.col_ptr), _p(X.row_idx),
                       _p(omega), _p(lam), float(tau), _p(v), _p(out), _p(work))
    return out


def build_b(X, omega, z, lam, tau, eta, delta):
    """Right-hand side b of Prop. 2.1, Eq. 2.3."""
    lib = _load()
    omega, z, lam, eta, delta = map(_f64, (omega, z, lam, eta, delta))
    b = np.empty(X.p)
    work = np.empty(X.n + X.p + 1)
    lib.oracle_build_b(X.n, X.p, _p(X.col_ptr), _p(X.row_idx), _p(omega), _p(z), _p(lam),
                       float(tau), _p(eta), _p(delta), _p(b), _p(work))
    return b


def x_mul_comp(X, v):
    """X v with each row sum accumulated by compensated summation."""
    lib = _load()
    v = _f64(v)
    out = np.empty(X.n)
    lib.oracle_x_mul_comp(X.n, _p(X.row_ptr), _p(X.col_idx), _p(v), _p(out))
    return out


def xt_mul_comp(X, w):
    """X^T w with each column sum accumulated by compensated summation."""
    lib = _load()
    w = _f64(w)
    out = np.empty(X.p)
    lib.oracle_xt_mul_comp(X.p, _p(X.col_ptr), _p(X.row_idx), _p(w), _p(out))
    return out


def dot_comp(a, b):
    """a . b with the rounded products summed by compensated summation."""
    lib = _load()
    a, b = _f64(a), _f64(b)
    return float(lib.oracle_dot_comp(a.size, _p(a), _p(b)))


def phi_diag(X, omega, lam, tau):
    """diag(Phi) = X^T omega + tau^-2 lambda^-2 for binary X: the Jacobi
    preconditioner's M (Sec. 2.4)."""
    lib = _load()
    omega, lam = _f64(omega), _f64(lam)
    out = np.empty(X.p)
    lib.oracle_phi_diag(X.p, _p(X.col_ptr), _p(X.row_idx), _p(omega), _p(lam), float(tau), _p(out))
    return out


def pcg(X, omega, lam, tau, b, *, tol=1e-6, stop_rule=STOP_RMS, max_iter=10_000,
        fixed_iters=0, want_hist=False, minv=None, beta0=None, sums="plain", vec="f64"):
    """Preconditioned CG (Algorithm S1 in PCG form).

    Defaults: the prior preconditioner M^-1 = tau^2 Lambda^2 (Sec. 2.4), beta_0 = 0
    (Sec. 2.7) and plain left-to-right sums.  ``minv`` gives another diagonal
    M^-1 (the Jacobi preconditioner: 1 / diag(Phi)); ``beta0`` an initial
    vector (Sec. S4.1); ``sums="compensated"`` accumulates the products' and
    the dot products' sums by compensated summation (``"float32"``: the
    products' sums left to right in float32, the dot products compensated); ``vec`` ("f64",
    "f32x2": float pairs of about 48 bits, "f32") is the storage format of
    the products' operands and results (s, omega, u and the product X^T u).  The stop rule tests
    ||tau lambda (.) r|| (Eq. S2) whatever the preconditioner.

    Returns (beta, iters, resid, status[, hist of the stop quantity]).
    ``fixed_iters > 0`` runs exactly that many iterations with no stop test.
    """
    lib = _load()
    omega, lam, b = _f64(omega), _f64(lam), _f64(b)
    beta = np.empty(X.p)
    iters = ctypes.c_int(0)
    resid = ctypes.c_double(0.0)
    hist = np.full(max(max_iter, fixed_iters) + 1, np.nan) if want_hist else None
    hp = _p(hist) if want_hist else None
    if minv is None and beta0 is None and sums == "plain" and vec == "f64":
        st = lib.oracle_pcg(X.n, X.p, _p(X.row_ptr), _p(X.col_idx), _p(X.col_ptr), _p(X.row_idx),
                            _p(omega), _p(lam), float(tau), _p(b), float(tol), int(stop_rule),
                            int(max_iter), int(fixed_iters), _p(beta), ctypes.byref(iters),
                            ctypes.byref(resid), hp)
    else:
        mv = _f64(minv) if minv is not None else None
        b0 = _f64(beta0) if beta0 is not None else None
        st = lib.oracle_pcg_ex(X.n, X.p, _p(X.row_ptr), _p(X.col_idx), _p(X.col_ptr),
                               _p(X.row_idx), _p(omega), _p(lam), float(tau), _p(b),
                               _p(mv) if mv is not None else None,
                               _p(b0) if b0 is not None else None,
                               float(tol), int(stop_rule), int(max_iter), int(fixed_iters),
                               _SUMS[sums], _VECS[vec], _p(beta), ctypes.byref(iters),
                               ctypes.byref(resid), hp)
    out = (beta, iters.value, resid.value, st)
    if want_hist:
        out = out + (hist[: iters.value + 1],)
    return out


def draw_beta_lsqr(X, omega, z, lam, tau, eta, delta, *, tol=1e-6, stop_rule=STOP_RMS,
                   max_iter=10_000, sums="plain"):
    """The draw of Prop. 2.1 by LSQR on the least-squares form (Sec. S7.1, Eq.
    S6), right-preconditioned by diag(tau lambda); stop rule Eq. S2 on LSQR's
    ||A^T r|| = ||tau lambda (.) (b - Phi beta)||.  Returns (beta, iters,
    resid, status)."""
    lib = _load()
    omega, z, lam, eta, delta = map(_f64, (omega, z, lam, eta, delta))
    beta = np.empty(X.p)
    iters = ctypes.c_int(0)
    resid = ctypes.c_double(0.0)
    st = lib.oracle_lsqr(X.n, X.p, _p(X.row_ptr), _p(X.col_idx), _p(X.col_ptr), _p(X.row_idx),
                         _p(omega), _p(z), _p(lam), float(tau), _p(eta), _p(delta), float(tol),
                         int(stop_rule), int(max_iter), _SUMS[sums], _p(beta), ctypes.byref(iters),
                         ctypes.byref(resid))
    return beta, iters.value, resid.value, st


# ---------------------------------------------------------------------------
# The rest of the Gibbs cycle of Sec. S1 (horseshoe prior, Polya-Gamma
# augmentation; see pcg_oracle.c): counter-based random numbers (Philox4x32-10)
# keyed by a 64-bit seed, one counter per (element, stream, Gibbs step).
# ---------------------------------------------------------------------------
STREAM_XI, STREAM_TAU, STREAM_NU, STREAM_LAMBDA, STREAM_OMEGA, STREAM_ETA, STREAM_DELTA = 1, 2, 3, 4, 5, 6, 7


def philox(ctr, key):
    """One Philox4x32-10 block: 4 counter words and 2 key words -> 4 words."""
    lib = _load()
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.empty(4, dtype=np.uint32)
    lib.oracle_philox(_p(c), _p(k), _p(out))
    return out


def pg_series(x, t, terms=60):
    """The J*(1, 0) density at x by the alternating series of the sampler,
    in the small-x form (x <= t) or the large-x form (x > t)."""
    return float(_load().oracle_pg_series(float(x), float(t), int(terms)))


def rng_draws(kind, m, seed, index, stream, step, a=1.0):
    """m successive draws of one counter: kind "uniform", "exp", "normal" or
    "gamma" (shape a >= 1)."""
    lib = _load()
    out = np.empty(m)
    code = {"uniform": 0, "exp": 1, "normal": 2, "gamma": 3}[kind]
    lib.oracle_rng_draws(code, m, int(seed), int(index), int(stream), int(step), float(a), _p(out))
    return out


def pg1(c, seed, stream=STREAM_OMEGA, step=0):
    """PolyaGamma(1, c_k) for each k, element k drawing from counter k."""
    lib = _load()
    c = _f64(c)
    out = np.empty(c.size)
    lib.oracle_pg1(c.size, _p(c), int(seed), int(stream), int(step), _p(out))
    return out


def gibbs_scales(beta, lam, nu, tau, xi, seed, step):
    """Steps 1-2 of Sec. S1 (horseshoe, auxiliary nu and xi): returns
    (lambda, nu, tau, xi) after the update."""
    lib = _load()
    beta = _f64(beta)
    lam, nu = _f64(lam).copy(), _f64(nu).copy()
    t, x = ctypes.c_double(tau), ctypes.c_double(xi)
    lib.oracle_gibbs_scales(beta.size, _p(beta), _p(lam), _p(nu), ctypes.byref(t), ctypes.byref(x),
                            int(seed), int(step))
    return lam, nu, t.value, x.value


def gibbs_omega(X, y, beta, seed, step):
    """Step 3 of Sec. S1 and step 4's Gaussian vectors: omega ~ PG(1, X beta),
    z = (y - 1/2) / omega, eta ~ N(0, I_n), delta ~ N(0, I_p)."""
    lib = _load()
    y, beta = _f64(y), _f64(beta)
    omega, z, eta, delta = np.empty(X.n), np.empty(X.n), np.empty(X.n), np.empty(X.p)
    lib.oracle_gibbs_omega(X.n, X.p, _p(X.row_ptr), _p(X.col_idx), _p(y), _p(beta), int(seed), int(step),
                           _p(omega), _p(z), _p(eta), _p(delta))
    return omega, z, eta, delta


def gibbs_step(X, y, beta, lam, nu, tau, xi, seed, step, *, tol=1e-6, stop_rule=STOP_RMS,
               max_iter=10_000, draw="chol", **pcg_kw):
    """One cycle of the Gibbs sampler of Sec. S1: tau, then lambda, then
    omega, then beta (Prop. 2.1: by Cholesky, draw="chol", or by the oracle's
    PCG, draw="cg").  Returns a dict with the new state and the beta draw's
    iteration count."""
    lam, nu, tau, xi = gibbs_scales(beta, lam, nu, tau, xi, seed, step)
    omega, z, eta, delta = gibbs_omega(X, y, beta, seed, step)
    k = 0
    if draw == "chol":
        beta = draw_beta_chol(X, omega, z, lam, tau, eta, delta)
    else:
        beta, k, _, st = draw_beta_cg(X, omega, z, lam, tau, eta, delta, tol=tol, stop_rule=stop_rule,
                                      max_iter=max_iter, **pcg_kw)
    return dict(beta=beta, lam=lam, nu=nu, tau=tau, xi=xi, omega=omega, z=z, eta=eta, delta=delta, iters=k)


def dense_phi(X, omega, lam, tau):
    """Dense Phi = X^T Omega X + tau^-2 Lambda^-2 (Eq. 1.2)."""
    lib = _load()
    omega, lam = _f64(omega), _f64(lam)
    phi = np.empty((X.p, X.p))
    lib.oracle_dense_phi(X.n, X.p, _p(X.row_ptr), _p(X.col_idx), _p(omega), _p(lam),
                         float(tau), _p(phi))
    return phi


def cholesky(a):
    """Lower Cholesky factor of an SPD matrix (plain column algorithm)."""
    lib = _load()
    l = np.array(a, dtype=np.float64, order="C", copy=True)
    rc = lib.oracle_cholesky(l.shape[0], _p(l))
    if rc != 0:
        raise np.linalg.LinAlgError(f"matrix not positive definite at column {-1 - rc}")
    return l


def chol_solve(l, b):
    """x = (L L^T)^-1 b."""
    lib = _load()
    b = _f64(b)
    x = np.empty_like(b)
    lib.oracle_chol_solve(l.shape[0], _p(l), _p(b), _p(x))
    return x


def draw_beta_chol(X, omega, z, lam, tau, eta, delta):
    """Direct sampler: b by Eq. 2.3, then beta = Phi^-1 b by dense Cholesky."""
    b = build_b(X, omega, z, lam, tau, eta, delta)
    l = cholesky(dense_phi(X, omega, lam, tau))
    return chol_solve(l, b)


def draw_beta_cg(X, omega, z, lam, tau, eta, delta, *, tol=1e-6, stop_rule=STOP_RMS,
                 max_iter=10_000, fixed_iters=0, **pcg_kw):
    """CG sampler of Prop. 2.1: b by Eq. 2.3, then PCG on Eq. 2.4 (``pcg_kw``:
    the preconditioner, initial vector and summation options of ``pcg``).

    Returns (beta, iters, resid, status)."""
    b = build_b(X, omega, z, lam, tau, eta, delta)
    return pcg(X, omega, lam, tau, b, tol=tol, stop_rule=stop_rule, max_iter=max_iter,
               fixed_iters=fixed_iters, **pcg_kw)


def adjoint_from_g(X, omega, z, lam, tau, eta, delta, beta, g, mode="draw"):
    """Gradient of L = c^T beta given beta = Phi^-1 b and g = Phi^-1 c.

    beta = Phi^-1 b with Phi = X^T Omega X + diag(d), d_j = tau^-2 lambda_j^-2,
    so dL = g^T db - g^T dPhi beta (Phi symmetric).  Hence, through Phi:
        dL/domega_i     = -(X g)_i (X beta)_i
        dL/dlog lambda_j = 2 d_j g_j beta_j        (dd_j/dlog lambda_j = -2 d_j)
        dL/dlog tau      = sum_j 2 d_j g_j beta_j
        dL/db            = g.
    In "draw" mode b is built inside by Eq. 2.3 from (z, eta, delta) held
    fixed, which adds, through b:
        dL/domega_i     += (X g)_i (z_i + eta_i / (2 sqrt(omega_i)))
        dL/dlog lambda_j += -g_j delta_j / (tau lambda_j)
        dL/dlog tau      += -sum_j g_j delta_j / (tau lambda_j).
    Returns dict(b=, omega=, log_lambda=, log_tau=).
    """
    omega, z, lam, eta, delta, beta, g = map(_f64, (omega, z, lam, eta, delta, beta, g))
    d = 1.0 / (tau * tau * lam * lam)
    xg = x_mul(X, g)
    xb = x_mul(X, beta)
    g_omega = -xg * xb
    g_loglam = 2.0 * d * g * beta
    if mode == "draw":
        g_omega = g_omega + xg * (z + eta / (2.0 * np.sqrt(omega)))
        g_loglam = g_loglam - g * delta / (tau * lam)
    elif mode != "solve":
        raise ValueError(mode)
    return dict(b=g.copy(), omega=g_omega, log_lambda=g_loglam, log_tau=float(g_loglam.sum()))


def adjoint_chol(X, omega, z, lam, tau, eta, delta, c, mode="draw"):
    """Dense-Cholesky reference gradient: beta and g = Phi^-1 c by Cholesky."""
    b = build_b(X, omega, z, lam, tau, eta, delta)
    l = cholesky(dense_phi(X, omega, lam, tau))
    beta = chol_solve(l, b)
    g = chol_solve(l, c)
    return beta, adjoint_from_g(X, omega, z, lam, tau, eta, delta, beta, g, mode)


def adjoint_cg(X, omega, z, lam, tau, eta, delta, c, *, tol=1e-12, stop_rule=STOP_RMS,
               max_iter=10_000, mode="draw"):
    """Gradient with beta and g = Phi^-1 c both by the oracle's PCG."""
    b = build_b(X, omega, z, lam, tau, eta, delta)
    beta = pcg(X, omega, lam, tau, b, tol=tol, stop_rule=stop_rule, max_iter=max_iter)[0]
    g = pcg(X, omega, lam, tau, c, tol=tol, stop_rule=stop_rule, max_iter=max_iter)[0]
    return beta, adjoint_from_g(X, omega, z, lam, tau, eta, delta, beta, g, mode)


# ---------------------------------------------------------------------------
# Unshrunk coefficients (Sec. S4.3).  Coefficients 0 .. q1-1 take independent
# priors N(0, sigma_j^2) (sigma_j = infinity, precision 0, for a flat prior)
# instead of the shrinkage prior, so Phi's diagonal prior term is sigma_j^-2
# for them; the preconditioner uses separate scales gamma_j, M = diag(gamma^-2,
# tau^-2 Lambda^-2).  Plain numpy on the dense design: for small cases only.
# ---------------------------------------------------------------------------
def prior_terms_unshrunk(lam, tau, prior_prec, gamma):
    """Per coefficient: prior precision d, its square root (the prior term of
    Eq. 2.3, sigma_j^-1 delta_j for the unshrunk ones) and the preconditioner
    variance m = M^-1 (gamma_j^2 for the unshrunk ones, tau^2 lambda_j^2 after)."""
    lam = _f64(lam)
    prior_prec = np.asarray(prior_prec, dtype=np.float64)
    q1 = prior_prec.size
    d = 1.0 / (tau * lam) ** 2
    sd = 1.0 / (tau * lam)
    m = (tau * lam) ** 2
    d[:q1] = prior_prec
    sd[:q1] = np.sqrt(prior_prec)
    if gamma is not None:
        m[:q1] = np.asarray(gamma, dtype=np.float64) ** 2
    return d, sd, m


def build_b_unshrunk(X, omega, z, lam, tau, eta, delta, prior_prec):
    """Eq. 2.3 with the prior of Sec. S4.3: b = X^T Omega z + X^T Omega^1/2 eta
    + diag(d)^1/2 delta, d the prior precision of each coefficient."""
    omega, z, eta, delta = map(_f64, (omega, z, eta, delta))
    _, sd, _ = prior_terms_unshrunk(lam, tau, prior_prec, None)
    xd = X.dense()
    return xd.T @ (omega * z + np.sqrt(omega) * eta) + sd * delta


def dense_phi_unshrunk(X, omega, lam, tau, prior_prec):
    """Phi of Sec. S4.3: X^T Omega X + diag(sigma^-2 (unshrunk), tau^-2 lambda^-2)."""
    d, _, _ = prior_terms_unshrunk(lam, tau, prior_prec, None)
    xd = X.dense()
    return xd.T @ (_f64(omega)[:, None] * xd) + np.diag(d)


def draw_beta_chol_unshrunk(X, omega, z, lam, tau, eta, delta, prior_prec):
    """Direct draw with unshrunk coefficients: b as above, beta = Phi^-1 b
    (numpy Cholesky)."""
    b = build_b_unshrunk(X, omega, z, lam, tau, eta, delta, prior_prec)
    l = np.linalg.cholesky(dense_phi_unshrunk(X, omega, lam, tau, prior_prec))
    return np.linalg.solve(l.T, np.linalg.solve(l, b))


def stored(vec, x):
    """x held in a storage format: "f64" as is, "f32x2" a pair of float32
    (hi = float32(x), lo = float32(x - hi), value hi + lo), "f32" one float32
    (the same formats as the C oracle's ORACLE_VEC_*)."""
    x = _f64(x)
    if vec == "f32x2":
        hi = x.astype(np.float32).astype(np.float64)
        return hi + (x - hi).astype(np.float32).astype(np.float64)
    if vec == "f32":
        return x.astype(np.float32).astype(np.float64)
    return x


def pcg_unshrunk(X, omega, lam, tau, b, prior_prec, gamma, *, tol=1e-6, stop_rule=STOP_RMS,
                 max_iter=10_000, sums="plain", vec="f64"):
    """PCG from beta_0 = 0 (Algorithm S1 in PCG form) on Phi of Sec. S4.3 with
    M^-1 = diag(gamma^2, tau^2 Lambda^2); stop rule Eq. S2 on rho = r . (M^-1 r).
    ``sums="compensated"`` accumulates the products' row and column sums and
    the dot products by compensated summation (else the C oracle's plain
    sums and numpy's dot); ``vec`` holds the products' operands and results
    in a storage format (``stored``).  Returns (beta, iters, resid, status)."""
    omega, b = _f64(omega), _f64(b)
    d, _, m = prior_terms_unshrunk(lam, tau, prior_prec, gamma)
    p = b.size
    xm, xtm = (x_mul_comp, xt_mul_comp) if sums == "compensated" else (x_mul, xt_mul)
    dotf = dot_comp if sums == "compensated" else (lambda a, c: float(a @ c))
    om_s = stored(vec, omega)
    beta = np.zeros(p)
    r = b.copy()
    zz = m * r
    s = zz.copy()
    rho = dotf(r, zz)
    rho0 = rho

    def resid(rh):
        return np.sqrt(rh / p) if stop_rule == STOP_RMS else np.sqrt(rh / rho0)

    if resid(rho) <= tol:
        return beta, 0, resid(rho), OK
    for k in range(1, max_iter + 1):
        u = stored(vec, stored(vec, xm(X, stored(vec, s))) * om_s)
        v = stored(vec, xtm(X, u)) + d * s
        sigma = dotf(s, v)
        if not (sigma > 0.0):
            return beta, k, resid(rho), BREAKDOWN
        alpha = rho / sigma
        beta = beta + alpha * s
        r = r - alpha * v
        zz = m * r
        rho_new = dotf(r, zz)
        if resid(rho_new) <= tol:
            return beta, k, resid(rho_new), OK
        s = zz + (rho_new / rho) * s
        rho = rho_new
    return beta, max_iter, resid(rho), MAXITER
