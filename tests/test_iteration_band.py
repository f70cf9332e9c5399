"""CPU pins for the reference band of iteration counts (tests/iteration_band.py).

These record, as checks, the facts the parity tests' iteration criterion rests
on: the compensated oracle does not depend on summation order; on config 2
its count still moves by several iterations under one-ulp changes of omega
and lambda; and the plain oracle's left-to-right sums add iterations on top.
The numbers were measured with the committed oracle (compensated band
[130, 135], plain [138, 145] on config 2; config 1 takes 27 in every run).
"""
import numpy as np

from oracle import oracle as O
from paper_1810_12437_gb300 import inputs
from tests.iteration_band import problem_band


def test_relabel_is_the_same_problem():
    """inputs.relabel permutes rows and columns: the Cholesky draw of the
    relabelled problem, read back through the column permutation, is the
    original draw."""
    P = inputs.make_problem(300, 40, -1.5, -0.5, seed=3, tau=0.1)
    Q, rows, cols = inputs.relabel(P, 11)
    assert Q.X.nnz == P.X.nnz
    assert np.array_equal(Q.X.dense()[np.ix_(rows, cols)], P.X.dense())
    a = O.draw_beta_chol(P.X, P.omega, P.z, P.lam, P.tau, P.eta, P.delta)
    b = O.draw_beta_chol(Q.X, Q.omega, Q.z, Q.lam, Q.tau, Q.eta, Q.delta)
    assert np.linalg.norm(b[cols] - a) <= 1e-12 * np.linalg.norm(a)


def test_config1_count_is_stable():
    """Config 1 (relative stop 1e-10) is well enough conditioned that every
    run, plain or compensated, perturbed or not, takes the same count."""
    P = inputs.config1()
    kw = dict(tol=1e-10, stop_rule=O.STOP_RELATIVE)
    comp = problem_band(P, **kw)
    plain = problem_band(P, sums="plain", **kw)
    assert comp.lo == comp.hi == plain.lo == plain.hi == 27


def test_config2_band_and_plain_sum_bias():
    """Config 2 (paper RMS stop 1e-6): the compensated count moves under
    one-ulp perturbations (band of width >= 2 inside [128, 138]); the plain
    sums' counts lie above the compensated band on average by at least 4."""
    P = inputs.config2()
    comp = problem_band(P)
    plain = problem_band(P, sums="plain")
    assert 128 <= comp.lo and comp.hi <= 138 and comp.hi - comp.lo >= 2, comp
    assert np.mean(plain.counts) - np.mean(comp.counts) >= 4, (plain, comp)


def test_compensated_count_does_not_depend_on_order():
    """Relabelling rows and columns changes every sum's order.  The
    compensated oracle's count is unchanged by it; the plain oracle's count
    changes."""
    P = inputs.config2()
    b = O.build_b(P.X, P.omega, P.z, P.lam, P.tau, P.eta, P.delta)
    base_c = O.pcg(P.X, P.omega, P.lam, P.tau, b, sums="compensated")[1]
    base_p = O.pcg(P.X, P.omega, P.lam, P.tau, b)[1]
    plain_counts = []
    for seed in (1, 2, 3):
        Q, _, cols = inputs.relabel(P, seed)
        bq = np.empty_like(b)
        bq[cols] = b
        assert O.pcg(Q.X, Q.omega, Q.lam, Q.tau, bq, sums="compensated")[1] == base_c
        plain_counts.append(O.pcg(Q.X, Q.omega, Q.lam, Q.tau, bq)[1])
    assert any(k != base_p for k in plain_counts), (base_p, plain_counts)
