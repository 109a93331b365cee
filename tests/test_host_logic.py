"""Host-side logic of the CUDA library, run without a GPU through its host-only C calls and
compared with the oracle:

* ch_lim_schedule (p, parameter order and a_m of Fig. 1 as the GPU path uses them): p equals the oracle's
  Eq. (p), the parameter order equals the oracle's, and the schedule applied to scalar
  modes mu in [0, lambda_max] (the step y <- (y + tau a_m y - tau mu y) / (1 + tau a_m)
  of Fig. 1) reproduces the oracle's LIM step on the 1 x 1 problem.
* ch_lambda_max_bound (the spectral bound of Fig. 1 in the closed form the GPU uses) equals the oracle's
  ||A_hat||_1 formed column by column.
"""
import ctypes

import numpy as np
import pytest

from paper_2502_14589_gb300 import inputs


@pytest.fixture(scope="module")
def ch():
    from paper_2502_14589_gb300 import build, ch as chmod
    build.build()
    chmod.load()
    return chmod


TAU_LAMBDA = [0.5, 1.0, 1.5, 4.0, 30.0, 700.0, 2.5e3, 1e5, 3e7]


@pytest.mark.parametrize("x", TAU_LAMBDA)
def test_lim_schedule_matches_the_oracle(ch, oracle, x):
    lmax = 2.7e6
    tau = x / lmax
    p, order, a = ch.ch_lim_schedule(tau, lmax)
    assert p == oracle.cheb_order(tau, lmax)
    assert np.array_equal(order - 1, oracle.lim_order(p))
    assert a[0] == 0.0 and np.all(np.diff(a) > 0) and a[-1] <= 2 * lmax
    # the schedule on scalar modes against the oracle's LIM step on the 1 x 1 problem
    for mu in np.linspace(0.0, lmax, 7):
        y = 1.0
        seq = list(order) + list(order[1:])
        for m in seq:
            am = a[m - 1]
            y = (1.0 + tau * am * y + tau * (0.0 - mu * y)) / (1.0 + tau * am)
        yo, po = oracle.lim_dense(np.array([[mu]]), np.zeros(1), np.ones(1), tau, lmax)
        assert po == p
        assert abs(y - yo[0]) <= 1e-12 * max(1.0, abs(yo[0]))


@pytest.mark.parametrize("dim,n", [(2, (8, 8)), (2, (12, 7)), (3, (6, 5, 7)), (3, (4, 4, 4)),
                                   (2, (4, 9))])
@pytest.mark.parametrize("eyre", [0, 1])
def test_lambda_max_bound_matches_the_oracle(ch, oracle, dim, n, eyre):
    for seed, (lo, hi) in enumerate([(-0.05, 0.05), (-1.0, 1.0), (0.3, 0.9)]):
        y = inputs.initial_state(n, 50 + seed, lo, hi, 0.0 if lo < 0 else 0.6)
        y2 = y * y
        lb = ch.ch_lambda_max_bound(dim, n, 0.04, float(y2.min()), float(y2.max()), eyre)
        ref = oracle.lambda_max(oracle.Grid(dim, n, 0.04, eyre=bool(eyre)), y)
        assert lb == pytest.approx(ref, rel=1e-13)


def test_host_calls_report_invalid_arguments(ch):
    lib = ch.load()
    p = ctypes.c_int()
    assert lib.ch_lim_schedule(float("inf"), 1.0, 0, ctypes.byref(p), None, None) == ch.CH_EINVAL
    assert lib.ch_lim_schedule(1e-3, float("nan"), 0, ctypes.byref(p), None, None) == ch.CH_EINVAL
    assert lib.ch_lim_schedule(1e-3, float("inf"), 0, ctypes.byref(p), None, None) == ch.CH_ENONFINITE
    assert lib.ch_lim_schedule(1.0, 1e16, 0, ctypes.byref(p), None, None) == ch.CH_EINVAL  # p > 10^6
    assert lib.ch_lim_schedule(1e-3, 2.7e6, 0, ctypes.byref(p), None, None) == ch.CH_OK and p.value > 2
    buf = (ctypes.c_int * 2)()
    assert lib.ch_lim_schedule(1e-3, 2.7e6, 2, ctypes.byref(p), buf, None) == ch.CH_EINVAL
    out = ctypes.c_double()
    n = (ctypes.c_int64 * 3)(3, 8, 1)
    assert lib.ch_lambda_max_bound(2, n, 0.04, 0, 0.0, 1.0, ctypes.byref(out)) == ch.CH_EINVAL
    n = (ctypes.c_int64 * 3)(8, 8, 1)
    assert lib.ch_lambda_max_bound(2, n, 0.04, 0, 0.5, 0.1, ctypes.byref(out)) == ch.CH_EINVAL
    assert lib.ch_lambda_max_bound(2, n, 0.04, 0, 0.1, 0.5, ctypes.byref(out)) == ch.CH_OK
