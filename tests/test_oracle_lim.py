"""Pins of the oracle's LIM step (Sec. 3.1, Fig. 1) by properties the method must have:
p = 1 is explicit Euler; every iteration has the implicit-Euler solution of Eq. (EBlin) as
its fixed point, so modes at the nodes a_m come out exactly implicit Euler; the step is
stable on [0, lambda_max]; the scheme has order 1."""
import numpy as np
import pytest
import scipy.linalg

from _dense import dense_Ahat, dense_ghat
from paper_2502_14589_gb300 import inputs


def nodes(p, lmax):
    """a_m of Fig. 1 (natural order)."""
    beta = np.cos(np.pi * (2 * np.arange(1, p + 1) - 1) / (2 * p))
    z1 = beta[0]
    return lmax / (1 + z1) * (z1 - beta)


def test_p1_is_explicit_euler(oracle):
    rng = np.random.default_rng(0)
    N = 20
    M = rng.standard_normal((N, N)); M = M @ M.T
    lmax = np.abs(M).sum(axis=0).max()
    tau = 0.9 / lmax
    g = rng.standard_normal(N); y = rng.standard_normal(N)
    out, p = oracle.lim_dense(M, g, y, tau, lmax)
    assert p == 1
    np.testing.assert_allclose(out, y + tau * (g - M @ y), rtol=0, atol=1e-14 * np.abs(y).max())


@pytest.mark.parametrize("taulam", [3.0, 40.0, 900.0, 2.5e4])
def test_modes_at_nodes_are_implicit_euler(oracle, taulam):
    lmax = 1.0e3
    tau = taulam / lmax
    p = oracle.cheb_order(tau, lmax)
    a = nodes(p, lmax)
    lam = np.concatenate([a, [0.0]])
    rng = np.random.default_rng(1)
    g = rng.standard_normal(lam.size); y = rng.standard_normal(lam.size)
    out, p2 = oracle.lim_dense(np.diag(lam), g, y, tau, lmax)
    assert p2 == p
    ie = (y + tau * g) / (1 + tau * lam)          # implicit Euler, Eq. (EBlin)
    tol = 1e-14 * max(taulam, 1.0)                # rounding grows like u * tau lambda_max
    np.testing.assert_allclose(out, ie, rtol=tol, atol=tol * np.abs(ie).max())


@pytest.mark.parametrize("taulam", [2.0, 50.0, 1e3, 1e5])
def test_stability_on_zero_to_lambda_max(oracle, taulam):
    lmax = 10.0
    tau = taulam / lmax
    lam = np.linspace(0.0, lmax, 2001)
    out, p = oracle.lim_dense(np.diag(lam), np.zeros(lam.size), np.ones(lam.size), tau, lmax)
    assert np.all(np.abs(out) <= 1.0 + 1e-12), (p, np.abs(out).max())
    assert abs(out[0] - 1.0) < 1e-14                # lambda = 0 mode is kept


def test_order_one_on_dense_ch_jacobian(oracle):
    """Local error against the exact linear solution of Eq. (IVPlin) is O(tau^2)."""
    n = (6, 6); eps = 0.08
    y = inputs.initial_state(n, 4, -0.7, 0.7)
    M = dense_Ahat(n, y, eps); g = dense_ghat(n, y)
    lmax = np.abs(M).sum(axis=0).max()
    errs = []
    for tau in [0.4 / lmax * 2 ** -k for k in range(3)]:
        N = M.shape[0]
        aug = np.zeros((N + 1, N + 1)); aug[:N, :N] = -tau * M; aug[:N, N] = tau * (g - M @ y)
        exact = y + scipy.linalg.expm(aug)[:N, N]
        out, p = oracle.lim_dense(M, g, y, tau, lmax)
        errs.append(np.linalg.norm(out - exact))
    r = [errs[k] / errs[k + 1] for k in range(2)]
    assert all(3.5 < x < 4.5 for x in r), r


def test_grid_lim_matches_dense_lim(oracle):
    """or_lim_step on the grid = the LIM core on the dense A_hat, g_hat, ||A_hat||_1."""
    n = (7, 6); eps = 0.06
    for eyre in (False, True):
        gr = oracle.Grid(2, n, eps, eyre=eyre)
        y = inputs.initial_state(n, 9, -0.9, 0.9)
        M = dense_Ahat(n, y, eps, eyre); gv = dense_ghat(n, y, eyre)
        lmax = np.abs(M).sum(axis=0).max()
        tau = 37.0 / lmax
        out, p, lm, mv = oracle.lim_step(gr, y, tau)
        ref, p2 = oracle.lim_dense(M, gv, y, tau, lmax)
        assert p == p2 and mv == 2 * p - 1
        assert abs(lm - lmax) < 1e-13 * lmax
        np.testing.assert_allclose(out, ref, rtol=0, atol=1e-11 * np.abs(ref).max())


def _alphas(p, X):
    beta = np.cos(np.pi * (2 * np.arange(1, p + 1) - 1) / (2 * p))
    return X / (1 + beta[0]) * (beta[0] - beta)


def _growth_times_tail(p, X, order, npts):
    """max over iterations k of (1 + X max|head_k|) * max|tail after k|: rounding errors of
    size ~ u X |iterate| made at iteration k, amplified by the factors still to come."""
    a = _alphas(p, X)
    x = np.linspace(0, X, npts)
    seq = list(order) + list(order[1:])
    Q = np.array([(a[m] - x) / (1 + a[m]) for m in seq])
    n = len(seq)
    H = np.ones(n + 1); h = np.ones_like(x)
    for k in range(n):
        h = h * Q[k]; H[k + 1] = np.abs(h).max()
    T = np.ones(n + 1); t = np.ones_like(x)
    for k in range(n - 1, -1, -1):
        T[k] = np.abs(t).max(); t = t * Q[k]
    return max((1 + X * H[k]) * T[k] for k in range(n))


@pytest.mark.parametrize("p", [1, 2, 3, 5, 8, 21, 40, 64, 125])
def test_lim_order_keeps_roundoff_growth_near_square_of_tau_lambda(oracle, p):
    """Fig. 1, ordered set: the order starts with beta_1 and is a permutation; its rounding-error
    growth stays within 3 (tau lambda_max)^2, whereas the natural order exceeds 1e13 at
    p = 21 and overflows double precision beyond p ~ 150."""
    order = oracle.lim_order(p)
    assert order[0] == 0 and sorted(order) == list(range(p))
    Xp = np.tan(np.pi / 2 - np.pi / (4 * p)) ** 2
    J = _growth_times_tail(p, Xp, order, 40 * p + 1)
    assert J <= 3 * max(Xp, 1.0) ** 2
    if p == 21:
        assert _growth_times_tail(p, Xp, list(range(p)), 40 * p + 1) > 1e12


@pytest.mark.parametrize("taulam", [3e3, 1e5])
def test_lim_large_p_matches_product_formula(oracle, taulam):
    """With many Chebyshev factors the step must still equal, up to round-off, the exact
    error propagation y_IE + prod_m q_m(tau lam) (y^n - y_IE) of the two sweeps."""
    lmax = 1.0
    tau = taulam / lmax
    lam = np.linspace(0.0, lmax, 513)
    rng = np.random.default_rng(4)
    g = rng.standard_normal(lam.size); y = rng.standard_normal(lam.size)
    out, p = oracle.lim_dense(np.diag(lam), g, y, tau, lmax)
    a = _alphas(p, lmax)
    R = np.ones_like(lam)
    for m in list(range(p)) + list(range(1, p)):
        R = R * (tau * a[m] - tau * lam) / (1 + tau * a[m])
    ie = (y + tau * g) / (1 + tau * lam)
    ref = ie + R * (y - ie)
    assert np.linalg.norm(out - ref) <= 1e-10 * np.linalg.norm(ref)
