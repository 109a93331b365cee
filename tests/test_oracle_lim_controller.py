"""Pins of the oracle's adaptive LIM path (Sec. 3.3: Fig. 3 with Eqs. LIMest and LIMdt)
against things other than the oracle's own formulas.

1. Eq. (LIMest) estimates the local error of the LIM step.  The predictor-corrector pair
   (LIM, order 1; implicit trapezoidal rule, order 2) gives est = O(tau^2), the relative local
   error of the step, for small tau: here est is compared with the true relative local error
   ||y_LIM - y(tau)|| / ||y(tau)||, y(tau) the exact solution of Eq. (IVP) from y^n computed by
   classical RK4 with 400 substeps, and their ratio must tend to 1 like O(tau).

2. Fig. 3 on a single Fourier mode about a constant state, y = ubar + c cos(2 pi k.x) with
   c = 1e-6.  To first order in c every operator of the method acts on the mode by a scalar:
   A by the symbol lambda_k = sum_a 4 s_a sin^2(pi k_a / n_a), A_hat by
   mu = lambda_k (3 ubar^2 - 1 + eps^2 lambda_k) after the constant part cancels against
   g_hat, f by -mu, ||A_hat||_1 by the closed column sum of the periodic 13-point operator at
   d = 3 (ubar -+ |c|)^2 - 1, and ||y_PC|| by |ubar| sqrt(N) (the mode is orthogonal to the
   constant).  A scalar recurrence built from those facts (Fig. 1's iteration on c, y_PC of
   Eq. LIMest, est, Eq. LIMdt, the clip to T of Fig. 3) must give the oracle's step sizes,
   estimates and Chebyshev orders step by step, the last step clipped to end at T.

Reading of the paper recorded with these pins: y_PC is formed from f(y^{n+1}) of the LIM
solution of the same step (Fig. 3 computes y^{n+1} in step 7, then y_PC and est in step 8);
lambda_max belongs to y^n and is formed afresh every step (step 6 forms A_hat_n, Fig. 1 step 1
takes its norm); est and tau_new use the step actually taken, after the clip of steps 3-4.
"""
import math

import numpy as np
import pytest

from paper_2502_14589_gb300 import inputs


def _rk4(oracle, g, y, T, m):
    h = T / m
    for _ in range(m):
        k1 = oracle.rhs(g, y)
        k2 = oracle.rhs(g, y + 0.5 * h * k1)
        k3 = oracle.rhs(g, y + 0.5 * h * k2)
        k4 = oracle.rhs(g, y + h * k3)
        y = y + (h / 6.0) * (k1 + 2.0 * k2 + 2.0 * k3 + k4)
    return y


def test_estimate_tends_to_the_true_local_error(oracle):
    n, eps = (16, 12), 0.05
    g = oracle.Grid(2, n, eps)
    y0 = 0.3 + 0.2 * inputs.initial_state(n, 3, -1.0, 1.0)
    lm = oracle.lambda_max(g, y0)
    gaps, ests = [], []
    for x in (0.4, 0.2, 0.1, 0.05):            # tau * lambda_max
        tau = x / lm
        y1, p, _, _ = oracle.lim_step(g, y0, tau)
        est = oracle.estimate(g, y0, y1, tau)
        yr = _rk4(oracle, g, y0, tau, 400)
        true = np.linalg.norm(y1 - yr) / np.linalg.norm(yr)
        gaps.append(abs(est / true - 1.0))
        ests.append(est)
    assert gaps[-1] < 0.02
    for a, b in zip(gaps, gaps[1:]):           # the ratio approaches 1 like O(tau)
        assert 0.4 < b / a < 0.6
    for a, b in zip(ests, ests[1:]):           # est = O(tau^2): a quarter per halving
        assert 0.2 < b / a < 0.3


def _column_sum_periodic(s, eps, d):
    """Closed column sum of the periodic 2D A_hat = A (d I + eps^2 A) (n_a >= 5): the centre,
    the four axis neighbours, the four second neighbours and the four diagonal neighbours."""
    sigma = 2.0 * (s[0] + s[1])
    r = abs(d * sigma + eps ** 2 * (sigma ** 2 + 2.0 * (s[0] ** 2 + s[1] ** 2)))
    r += sum(2.0 * sa * abs(d + 2.0 * eps ** 2 * sigma) for sa in s)
    r += sum(2.0 * eps ** 2 * sa * sa for sa in s) + 8.0 * eps ** 2 * s[0] * s[1]
    return r


def _mode_model(oracle, n, eps, ubar, c0, k, T, tau0, tol):
    s = [float(m) ** 2 for m in n]
    lam = sum(4.0 * s[a] * math.sin(math.pi * k[a] / n[a]) ** 2 for a in range(2))
    mu = lam * (3.0 * ubar ** 2 - 1.0 + eps ** 2 * lam)
    t, tau, c = 0.0, tau0, c0
    taus, ests, ps = [], [], []
    while t < T:
        clipped = t + tau > T
        if clipped:
            tau = T - t
        lmax = max(_column_sum_periodic(s, eps, 3.0 * (ubar - abs(c)) ** 2 - 1.0),
                   _column_sum_periodic(s, eps, 3.0 * (ubar + abs(c)) ** 2 - 1.0))
        p = math.ceil((math.pi / 4) / (math.pi / 2 - math.atan(math.sqrt(tau * lmax))))
        beta = [math.cos(math.pi * (2 * i - 1) / (2 * p)) for i in range(1, p + 1)]
        a = [lmax / (1.0 + beta[0]) * (beta[0] - b) for b in beta]
        order = oracle.lim_order(p)               # the factors commute: order only moves rounding
        cp = c
        for sweep in range(2):
            for idx in range(0 if sweep == 0 else 1, p):
                am = a[order[idx]]
                cp = (c + tau * am * cp - tau * mu * cp) / (1.0 + tau * am)
        cpc = c - 0.5 * tau * mu * (c + cp)       # y_PC on the mode
        est = abs(cp - cpc) / (abs(ubar) * math.sqrt(2.0))
        taus.append(tau); ests.append(est); ps.append(p)
        t = T if clipped else t + tau
        tau = tol / est * tau
        c = cp
    return np.array(taus), np.array(ests), np.array(ps)


@pytest.mark.parametrize("ubar,k,x0,steps,tol", [(0.6, (3, 2), 20.0, 12.0, 3e-9),
                                                 (0.45, (1, 4), 6.0, 20.0, 1e-9)])
def test_adaptive_lim_follows_the_fourier_mode_model(oracle, ubar, k, x0, steps, tol):
    n, eps, c0 = (24, 20), 0.05, 1e-6
    i0, i1 = np.meshgrid(np.arange(n[0]), np.arange(n[1]), indexing="xy")
    mode = np.cos(2 * np.pi * (k[0] * i0 / n[0] + k[1] * i1 / n[1])).reshape(-1)
    y0 = ubar + c0 * mode
    g = oracle.Grid(2, n, eps)
    tau0 = x0 / oracle.lambda_max(g, y0)
    T = steps * tau0
    rc, y, t, st, rec = oracle.integrate(g, y0, "lim", True, T, tau0, tol=tol)
    assert rc == 0 and t == T
    mt, me, mp = _mode_model(oracle, n, eps, ubar, c0, k, T, tau0, tol)
    assert st["steps"] == len(mt) >= 4
    np.testing.assert_array_equal(rec["p"], mp)
    np.testing.assert_allclose(rec["tau"], mt, rtol=1e-4)
    np.testing.assert_allclose(rec["est"], me, rtol=1e-3)
    assert rec["tau"][-1] < mt[-2] * tol / me[-2]         # the last step was clipped to end at T
