"""Pins of the oracle's time-stepping drivers (Figs. 3 and 4, constant-step forms) by the
laws of Sec. 2 (Eqs. Ee, m), the linearised Fourier dynamics about a constant state, and
the convergence orders of Sec. 3.1 (LIM order 1) and Prop. 3 (EE2 order 2)."""
import numpy as np
import pytest

from _dense import symbol_A
from paper_2502_14589_gb300 import inputs


def test_mass_is_conserved(oracle):
    n = (32, 32)
    g = oracle.Grid(2, n, 0.05)
    y0 = inputs.initial_state(n, 0, -0.05, 0.05, mean=0.2)
    for scheme, adaptive in [("ee2", False), ("lim", False), ("ee2", True), ("lim", True)]:
        rc, y, t, st, rec = oracle.integrate(g, y0, scheme, adaptive, 2e-5, 1e-6, tol=1e-5,
                                             tol_phi=1e-8 if not adaptive else -1.0)
        assert rc == 0 and t == 2e-5
        assert abs(oracle.mass(g, y) - oracle.mass(g, y0)) < 1e-13


@pytest.mark.parametrize("scheme", ["ee2", "lim"])
def test_energy_does_not_increase(oracle, scheme):
    """Eq. (Ee): the discrete energy is a Lyapunov function of the semi-discrete IVP."""
    n = (24, 24)
    g = oracle.Grid(2, n, 0.05)
    y = inputs.initial_state(n, 1, -0.05, 0.05)
    E = [oracle.energy(g, y)]
    for k in range(15):
        rc, y, t, st, rec = oracle.integrate(g, y, scheme, False, 2e-6, 2e-6, tol_phi=1e-10)
        assert rc == 0
        E.append(oracle.energy(g, y))
    E = np.array(E)
    assert np.all(np.diff(E) <= 1e-12 * np.abs(E[:-1]))
    assert E[-1] < E[0]


@pytest.mark.parametrize("ubar,k", [(0.6, (3, 0)), (0.0, (1, 2)), (0.0, (5, 4))])
def test_linearised_fourier_mode(oracle, ubar, k):
    """About a constant ubar, a mode of amplitude delta evolves as
    exp(-lam_k (3 ubar^2 - 1 + eps^2 lam_k) t) to O(delta) (decay for ubar = 0.6, growth for
    ubar = 0 with lam_k < 1/eps^2)."""
    n = (16, 16); eps = 0.02
    g = oracle.Grid(2, n, eps)
    x = np.arange(n[0]) / n[0]; yy = np.arange(n[1]) / n[1]
    mode = np.cos(2 * np.pi * (k[0] * x[None, :] + k[1] * yy[:, None])).reshape(-1)
    delta = 1e-9
    y0 = ubar + delta * mode
    lam = symbol_A(n)[k[1], k[0]]
    rate = -lam * (3 * ubar ** 2 - 1 + eps ** 2 * lam)
    T = 0.3 / abs(rate)
    rc, y, t, st, rec = oracle.integrate(g, y0, "ee2", False, T, T / 8, tol_phi=1e-12)
    assert rc == 0
    amp = np.dot(y - ubar, mode) / np.dot(mode, mode)
    assert abs(amp / delta - np.exp(rate * T)) < 1e-6 * np.exp(abs(rate) * T)


def _conv(oracle, scheme, taus, ref_tau, n=(12, 12), eps=0.08, T=4e-4):
    g = oracle.Grid(2, n, eps)
    y0 = inputs.initial_state(n, 3, -0.3, 0.3)
    rc, yref, *_ = oracle.integrate(g, y0, scheme, False, T, ref_tau, tol_phi=1e-13, mmax=60)
    assert rc == 0
    errs = []
    for tau in taus:
        rc, y, *_ = oracle.integrate(g, y0, scheme, False, T, tau, tol_phi=1e-13, mmax=60)
        assert rc == 0
        errs.append(np.linalg.norm(y - yref) / np.linalg.norm(yref))   # Eq. (acc_reached)
    return np.array(errs)


def test_ee2_is_second_order(oracle):
    """Prop. 3: local error O(tau^3), global order 2 (nonstiff regime here)."""
    errs = _conv(oracle, "ee2", [1e-4, 5e-5, 2.5e-5], 2.5e-5 / 16)
    ratios = errs[:-1] / errs[1:]
    assert np.all((ratios > 3.3) & (ratios < 4.7)), ratios


def test_lim_is_first_order(oracle):
    """Sec. 3.1: LIM has order 1."""
    errs = _conv(oracle, "lim", [2e-5, 1e-5, 5e-6], 5e-6 / 32)
    ratios = errs[:-1] / errs[1:]
    assert np.all((ratios > 1.7) & (ratios < 2.4)), ratios


def test_adaptive_controllers_follow_eq_eedt_and_eq_limdt(oracle):
    """The step-size update of Figs. 3/4 from the recorded (tau, est): EE2 tau_new = min(5/4 tau,
    sqrt(tol/est) tau) (Eq. EEdt); LIM tau_new = tol/est tau (Eq. LIMdt); the last step ends at T."""
    n = (24, 24); T = 1e-4; tol = 1e-5
    g = oracle.Grid(2, n, 0.03)
    y0 = inputs.initial_state(n, 8, -0.05, 0.05)
    for scheme in ("ee2", "lim"):
        rc, y, t, st, rec = oracle.integrate(g, y0, scheme, True, T, 1e-7, tol=tol)
        assert rc == 0 and t == T and st["steps"] == len(rec["tau"])
        tau, est = rec["tau"], rec["est"]
        if scheme == "ee2":
            nxt = np.minimum(1.25 * tau, np.sqrt(tol / est) * tau)
        else:
            nxt = tol / est * tau
        # every step but the last (which is clipped to T) takes the controller's tau
        shrunk = rec["shrunk"][1:-1].astype(bool)
        assert np.allclose(tau[1:-1][~shrunk], nxt[:-2][~shrunk], rtol=1e-14)
        assert abs(tau.sum() - T) < 1e-12 * T


@pytest.mark.parametrize("scheme,order", [("ee2", 3), ("lim", 2)])
def test_estimate_scales_with_local_error_order(oracle, scheme, order):
    """Eq. (LIMest): y_PC is the explicit trapezoidal corrector, so est for an EE2 step (local
    error O(tau^3), Prop. 3) scales like tau^3 and for a LIM step (order 1) like tau^2."""
    n = (12, 12)
    g = oracle.Grid(2, n, 0.08)
    y = inputs.initial_state(n, 5, -0.3, 0.3)
    ests = []
    for tau in (4e-6, 2e-6, 1e-6):
        if scheme == "ee2":
            rc, y1, taken, j, st = oracle.ee_step(g, y, tau, tol_phi_fixed=1e-13, mmax=60)
        else:
            y1, *_ = oracle.lim_step(g, y, tau)
        ests.append(oracle.estimate(g, y, y1, tau))
    r = np.array(ests[:-1]) / np.array(ests[1:])
    assert np.all(np.abs(np.log2(r) - order) < 0.35), r
