"""Pins of the oracle's matrix exponential, projected phi (Eqs. phi, yt_m), Arnoldi process
(Eq. Arn), residual identity (Eq. rm) and EE2 Krylov step (Fig. 2, Eq. yt) against scipy,
eigendecompositions, closed forms and the dense augmented-matrix exponential."""
import numpy as np
import pytest
import scipy.linalg

from _dense import dense_Ahat, dense_ghat
from paper_2502_14589_gb300 import inputs


@pytest.mark.parametrize("n", [1, 2, 5, 17, 31])
@pytest.mark.parametrize("scale", [1e-4, 0.5, 3.0, 40.0, 700.0])
def test_expm_matches_scipy(oracle, n, scale):
    rng = np.random.default_rng(n)
    M = rng.standard_normal((n, n))
    M = np.triu(M, -1)                                 # Hessenberg, like H_j
    M = -scale * (M @ M.T + 0.1 * np.eye(n)) / max(1, n) if scale > 1 else scale * M
    E = oracle.expm(M)
    R = scipy.linalg.expm(M)
    assert np.linalg.norm(E - R) <= 1e-12 * max(np.linalg.norm(R), 1e-300) + 1e-300


def test_phi_closed_forms(oracle):
    # j = 1: u = s phi(-s h) = (1 - exp(-s h)) / h
    for h, s in [(2.0, 0.1), (1e3, 1.0), (-0.5, 2.0), (1e-12, 3.0)]:
        u = oracle.phi_e1(np.array([[h]]), 1, s)
        ref = (1 - np.exp(-s * h)) / h if abs(s * h) > 1e-8 else s * (1 - s * h / 2)
        assert abs(u[0] - ref) <= 1e-14 * abs(ref)
    # phi(0) = 1: H = 0 gives u = s e_1
    u = oracle.phi_e1(np.zeros((4, 4)), 4, 0.7)
    np.testing.assert_allclose(u, [0.7, 0, 0, 0], atol=1e-16)


def test_phi_matches_eigendecomposition(oracle):
    rng = np.random.default_rng(3)
    j = 12
    lam = np.sort(rng.uniform(0.01, 50.0, j))
    Q = rng.standard_normal((j, j))
    H = Q @ np.diag(lam) @ np.linalg.inv(Q)
    s = 0.3
    u = oracle.phi_e1(H, j, s)
    z = -s * lam
    phi = np.expm1(z) / z
    ref = s * (Q @ (phi * np.linalg.solve(Q, np.eye(j)[:, 0])))
    assert np.linalg.norm(u - ref) <= 1e-11 * np.linalg.norm(ref)


def _ch_dense(n=(6, 5), eps=0.07, seed=2, amp=0.8):
    y = inputs.initial_state(n, seed, -amp, amp)
    return y, dense_Ahat(n, y, eps), dense_ghat(n, y)


def test_arnoldi_relation_and_orthonormality(oracle):
    y, M, g = _ch_dense()
    v1 = g - M @ y
    m = 12
    V, H = oracle.arnoldi_dense(M, v1, m)
    Vm = V[:m].T; Vm1 = V.T
    assert np.linalg.norm(Vm1.T @ Vm1 - np.eye(m + 1)) < 1e-10
    assert np.linalg.norm(M @ Vm - Vm1 @ H) <= 1e-12 * np.linalg.norm(M) * np.sqrt(m)
    assert np.allclose(np.tril(H, -2), 0.0)          # upper Hessenberg


@pytest.mark.parametrize("t", [1e-3, 0.05, 0.3])
def test_residual_identity_eq_rm(oracle, t):
    """||r_m(t)|| of Eq. (rm) formed explicitly equals beta h_{m+1,m} t |e_m^T phi(-tH) e_1|."""
    y, M, g = _ch_dense()
    v1 = g - M @ y
    beta = np.linalg.norm(v1)
    m = 8
    V, H = oracle.arnoldi_dense(M, v1, m)
    Vm = V[:m].T
    u = oracle.phi_e1(H[:m, :m], m, t)                 # t phi(-t H) e_1
    ym = y + Vm @ (beta * u)
    dym = Vm @ (beta * scipy.linalg.expm(-t * H[:m, :m])[:, 0])   # d/dt [t phi(-tH)] = exp(-tH)
    r = -M @ ym + g - dym
    ident = beta * H[m, m - 1] * abs(u[m - 1])
    floor = 1e-13 * (np.linalg.norm(M) * np.linalg.norm(ym) + np.linalg.norm(g))  # rounding of r
    assert abs(np.linalg.norm(r) - ident) <= 1e-8 * ident + floor
    if t >= 0.05:
        assert ident > 100 * floor          # the identity is tested above the rounding level


@pytest.mark.parametrize("tau", [1e-5, 1e-4, 1e-3])
def test_krylov_step_equals_augmented_expm(oracle, tau):
    """Eq. (yt): y(t_n+tau) = y^n + tau phi(-tau A_hat)(g_hat - A_hat y^n), from the dense
    augmented (N+1) x (N+1) exponential; Krylov with m_max = N and tol_phi = 1e-14."""
    y, M, g = _ch_dense()
    N = M.shape[0]
    aug = np.zeros((N + 1, N + 1)); aug[:N, :N] = -tau * M; aug[:N, N] = tau * (g - M @ y)
    exact = y + scipy.linalg.expm(aug)[:N, N]
    rc, out, taken, j = oracle.krylov_dense(M, g, y, tau, 1e-14, N)
    assert rc == 0 and taken == tau
    assert np.linalg.norm(out - exact) <= 1e-12 * np.linalg.norm(exact)


def test_krylov_shrinks_step_and_meets_tolerance(oracle):
    """Fig. 2, step trace: at j = m_max the step is cut to an admissible tau < tau0 and the
    Krylov solution then satisfies Eq. (phi_stop) against the exact linear solution."""
    y, M, g = _ch_dense()
    N = M.shape[0]
    tau0 = 5e-3; tol = 1e-6; mmax = 4
    rc, out, taken, j = oracle.krylov_dense(M, g, y, tau0, tol, mmax)
    assert rc == 0 and j == mmax and 0 < taken < tau0
    aug = np.zeros((N + 1, N + 1)); aug[:N, :N] = -taken * M; aug[:N, N] = taken * (g - M @ y)
    exact = y + scipy.linalg.expm(aug)[:N, N]
    beta = np.linalg.norm(g - M @ y)
    assert np.linalg.norm(out - exact) < 100 * tol * beta * taken
    # Maximality at the trace's resolution: halving from tau0 stops at the first admissible
    # lo0 = tau0 / 2^k, and 12 bisections of [lo0, 2 lo0] leave an inadmissible end within
    # lo0 / 2^12 <= taken / 2^12 of the step; a run started just beyond it must be cut.
    for tau0_, tol_, mmax_ in [(tau0, tol, mmax), (3e-3, 1e-7, 5), (1e-2, 1e-6, 3), (5e-3, 1e-8, 6)]:
        rc, _, taken, j = oracle.krylov_dense(M, g, y, tau0_, tol_, mmax_)
        assert rc == 0 and j == mmax_ and 0 < taken < tau0_
        start = taken * (1 + 2.0 ** -12)
        rc2, _, taken2, _ = oracle.krylov_dense(M, g, y, start, tol_, mmax_)
        assert rc2 == 0 and taken2 < start


def test_grid_ee_step_linear_restart_matches_exact(oracle):
    """Constant-step EE2 with linear RT restarting covers the whole tau (Sec. 4.1 end)."""
    n = (6, 5); eps = 0.07
    g = oracle.Grid(2, n, eps)
    y = inputs.initial_state(n, 2, -0.8, 0.8)
    M = dense_Ahat(n, y, eps); gv = dense_ghat(n, y)
    N = M.shape[0]
    tau = 4e-3
    aug = np.zeros((N + 1, N + 1)); aug[:N, :N] = -tau * M; aug[:N, N] = tau * (gv - M @ y)
    exact = y + scipy.linalg.expm(aug)[:N, N]
    rc, out, taken, j, st = oracle.ee_step(g, y, tau, tol_phi_fixed=1e-10, mmax=5, linear_restart=True)
    assert rc == 0 and taken == tau and st["restarts"] >= 1
    assert np.linalg.norm(out - exact) <= 1e-7 * np.linalg.norm(exact)


def test_tol_phi_cases(oracle):
    """Eq. (tol_phi) on hand-worked cases: each of the four terms can be the active one."""
    assert oracle.tol_phi(1.0, 1.0, 1e-6) == pytest.approx(1e-5)      # 10 tol
    assert oracle.tol_phi(1.0, 1.0, 1.0) == pytest.approx(0.1)        # 1/10 and ||g||/(10 beta)
    assert oracle.tol_phi(1e-3, 1.0, 1.0) == pytest.approx(1e-4)      # ||g||/(10 beta)
    assert oracle.tol_phi(1.0, 1.0, 1e-10) == pytest.approx(1e-7)     # floor
