"""Pins of the oracle's spatial operators (Sec. 2 Eq. IVP; Sec. 3 Eqs. A_g, J, A_g_cs, p;
the spectral bound of Fig. 1) against Fourier symbols, dense matrices, finite differences and the LIM
matvec counts the paper prints in Tables 1 and 2."""
import os

import numpy as np
import pytest

from _dense import dense_A, dense_Ahat, dense_ghat, shape_of, spectral_A, symbol_A
from paper_2502_14589_gb300 import inputs

GRIDS = [(2, (8, 8)), (2, (12, 7)), (2, (16, 16)), (3, (6, 6, 6)), (3, (5, 7, 9))]


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("dim,n", GRIDS)
def test_A_matches_fourier_symbol_and_dense(oracle, dim, n):
    g = oracle.Grid(dim, n, 0.05)
    v = inputs.initial_state(n, 7, -1, 1)
    Av = oracle.apply_A(g, v)
    assert rel(Av, spectral_A(n, v)) < 1e-13
    if g.N <= 400:
        assert rel(Av, dense_A(n) @ v) < 1e-14
    # mass: columns of A sum to zero, so sum(A v) = 0
    assert abs(Av.sum()) < 1e-12 * np.abs(Av).sum()


@pytest.mark.parametrize("dim,n", GRIDS)
def test_rhs_matches_spectral_evaluation(oracle, dim, n):
    eps = 0.03
    g = oracle.Grid(dim, n, eps)
    y = inputs.initial_state(n, 3, -0.8, 0.8)
    f = oracle.rhs(g, y)
    lam = symbol_A(n)
    Y = np.fft.fftn(y.reshape(shape_of(n)))
    mu = np.fft.fftn((y ** 3 - y).reshape(shape_of(n))) + eps ** 2 * lam * Y
    ref = -np.real(np.fft.ifftn(lam * mu)).reshape(-1)
    assert rel(f, ref) < 1e-12


@pytest.mark.parametrize("dim,n", GRIDS)
@pytest.mark.parametrize("eyre", [False, True])
def test_jacvec_is_minus_jacobian_of_rhs(oracle, dim, n, eyre):
    """f is cubic in y, so the central difference is exact up to the delta^2 v^3 term:
    (f(y+dv) - f(y-dv)) / 2d = -A(J + eps^2 A) v - d^2 A(v^3)."""
    eps = 0.04
    g = oracle.Grid(dim, n, eps)
    y = inputs.initial_state(n, 11, -0.9, 0.9)
    v = inputs.initial_state(n, 12, -1, 1)
    d = 1e-3
    fd = (oracle.rhs(g, y + d * v) - oracle.rhs(g, y - d * v)) / (2 * d)
    jac = -(fd + d * d * oracle.apply_A(g, v ** 3))
    if eyre:  # Eq. (A_g_cs) adds A v
        jac = jac + oracle.apply_A(g, v)
    ge = oracle.Grid(dim, n, eps, eyre=eyre)
    w = oracle.jacvec(ge, y, v)
    assert rel(w, jac) < 1e-9
    if g.N <= 400:
        assert rel(w, dense_Ahat(n, y, eps, eyre) @ v) < 1e-13


@pytest.mark.parametrize("dim,n", GRIDS)
@pytest.mark.parametrize("eyre", [False, True])
def test_ghat_minus_Ahat_y_is_rhs(oracle, dim, n, eyre):
    """Algebra of Eq. (A_g) / (A_g_cs): g_hat - A_hat y = -A(F'(y) + eps^2 A y) = f(y)."""
    g = oracle.Grid(dim, n, 0.05, eyre=eyre)
    y = inputs.initial_state(n, 5, -1, 1)
    gh = oracle.ghat(g, y)
    assert rel(gh, dense_ghat(n, y, eyre) if g.N <= 400 else gh) < 1e-13
    assert rel(gh - oracle.jacvec(g, y, y), oracle.rhs(g, y)) < 1e-12


@pytest.mark.parametrize("dim,n", [(2, (3, 3)), (2, (4, 6)), (2, (5, 5)), (2, (8, 6)),
                                   (3, (3, 4, 5)), (3, (5, 5, 5)), (3, (6, 5, 7))])
@pytest.mark.parametrize("eyre", [False, True])
def test_lambda_max_is_dense_one_norm(oracle, dim, n, eyre):
    """Fig. 1, spectral bound: lambda_max = max_j sum_i |a_ij|, also on grids whose +-2 offsets alias."""
    eps = 0.07
    g = oracle.Grid(dim, n, eps, eyre=eyre)
    y = inputs.initial_state(n, 21, -1.1, 1.1)
    M = dense_Ahat(n, y, eps, eyre)
    ref = np.abs(M).sum(axis=0).max()
    assert abs(oracle.lambda_max(g, y) - ref) <= 1e-13 * ref


@pytest.mark.parametrize("dim,n", [(2, (6, 5)), (3, (4, 5, 6))])
def test_column_abs_sum_is_dense_column_sum(oracle, dim, n):
    """One column of the bound of Fig. 1: the absolute sum of every column of A_hat."""
    eps = 0.07
    g = oracle.Grid(dim, n, eps)
    y = inputs.initial_state(n, 22, -1.1, 1.1)
    ref = np.abs(dense_Ahat(n, y, eps, False)).sum(axis=0)
    got = np.array([oracle.column_abs_sum(g, y, j) for j in range(ref.size)])
    assert np.allclose(got, ref, rtol=1e-13, atol=0)


def _golden_counts():
    path = os.path.join(os.path.dirname(__file__), "golden", "paper_lim_counts.txt")
    rows = []
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        f = line.split()
        rows.append((int(f[0]), float(f[1]), int(f[2]), int(f[3]), f[4]))
    return rows


@pytest.mark.parametrize("row", _golden_counts(), ids=lambda r: f"n{r[0]}-tau{r[1]}-eyre{r[2]}")
def test_lim_matvec_counts_printed_in_paper(oracle, row):
    """Tables 1 and 2 (LIM columns): T/tau steps of 2p-1 matvecs with p from Eq. (p) and
    lambda_max = ||A_hat||_1 (Fig. 1).  The paper's domain (0,64)^2 with h = 64/n is mapped to the
    unit square by x' = x/64, t' = t/64^2, eps' = eps/64, which leaves tau*lambda_max fixed."""
    n, tau, eyre, printed, kind = row
    eps4 = 1.0 * 4 / (2 * np.sqrt(2) * np.arctanh(0.9))     # Eq. (eps), h = 1, m = 4
    g = oracle.Grid(2, n, eps4 / 64, eyre=bool(eyre))
    tau_unit = tau / 64 ** 2
    steps = int(round(1000 / tau))
    counts = [steps * (2 * oracle.cheb_order(tau_unit, oracle.lambda_max(g, np.full(n * n, c))) - 1)
              for c in (0.0, 1.0)]                           # d = 3y^2 - 1 at its two ends
    if kind == "exact":
        assert counts[0] == counts[1] == printed
    else:
        assert min(counts) <= printed <= max(counts)


@pytest.mark.parametrize("x", [1e-6, 0.3, 1.0, 2.0, 10.0, 1e2, 1e4, 1e6, 1e8])
def test_cheb_order_against_eq_p_est(oracle, x):
    """Eq. (p_est): the unrounded order is at most (pi/4) sqrt(x+1) and approaches it;
    tau*lambda_max <= 1 gives p = 1 (LIM reduces to explicit Euler, Sec. 3.1)."""
    p = oracle.cheb_order(x, 1.0)
    bound = np.pi / 4 * np.sqrt(x + 1)
    assert p <= np.ceil(bound)
    assert p >= bound - 1.0 - 0.05 * bound
    if x <= 1.0:
        assert p == 1


def test_energy_and_mass_closed_forms(oracle):
    n = (32, 16)
    eps = 0.1
    g = oracle.Grid(2, n, eps)
    c = 0.3
    y = np.full(g.N, c)
    assert abs(oracle.energy(g, y) - 0.25 * (1 - c * c) ** 2) < 1e-13
    assert abs(oracle.mass(g, y) - c) < 1e-13
    # single x-mode: energy gradient part = eps^2/2 * a^2 * (2 sin(pi/n)/h)^2 * 1/2
    a = 1e-3
    x = (np.arange(n[0]) + 0.0) / n[0]
    y = (a * np.cos(2 * np.pi * x))[None, :].repeat(n[1], axis=0).reshape(-1)
    grad = 0.5 * eps ** 2 * a ** 2 * (2 * np.sin(np.pi / n[0]) * n[0]) ** 2 * 0.5
    Fsum = np.mean(0.25 * (1 - y ** 2) ** 2)
    assert abs(oracle.energy(g, y) - (Fsum + grad)) < 1e-14


@pytest.mark.parametrize("dim,n", [(2, (6, 6)), (2, (7, 5)), (3, (4, 5, 3))])
def test_jacobian_spectrum_follows_propositions_1_and_2(oracle, dim, n):
    """Sec. 3, Propositions 1 and 2, on the oracle's A_hat assembled column by column from its
    Jacobian action: the eigenvalues are real and coincide with those of the symmetric
    A^{1/2}(J + eps^2 A)A^{1/2} (A^{1/2} from the test's own dense Laplacian); A_hat has no
    more negative (positive) eigenvalues than J + eps^2 A; with the Eyre term (Eq. A_g_cs)
    every eigenvalue is nonnegative, so I + tau A_hat is nonsingular."""
    eps = 0.1
    y = inputs.initial_state(n, 21, -0.6, 0.6)
    A = dense_A(n)
    lam, Q = np.linalg.eigh(A)
    sqrtA = (Q * np.sqrt(np.clip(lam, 0.0, None))) @ Q.T
    N = y.size
    for eyre in (False, True):
        g = oracle.Grid(dim, n, eps, eyre=eyre)
        M = np.column_stack([oracle.jacvec(g, y, np.eye(N)[:, k]) for k in range(N)])
        B = np.diag(3 * y ** 2 - 1 + (1.0 if eyre else 0.0)) + eps ** 2 * A
        ev = np.linalg.eigvals(M)
        scale = np.abs(ev).max()
        assert np.abs(ev.imag).max() < 1e-9 * scale
        ev = np.sort(ev.real)
        ev_sym = np.linalg.eigvalsh(sqrtA @ B @ sqrtA)
        assert np.abs(ev - ev_sym).max() < 1e-9 * scale
        eB = np.linalg.eigvalsh(B)
        cut = 1e-9 * scale
        assert (ev < -cut).sum() <= (eB < -cut).sum()
        assert (ev > cut).sum() <= (eB > cut).sum()
        if eyre:
            assert ev.min() > -cut
            assert np.linalg.eigvals(np.eye(N) + 1e-3 * M).real.min() >= 1.0 - 1e-9
        else:
            assert ev.min() < -cut       # this y makes J + eps^2 A indefinite: A_hat is too
