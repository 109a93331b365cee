"""Pins of the oracle's homogeneous Neumann discretisation: the boundary conditions of
Eq. (CH) on the cell-centred nodes of Sec. 5.1, x_i = (i - 1/2) h, the paper's own
test setting.

* The cell-centred Neumann Laplacian is diagonalised by the type-II discrete cosine
  transform, with eigenvalues sum_a (4 / h_a^2) sin^2(pi k_a / (2 n_a)); this fixes A,
  f and the linearised cosine-mode dynamics independently of the oracle's loops.
* A dense matrix assembled here from the one-dimensional stencil (diagonal 1 instead of 2
  in the first and last rows) pins A, A_hat and ||A_hat||_1.
* Eq. (Ediscr) sums the n - 1 interior differences per axis, which is the Neumann form:
  a cosine mode gives its gradient energy in closed form.
* The LIM matvec counts printed in Tables 1 and 2 hold on the paper's own Neumann grid.
"""
import os

import numpy as np
import pytest
import scipy.fft

from paper_2502_14589_gb300 import inputs

GRIDS = [(2, (8, 8)), (2, (7, 12)), (3, (5, 6, 4)), (2, (2, 3))]


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def shape_of(n):
    return tuple(reversed(n))


def neumann_symbol(n):
    dim = len(n)
    lam = np.zeros(shape_of(n))
    for a in range(dim):
        ax = dim - 1 - a
        k = np.arange(n[a])
        la = 4.0 * float(n[a]) ** 2 * np.sin(np.pi * k / (2 * n[a])) ** 2
        sh = [1] * dim
        sh[ax] = n[a]
        lam = lam + la.reshape(sh)
    return lam


def dct_apply(n, lam_fn, v):
    V = scipy.fft.dctn(v.reshape(shape_of(n)), type=2, norm="ortho")
    return scipy.fft.idctn(lam_fn * V, type=2, norm="ortho").reshape(-1)


def dense_neumann_A(n):
    """Kronecker sum of the 1D cell-centred Neumann second differences (x fastest)."""
    def one(m):
        D = 2.0 * np.eye(m) - np.eye(m, k=1) - np.eye(m, k=-1)
        D[0, 0] -= 1.0
        D[-1, -1] -= 1.0
        return float(m) ** 2 * D
    A = np.zeros((1, 1))
    for a in reversed(range(len(n))):     # slowest axis first in the Kronecker product
        Da = one(n[a])
        A = np.kron(A, np.eye(n[a])) + np.kron(np.eye(A.shape[0]), Da) if A.size > 1 else Da
    return A


@pytest.mark.parametrize("dim,n", GRIDS)
def test_neumann_A_matches_dct_symbol_and_dense(oracle, dim, n):
    g = oracle.Grid(dim, n, 0.05, bc="neumann")
    v = inputs.initial_state(n, 7, -1, 1)
    Av = oracle.apply_A(g, v)
    assert rel(Av, dct_apply(n, neumann_symbol(n), v)) < 1e-13
    A = dense_neumann_A(n)
    assert np.allclose(A, A.T)
    assert rel(Av, A @ v) < 1e-14
    assert abs(Av.sum()) < 1e-12 * np.abs(Av).sum()         # zero column sums: mass
    # the boundary really differs from the periodic operator
    assert rel(Av, oracle.apply_A(oracle.Grid(dim, n, 0.05), v)) > 1e-3


@pytest.mark.parametrize("dim,n", GRIDS[:3])
def test_neumann_rhs_by_cosine_transform(oracle, dim, n):
    """Eq. (IVP): f = -A (F'(y) + eps^2 A y), both products through the DCT."""
    eps = 0.03
    g = oracle.Grid(dim, n, eps, bc="neumann")
    y = inputs.initial_state(n, 3, -0.8, 0.8)
    lam = neumann_symbol(n)
    mu = (y ** 3 - y) + eps ** 2 * dct_apply(n, lam, y)
    assert rel(oracle.rhs(g, y), -dct_apply(n, lam, mu)) < 1e-12
    assert abs(oracle.rhs(g, y).sum()) < 1e-11 * np.abs(oracle.rhs(g, y)).sum()


@pytest.mark.parametrize("dim,n", GRIDS)
@pytest.mark.parametrize("eyre", [False, True])
def test_neumann_jacobian_and_one_norm(oracle, dim, n, eyre):
    """Eqs. (A_g) / (A_g_cs) against the dense A_hat; g_hat - A_hat y = f; the bound of
    Fig. 1, lambda_max = ||A_hat||_1 against the dense column sums."""
    eps = 0.06
    g = oracle.Grid(dim, n, eps, eyre=eyre, bc="neumann")
    y = inputs.initial_state(n, 11, -0.9, 0.9)
    v = inputs.initial_state(n, 12, -1, 1)
    A = dense_neumann_A(n)
    M = A @ (np.diag(3 * y ** 2 - 1 + (1.0 if eyre else 0.0)) + eps ** 2 * A)
    assert rel(oracle.jacvec(g, y, v), M @ v) < 1e-13
    gh = A @ (2 * y ** 3 + (y if eyre else 0.0))
    assert rel(oracle.ghat(g, y), gh) < 1e-13
    assert rel(oracle.ghat(g, y) - oracle.jacvec(g, y, y), oracle.rhs(g, y)) < 1e-12
    assert oracle.lambda_max(g, y) == pytest.approx(np.abs(M).sum(axis=0).max(), rel=1e-13)


def test_neumann_energy_of_a_cosine_mode(oracle):
    """Eq. (Ediscr) with its n - 1 interior differences per axis: for y = c + a cos(pi k x / L)
    on cell centres, sum_i (y_{i+1} - y_i)^2 = 2 n a^2 sin^2(pi k / (2 n)) per grid line."""
    n = (24, 10); eps = 0.07; c = 0.2; a = 0.3; k = 5
    g = oracle.Grid(2, n, eps, bc="neumann")
    x = (np.arange(n[0]) + 0.5) / n[0]
    row = c + a * np.cos(np.pi * k * x)
    y = np.tile(row, n[1])
    h2 = 1.0 / (n[0] * n[1])
    grad = 0.5 * eps ** 2 * n[1] * (2 * n[0] * a ** 2 * np.sin(np.pi * k / (2 * n[0])) ** 2) * n[0] ** 2
    F = 0.25 * (1 - y ** 2) ** 2
    assert oracle.energy(g, y) == pytest.approx(h2 * (F.sum() + grad), rel=1e-13)
    assert oracle.mass(g, y) == pytest.approx(c, rel=1e-13)


@pytest.mark.parametrize("ubar,k", [(0.6, (3, 0)), (0.0, (1, 2))])
def test_neumann_linearised_cosine_mode(oracle, ubar, k):
    """About a constant ubar a cosine mode of amplitude delta evolves as
    exp(-lam_k (3 ubar^2 - 1 + eps^2 lam_k) t) to O(delta), lam_k the Neumann eigenvalue."""
    n = (16, 12); eps = 0.02
    g = oracle.Grid(2, n, eps, bc="neumann")
    x = (np.arange(n[0]) + 0.5) / n[0]; yy = (np.arange(n[1]) + 0.5) / n[1]
    mode = (np.cos(np.pi * k[1] * yy)[:, None] * np.cos(np.pi * k[0] * x)[None, :]).reshape(-1)
    delta = 1e-9
    lam = neumann_symbol(n)[k[1], k[0]]
    rate = -lam * (3 * ubar ** 2 - 1 + eps ** 2 * lam)
    T = 0.3 / abs(rate)
    rc, y, t, st, rec = oracle.integrate(g, ubar + delta * mode, "ee2", False, T, T / 8, tol_phi=1e-12)
    assert rc == 0
    amp = np.dot(y - ubar, mode) / np.dot(mode, mode)
    assert abs(amp / delta - np.exp(rate * T)) < 1e-6 * np.exp(abs(rate) * T)


@pytest.mark.parametrize("scheme", ["ee2", "lim"])
def test_neumann_mass_and_energy_laws(oracle, scheme):
    """Eqs. (m), (Ee) under the Neumann conditions: adaptive runs keep the mass and never
    raise the energy from step to step."""
    n = (20, 16)
    g = oracle.Grid(2, n, 0.05, bc="neumann")
    y = inputs.initial_state(n, 4, -0.05, 0.05, mean=0.1)
    m0 = oracle.mass(g, y)
    E = [oracle.energy(g, y)]
    for _ in range(8):
        rc, y, t, st, rec = oracle.integrate(g, y, scheme, True, 4e-6, 1e-7, tol=1e-6)
        assert rc == 0 and t == 4e-6
        E.append(oracle.energy(g, y))
        assert abs(oracle.mass(g, y) - m0) < 1e-14
    E = np.array(E)
    assert np.all(np.diff(E) <= 1e-12 * np.abs(E[:-1]))
    assert E[-1] < E[0]


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
def test_lim_counts_on_the_papers_neumann_grid(oracle, row):
    """Tables 1 and 2 (LIM columns) on the paper's own grid: Neumann, cell-centred, (0,64)^2
    with h = 64/n, mapped to the unit square by x' = x/64, t' = t/64^2, eps' = eps/64.
    lambda_max = ||A_hat||_1 over all columns, boundary ones included."""
    n, tau, eyre, printed, kind = row
    eps4 = 4 / (2 * np.sqrt(2) * np.arctanh(0.9))            # Eq. (eps), h = 1, m = 4
    g = oracle.Grid(2, n, eps4 / 64, eyre=bool(eyre), bc="neumann")
    tau_unit = tau / 64 ** 2
    steps = int(round(1000 / tau))
    counts = [steps * (2 * oracle.cheb_order(tau_unit, oracle.lambda_max(g, np.full(n * n, c))) - 1)
              for c in (0.0, 1.0)]
    if kind == "exact":
        assert counts[0] == counts[1] == printed
    else:
        assert min(counts) <= printed <= max(counts)



def _dense_neumann_ahat(n, y, eps, eyre):
    A = dense_neumann_A(n)
    return A @ (np.diag(3 * y ** 2 - 1 + (1.0 if eyre else 0.0)) + eps ** 2 * A), A


@pytest.mark.parametrize("eyre", [False, True])
def test_neumann_lim_step_equals_dense_lim(oracle, eyre):
    """Fig. 1 on the Neumann grid equals the LIM core on the dense A_hat, g_hat, ||A_hat||_1."""
    n = (7, 6); eps = 0.06
    g = oracle.Grid(2, n, eps, eyre=eyre, bc="neumann")
    y = inputs.initial_state(n, 9, -0.9, 0.9)
    M, A = _dense_neumann_ahat(n, y, eps, eyre)
    gv = A @ (2 * y ** 3 + (y if eyre else 0.0))
    lmax = np.abs(M).sum(axis=0).max()
    tau = 37.0 / lmax
    out, p, lm, mv = oracle.lim_step(g, y, tau)
    ref, p2 = oracle.lim_dense(M, gv, y, tau, lmax)
    assert p == p2 and mv == 2 * p - 1
    assert abs(lm - lmax) < 1e-13 * lmax
    np.testing.assert_allclose(out, ref, rtol=0, atol=1e-11 * np.abs(ref).max())


@pytest.mark.parametrize("linear_restart,mmax", [(False, 30), (True, 5)])
def test_neumann_ee_step_equals_augmented_exponential(oracle, linear_restart, mmax):
    """Eq. (yt) on the Neumann grid: y^n + tau phi(-tau A_hat)(g_hat - A_hat y^n) from the
    dense (N+1) x (N+1) augmented exponential, with and without linear restarting."""
    import scipy.linalg
    n = (6, 5); eps = 0.07
    g = oracle.Grid(2, n, eps, bc="neumann")
    y = inputs.initial_state(n, 2, -0.8, 0.8)
    M, A = _dense_neumann_ahat(n, y, eps, False)
    gv = A @ (2 * y ** 3)
    N = M.shape[0]
    tau = 2e-3 if linear_restart else 1e-4
    aug = np.zeros((N + 1, N + 1)); aug[:N, :N] = -tau * M; aug[:N, N] = tau * (gv - M @ y)
    exact = y + scipy.linalg.expm(aug)[:N, N]
    rc, out, taken, j, st = oracle.ee_step(g, y, tau, tol_phi_fixed=1e-11, mmax=mmax,
                                           linear_restart=linear_restart)
    assert rc == 0 and taken == tau
    if linear_restart:
        assert st["restarts"] >= 1
    assert np.linalg.norm(out - exact) <= 1e-8 * np.linalg.norm(exact)


def test_neumann_jacobian_spectrum_follows_propositions_1_and_2(oracle):
    """Sec. 3, Propositions 1 and 2 with the Neumann A (also symmetric positive
    semidefinite): real eigenvalues equal to those of A^{1/2}(J + eps^2 A)A^{1/2}; only
    nonnegative ones with the Eyre term."""
    n = (6, 5); eps = 0.1
    y = inputs.initial_state(n, 21, -0.6, 0.6)
    A = dense_neumann_A(n)
    lam, Q = np.linalg.eigh(A)
    sqrtA = (Q * np.sqrt(np.clip(lam, 0.0, None))) @ Q.T
    N = y.size
    for eyre in (False, True):
        g = oracle.Grid(2, n, eps, eyre=eyre, bc="neumann")
        M = np.column_stack([oracle.jacvec(g, y, np.eye(N)[:, k]) for k in range(N)])
        B = np.diag(3 * y ** 2 - 1 + (1.0 if eyre else 0.0)) + eps ** 2 * A
        ev = np.linalg.eigvals(M)
        scale = np.abs(ev).max()
        assert np.abs(ev.imag).max() < 1e-9 * scale
        assert np.abs(np.sort(ev.real) - np.linalg.eigvalsh(sqrtA @ B @ sqrtA)).max() < 1e-9 * scale
        if eyre:
            assert ev.real.min() > -1e-9 * scale
