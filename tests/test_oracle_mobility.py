"""Pins of the oracle's variable-mobility form (the Remark on Eq. CHmob): the outer operator
A becomes A_M(y^n), a discretisation of -div(M grad .) frozen over the step, so that
A_hat = A_M (J + eps^2 A) and g_hat = A_M (J y - F'(y)).

* A_M is assembled here independently as sum_a (1/h_a^2) D_a^T diag(face mobility) D_a
  from forward-difference matrices D_a (periodic, or Neumann with no flux through the
  boundary faces), the face mobility being the mean of the two nodes;
* unit mobility gives back the constant-mobility operators;
* A_M is symmetric positive semidefinite with zero column sums (mass), so the Jacobian
  keeps the spectral properties of Propositions 1 and 2 (the Remark after them);
* one EE2 step equals the dense augmented exponential of Eq. (yt) with these A_hat, g_hat;
* steps with the mobility re-frozen at every y^n keep the mass and lower the energy.
"""
import numpy as np
import pytest
import scipy.linalg

from paper_2502_14589_gb300 import inputs


def shape_of(n):
    return tuple(reversed(n))


def forward_differences(n, bc):
    """D_a (one per axis): (D_a v)_i = v_{i+e_a} - v_i; Neumann: 0 on the last layer."""
    dim = len(n)
    N = int(np.prod(n))
    idx = np.arange(N).reshape(shape_of(n))
    Ds = []
    for a in range(dim):
        ax = dim - 1 - a
        D = np.zeros((N, N))
        nb = np.roll(idx, -1, axis=ax).reshape(-1)
        rows = np.arange(N)
        keep = np.ones(N, bool)
        if bc == "neumann":
            last = np.take(idx, [n[a] - 1], axis=ax).reshape(-1)
            keep[last] = False
        D[rows[keep], nb[keep]] += 1.0
        D[rows[keep], rows[keep]] -= 1.0
        Ds.append((a, D, nb))
    return Ds


def dense_AM(n, bc, m):
    AM = np.zeros((m.size, m.size))
    for a, D, nb in forward_differences(n, bc):
        face = 0.5 * (m + m[nb])
        AM += float(n[a]) ** 2 * D.T @ np.diag(face) @ D
    return AM


CASES = [(2, (7, 6), "periodic"), (2, (7, 6), "neumann"), (3, (4, 5, 3), "periodic"),
         (3, (4, 5, 3), "neumann")]


@pytest.mark.parametrize("dim,n,bc", CASES)
def test_mobility_operators_match_dense_flux_form(oracle, dim, n, bc):
    eps = 0.05
    y = inputs.initial_state(n, 31, -0.7, 0.7)
    m = 1.0 - y ** 2                                    # a typical degenerate-type mobility
    AM = dense_AM(n, bc, m)
    A = dense_AM(n, bc, np.ones_like(m))
    assert np.allclose(AM, AM.T) and np.abs(AM.sum(axis=0)).max() < 1e-10 * np.abs(AM).max()
    assert np.linalg.eigvalsh(AM).min() > -1e-10 * np.abs(AM).max()
    v = inputs.initial_state(n, 32, -1, 1)
    for eyre in (False, True):
        g = oracle.Grid(dim, n, eps, eyre=eyre, bc=bc, mobility=m)
        Mhat = AM @ (np.diag(3 * y ** 2 - 1 + (1.0 if eyre else 0.0)) + eps ** 2 * A)
        ghat = AM @ (2 * y ** 3 + (y if eyre else 0.0))
        rel = lambda a, b: np.linalg.norm(a - b) / np.linalg.norm(b)
        assert rel(oracle.jacvec(g, y, v), Mhat @ v) < 1e-13
        assert rel(oracle.ghat(g, y), ghat) < 1e-13
        assert rel(oracle.rhs(g, y), -AM @ (y ** 3 - y + eps ** 2 * A @ y)) < 1e-13
        assert oracle.lambda_max(g, y) == pytest.approx(np.abs(Mhat).sum(axis=0).max(), rel=1e-13)
    # the constant-mobility operators are the unit-mobility case
    g1 = oracle.Grid(dim, n, eps, bc=bc, mobility=np.ones(y.size))
    g0 = oracle.Grid(dim, n, eps, bc=bc)
    assert np.allclose(oracle.jacvec(g1, y, v), oracle.jacvec(g0, y, v), rtol=0,
                       atol=1e-13 * np.abs(oracle.jacvec(g0, y, v)).max())
    assert oracle.lambda_max(g1, y) == pytest.approx(oracle.lambda_max(g0, y), rel=1e-14)


@pytest.mark.parametrize("bc", ["periodic", "neumann"])
def test_mobility_jacobian_spectrum_follows_the_remark(oracle, bc):
    """Propositions 1 and 2 stay valid with a symmetric positive semidefinite A_M: real
    eigenvalues, equal to those of A_M^{1/2}(J + eps^2 A)A_M^{1/2}; nonnegative with Eyre."""
    n = (6, 5); eps = 0.1
    y = inputs.initial_state(n, 33, -0.6, 0.6)
    m = 1.0 - y ** 2
    AM = dense_AM(n, bc, m)
    A = dense_AM(n, bc, np.ones_like(m))
    lam, Q = np.linalg.eigh(AM)
    root = (Q * np.sqrt(np.clip(lam, 0.0, None))) @ Q.T
    N = y.size
    for eyre in (False, True):
        g = oracle.Grid(2, n, eps, eyre=eyre, bc=bc, mobility=m)
        Mhat = np.column_stack([oracle.jacvec(g, y, np.eye(N)[:, k]) for k in range(N)])
        B = np.diag(3 * y ** 2 - 1 + (1.0 if eyre else 0.0)) + eps ** 2 * A
        ev = np.linalg.eigvals(Mhat)
        scale = np.abs(ev).max()
        assert np.abs(ev.imag).max() < 1e-9 * scale
        assert np.abs(np.sort(ev.real) - np.linalg.eigvalsh(root @ B @ root)).max() < 1e-9 * scale
        if eyre:
            assert ev.real.min() > -1e-9 * scale


@pytest.mark.parametrize("bc", ["periodic", "neumann"])
def test_mobility_ee_step_equals_augmented_exponential(oracle, bc):
    n = (6, 5); eps = 0.07
    y = inputs.initial_state(n, 34, -0.8, 0.8)
    m = 1.0 - y ** 2
    AM = dense_AM(n, bc, m)
    A = dense_AM(n, bc, np.ones_like(m))
    Mhat = AM @ (np.diag(3 * y ** 2 - 1) + eps ** 2 * A)
    gv = AM @ (2 * y ** 3)
    N = y.size
    tau = 2e-4
    aug = np.zeros((N + 1, N + 1)); aug[:N, :N] = -tau * Mhat; aug[:N, N] = tau * (gv - Mhat @ y)
    exact = y + scipy.linalg.expm(aug)[:N, N]
    g = oracle.Grid(2, n, eps, bc=bc, mobility=m)
    rc, out, taken, j, st = oracle.ee_step(g, y, tau, tol_phi_fixed=1e-12, mmax=N)
    assert rc == 0 and taken == tau
    assert np.linalg.norm(out - exact) <= 1e-10 * np.linalg.norm(exact)


@pytest.mark.parametrize("scheme", ["ee2", "lim"])
def test_mobility_steps_keep_mass_and_lower_energy(oracle, scheme):
    """Mobility M(c) = 1 - c^2 re-frozen at every y^n (as the Remark prescribes): the mass is
    kept and the energy of Eq. (Ee) decreases from step to step."""
    n = (20, 16); eps = 0.05
    g0 = oracle.Grid(2, n, eps, bc="neumann")
    y = inputs.initial_state(n, 35, -0.05, 0.05, mean=0.1)
    m0 = oracle.mass(g0, y)
    E = [oracle.energy(g0, y)]
    tau = 2e-7
    for _ in range(10):
        g = oracle.Grid(2, n, eps, bc="neumann", mobility=1.0 - y ** 2)
        if scheme == "ee2":
            rc, y, taken, j, st = oracle.ee_step(g, y, tau, tol_phi_fixed=1e-10, mmax=30,
                                                 linear_restart=True)
            assert rc == 0
        else:
            y, p, lm, mv = oracle.lim_step(g, y, tau)
            assert p >= 1
        assert abs(oracle.mass(g0, y) - m0) < 1e-14
        E.append(oracle.energy(g0, y))
    E = np.array(E)
    assert np.all(np.diff(E) <= 1e-12 * np.abs(E[:-1])) and E[-1] < E[0]


@pytest.mark.parametrize("bc", ["periodic", "neumann"])
def test_mobility_estimate_uses_the_mobility_operator(oracle, bc):
    """Eq. (LIMest) with the outer A replaced by A_M (the corrector is the trapezoidal rule of
    the same semi-discrete system)."""
    n = (7, 6); eps = 0.05; tau = 3e-6
    y0 = inputs.initial_state(n, 36, -0.5, 0.5)
    y1 = y0 + 1e-3 * inputs.initial_state(n, 37, -1, 1)
    m = 1.0 - y0 ** 2
    AM = dense_AM(n, bc, m)
    A = dense_AM(n, bc, np.ones_like(m))
    fp = lambda c: c ** 3 - c
    ypc = y0 - 0.5 * tau * AM @ (fp(y0) + fp(y1) + eps ** 2 * A @ (y0 + y1))
    ref = np.linalg.norm(y1 - ypc) / np.linalg.norm(ypc)
    g = oracle.Grid(2, n, eps, bc=bc, mobility=m)
    assert oracle.estimate(g, y0, y1, tau) == pytest.approx(ref, rel=1e-12)
