"""Mixed precision (FP32 Krylov basis and stencil arithmetic, FP64 solution, reductions,
Hessenberg matrix, projected phi and control) against the FP64 oracle.  The tolerance of a
single Krylov step comes from the arithmetic: FP32 basis vectors perturb A_hat by about
u32 ||A_hat||, which moves the increment by about u32 * tau * lambda_max relative to it."""
import numpy as np
import pytest

from paper_2502_14589_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def ch():
    from paper_2502_14589_gb300 import build, ch as chmod
    build.build()
    chmod.load()
    return chmod


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


@pytest.mark.parametrize("dim,n,eps,tau", [(2, (128, 128), 0.02, 2e-7), (2, (256, 256), 0.01, 2e-8),
                                           (3, (32, 32, 32), 0.03, 1e-6),
                                           (2, (1024, 1024), 0.01, 1e-8),     # resident FP32 iteration
                                           (3, (144, 144, 144), 0.02, 1e-7),  # streaming FP32 iteration
                                           # streaming, the last tile ending inside a warp
                                           (2, (1400, 900), 0.01, 1e-8), (3, (110, 110, 105), 0.02, 1e-7),
                                           (2, (37, 53), 0.03, 1e-6),         # rows not a multiple of 4,
                                           (3, (10, 9, 11), 0.05, 1e-5)])     # partial last group
def test_mixed_krylov_step(ch, oracle, dim, n, eps, tau):
    y = inputs.initial_state(n, 3, -0.05, 0.05)
    og = oracle.Grid(dim, n, eps)
    lmax = oracle.lambda_max(og, y)
    with ch.Grid(dim, n, eps, ch.CH_MIXED) as G:
        yn = torch.empty(G.N, dtype=torch.float64, device="cuda")
        tu, st = ch.ch_phi_krylov(G.h, dev(y), tau, 1e-7, 30, 0, yn)
        yg = host(yn)
        _, m1 = ch.ch_energy_mass(G.h, yn)
        _, m0 = ch.ch_energy_mass(G.h, dev(y))
    rc, yo, to, jo, sto = oracle.ee_step(og, y, tu, tol_phi_fixed=1e-7, mmax=30)
    inc = np.linalg.norm(yo - y)
    err = np.linalg.norm(yg - yo) / inc
    bound = 50 * U32 * max(tau * lmax, 1.0)
    print(f"mixed Krylov step n={n} tau*lmax={tau * lmax:.3g} increment rel err={err:.2e} bound={bound:.2e}")
    assert err < bound
    assert abs(m1 - m0) < 1e-13


@pytest.mark.parametrize("dim,n,eps,T", [(2, (96, 96), 0.02, 1e-4), (3, (24, 24, 24), 0.04, 1e-4)])
def test_mixed_adaptive_error_at_T(ch, oracle, dim, n, eps, T):
    """Adaptive EE2 in mixed precision: relative L2 error at T against the FP64 oracle run
    of the same scheme and tolerance, stated and held to the 1e-5 target."""
    y0 = inputs.initial_state(n, 1, -0.05, 0.05)
    with ch.Grid(dim, n, eps, ch.CH_MIXED) as G:
        y = dev(y0)
        st = ch.ch_integrate(G.h, ch.make_params("ee2", True, T, 1e-7, 1e-6, 30), y)
        yg = host(y)
    rc, yo, t, sto, rec = oracle.integrate(oracle.Grid(dim, n, eps), y0, "ee2", True, T, 1e-7,
                                           tol=1e-6, mmax=30)
    err = np.linalg.norm(yg - yo) / np.linalg.norm(yo)
    print(f"mixed adaptive EE2 n={n}: steps {st['steps']} vs {sto['steps']}, error at T {err:.2e}")
    assert st["t"] == T
    assert err < 1e-5
    assert abs(yg.mean() - y0.mean()) < 1e-13


def test_mixed_grid_lim_runs_fp64(ch, oracle):
    """LIM iterations amplify rounding by ~ (tau lambda_max)^2, so a mixed grid keeps them in
    FP64: the result matches the FP64 oracle to FP64 parity."""
    n = (64, 64)
    y = inputs.initial_state(n, 2, -0.05, 0.05)
    with ch.Grid(2, n, 0.05, ch.CH_MIXED) as G:
        yn = torch.empty(64 * 64, dtype=torch.float64, device="cuda")
        p, lm = ch.ch_lim_step(G.h, dev(y), 3e-6, yn)
        yg = host(yn)
    yo, po, lo, _ = oracle.lim_step(oracle.Grid(2, n, 0.05), y, 3e-6)
    assert p == po
    assert np.linalg.norm(yg - yo) / np.linalg.norm(yo) < 1e-12


def test_mixed_krylov_beyond_31_dimensions(ch, oracle):
    """A run that needs more than 31 Krylov dimensions (128^2, tau lambda_max ~ 100, m_max 40):
    the FP32 basis uses the Gram-corrected iteration up to j = 31 and the sequential passes
    after it, in the same run."""
    n, eps, tau, tphi = (128, 128), 0.02, 1.5e-5, 1e-7
    y = inputs.initial_state(n, 3, -0.05, 0.05)
    og = oracle.Grid(2, n, eps)
    lmax = oracle.lambda_max(og, y)
    with ch.Grid(2, n, eps, ch.CH_MIXED, mmax_capacity=40) as G:
        yn = torch.empty(G.N, dtype=torch.float64, device="cuda")
        tu, st = ch.ch_phi_krylov(G.h, dev(y), tau, tphi, 40, 0, yn)
        yg = host(yn)
    print(f"mixed run with m_max 40: tau={tu:.3g} matvecs={st['matvecs']}")
    assert st["matvecs"] > 32
    rc, yo, _, _, _ = oracle.ee_step(og, y, tu, tol_phi_fixed=tphi, mmax=40)
    assert rc == 0
    assert np.linalg.norm(yg - yo) / np.linalg.norm(yo - y) < 50 * U32 * max(tu * lmax, 1.0)
    assert abs(yg.mean() - y.mean()) < 1e-13


@pytest.mark.parametrize("dim,n,tau,eyre", [(2, (64, 64), 3e-7, 0), (2, (50, 70), 2e-6, 1), (3, (24, 20, 16), 5e-7, 0)])
def test_mixed_lim_step_in_increment_form(ch, oracle, dim, n, tau, eyre):
    """Fig. 1 on a mixed-precision grid runs on the FP32 increment d = y_prev - y^n (when the
    rounding growth 3 (tau lambda_max)^2 u32 is small): the step agrees with the oracle's to
    the FP32 bound relative to the increment, with the same p, and keeps the mass."""
    eps = 0.05
    y = inputs.initial_state(n, 8, -0.05, 0.05)
    og = oracle.Grid(dim, n, eps, eyre=bool(eyre))
    yo, po, lo, _ = oracle.lim_step(og, y, tau)
    assert 3 * (tau * lo) ** 2 * U32 <= 1e-5          # the increment form applies
    with ch.Grid(dim, n, eps, ch.CH_MIXED) as G:
        yn = torch.empty(G.N, dtype=torch.float64, device="cuda")
        p, lm = ch.ch_lim_step(G.h, dev(y), tau, yn, eyre)
        yg = host(yn)
    assert p == po
    assert np.linalg.norm(yg - yo) / np.linalg.norm(yo - y) < 50 * U32 * max(3 * (tau * lo) ** 2, 1.0)
    assert abs(yg.mean() - y.mean()) < 1e-14


@pytest.mark.parametrize("dim,n,eps,T", [(2, (64, 64), 0.05, 2e-4), (3, (16, 16, 16), 0.05, 1e-4)])
def test_mixed_adaptive_lim_error_at_T(ch, oracle, dim, n, eps, T):
    """Adaptive LIM (Fig. 3) on a mixed-precision grid: every step whose tau lambda_max allows
    it runs the FP32 increment form; the solution at T agrees with the FP64 oracle's to 1e-5
    and the mass is kept."""
    y0 = inputs.initial_state(n, 4, -0.05, 0.05)
    with ch.Grid(dim, n, eps, ch.CH_MIXED) as G:
        y = dev(y0)
        st = ch.ch_integrate(G.h, ch.make_params("lim", True, T, 1e-8, 1e-6), y)
        yg = host(y)
    rc, yo, to, sto, _ = oracle.integrate(oracle.Grid(dim, n, eps), y0, "lim", True, T, 1e-8, tol=1e-6)
    assert rc == 0 and st["t"] == T
    assert np.linalg.norm(yg - yo) / np.linalg.norm(yo) < 1e-5
    assert abs(yg.mean() - y0.mean()) < 1e-13
