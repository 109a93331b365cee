"""GPU-vs-oracle parity of the paper's own boundary conditions and of the variable-mobility
form, through the C ABI, element by element on the same seeded inputs.

* Homogeneous Neumann conditions on cell-centred nodes (Eq. CH, Sec. 5.1): every call of
  the FP64 path at 1e-12 per kernel and per step, identical step sequences, the spectral
  bound of Fig. 1 from explicitly formed columns (boundary columns included), and the LIM
  matvec counts printed in Tables 1 and 2 reproduced by whole constant-step runs on the GPU.
* Variable mobility (the Remark on Eq. CHmob): A_M(y^n) as the outer operator with face
  mobilities (M_i + M_j)/2, on periodic and Neumann grids, with M frozen per step.
* Mixed precision on both forms: error within the FP32 bound, mass kept to FP64 rounding.
"""
import os

import numpy as np
import pytest

from paper_2502_14589_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def rel(a, b):
    a = np.asarray(a); b = np.asarray(b)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.fixture(scope="module")
def ch():
    from paper_2502_14589_gb300 import build, ch as chmod
    build.build()
    chmod.load()
    assert torch.cuda.is_available()
    return chmod


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def mobility_of(y):
    """The degenerate mobility M(c) = 1 - c^2 of the Remark on Eq. (CHmob), at the nodes,
    taken as 0 where |c| > 1 (M >= 0 keeps A_M positive semidefinite)."""
    return np.maximum(1.0 - np.asarray(y) ** 2, 0.0)


NGRIDS = [(2, (64, 64)), (2, (37, 53)), (3, (16, 16, 16)), (3, (5, 7, 9)), (2, (4, 6))]
# (bc, mobility) forms beyond the periodic constant-mobility one
FORMS = [("neumann", False), ("periodic", True), ("neumann", True)]


def grids(ch, oracle, dim, n, eps, bc, mob, y_lin, eyre=False, precision=None, mmax=30):
    M = mobility_of(y_lin) if mob else None
    og = oracle.Grid(dim, n, eps, eyre=eyre, bc=bc, mobility=M)
    G = ch.Grid(dim, n, eps, ch.CH_FP64 if precision is None else precision, mmax, bc=bc,
                variable_mobility=mob)
    if mob:
        ch.ch_set_mobility(G.h, dev(M))
    return G, og


@pytest.mark.parametrize("bc,mob", FORMS)
@pytest.mark.parametrize("dim,n", NGRIDS)
def test_rhs_jacvec_norms(ch, oracle, dim, n, bc, mob):
    eps = 0.03
    y = inputs.initial_state(n, 1, -0.6, 0.6)
    v = inputs.initial_state(n, 3, -1.0, 1.0)
    G, og = grids(ch, oracle, dim, n, eps, bc, mob, y)
    with G:
        f = torch.empty(G.N, dtype=torch.float64, device="cuda")
        nf, ng = ch.ch_rhs(G.h, dev(y), f, 0, want_norms=True)
        fo = oracle.rhs(og, y)
        assert rel(host(f), fo) < 1e-12
        assert abs(nf - np.linalg.norm(fo)) <= 1e-12 * np.linalg.norm(fo)
        gh = oracle.ghat(og, y)
        assert abs(ng - np.linalg.norm(gh)) <= 1e-12 * np.linalg.norm(gh)
        for eyre in (0, 1):
            w = torch.empty(G.N, dtype=torch.float64, device="cuda")
            ch.ch_jacvec(G.h, dev(y), dev(v), w, eyre)
            oge = oracle.Grid(dim, n, eps, eyre=bool(eyre), bc=bc, mobility=mobility_of(y) if mob else None)
            assert rel(host(w), oracle.jacvec(oge, y, v)) < 1e-12


@pytest.mark.parametrize("bc,mob", FORMS)
@pytest.mark.parametrize("dim,n", NGRIDS)
@pytest.mark.parametrize("eyre", [0, 1])
def test_lambda_max_by_explicit_columns(ch, oracle, dim, n, bc, mob, eyre):
    """Fig. 1's ||A_hat||_1 over every column, boundary columns included."""
    eps = 0.02
    y = inputs.initial_state(n, 4, -1.0, 1.0)
    G, og = grids(ch, oracle, dim, n, eps, bc, mob, y, eyre=bool(eyre))
    with G:
        lm = ch.ch_lambda_max(G.h, dev(y), eyre)
    ref = oracle.lambda_max(og, y)
    assert abs(lm - ref) <= 1e-13 * ref


@pytest.mark.parametrize("bc,mob", FORMS)
@pytest.mark.parametrize("dim,n", [(2, (64, 64)), (3, (12, 10, 14))])
def test_estimate_energy_mass(ch, oracle, dim, n, bc, mob):
    eps = 0.05
    y0 = inputs.initial_state(n, 5, -0.3, 0.3, mean=0.1)
    G, og = grids(ch, oracle, dim, n, eps, bc, mob, y0)
    y1, *_ = oracle.lim_step(og, y0, 1e-6)
    with G:
        est = ch.ch_estimate(G.h, dev(y0), dev(y1), 1e-6)
        e, m = ch.ch_energy_mass(G.h, dev(y1))
    assert abs(est - oracle.estimate(og, y0, y1, 1e-6)) <= 1e-11 * est
    assert abs(e - oracle.energy(og, y1)) <= 1e-13 * abs(e)
    assert abs(m - oracle.mass(og, y1)) <= 1e-13


@pytest.mark.parametrize("bc,mob", FORMS)
@pytest.mark.parametrize("dim,n,tau,eyre", [(2, (64, 64), 3e-5, 0), (2, (50, 70), 1e-4, 1),
                                            (3, (14, 12, 10), 2e-5, 0)])
def test_lim_step(ch, oracle, dim, n, tau, eyre, bc, mob):
    eps = 0.05
    y = inputs.initial_state(n, 8, -0.05, 0.05)
    G, og = grids(ch, oracle, dim, n, eps, bc, mob, y, eyre=bool(eyre))
    with G:
        yn = torch.empty(G.N, dtype=torch.float64, device="cuda")
        p, lm = ch.ch_lim_step(G.h, dev(y), tau, yn, eyre)
        yg = host(yn)
    yo, po, lo, _ = oracle.lim_step(og, y, tau)
    assert p == po and abs(lm - lo) <= 1e-13 * lo
    assert rel(yg, yo) < 1e-12


@pytest.mark.parametrize("bc,mob", FORMS)
@pytest.mark.parametrize("dim,n,tau,mmax,lin", [(2, (64, 64), 1e-6, 30, 0), (2, (48, 40), 2e-5, 6, 0),
                                                (3, (12, 12, 12), 1e-5, 30, 0), (2, (40, 44), 2e-5, 5, 1),
                                                (3, (10, 9, 11), 3e-5, 8, 1)])
def test_phi_krylov(ch, oracle, dim, n, tau, mmax, lin, bc, mob):
    """Fig. 2: nonlinear residual-time step choice (the step may be cut) and linear
    restarting over the whole step."""
    eps, tol_phi = 0.05, 1e-8
    y = inputs.initial_state(n, 6, -0.05, 0.05)
    G, og = grids(ch, oracle, dim, n, eps, bc, mob, y)
    with G:
        yn = torch.empty(G.N, dtype=torch.float64, device="cuda")
        tu, st = ch.ch_phi_krylov(G.h, dev(y), tau, tol_phi, mmax, lin, yn)
        yg = host(yn)
    rc, yo, to, jo, sto = oracle.ee_step(og, y, tau, tol_phi_fixed=tol_phi, mmax=mmax, linear_restart=bool(lin))
    assert rc == 0
    assert tu == pytest.approx(to, rel=1e-12, abs=0)
    assert st["matvecs"] == sto["matvecs"] and st["restarts"] == sto["restarts"]
    assert rel(yg, yo) < 1e-12


@pytest.mark.parametrize("bc,mob", FORMS)
@pytest.mark.parametrize("scheme", ["ee2", "lim"])
def test_adaptive_integration(ch, oracle, scheme, bc, mob):
    """Figs. 3/4 with the mobility frozen at y^0 for the run: identical step sequence and
    the same solution at T."""
    dim, n, eps, T = 2, (48, 40), 0.03, 2e-4
    y0 = inputs.initial_state(n, 3, -0.05, 0.05)
    G, og = grids(ch, oracle, dim, n, eps, bc, mob, y0)
    cap = 100000
    with G:
        ch.ch_set_record_capacity(G.h, cap)
        y = dev(y0)
        st = ch.ch_integrate(G.h, ch.make_params(scheme, True, T, 1e-7, 1e-5, 30), y)
        rec = ch.ch_get_records(G.h, cap)
        yg = host(y)
    rc, yo, to, sto, reco = oracle.integrate(og, y0, scheme, True, T, 1e-7, tol=1e-5, mmax=30, max_rec=cap)
    assert rc == 0
    assert st["steps"] == sto["steps"] and st["matvecs"] == sto["matvecs"]
    np.testing.assert_array_equal(rec["jexit"], reco["jexit"])
    np.testing.assert_array_equal(rec["p"], reco["p"])
    # LIM's tau_new = (tol/est) tau carries est's rounding (a difference of nearly equal
    # vectors) into every later step: over ~200 steps it reaches ~1e-9 relative
    np.testing.assert_allclose(rec["tau"][:-1], reco["tau"][:-1], rtol=1e-8)
    assert rel(yg, yo) < 1e-10


@pytest.mark.parametrize("bc", ["periodic", "neumann"])
def test_mobility_refrozen_every_step(ch, oracle, bc):
    """The Remark on Eq. (CHmob) freezes A_M at y^n: ten EE2 steps and ten LIM steps with
    M = 1 - (y^n)^2 set before each step, each step against the oracle's step from the
    oracle's own previous state."""
    dim, n, eps, tau = 2, (40, 36), 0.04, 2e-5
    y0 = inputs.initial_state(n, 9, -0.5, 0.5)
    prm = None
    with ch.Grid(dim, n, eps, bc=bc, variable_mobility=True) as G:
        prm = ch.make_params("ee2", False, tau, tau, 1e-6, 30, tol_phi=1e-8)
        for scheme in ("ee2", "lim"):
            yg = dev(y0); yo = y0.copy()
            nxt = torch.empty_like(yg)
            for k in range(10):
                ch.ch_set_mobility(G.h, dev(mobility_of(host(yg))))
                og = oracle.Grid(dim, n, eps, bc=bc, mobility=mobility_of(yo))
                if scheme == "ee2":
                    ch.ch_ee_step(G.h, yg, tau, prm, nxt)
                    rc, yo_next, *_ = oracle.ee_step(og, yo, tau, tol_phi_fixed=1e-8, mmax=30, linear_restart=True)
                    assert rc == 0
                else:
                    ch.ch_lim_step(G.h, yg, tau, nxt)
                    yo_next, *_ = oracle.lim_step(og, yo, tau)
                yg.copy_(nxt); yo = yo_next
                assert rel(host(yg), yo) < 1e-11, (scheme, k)
            assert abs(host(yg).mean() - y0.mean()) < 1e-14


@pytest.mark.parametrize("bc,mob", FORMS)
def test_mixed_precision_forms(ch, oracle, bc, mob):
    """Mixed precision (FP32 basis and stages) on these operators: the run reaches T with
    relative error <= 1e-5 against the FP64 oracle, and the mass is kept."""
    dim, n, eps, T = 2, (64, 48), 0.03, 2e-5
    y0 = inputs.initial_state(n, 2, -0.05, 0.05)
    G, og = grids(ch, oracle, dim, n, eps, bc, mob, y0, precision=ch.CH_MIXED)
    with G:
        y = dev(y0)
        st = ch.ch_integrate(G.h, ch.make_params("ee2", True, T, 1e-7, 1e-5, 30), y)
        yg = host(y)
    rc, yo, *_ = oracle.integrate(og, y0, "ee2", True, T, 1e-7, tol=1e-5, mmax=30)
    assert rc == 0 and st["t"] == T
    assert rel(yg, yo) < 1e-5
    assert abs(yg.mean() - y0.mean()) < 1e-13


def _golden_counts():
    path = os.path.join(os.path.dirname(__file__), "golden", "paper_lim_counts.txt")
    rows = []
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        f = line.split()
        rows.append((int(f[0]), float(f[1]), int(f[2]), int(f[3]), f[4]))
    return rows


# The exact rows of Tables 1 and 2 with at most 16000 steps (each run is whole on the GPU)
GPU_ROWS = [r for r in _golden_counts() if r[4] == "exact" and 1000 / r[1] <= 16000]


@pytest.mark.parametrize("row", GPU_ROWS, ids=lambda r: f"n{r[0]}-tau{r[1]}-eyre{r[2]}")
def test_papers_lim_counts_on_the_gpu(ch, oracle, row):
    """Tables 1 and 2 (LIM columns): constant-step LIM over the paper's whole run, on the
    paper's Neumann grid (0,64)^2 with cell-centred nodes mapped to the unit square by
    x' = x/64, t' = t/64^2, eps' = eps/64, from a U(-0.01, 0.01) start (Sec. 5.1).  The
    GPU's own matvec count must equal the printed one."""
    n, tau, eyre, printed, kind = row
    eps4 = 4 / (2 * np.sqrt(2) * np.arctanh(0.9))            # Eq. (eps), h = 1, m = 4
    y0 = inputs.initial_state((n, n), 0, -0.01, 0.01)
    with ch.Grid(2, (n, n), eps4 / 64, bc="neumann") as G:
        y = dev(y0)
        T = 1000 / 64 ** 2
        st = ch.ch_integrate(G.h, ch.make_params("lim", False, T, tau / 64 ** 2, 1e-6, 30, eyre=bool(eyre)), y)
        yg = host(y)
    assert st["steps"] == int(round(1000 / tau))
    assert st["matvecs"] == printed
    assert np.all(np.isfinite(yg)) and abs(yg.mean() - y0.mean()) < 1e-12
    if n == 64 and tau == 0.5 and not eyre:          # the whole run against the oracle too
        rc, yo, *_ = oracle.integrate(oracle.Grid(2, (n, n), eps4 / 64, bc="neumann"), y0, "lim", False,
                                      T, tau / 64 ** 2)
        assert rc == 0 and rel(yg, yo) < 1e-9
