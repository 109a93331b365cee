"""GPU-vs-oracle parity of every C-ABI call (FP64 path), element by element on the same
seeded inputs.  Tolerances: 1e-12 relative L2 per kernel and per step, 1e-10 after 100
constant steps, identical step sequences (Krylov j at exit, restarts, step cuts, LIM p)."""
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


GRIDS = [(2, (64, 64)), (2, (37, 53)), (2, (128, 96)), (3, (16, 16, 16)), (3, (5, 7, 9)),
         (3, (24, 20, 33)), (2, (4, 4)), (3, (4, 5, 4))]


@pytest.mark.parametrize("dim,n", GRIDS)
def test_rhs_and_norms(ch, oracle, dim, n):
    eps = 0.03
    y = inputs.initial_state(n, 1, -0.6, 0.6)
    with ch.Grid(dim, n, eps) as G:
        f = torch.empty(G.N, dtype=torch.float64, device="cuda")
        nf, ng = ch.ch_rhs(G.h, dev(y), f, 0, want_norms=True)
        og = oracle.Grid(dim, n, eps)
        fo = oracle.rhs(og, y)
        assert rel(host(f), fo) < 1e-12
        assert abs(nf - np.linalg.norm(fo)) < 1e-12 * np.linalg.norm(fo)
        gh = oracle.ghat(og, y)
        assert abs(ng - np.linalg.norm(gh)) < 1e-12 * np.linalg.norm(gh)


@pytest.mark.parametrize("dim,n", GRIDS)
@pytest.mark.parametrize("eyre", [0, 1])
def test_jacvec(ch, oracle, dim, n, eyre):
    eps = 0.04
    y = inputs.initial_state(n, 2, -0.9, 0.9)
    v = inputs.initial_state(n, 3, -1.0, 1.0)
    with ch.Grid(dim, n, eps) as G:
        w = torch.empty(G.N, dtype=torch.float64, device="cuda")
        ch.ch_jacvec(G.h, dev(y), dev(v), w, eyre)
        wo = oracle.jacvec(oracle.Grid(dim, n, eps, eyre=bool(eyre)), y, v)
        assert rel(host(w), wo) < 1e-12


@pytest.mark.parametrize("dim,n", GRIDS)
@pytest.mark.parametrize("eyre", [0, 1])
def test_lambda_max(ch, oracle, dim, n, eyre):
    eps = 0.02
    y = inputs.initial_state(n, 4, -1.2, 1.2)
    with ch.Grid(dim, n, eps) as G:
        lm = ch.ch_lambda_max(G.h, dev(y), eyre)
    ref = oracle.lambda_max(oracle.Grid(dim, n, eps, eyre=bool(eyre)), y)
    assert abs(lm - ref) <= 1e-13 * ref


@pytest.mark.parametrize("dim,n", [(2, (64, 64)), (3, (12, 10, 14))])
def test_estimate_energy_mass(ch, oracle, dim, n):
    eps = 0.05
    og = oracle.Grid(dim, n, eps)
    y0 = inputs.initial_state(n, 5, -0.3, 0.3, mean=0.1)
    y1, *_ = oracle.lim_step(og, y0, 1e-6)
    with ch.Grid(dim, n, eps) as G:
        est = ch.ch_estimate(G.h, dev(y0), dev(y1), 1e-6)
        e, m = ch.ch_energy_mass(G.h, dev(y1))
    assert abs(est - oracle.estimate(og, y0, y1, 1e-6)) <= 1e-11 * est
    assert abs(e - oracle.energy(og, y1)) <= 1e-13 * abs(e)
    assert abs(m - oracle.mass(og, y1)) <= 1e-13


@pytest.mark.parametrize("dim,n,tau,mmax", [(2, (64, 64), 1e-6, 30), (2, (48, 40), 3e-6, 30),
                                            (3, (12, 12, 12), 1e-5, 30), (2, (64, 64), 2e-5, 6),
                                            (2, (33, 31), 5e-6, 1)])
def test_phi_krylov_nonlinear_rt(ch, oracle, dim, n, tau, mmax):
    """Fig. 2 with the step choice of Eq. (phi_stop): same tau (also when cut) and y_next."""
    eps = 0.05
    y = inputs.initial_state(n, 6, -0.05, 0.05)
    tol_phi = 1e-8
    with ch.Grid(dim, n, eps, mmax_capacity=30) as G:
        yn = torch.empty(G.N, dtype=torch.float64, device="cuda")
        tu, st = ch.ch_phi_krylov(G.h, dev(y), tau, tol_phi, mmax, 0, yn)
    rc, yo, to, jo, sto = oracle.ee_step(oracle.Grid(dim, n, eps), y, tau, tol_phi_fixed=tol_phi,
                                         mmax=mmax, linear_restart=False)
    assert rc == 0
    assert tu == pytest.approx(to, rel=1e-12, abs=0)
    assert st["matvecs"] == sto["matvecs"]
    assert rel(host(yn), yo) < 1e-12


@pytest.mark.parametrize("n,tau,precision", [((40, 52), 4e-4, "fp64"), ((64, 64), 1.5e-4, "fp64"),
                                             ((64, 64), 3e-4, "fp64"), ((64, 64), 1.5e-4, "mixed")])
def test_phi_krylov_beyond_64_dimensions(ch, oracle, n, tau, precision):
    """The EE2(100) configuration of Sec. 5: m_max = 100 (Krylov runs ending at j = 65, 76 and
    at m_max with the step trace), where each dimension's projected phi (n = j + 1 > 64) works
    from global memory on one CTA.  FP64 is element by element; the mixed run (FP32 basis) is
    held to its FP32 bound against the oracle run of the step it took."""
    eps, tol_phi, mmax = 0.05, 1e-8, 100
    y = inputs.initial_state(n, 6, -0.05, 0.05)
    og = oracle.Grid(2, n, eps)
    prec = ch.CH_FP64 if precision == "fp64" else ch.CH_MIXED
    with ch.Grid(2, n, eps, prec, mmax_capacity=mmax) as G:
        yn = torch.empty(G.N, dtype=torch.float64, device="cuda")
        tu, st = ch.ch_phi_krylov(G.h, dev(y), tau, tol_phi, mmax, 0, yn)
        yg = host(yn)
    rc, yo, to, jo, sto = oracle.ee_step(og, y, tu if precision == "mixed" else tau,
                                         tol_phi_fixed=tol_phi, mmax=mmax, linear_restart=False)
    assert rc == 0
    assert st["matvecs"] > 65
    if precision == "fp64":
        assert tu == pytest.approx(to, rel=1e-12, abs=0)
        assert st["matvecs"] == sto["matvecs"]
        assert rel(yg, yo) < 1e-12
    else:
        lmax = oracle.lambda_max(og, y)
        assert np.linalg.norm(yg - yo) / np.linalg.norm(yo - y) < 50 * 2.0 ** -24 * max(tu * lmax, 1.0)
        assert abs(yg.mean() - y.mean()) < 1e-13


@pytest.mark.parametrize("dim,n,tau,mmax", [(2, (64, 64), 1e-6, 30), (2, (40, 44), 2e-5, 5),
                                            (3, (10, 9, 11), 3e-5, 8)])
def test_phi_krylov_linear_restart(ch, oracle, dim, n, tau, mmax):
    eps = 0.05
    y = inputs.initial_state(n, 7, -0.05, 0.05)
    with ch.Grid(dim, n, eps) as G:
        yn = torch.empty(G.N, dtype=torch.float64, device="cuda")
        tu, st = ch.ch_phi_krylov(G.h, dev(y), tau, 1e-8, mmax, 1, yn)
    rc, yo, to, jo, sto = oracle.ee_step(oracle.Grid(dim, n, eps), y, tau, tol_phi_fixed=1e-8,
                                         mmax=mmax, linear_restart=True)
    assert rc == 0 and tu == tau
    assert st["restarts"] == sto["restarts"] and st["matvecs"] == sto["matvecs"]
    assert rel(host(yn), yo) < 1e-12


@pytest.mark.parametrize("dim,n,tau,eyre", [(2, (64, 64), 1e-6, 0), (2, (64, 64), 3e-5, 0),
                                            (2, (50, 70), 1e-4, 1), (3, (14, 12, 10), 2e-5, 0),
                                            (2, (64, 64), 1e-12, 0)])
def test_lim_step(ch, oracle, dim, n, tau, eyre):
    eps = 0.05
    y = inputs.initial_state(n, 8, -0.05, 0.05)
    with ch.Grid(dim, n, eps) as G:
        yn = torch.empty(G.N, dtype=torch.float64, device="cuda")
        p, lm = ch.ch_lim_step(G.h, dev(y), tau, yn, eyre)
    yo, po, lo, mvo = oracle.lim_step(oracle.Grid(dim, n, eps, eyre=bool(eyre)), y, tau)
    assert p == po
    assert abs(lm - lo) <= 1e-13 * lo
    r = rel(host(yn), yo)
    print(f"LIM step n={n} tau={tau} p={p} tau*lmax={tau * lm:.3g} rel={r:.3e}")
    assert r < 1e-12


def _run_both(ch, oracle, dim, n, eps, y0, scheme, adaptive, T, tau0, tol=1e-6, mmax=30,
              tol_phi=-1.0, eyre=False, cap=200000):
    with ch.Grid(dim, n, eps, mmax_capacity=max(mmax, 1)) as G:
        ch.ch_set_record_capacity(G.h, cap)
        y = dev(y0)
        prm = ch.make_params(scheme, adaptive, T, tau0, tol, mmax, tol_phi, eyre)
        st = ch.ch_integrate(G.h, prm, y)
        rec = ch.ch_get_records(G.h, cap)
        yg = host(y)
    rc, yo, to, sto, reco = oracle.integrate(oracle.Grid(dim, n, eps, eyre=eyre), y0, scheme,
                                             adaptive, T, tau0, tol=tol, mmax=mmax, tol_phi=tol_phi,
                                             max_rec=cap)
    assert rc == 0
    return yg, st, rec, yo, sto, reco


@pytest.mark.parametrize("scheme", ["ee2", "lim"])
@pytest.mark.parametrize("seed", [0, 1])
def test_config0_constant_steps(ch, oracle, scheme, seed):
    """2D periodic 64x64, eps 0.05, U[-0.05,0.05] zero-mean, 100 steps of tau = 1e-6;
    EE2 with m_max = 30 and restart residual tolerance 1e-8; LIM with the same tau."""
    wl = inputs.WORKLOADS["c0_2d64_const"]
    y0 = inputs.initial_state((64, 64), seed, wl["lo"], wl["hi"])
    yg, st, rec, yo, sto, reco = _run_both(ch, oracle, 2, (64, 64), wl["eps"], y0, scheme, False,
                                           wl["T"], wl["tau0"], mmax=30, tol_phi=wl["tol_phi"])
    assert st["steps"] == sto["steps"] == 100
    assert st["matvecs"] == sto["matvecs"]
    np.testing.assert_array_equal(rec["jexit"], reco["jexit"])
    np.testing.assert_array_equal(rec["restarts"], reco["restarts"])
    np.testing.assert_array_equal(rec["p"], reco["p"])
    assert rel(yg, yo) < 1e-10


@pytest.mark.parametrize("scheme", ["ee2", "lim"])
@pytest.mark.parametrize("dim,n,eps,T", [(2, (48, 48), 0.02, 2e-4), (3, (12, 12, 12), 0.05, 2e-4)])
def test_adaptive_step_sequence(ch, oracle, scheme, dim, n, eps, T):
    """Figs. 3/4: identical accepted-step sequence and matching solution at T."""
    y0 = inputs.initial_state(n, 3, -0.05, 0.05)
    yg, st, rec, yo, sto, reco = _run_both(ch, oracle, dim, n, eps, y0, scheme, True, T, 1e-7, tol=1e-5)
    assert st["steps"] == sto["steps"]
    assert st["matvecs"] == sto["matvecs"]
    np.testing.assert_array_equal(rec["jexit"], reco["jexit"])
    np.testing.assert_array_equal(rec["shrunk"], reco["shrunk"])
    np.testing.assert_array_equal(rec["p"], reco["p"])
    # Every tau carries the rounding of est (a difference of nearly equal vectors, relative
    # error ~ u/est ~ 1e-11 at tol 1e-5), and LIM's tau_new = (tol/est) tau compounds it over
    # the run; the last step T - t inherits the accumulated absolute difference of t.
    np.testing.assert_allclose(rec["tau"][:-1], reco["tau"][:-1], rtol=1e-9)
    assert abs(rec["tau"][-1] - reco["tau"][-1]) <= 1e-8 * T
    assert abs(st["t"] - T) <= 1e-15 * T
    assert rel(yg, yo) < 1e-10


def test_stationary_state_beta_zero(ch, oracle):
    """beta = 0 at a constant state: y^{n+1} = y^n exactly, tau kept / grown by the controller."""
    n = (32, 32)
    y0 = np.full(32 * 32, 0.3)
    with ch.Grid(2, n, 0.05) as G:
        y = dev(y0)
        yn = torch.empty_like(y)
        tu, st = ch.ch_phi_krylov(G.h, y, 1e-5, 1e-8, 30, 0, yn)
        assert tu == 1e-5
        assert np.array_equal(host(yn), y0)


def test_errors_are_reported(ch):
    with pytest.raises(ch.CHError) as e:
        ch.Grid(2, (3, 64), 0.05)
    assert e.value.status == ch.CH_EINVAL
    with pytest.raises(ch.CHError):
        ch.Grid(2, (64, 64), -1.0)
    with ch.Grid(2, (16, 16), 0.05) as G:
        y = dev(np.full(256, np.nan))
        with pytest.raises(ch.CHError) as e:
            ch.ch_integrate(G.h, ch.make_params("ee2", True, 1e-5, 1e-7, 1e-6), y)
        assert e.value.status == ch.CH_ENONFINITE
        # the grid stays usable after a reported failure
        y = dev(inputs.initial_state((16, 16), 0))
        st = ch.ch_integrate(G.h, ch.make_params("lim", True, 1e-6, 1e-8, 1e-5), y)
        assert st["t"] == 1e-6


def test_binding_checks_vector_lengths(ch):
    """The C functions cannot see the length of a caller's buffer; the binding refuses a
    vector shorter than the grid (or the batch layout) before any launch."""
    z = lambda k: torch.zeros(k, dtype=torch.float64, device="cuda")
    with ch.Grid(2, (16, 16), 0.05) as G:
        y = dev(inputs.initial_state((16, 16), 0))
        with pytest.raises(ValueError):
            ch.ch_rhs(G.h, z(255), z(256))
        with pytest.raises(ValueError):
            ch.ch_jacvec(G.h, y, y, z(100))
        with pytest.raises(ValueError):
            ch.ch_integrate(G.h, ch.make_params("lim", True, 1e-6, 1e-8, 1e-5), z(200))
        f = z(300)                                  # longer buffers are fine
        ch.ch_rhs(G.h, y, f)
        ref = z(256)
        ch.ch_rhs(G.h, y, ref)
        assert torch.equal(f[:256], ref)
    h = ch.ch_create_batch(2, [16, 24], [0.05, 0.04], ch.CH_FP64, 30)
    try:
        offs, _ = ch.ch_batch_layout(h, 2)
        with pytest.raises(ValueError):
            ch.ch_integrate_batch(h, ch.make_params("ee2", True, 1e-6, 1e-7, 1e-5), z(offs[-1] - 1), 2)
    finally:
        ch.ch_destroy_batch(h)
    with pytest.raises(ValueError):
        ch.ch_energy_mass_noalloc(2, (16, 16), 0.05, z(255), z(2))


def test_step_sizes_are_validated(ch):
    """Step sizes that are zero, negative, infinite or NaN are refused before any work, and a
    LIM step from a non-finite state reports the non-finite lambda_max."""
    with ch.Grid(2, (16, 16), 0.05) as G:
        y = dev(inputs.initial_state((16, 16), 0))
        yn = torch.empty_like(y)
        prm = ch.make_params("ee2", True, 1e-5, 1e-7, 1e-6)
        for tau in (0.0, -1e-6, float("inf"), float("nan")):
            for call in (lambda: ch.ch_lim_step(G.h, y, tau, yn),
                         lambda: ch.ch_ee_step(G.h, y, tau, prm, yn),
                         lambda: ch.ch_phi_krylov(G.h, y, tau, 1e-8, 30, 0, yn)):
                with pytest.raises(ch.CHError) as e:
                    call()
                assert e.value.status == ch.CH_EINVAL
        with pytest.raises(ch.CHError) as e:
            ch.ch_lim_step(G.h, dev(np.full(256, np.nan)), 1e-6, yn)
        assert e.value.status == ch.CH_ENONFINITE
        p, _ = ch.ch_lim_step(G.h, y, 1e-6, yn)       # the grid stays usable
        assert p >= 1


@pytest.mark.parametrize("scheme", ["ee2", "lim"])
def test_checkpoint_resume_is_bit_identical(ch, scheme):
    """Stop after k steps (max_steps), read (t, tau_next), resume: same bits as one run."""
    n = (40, 40)
    y0 = inputs.initial_state(n, 9)
    with ch.Grid(2, n, 0.03) as G:
        ya = dev(y0)
        full = ch.ch_integrate(G.h, ch.make_params(scheme, True, 2e-4, 1e-7, 1e-5), ya)
        k = full["steps"] // 2
        yb = dev(y0)
        with pytest.raises(ch.CHError) as e:
            ch.ch_integrate(G.h, ch.make_params(scheme, True, 2e-4, 1e-7, 1e-5, max_steps=k), yb)
        assert e.value.status == ch.CH_ENOTCONV
        t, tau = ch.ch_get_state(G.h)
        assert 0 < t < 2e-4
        ch.ch_set_state(G.h, t, tau)
        rest = ch.ch_integrate(G.h, ch.make_params(scheme, True, 2e-4, 1e-7, 1e-5), yb)
        assert rest["steps"] == full["steps"] - k and rest["t"] == 2e-4
        assert np.array_equal(host(ya), host(yb))


# ---- full-size configuration (2D periodic 1024 x 1024, eps 0.01) -------------------------
@pytest.fixture(scope="module")
def c1():
    wl = inputs.WORKLOADS["c1_2d1024_adaptive"]
    return wl, inputs.initial_state((1024, 1024), 0, wl["lo"], wl["hi"])


def test_full_size_operators(ch, oracle, c1):
    wl, y = c1
    n = (1024, 1024)
    og = oracle.Grid(2, n, wl["eps"])
    with ch.Grid(2, n, wl["eps"]) as G:
        f = torch.empty(G.N, dtype=torch.float64, device="cuda")
        ch.ch_rhs(G.h, dev(y), f)
        assert rel(host(f), oracle.rhs(og, y)) < 1e-12
        v = inputs.initial_state(n, 1, -1, 1)
        ch.ch_jacvec(G.h, dev(y), dev(v), f)
        assert rel(host(f), oracle.jacvec(og, y, v)) < 1e-12
        assert ch.ch_lambda_max(G.h, dev(y)) == pytest.approx(oracle.lambda_max(og, y), rel=1e-13)


def test_full_size_first_steps(ch, oracle, c1):
    """First adaptive EE2 step and a LIM step at tau0 on the full 1024^2 grid."""
    wl, y = c1
    n = (1024, 1024)
    og = oracle.Grid(2, n, wl["eps"])
    with ch.Grid(2, n, wl["eps"]) as G:
        yn = torch.empty(G.N, dtype=torch.float64, device="cuda")
        prm = ch.make_params("ee2", True, wl["T"], wl["tau0"], wl["tol"], 30)
        tu, est = ch.ch_ee_step(G.h, dev(y), wl["tau0"], prm, yn)
        rc, yo, to, jo, sto = oracle.ee_step(og, y, wl["tau0"], tol=wl["tol"], mmax=30)
        assert tu == pytest.approx(to, rel=1e-12)
        assert rel(host(yn), yo) < 1e-12
        assert est == pytest.approx(oracle.estimate(og, y, yo, to), rel=1e-9)
        p, lm = ch.ch_lim_step(G.h, dev(y), wl["tau0"], yn)
        yl, pl, ll, _ = oracle.lim_step(og, y, wl["tau0"])
        assert p == pl
        assert rel(host(yn), yl) < 1e-12


@pytest.mark.parametrize("env", [{"CH_NO_FUSED_ARNOLDI": "1"}, {"CH_NO_GRAPHS": "1"},
                                 {"CH_NO_FUSED_ARNOLDI": "1", "CH_NO_GRAPHS": "1"},
                                 {"CH_ARNOLDI_MGS": "1"}])
@pytest.mark.parametrize("dim,n,tau", [(2, (64, 64), 1e-6), (3, (10, 9, 11), 3e-5)])
def test_launch_variants_match_oracle(ch, oracle, monkeypatch, env, dim, n, tau):
    """Arnoldi iterations as separate kernels, and without CUDA graphs (both read when a grid
    is created), give the same Krylov run as the oracle."""
    for k, v in env.items():
        monkeypatch.setenv(k, v)
    eps = 0.05
    y = inputs.initial_state(n, 6, -0.05, 0.05)
    with ch.Grid(dim, n, eps, mmax_capacity=30) as G:
        yn = torch.empty(G.N, dtype=torch.float64, device="cuda")
        tu, st = ch.ch_phi_krylov(G.h, dev(y), tau, 1e-8, 30, 0, yn)
    rc, yo, to, jo, sto = oracle.ee_step(oracle.Grid(dim, n, eps), y, tau, tol_phi_fixed=1e-8,
                                         mmax=30, linear_restart=False)
    assert rc == 0
    assert tu == pytest.approx(to, rel=1e-12, abs=0)
    assert st["matvecs"] == sto["matvecs"]
    assert rel(host(yn), yo) < 1e-12


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_kernel_bench_classes(ch, precision):
    """Every kernel class the micro-benchmark supports runs and reports its work."""
    prec = ch.CH_FP64 if precision == "fp64" else ch.CH_MIXED
    n = (256, 256)
    with ch.Grid(2, n, 0.02, prec, mmax_capacity=30) as G:
        y = dev(inputs.initial_state(n, 3))
        ch.ch_integrate(G.h, ch.make_params("ee2", True, 1e-6, 1e-7, 1e-6, 30), y)
        classes = ["arnoldi", "tstage", "wstage", "mgs"]
        if precision == "fp64":
            classes += ["resid1", "lim2", "rhs1", "rhs2"]
        for cls in classes:
            kb = ch.ch_bench_kernel(G.h, cls, 5)
            assert kb["avg_us"] > 0 and kb["bytes"] > 0 and kb["flops"] > 0, cls


@pytest.mark.parametrize("dim,n,tau", [
    (2, (1100, 1100), 2e-8),      # 8 elements per thread: largest resident FP64 iteration
    (3, (112, 112, 112), 1e-7),   # beyond it: the streaming iteration kernel
])
def test_arnoldi_kernel_forms_at_size(ch, oracle, dim, n, tau):
    """The resident and the streaming form of the fused Arnoldi iteration against the oracle
    on grids of more than a million points (one Krylov run of Fig. 2 with Eq. phi_stop)."""
    eps = 0.02
    y = inputs.initial_state(n, 9, -0.05, 0.05)
    with ch.Grid(dim, n, eps, mmax_capacity=30) as G:
        yn = torch.empty(G.N, dtype=torch.float64, device="cuda")
        tu, st = ch.ch_phi_krylov(G.h, dev(y), tau, 1e-8, 30, 0, yn)
    rc, yo, to, jo, sto = oracle.ee_step(oracle.Grid(dim, n, eps), y, tau, tol_phi_fixed=1e-8,
                                         mmax=30, linear_restart=False)
    assert rc == 0
    assert tu == pytest.approx(to, rel=1e-12, abs=0)
    assert st["matvecs"] == sto["matvecs"]
    assert rel(host(yn), yo) < 1e-12


@pytest.mark.parametrize("dim,n,tau,mmax,lin", [(2, (64, 64), 1e-5, 30, 0), (3, (12, 12, 12), 3e-5, 30, 0),
                                                (2, (48, 40), 4e-5, 6, 1), (2, (64, 64), 2e-4, 30, 0)])
def test_phi_krylov_eyre(ch, oracle, dim, n, tau, mmax, lin):
    """Eq. (A_g_cs): the Krylov run of Fig. 2 on the Eyre-split A_hat, g_hat (Sec. 4.3),
    with the step choice of Eq. (phi_stop) or linear restarting."""
    eps, tol_phi = 0.05, 1e-8
    y = inputs.initial_state(n, 11, -0.4, 0.4)
    with ch.Grid(dim, n, eps) as G:
        yn = torch.empty(G.N, dtype=torch.float64, device="cuda")
        tu, st = ch.ch_phi_krylov(G.h, dev(y), tau, tol_phi, mmax, lin, yn, eyre=1)
    rc, yo, to, jo, sto = oracle.ee_step(oracle.Grid(dim, n, eps, eyre=True), y, tau, tol_phi_fixed=tol_phi,
                                         mmax=mmax, linear_restart=bool(lin))
    assert rc == 0
    assert tu == pytest.approx(to, rel=1e-12, abs=0)
    assert st["matvecs"] == sto["matvecs"] and st["restarts"] == sto["restarts"]
    assert rel(host(yn), yo) < 1e-12


@pytest.mark.parametrize("adaptive", [False, True])
def test_eyre_ee2_integration(ch, oracle, adaptive):
    """EE2 with the Eyre splitting (Sec. 4.3, the EE2 column of Table 2), constant steps with
    linear restarting and adaptive steps by Fig. 4: identical step sequence and solution."""
    n, eps = (48, 48), 0.03
    y0 = inputs.initial_state(n, 12, -0.05, 0.05)
    if adaptive:
        args = dict(T=2e-4, tau0=1e-7, tol=1e-5)
    else:
        args = dict(T=4e-5, tau0=4e-6, tol=1e-5, tol_phi=1e-8)
    yg, st, rec, yo, sto, reco = _run_both(ch, oracle, 2, n, eps, y0, "ee2", adaptive, args["T"], args["tau0"],
                                           tol=args["tol"], tol_phi=args.get("tol_phi", -1.0), eyre=True)
    assert st["steps"] == sto["steps"] and st["matvecs"] == sto["matvecs"]
    np.testing.assert_array_equal(rec["jexit"], reco["jexit"])
    np.testing.assert_array_equal(rec["restarts"], reco["restarts"])
    np.testing.assert_array_equal(rec["shrunk"], reco["shrunk"])
    assert rel(yg, yo) < 1e-10


def test_ee2_mmax100_constant_steps_with_restarts(ch, oracle):
    """The EE2(m_max = 100) configuration of Table 1 on a periodic grid: constant steps,
    linear residual-time restarting once a run reaches m_max, identical restarts and
    solution (projected phi beyond 64 dimensions works from global memory)."""
    n, eps = (40, 52), 0.05
    y0 = inputs.initial_state(n, 6, -0.05, 0.05)
    yg, st, rec, yo, sto, reco = _run_both(ch, oracle, 2, n, eps, y0, "ee2", False, 1.2e-3, 4e-4, mmax=100,
                                           tol_phi=1e-8)
    assert st["steps"] == sto["steps"] == 3
    assert st["matvecs"] == sto["matvecs"] and max(rec["jexit"]) > 64
    np.testing.assert_array_equal(rec["jexit"], reco["jexit"])
    np.testing.assert_array_equal(rec["restarts"], reco["restarts"])
    assert rel(yg, yo) < 1e-10


@pytest.mark.parametrize("dim,n,tau", [(2, (512, 1024), 3e-8), (2, (256, 192), 2e-6), (3, (64, 64, 64), 1e-6)])
def test_fp64_gram_iteration_against_sequential_passes(ch, oracle, monkeypatch, dim, n, tau):
    """FP64 grids of up to 512K points compute the coefficients of Fig. 2's modified
    Gram-Schmidt through the Gram identity h_kj = c_k - sum_{i<k} G_ki h_ij (three grid
    synchronisations per iteration); larger ones, or CH_ARNOLDI_MGS=1, run the passes one
    by one.  Both forms give the oracle's Krylov run: the same step, the same exit
    dimension and y within 1e-12."""
    eps, tol_phi = 0.01 if dim == 2 else 0.02, 1e-8
    y = inputs.initial_state(n, 6, -0.05, 0.05)
    out = {}
    for mgs in ("0", "1"):
        monkeypatch.setenv("CH_ARNOLDI_MGS", mgs)
        with ch.Grid(dim, n, eps, mmax_capacity=30) as G:
            yn = torch.empty(G.N, dtype=torch.float64, device="cuda")
            tu, st = ch.ch_phi_krylov(G.h, dev(y), tau, tol_phi, 30, 0, yn)
            out[mgs] = (tu, st["matvecs"], host(yn))
    rc, yo, to, jo, sto = oracle.ee_step(oracle.Grid(dim, n, eps), y, tau, tol_phi_fixed=tol_phi, mmax=30,
                                         linear_restart=False)
    assert rc == 0
    for mgs, (tu, mv, yg) in out.items():
        assert tu == pytest.approx(to, rel=1e-12, abs=0), mgs
        assert mv == sto["matvecs"], mgs
        assert rel(yg, yo) < 1e-12, mgs
