"""Batched adaptive EE2 (many independent instances of uneven size and eps in one launch
sequence) against the oracle run of every instance on its own."""
import numpy as np
import pytest

from paper_2502_14589_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ch():
    from paper_2502_14589_gb300 import build, ch as chmod
    build.build()
    chmod.load()
    return chmod


def run_batch(ch, dim, sizes, eps, y0s, precision, T, tol=1e-5, tau0=1e-7, mmax=30):
    h = ch.ch_create_batch(dim, sizes, eps, precision, mmax)
    try:
        offs, chunk = ch.ch_batch_layout(h, len(sizes))
        y = torch.zeros(offs[-1], dtype=torch.float64, device="cuda")
        for i, y0 in enumerate(y0s):
            y[offs[i]:offs[i] + y0.size] = torch.from_numpy(y0).cuda()
        st = ch.ch_integrate_batch(h, ch.make_params("ee2", True, T, tau0, tol, mmax), y, len(sizes))
        torch.cuda.synchronize()
        yh = y.cpu().numpy()
        return [yh[offs[i]:offs[i] + y0s[i].size] for i in range(len(sizes))], st, chunk
    finally:
        ch.ch_destroy_batch(h)


def oracle_run(oracle, dim, n, eps, y0, T, tol=1e-5, tau0=1e-7, mmax=30):
    rc, y, t, st, rec = oracle.integrate(oracle.Grid(dim, n, eps), y0, "ee2", True, T, tau0,
                                         tol=tol, mmax=mmax)
    assert rc == 0
    return y, st


def test_fp64_batch_matches_oracle_per_instance(ch, oracle):
    sides = [24, 32, 40, 48, 36, 20]
    eps = [0.02, 0.05, 0.03, 0.04, 0.025, 0.045]
    y0s = [inputs.initial_state((s, s), 10 + i) for i, s in enumerate(sides)]
    T = 3e-5
    ys, st, chunk = run_batch(ch, 2, sides, eps, y0s, ch.CH_FP64, T)
    for i, s in enumerate(sides):
        yo, sto = oracle_run(oracle, 2, (s, s), eps[i], y0s[i], T)
        err = np.linalg.norm(ys[i] - yo) / np.linalg.norm(yo)
        assert st[i]["t"] == T
        assert st[i]["steps"] == sto["steps"], (i, st[i], sto)
        assert st[i]["matvecs"] == sto["matvecs"], (i, st[i], sto)
        assert err < 1e-10, (i, err)


def test_mixed_batch_error_at_T(ch, oracle):
    sides = [32, 64, 48, 96]
    eps = [0.02, 0.04, 0.03, 0.01]
    y0s = [inputs.initial_state((s, s), 20 + i) for i, s in enumerate(sides)]
    T = 3e-5
    ys, st, chunk = run_batch(ch, 2, sides, eps, y0s, ch.CH_MIXED, T, tol=1e-6)
    for i, s in enumerate(sides):
        yo, sto = oracle_run(oracle, 2, (s, s), eps[i], y0s[i], T, tol=1e-6)
        err = np.linalg.norm(ys[i] - yo) / np.linalg.norm(yo)
        print(f"mixed batch instance {i} side {s}: steps {st[i]['steps']} vs {sto['steps']}, error at T {err:.2e}")
        assert st[i]["t"] == T
        assert err < 1e-5
        assert abs(ys[i].mean() - y0s[i].mean()) < 1e-13


@pytest.mark.parametrize("dim,sizes,eps", [
    (2, [(36, 36), (50, 50), (100, 100), (44, 60)], [0.03, 0.02, 0.015, 0.04]),
    (3, [(12, 12, 12), (16, 12, 20), (10, 10, 10)], [0.05, 0.04, 0.06])])
def test_mixed_batch_grouped_and_scalar_rows(ch, oracle, dim, sizes, eps):
    """Instances whose rows hold a multiple of four points take the 16-byte grouped kernels
    (a chunk's last tile ending inside a warp: 36^2 = 1296 points is 1024 + 272); the others
    (50, 10) take the scalar ones, in the same batch.  Each is held to the mixed bound."""
    y0s = [inputs.initial_state(n, 70 + i) for i, n in enumerate(sizes)]
    T = 3e-5 if dim == 2 else 2e-5
    ys, st, chunk = run_batch(ch, dim, [list(n) for n in sizes], eps, y0s, ch.CH_MIXED, T, tol=1e-6)
    for i, n in enumerate(sizes):
        yo, sto = oracle_run(oracle, dim, n, eps[i], y0s[i], T, tol=1e-6)
        err = np.linalg.norm(ys[i] - yo) / np.linalg.norm(yo)
        print(f"mixed batch instance {i} n={n}: steps {st[i]['steps']} vs {sto['steps']}, error at T {err:.2e}")
        assert st[i]["t"] == T
        assert err < 1e-5
        assert abs(ys[i].mean() - y0s[i].mean()) < 1e-13


def test_batch_3d_and_stationary_instance(ch, oracle):
    sides = [12, 16, 10]
    eps = [0.05, 0.04, 0.06]
    y0s = [inputs.initial_state((s, s, s), 30 + i) for i, s in enumerate(sides)]
    y0s[1] = np.full(16 ** 3, 0.25)                   # beta = 0: must stay put
    T = 2e-5
    ys, st, chunk = run_batch(ch, 3, sides, eps, y0s, ch.CH_FP64, T)
    assert np.array_equal(ys[1], y0s[1])
    for i in (0, 2):
        yo, sto = oracle_run(oracle, 3, (sides[i],) * 3, eps[i], y0s[i], T)
        assert st[i]["steps"] == sto["steps"]
        assert np.linalg.norm(ys[i] - yo) / np.linalg.norm(yo) < 1e-10


def test_batch_arguments_are_validated(ch):
    """Invalid run parameters are refused before any work, and the batch stays usable."""
    h = ch.ch_create_batch(2, [16, 24], [0.05, 0.04], ch.CH_FP64, 30)
    try:
        offs, _ = ch.ch_batch_layout(h, 2)
        y = torch.zeros(offs[-1], dtype=torch.float64, device="cuda")
        for i, s in enumerate((16, 24)):
            y[offs[i]:offs[i] + s * s] = torch.from_numpy(inputs.initial_state((s, s), 40 + i)).cuda()
        bad = [ch.make_params("ee2", True, float("inf"), 1e-7, 1e-5),
               ch.make_params("ee2", True, 1e-5, float("nan"), 1e-5),
               ch.make_params("ee2", True, 1e-5, float("inf"), 1e-5),
               ch.make_params("ee2", True, 1e-5, 1e-7, 0.0),
               ch.make_params("ee2", True, 1e-5, 1e-7, 1e-5, mmax=31),
               ch.make_params("lim", True, 1e-5, 1e-7, 1e-5),
               ch.make_params("ee2", False, 1e-5, 1e-7, 1e-5)]
        for prm in bad:
            with pytest.raises(ch.CHError) as e:
                ch.ch_integrate_batch(h, prm, y, 2)
            assert e.value.status == ch.CH_EINVAL
        st = ch.ch_integrate_batch(h, ch.make_params("ee2", True, 2e-6, 1e-7, 1e-5), y, 2)
        assert all(s["t"] == 2e-6 for s in st)
    finally:
        ch.ch_destroy_batch(h)


def _run_with_loop(ch, monkeypatch, host_loop, sizes, eps, y0s, precision, T, max_steps=10 ** 9):
    monkeypatch.setenv("CH_BATCH_HOST_LOOP", "1" if host_loop else "0")
    h = ch.ch_create_batch(2, sizes, eps, precision, 30)
    try:
        offs, _ = ch.ch_batch_layout(h, len(sizes))
        y = torch.zeros(offs[-1], dtype=torch.float64, device="cuda")
        for i, y0 in enumerate(y0s):
            y[offs[i]:offs[i] + y0.size] = torch.from_numpy(y0).cuda()
        l0 = ch.ch_batch_kernel_launches(h)
        status = ch.CH_OK
        try:
            st = ch.ch_integrate_batch(h, ch.make_params("ee2", True, T, 1e-7, 1e-5, 30, max_steps=max_steps),
                                       y, len(sizes))
        except ch.CHError as e:
            status, st = e.status, None
        torch.cuda.synchronize()
        yh = y.cpu().numpy()
        return [yh[offs[i]:offs[i] + y0s[i].size] for i in range(len(sizes))], st, status, \
            ch.ch_batch_kernel_launches(h) - l0
    finally:
        ch.ch_destroy_batch(h)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_device_driven_run_equals_host_driven_loop(ch, monkeypatch, precision):
    """The whole run as one graph launch (conditional while over steps, conditional nodes
    over Arnoldi iterations) gives bit for bit the same states and counters as the loop in
    which the host reads a device flag after every iteration."""
    sides = [24, 40, 64, 32]
    eps = [0.02, 0.04, 0.03, 0.05]
    y0s = [inputs.initial_state((s, s), 50 + i) for i, s in enumerate(sides)]
    prec = ch.CH_FP64 if precision == "fp64" else ch.CH_MIXED
    yd, sd, rcd, ld = _run_with_loop(ch, monkeypatch, False, sides, eps, y0s, prec, 2e-5)
    yh, sh, rch, lh = _run_with_loop(ch, monkeypatch, True, sides, eps, y0s, prec, 2e-5)
    assert rcd == rch == ch.CH_OK
    for i in range(len(sides)):
        assert np.array_equal(yd[i], yh[i]), i
        for k in ("steps", "matvecs", "krylov_iters", "tau_shrinks", "t", "tau_next"):
            assert sd[i][k] == sh[i][k], (i, k)
    assert ld > 0 and lh > 0


def test_device_driven_run_stops_at_max_steps(ch, monkeypatch):
    """max_steps batch steps are taken exactly (also an odd number: the graph's loop body
    holds two steps), the run reports CH_ENOTCONV and y holds the state reached, equal to
    the host-driven loop's."""
    sides = [32, 48]
    eps = [0.02, 0.03]
    y0s = [inputs.initial_state((s, s), 60 + i) for i, s in enumerate(sides)]
    yd, _, rcd, _ = _run_with_loop(ch, monkeypatch, False, sides, eps, y0s, ch.CH_MIXED, 1e-3, max_steps=7)
    yh, _, rch, _ = _run_with_loop(ch, monkeypatch, True, sides, eps, y0s, ch.CH_MIXED, 1e-3, max_steps=7)
    assert rcd == rch == ch.CH_ENOTCONV
    for a, b in zip(yd, yh):
        assert np.array_equal(a, b)


def _group_batch():
    """18 soft instances and 2 stiff ones (stiffness estimate 20x larger): two groups.  No
    instance exceeds 1024 points, so every chunk length the creation-time tuner may pick gives
    one chunk per instance and the same reduction order in every run."""
    sides = [16, 20, 24] * 6 + [32, 32]
    eps = [0.01 + 0.0005 * i for i in range(18)] + [0.05, 0.048]
    y0s = [inputs.initial_state((s, s), 80 + i) for i, s in enumerate(sides)]
    return sides, eps, y0s


def test_batch_scheduling_groups_fp64_match_oracle(ch, oracle, monkeypatch):
    """The stiff group runs concurrently with the rest; every instance still follows the
    oracle's step sequence exactly (steps and matvecs) and its state to 1e-10."""
    monkeypatch.setenv("CH_BATCH_GROUPS", "2")
    sides, eps, y0s = _group_batch()
    h = ch.ch_create_batch(2, sides, eps, ch.CH_FP64, 30)
    try:
        assert ch.ch_batch_groups(h) == 2
    finally:
        ch.ch_destroy_batch(h)
    T = 3e-5
    ys, st, chunk = run_batch(ch, 2, sides, eps, y0s, ch.CH_FP64, T)
    for i, s in enumerate(sides):
        yo, sto = oracle_run(oracle, 2, (s, s), eps[i], y0s[i], T)
        err = np.linalg.norm(ys[i] - yo) / np.linalg.norm(yo)
        assert st[i]["t"] == T
        assert st[i]["steps"] == sto["steps"], (i, st[i], sto)
        assert st[i]["matvecs"] == sto["matvecs"], (i, st[i], sto)
        assert err < 1e-10, (i, err)


def test_batch_scheduling_groups_mixed_device_equals_host_loop(ch, monkeypatch):
    """Concurrent groups (device-driven) and the host-driven loop running the groups one
    after the other give bit-identical states and counters; without CH_BATCH_GROUPS=2 the
    batch is one group."""
    monkeypatch.setenv("CH_BATCH_GROUPS", "2")
    sides, eps, y0s = _group_batch()
    yd, sd, rcd, _ = _run_with_loop(ch, monkeypatch, False, sides, eps, y0s, ch.CH_MIXED, 2e-5)
    yh, sh, rch, _ = _run_with_loop(ch, monkeypatch, True, sides, eps, y0s, ch.CH_MIXED, 2e-5)
    assert rcd == rch == 0
    for i in range(len(sides)):
        np.testing.assert_array_equal(yd[i], yh[i])
        assert sd[i]["steps"] == sh[i]["steps"] and sd[i]["matvecs"] == sh[i]["matvecs"]
    monkeypatch.delenv("CH_BATCH_GROUPS")
    h = ch.ch_create_batch(2, sides, eps, ch.CH_MIXED, 30)
    try:
        assert ch.ch_batch_groups(h) == 1
    finally:
        ch.ch_destroy_batch(h)
