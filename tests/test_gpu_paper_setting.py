"""The paper's own experiments (Sec. 5) run whole on the GPU and compared with the oracle:
the cell-centred homogeneous Neumann grid of Eq. (CH) on (0,64)^2 (mapped to the unit
square by x' = x/64, t' = t/64^2, eps' = eps/64), eps = eps_4 of Eq. (eps), T = 1000, a
U(-0.01, 0.01) start.

* Table 1's EE2(m_max = 100) with constant steps and linear residual-time restarting;
* the same with m_max = 10, where runs stop at m_max and restart within a step;
* Table 2's Eyre-stabilised EE2(30) (Eq. A_g_cs), constant steps;
* Table 3's adaptive EE2(30) (Fig. 4, tau_0 = 1).

Each run is compared with the oracle's run of the same setting: the step-by-step records
(Krylov dimension at exit, restarts, step cuts) up to their first difference, which must
not come before step 100; the total matvec count; the solution at T; and the count printed
in the paper within the seed spread of tests/golden/paper_ee2_counts.txt.  GPU and oracle
sum in different orders, and over thousands of steps with the paper's loose tolerances
(tol = 1e-2) the states drift apart far enough for a Krylov exit to fall on the other side
of resnorm <= tol_phi once (seen: step 196 of 2000 in the Eyre run, step ~100s of the
adaptive run), after which the runs follow different but equally admissible step
sequences.  Totals are then held to 1 % of the oracle's, the solution at T to 10 tol for
tol >= 1e-2 runs and to 1e-8 for the tol = 1e-6 runs.
"""
import numpy as np
import pytest

from paper_2502_14589_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

EPS4 = 4 / (2 * np.sqrt(2) * np.arctanh(0.9))       # Eq. (eps), h = 1, m = 4


@pytest.fixture(scope="module")
def ch():
    from paper_2502_14589_gb300 import build, ch as chmod
    build.build()
    chmod.load()
    return chmod


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300)


# (label, n, mode, tau(_0), tol, m_max, eyre, printed or None, rel spread of the printed count)
RUNS = [("Table1-EE2(100)", 64, "const", 0.25, 1e-6, 100, 0, 39138, 0.03),
        ("EE2(10)-restarts", 64, "const", 0.25, 1e-6, 10, 0, None, 0.0),
        ("Table2-Eyre-EE2(30)", 64, "const", 0.5, 1e-2, 30, 1, 13776, 0.01),
        ("Table3-adaptive-EE2(30)", 128, "adaptive", 1.0, 1e-2, 30, 0, 22800, 0.03)]


@pytest.mark.parametrize("run", RUNS, ids=[r[0] for r in RUNS])
def test_paper_ee2_runs_against_the_oracle(ch, oracle, run):
    label, n, mode, tau, tol, mmax, eyre, printed, spread = run
    y0 = inputs.initial_state((n, n), 0, -0.01, 0.01)
    T, tau_u = 1000 / 64 ** 2, tau / 64 ** 2
    cap = 100000
    with ch.Grid(2, (n, n), EPS4 / 64, mmax_capacity=mmax, bc="neumann") as G:
        ch.ch_set_record_capacity(G.h, cap)
        y = torch.from_numpy(y0).cuda()
        st = ch.ch_integrate(G.h, ch.make_params("ee2", mode == "adaptive", T, tau_u, tol, mmax, eyre=bool(eyre)), y)
        rec = ch.ch_get_records(G.h, cap)
        yg = y.cpu().numpy()
    og = oracle.Grid(2, (n, n), EPS4 / 64, eyre=bool(eyre), bc="neumann")
    rc, yo, to, sto, reco = oracle.integrate(og, y0, "ee2", mode == "adaptive", T, tau_u, tol=tol, mmax=mmax,
                                             max_rec=cap)
    assert rc == 0 and st["t"] == T
    if mode == "const":
        assert st["steps"] == sto["steps"] == int(round(1000 / tau))
    k = min(len(rec["jexit"]), len(reco["jexit"]))
    same = ((rec["jexit"][:k] == reco["jexit"][:k]) & (rec["restarts"][:k] == reco["restarts"][:k])
            & (rec["shrunk"][:k] == reco["shrunk"][:k]))
    first = k if same.all() else int(np.argmin(same))
    print(f"{label}: records identical for {first} of {k} steps; matvecs {st['matvecs']} vs {sto['matvecs']}; "
          f"rel at T {rel(yg, yo):.2e}")
    assert first >= min(k, 100)
    assert abs(st["matvecs"] - sto["matvecs"]) <= 1e-2 * sto["matvecs"]
    if label.startswith("EE2(10)"):
        assert sto["restarts"] > 0 and st["restarts"] > 0     # linear restarts were exercised
    assert rel(yg, yo) < (1e-8 if tol <= 1e-6 else 10 * tol)
    if printed is not None:          # Arnoldi products as the paper counts them (start vectors left out)
        arnoldi = st["matvecs"] - st["steps"] - st["restarts"]
        assert abs(arnoldi - printed) <= spread * printed, (arnoldi, printed)
