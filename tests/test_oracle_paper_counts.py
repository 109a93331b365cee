"""The oracle's EE2 on the paper's own test setting against the matvec counts printed in
Tables 1-3 (rows in tests/golden/paper_ee2_counts.txt).  The rows run concurrently (the
oracle's C routines keep no global state and ctypes releases the GIL during them)."""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

from paper_2502_14589_gb300 import inputs

EPS4 = 4 / (2 * np.sqrt(2) * np.arctanh(0.9))       # Eq. (eps), h = 1, m = 4


def _rows():
    path = os.path.join(os.path.dirname(__file__), "golden", "paper_ee2_counts.txt")
    rows = []
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        f = line.split()
        rows.append((f[0], int(f[1]), f[2], float(f[3]), float(f[4]), int(f[5]), int(f[6]),
                     int(f[7]), float(f[8])))
    return rows


ROWS = _rows()


def _run(oracle, row):
    src, n, mode, tau, tol, mmax, eyre, printed, rtol = row
    # the unit square: x' = x/64, t' = t/64^2, eps' = eps/64 keep tau*lambda_max and the
    # relative Krylov residual of Eq. (phi_stop) unchanged
    g = oracle.Grid(2, (n, n), EPS4 / 64, eyre=bool(eyre), bc="neumann")
    y0 = inputs.initial_state((n, n), 0, -0.01, 0.01)
    rc, y, t, st, rec = oracle.integrate(g, y0, "ee2", mode == "adaptive", 1000 / 64 ** 2,
                                         tau / 64 ** 2, tol=tol, mmax=mmax, max_rec=1)
    return rc, st


@pytest.fixture(scope="module")
def runs(oracle):
    with ThreadPoolExecutor(min(len(ROWS), max(1, os.cpu_count() or 1))) as ex:
        return dict(zip(range(len(ROWS)), ex.map(lambda r: _run(oracle, r), ROWS)))


@pytest.mark.parametrize("k", range(len(ROWS)),
                         ids=[f"{r[0]}-n{r[1]}-{r[2]}-tau{r[3]}-tol{r[4]}-m{r[5]}-eyre{r[6]}" for r in ROWS])
def test_ee2_matvecs_printed_in_the_paper(runs, k):
    src, n, mode, tau, tol, mmax, eyre, printed, rtol = ROWS[k]
    rc, st = runs[k]
    assert rc == 0
    if mode == "const":
        assert st["steps"] == int(round(1000 / tau))
    arnoldi = st["matvecs"] - st["steps"] - st["restarts"]
    assert abs(arnoldi - printed) <= rtol * printed, (arnoldi, printed)
