"""Mutation check of the oracle's pins: each case plants one plausible mistake (a sign, an
index, a dropped term or factor, a transposed operand, a wrong coefficient) in a copy of
ch_oracle.c, builds it, and runs the oracle's pin tests against that build through
CH_ORACLE_LIB.  Every mutant must make at least one pin fail; the unmodified copy must
pass them all.  The planted mistakes exist only in temporary copies on the CPU."""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "ch_oracle.c")
PINS = [os.path.join(ROOT, "tests", f) for f in
        ("test_oracle_operators.py", "test_oracle_krylov.py", "test_oracle_lim.py",
         "test_oracle_drivers.py", "test_oracle_neumann.py", "test_oracle_mobility.py",
         "test_oracle_lim_controller.py")]

# (name, original text, planted text): the original must occur exactly once in ch_oracle.c
MUTANTS = [
    ("A: sign of a neighbour", "- v[shift(g, i, a, +1)] - v[shift(g, i, a, -1)]",
     "- v[shift(g, i, a, +1)] + v[shift(g, i, a, -1)]"),
    ("A: neighbour offset", "- v[shift(g, i, a, -1)]);", "- v[shift(g, i, a, -2)]);"),
    ("F': dropped linear term", "return c * (c * c - 1.0);", "return c * c * c;"),
    ("J: sign of the identity", "return 3.0 * y * y - 1.0;", "return 3.0 * y * y + 1.0;"),
    ("f: eps instead of eps^2", "mu[i] = Fp(y[i]) + g->eps * g->eps * Ay[i];",
     "mu[i] = Fp(y[i]) + g->eps * Ay[i];"),
    ("g_hat: Eyre term dropped", "if (g->eyre) t[i] += yn[i];", "if (g->eyre) t[i] += 0.0;"),
    ("A_hat: Eyre term sign", "if (g->eyre) t[i] += v[i];", "if (g->eyre) t[i] -= v[i];"),
    ("lambda_max: |d_j| in the column", "dj * Me[k].val", "fabs(dj) * Me[k].val"),
    ("Eq. p: sqrt dropped", "atan(sqrt(tau * lambda_max))", "atan(tau * lambda_max)"),
    ("Fig. 1: sign of beta_m in a_m", "(z1 - beta[m - 1])", "(z1 + beta[m - 1])"),
    ("Fig. 1: y^n for y^(prev)", "tau * am * prev[i] +", "tau * am * yn[i] +"),
    ("Fig. 1: second sweep from m = 1", "(sweep == 0 ? 0 : 1)", "(sweep == 0 ? 0 : 0)"),
    ("Pade: coefficient denominator", "((double)(2 * m - k + 1) * k)", "((double)(2 * m - k) * k)"),
    ("expm: one squaring short", "for (int k = 0; k < sq; ++k) { mat_mul",
     "for (int k = 1; k < sq; ++k) { mat_mul"),
    ("phi: augmented column not scaled", "M[0 * n + j] = s;", "M[0 * n + j] = 1.0;"),
    ("phi: transposed H", "M[r * n + c] = -s * H[r * ldh + c];", "M[r * n + c] = -s * H[c * ldh + r];"),
    ("Fig. 2: v_1 sign", "V[i] = g[i] - w[i];", "V[i] = g[i] + w[i];"),
    ("Fig. 2: residual entry index", "return hnext * fabs(u[j - 1]);", "return hnext * fabs(u[0]);"),
    ("Fig. 2: subdiagonal not stored", "H[j * ldh + (j - 1)] = hnext;", "H[j * ldh + (j - 1)] = 0.0;"),
    ("Fig. 2: beta dropped in the combine", "* (beta * u[c]);", "* (u[c]);"),
    ("Fig. 2: trace quarters instead of halving", "hi = lo; lo = 0.5 * lo;", "hi = lo; lo = 0.25 * lo;"),
    ("Eq. tol_phi: factor 10 dropped", "norm_ghat / (10.0 * beta)", "norm_ghat / beta"),
    ("Eq. LIMest: full step in the corrector", "ypc[i] = yn[i] - 0.5 * tau * Asum[i];",
     "ypc[i] = yn[i] - tau * Asum[i];"),
    ("Eq. EEdt: square root dropped", "sqrt(prm->tol / est) * taken", "(prm->tol / est) * taken"),
    ("Eq. LIMdt: square root added", "? (prm->tol / est) * taken : taken;",
     "? sqrt(prm->tol / est) * taken : taken;"),
    ("Eq. LIMest: F'(y^n) twice in the corrector", "t[i] = Fp(yn[i]) + Fp(ynp1[i]) + g->eps * g->eps * Asum[i];",
     "t[i] = Fp(yn[i]) + Fp(yn[i]) + g->eps * g->eps * Asum[i];"),
    ("Eq. LIMest: y^n twice in the eps^2 A sum", "sum[i] = yn[i] + ynp1[i];", "sum[i] = yn[i] + yn[i];"),
    ("Fig. 3: next step scaled from tau0", "? (prm->tol / est) * taken : taken;",
     "? (prm->tol / est) * prm->tau0 : taken;"),
    ("Fig. 3: no clip to T", "if (t + tau > prm->T) { tau = prm->T - t; clipped = 1; }",
     "if (0) { tau = prm->T - t; clipped = 1; }"),
    ("energy: gradient term doubled", "0.5 * g->eps * g->eps * sG", "g->eps * g->eps * sG"),
    ("mass: cell volume dropped", "return vol * s;", "return s;"),
    ("Neumann: vertex-centred mirror at the low face", "if (i < 0) return -i - 1;",
     "if (i < 0) return -i;"),
    ("Neumann: vertex-centred mirror at the high face", "if (i >= n) return 2 * n - i - 1;",
     "if (i >= n) return 2 * n - i - 2;"),
    ("mobility: upwind face value instead of the mean",
     "0.5 * (M[i] + M[ip]) * (v[i] - v[ip])", "M[ip] * (v[i] - v[ip])"),
    ("mobility: one-sided face value in the column sums", "double mf = 0.5 * (M[c] + M[nb]);",
     "double mf = M[c];"),
    ("mobility: plain A in the estimate's outer product", "    or_apply_AM(g, t, Asum);",
     "    or_apply_A(g, t, Asum);"),
    ("mobility: plain A as the outer operator of A_hat", "    or_apply_AM(g, t, w);",
     "    or_apply_A(g, t, w);"),
    ("Neumann: periodic wrap kept", "i[a] = g->bc ? mirror(i[a] + off, g->n[a]) : wrap(i[a] + off, g->n[a]);",
     "i[a] = wrap(i[a] + off, g->n[a]);"),
]


def _build(dirpath, name, text):
    c = os.path.join(dirpath, f"{name}.c")
    so = os.path.join(dirpath, f"{name}.so")
    with open(c, "w") as fh:
        fh.write(text)
    subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-fno-fast-math",
                           "-ffp-contract=off", "-o", so, c, "-lm"])
    return so


def _run_pins(so, first_failure):
    env = dict(os.environ, CH_ORACLE_LIB=so)
    args = [sys.executable, "-m", "pytest", "-q", "-m", "not gpu", "-p", "no:cacheprovider"]
    if first_failure:
        args.append("-x")
    r = subprocess.run(args + PINS, cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    return r.returncode, r.stdout[-2000:]


@pytest.fixture(scope="module")
def source():
    return open(SRC).read()


@pytest.fixture(scope="module")
def outcomes(source, tmp_path_factory):
    """Build every copy and run the pins on each, a few copies at a time."""
    d = str(tmp_path_factory.mktemp("mutants"))
    jobs = [("control", source, False)]
    jobs += [(name, source.replace(orig, planted), True) for name, orig, planted in MUTANTS
             if source.count(orig) == 1]

    def run(k):
        key, text, first = jobs[k]
        return key, _run_pins(_build(d, f"copy{k}", text), first)

    workers = max(1, min(6, (os.cpu_count() or 2) // 2))
    with ThreadPoolExecutor(workers) as ex:
        return dict(ex.map(run, range(len(jobs))))


def test_unmodified_copy_passes_every_pin(outcomes):
    rc, out = outcomes["control"]
    assert rc == 0, out


@pytest.mark.parametrize("name,orig,planted", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_every_planted_mistake_fails_a_pin(source, outcomes, name, orig, planted):
    assert source.count(orig) == 1, f"mutation site not unique or gone: {orig!r}"
    rc, out = outcomes[name]
    assert rc == 1, f"{name}: no pin failed (pytest exit {rc})\n{out}"
