"""ctypes binding of the plain FP64 C oracle (ch_oracle.c).

Test infrastructure only: the test suite, ``__graft_entry__.smoke()`` and the CPU
baseline / reference arm of ``bench.py`` are the only callers.  Nothing in the CUDA
library imports this module, and this module imports nothing from the library.

Parity status of each oracle routine (what pins it, see tests/test_oracle_*.py):
  apply_A, rhs, ghat, jacvec   -- Fourier symbols (FFT), dense matrices, finite differences;
                                  Neumann grids: cosine-transform symbols, dense matrices;
                                  variable mobility: dense flux-form matrices
  lambda_max, cheb_order       -- dense ||A_hat||_1 and the LIM matvec counts printed in
                                  Tables 1 and 2 of the paper
  lim_step                     -- p = 1 reduces to explicit Euler; exact implicit-Euler modes
                                  at the Chebyshev nodes; stability on [0, lambda_max]; order 1
  expm, phi_e1                 -- scipy.linalg.expm, eigendecomposition, scalar closed form
  krylov / ee_step             -- dense augmented-matrix exponential of Eq. (yt); Arnoldi
                                  relation; residual identity of Eq. (rm); the EE2 matvec
                                  counts printed in Tables 1-3 (paper's Neumann setting)
  estimate, drivers            -- mass conservation, energy decrease, Fourier linear decay,
                                  convergence orders; adaptive EE2 also by Table 3's work;
                                  the adaptive LIM controller only by its printed formulas
Planted mistakes in copies of ch_oracle.c (tests/test_oracle_mutants.py) each fail a pin.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ch_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ch_oracle.c with gcc -O2 (no fast-math, single thread)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-fno-fast-math",
                               "-ffp-contract=off", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class OrGrid(C.Structure):
    _fields_ = [("dim", C.c_int), ("n", C.c_long * 3), ("eps", C.c_double), ("eyre", C.c_int),
                ("bc", C.c_int), ("mob", C.c_void_p)]


class OrStats(C.Structure):
    _fields_ = [("steps", C.c_long), ("matvecs", C.c_long), ("rhs_evals", C.c_long),
                ("krylov_iters", C.c_long), ("restarts", C.c_long), ("tau_shrinks", C.c_long),
                ("phi_evals", C.c_long), ("status", C.c_int)]


class OrParams(C.Structure):
    _fields_ = [("scheme", C.c_int), ("adaptive", C.c_int), ("T", C.c_double),
                ("tau0", C.c_double), ("tol", C.c_double), ("mmax", C.c_int),
                ("tol_phi", C.c_double), ("max_steps", C.c_long)]


class OrRecords(C.Structure):
    _fields_ = [("tau", C.POINTER(C.c_double)), ("jexit", C.POINTER(C.c_int)),
                ("restarts", C.POINTER(C.c_int)), ("shrunk", C.POINTER(C.c_int)),
                ("p", C.POINTER(C.c_int)), ("est", C.POINTER(C.c_double)),
                ("max_rec", C.c_long)]


_D = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")


def lib():
    """The oracle library.  CH_ORACLE_LIB names another build of ch_oracle.c to load instead
    (the mutation test compiles copies with planted mistakes and runs the pins on them)."""
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(os.environ.get("CH_ORACLE_LIB") or build())
            G = C.POINTER(OrGrid)
            sig = {
                "or_apply_A": (None, [G, _D, _D]),
                "or_rhs": (None, [G, _D, _D]),
                "or_ghat": (None, [G, _D, _D]),
                "or_jacvec": (None, [G, _D, _D, _D]),
                "or_lambda_max": (C.c_double, [G, _D]),
                "or_column_abs_sum": (C.c_double, [G, _D, C.c_long]),
                "or_cheb_order": (C.c_int, [C.c_double, C.c_double]),
                "or_lim_order": (C.c_int, [C.c_int, np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")]),
                "or_lim_step": (C.c_int, [G, _D, C.c_double, _D, C.POINTER(C.c_double),
                                          C.POINTER(C.c_long)]),
                "or_lim_dense": (C.c_int, [C.c_long, _D, _D, _D, C.c_double, C.c_double, _D]),
                "or_expm": (C.c_int, [C.c_int, _D, _D]),
                "or_phi_e1": (C.c_int, [C.c_int, _D, C.c_int, C.c_double, _D]),
                "or_krylov_dense": (C.c_int, [C.c_long, _D, _D, _D, C.c_double, C.c_double,
                                              C.c_int, _D, C.POINTER(C.c_double),
                                              C.POINTER(C.c_int)]),
                "or_arnoldi_dense": (C.c_int, [C.c_long, _D, _D, C.c_int, _D, _D]),
                "or_tol_phi": (C.c_double, [C.c_double, C.c_double, C.c_double]),
                "or_ee_step": (C.c_int, [G, _D, C.c_double, C.c_double, C.c_double, C.c_int,
                                         C.c_int, _D, C.POINTER(C.c_double), C.POINTER(C.c_int),
                                         C.POINTER(OrStats)]),
                "or_estimate": (C.c_double, [G, _D, _D, C.c_double]),
                "or_integrate": (C.c_int, [G, C.POINTER(OrParams), _D, C.POINTER(OrStats),
                                           C.POINTER(OrRecords), C.POINTER(C.c_double)]),
                "or_energy": (C.c_double, [G, _D]),
                "or_mass": (C.c_double, [G, _D]),
                "or_const_nsteps": (C.c_long, [C.c_double, C.c_double]),
                "or_const_tau": (C.c_double, [C.c_double, C.c_double, C.c_long]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


BCS = ("periodic", "neumann")


class Grid:
    """Grid on the unit square (dim=2) or cube (dim=3), h_a = 1/n_a, with periodic
    boundaries or the homogeneous Neumann conditions of Eq. (CH) on cell-centred nodes.
    `mobility`: None for unit mobility, else the nodal values M(y^n_i) >= 0 that make the
    outer operator A_M of the Remark on Eq. (CHmob)."""

    def __init__(self, dim: int, n, eps: float, eyre: bool = False, bc: str = "periodic",
                 mobility=None):
        n = [int(n)] * dim if np.isscalar(n) else [int(v) for v in n]
        assert dim in (2, 3) and len(n) == dim and bc in BCS
        self.dim, self.n, self.eps, self.eyre, self.bc = dim, tuple(n), float(eps), bool(eyre), bc
        nn = (n + [1, 1])[:3]
        self.N = int(np.prod(n))
        self._mob = None
        if mobility is not None:
            self._mob = np.ascontiguousarray(mobility, dtype=np.float64).reshape(-1)
            assert self._mob.size == self.N and np.all(self._mob >= 0.0)
        self._g = OrGrid(dim, (C.c_long * 3)(*nn), float(eps), int(eyre), BCS.index(bc),
                         None if self._mob is None else self._mob.ctypes.data)

    @property
    def shape(self):  # numpy shape, x fastest
        return tuple(reversed(self.n))

    def ptr(self):
        return C.byref(self._g)

    def _vec(self, y):
        y = np.ascontiguousarray(y, dtype=np.float64).reshape(-1)
        assert y.size == self.N
        return y


def _out(g):
    return np.empty(g.N, dtype=np.float64)


def apply_A(g: Grid, v):
    o = _out(g); lib().or_apply_A(g.ptr(), g._vec(v), o); return o


def rhs(g: Grid, y):
    o = _out(g); lib().or_rhs(g.ptr(), g._vec(y), o); return o


def ghat(g: Grid, y):
    o = _out(g); lib().or_ghat(g.ptr(), g._vec(y), o); return o


def jacvec(g: Grid, y, v):
    o = _out(g); lib().or_jacvec(g.ptr(), g._vec(y), g._vec(v), o); return o


def lambda_max(g: Grid, y) -> float:
    return lib().or_lambda_max(g.ptr(), g._vec(y))


def column_abs_sum(g: Grid, y, j: int) -> float:
    """Absolute sum of column j of A_hat_n (the spectral bound of Fig. 1, one column)."""
    return lib().or_column_abs_sum(g.ptr(), g._vec(y), int(j))


def cheb_order(tau: float, lmax: float) -> int:
    return lib().or_cheb_order(tau, lmax)


def lim_order(p: int):
    """0-based order of the Chebyshev parameters used by the LIM step (the ordered set of Fig. 1)."""
    o = np.zeros(p, dtype=np.int32)
    assert lib().or_lim_order(p, o) == 0
    return o


def lim_step(g: Grid, y, tau: float):
    o = _out(g); lm = C.c_double(); mv = C.c_long(0)
    p = lib().or_lim_step(g.ptr(), g._vec(y), tau, o, C.byref(lm), C.byref(mv))
    return o, p, lm.value, mv.value


def lim_dense(M, ghat_v, y, tau: float, lmax: float):
    M = np.ascontiguousarray(M, dtype=np.float64); N = M.shape[0]
    o = np.empty(N); p = lib().or_lim_dense(N, M, np.ascontiguousarray(ghat_v, dtype=np.float64),
                                            np.ascontiguousarray(y, dtype=np.float64), tau, lmax, o)
    return o, p


def expm(M):
    M = np.ascontiguousarray(M, dtype=np.float64); n = M.shape[0]
    E = np.empty_like(M); rc = lib().or_expm(n, M, E); assert rc == 0; return E


def phi_e1(H, j: int, s: float):
    """u = s phi(-s H_j) e_1 for the leading j x j block of H (row-major, any ld)."""
    H = np.ascontiguousarray(H, dtype=np.float64)
    u = np.empty(j); rc = lib().or_phi_e1(j, H, H.shape[1], s, u); assert rc == 0; return u


def krylov_dense(M, g_v, y0, tau0, tol_phi, mmax):
    M = np.ascontiguousarray(M, dtype=np.float64); N = M.shape[0]
    o = np.empty(N); tau = C.c_double(); j = C.c_int()
    rc = lib().or_krylov_dense(N, M, np.ascontiguousarray(g_v, dtype=np.float64),
                               np.ascontiguousarray(y0, dtype=np.float64), tau0, tol_phi, mmax,
                               o, C.byref(tau), C.byref(j))
    return rc, o, tau.value, j.value


def arnoldi_dense(M, v1, m):
    M = np.ascontiguousarray(M, dtype=np.float64); N = M.shape[0]
    V = np.empty((m + 1, N)); H = np.empty((m + 1, m))
    lib().or_arnoldi_dense(N, M, np.ascontiguousarray(v1, dtype=np.float64), m, V, H)
    return V, H


def tol_phi(norm_ghat, beta, tol):
    return lib().or_tol_phi(norm_ghat, beta, tol)


def ee_step(g: Grid, y, tau, tol=1e-6, tol_phi_fixed=-1.0, mmax=30, linear_restart=False):
    o = _out(g); taken = C.c_double(); j = C.c_int(); st = OrStats()
    rc = lib().or_ee_step(g.ptr(), g._vec(y), tau, tol, tol_phi_fixed, mmax, int(linear_restart),
                          o, C.byref(taken), C.byref(j), C.byref(st))
    return rc, o, taken.value, j.value, stats_dict(st)


def estimate(g: Grid, yn, ynp1, tau):
    return lib().or_estimate(g.ptr(), g._vec(yn), g._vec(ynp1), tau)


def energy(g: Grid, y):
    return lib().or_energy(g.ptr(), g._vec(y))


def mass(g: Grid, y):
    return lib().or_mass(g.ptr(), g._vec(y))


def const_nsteps(T, tau0):
    return lib().or_const_nsteps(T, tau0)


def stats_dict(st: OrStats):
    return {k: getattr(st, k) for k, _ in OrStats._fields_}


def integrate(g: Grid, y0, scheme: str, adaptive: bool, T: float, tau0: float, tol: float = 1e-6,
              mmax: int = 30, tol_phi: float = -1.0, max_steps: int = 10**7, max_rec: int = 100000):
    """Run Fig. 3 (LIM) / Fig. 4 (EE2) or their constant-step forms.  Returns
    (rc, y(T), t, stats, records)."""
    y = g._vec(y0).copy()
    prm = OrParams(0 if scheme == "ee2" else 1, int(adaptive), T, tau0, tol, mmax, tol_phi,
                   max_steps)
    st = OrStats()
    rec_arrays = dict(tau=np.zeros(max_rec), jexit=np.zeros(max_rec, np.int32),
                      restarts=np.zeros(max_rec, np.int32), shrunk=np.zeros(max_rec, np.int32),
                      p=np.zeros(max_rec, np.int32), est=np.zeros(max_rec))
    rec = OrRecords(rec_arrays["tau"].ctypes.data_as(C.POINTER(C.c_double)),
                    rec_arrays["jexit"].ctypes.data_as(C.POINTER(C.c_int)),
                    rec_arrays["restarts"].ctypes.data_as(C.POINTER(C.c_int)),
                    rec_arrays["shrunk"].ctypes.data_as(C.POINTER(C.c_int)),
                    rec_arrays["p"].ctypes.data_as(C.POINTER(C.c_int)),
                    rec_arrays["est"].ctypes.data_as(C.POINTER(C.c_double)), max_rec)
    t = C.c_double()
    rc = lib().or_integrate(g.ptr(), C.byref(prm), y, C.byref(st), C.byref(rec), C.byref(t))
    n = min(st.steps, max_rec)
    records = {k: v[:n].copy() for k, v in rec_arrays.items()}
    return rc, y, t.value, stats_dict(st), records
