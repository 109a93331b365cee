"""Thin ctypes binding of the C ABI in include/ch.h (libch.so, built by build.py).

Argument marshalling only: every step of the method runs in the CUDA kernels of libch.so.
Functions keep the C names; vector arguments are CUDA float64 contiguous torch tensors
(their device pointers are passed), scalars come back as Python numbers.  There is no
CPU path: if libch.so is missing or no GPU is present, the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os

from . import build as _build

_LIB = None

CH_OK, CH_EINVAL, CH_ENOMEM, CH_ECUDA, CH_ENOTCONV, CH_ENONFINITE, CH_ETIMEOUT = range(7)
CH_FP64, CH_MIXED = 0, 1
CH_EE2, CH_LIM = 0, 1
CH_BC_PERIODIC, CH_BC_NEUMANN = 0, 1
BCS = {"periodic": CH_BC_PERIODIC, "neumann": CH_BC_NEUMANN}
STATUS_NAMES = {0: "CH_OK", 1: "CH_EINVAL", 2: "CH_ENOMEM", 3: "CH_ECUDA", 4: "CH_ENOTCONV",
                5: "CH_ENONFINITE", 6: "CH_ETIMEOUT"}


class CHError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class ch_params(C.Structure):
    _fields_ = [("scheme", C.c_int), ("adaptive", C.c_int), ("T", C.c_double),
                ("tau0", C.c_double), ("tol", C.c_double), ("mmax", C.c_int),
                ("tol_phi", C.c_double), ("eyre", C.c_int), ("max_steps", C.c_int64)]


class ch_grid_options(C.Structure):
    _fields_ = [("bc", C.c_int), ("variable_mobility", C.c_int)]


class ch_stats(C.Structure):
    _fields_ = [("steps", C.c_int64), ("matvecs", C.c_int64), ("rhs_evals", C.c_int64),
                ("krylov_iters", C.c_int64), ("restarts", C.c_int64), ("tau_shrinks", C.c_int64),
                ("phi_evals", C.c_int64), ("t", C.c_double), ("tau_next", C.c_double),
                ("last_est", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_P = C.c_void_p
_D = C.c_double
_DP = C.POINTER(C.c_double)
_IP = C.POINTER(C.c_int)
_SIGS = {
    "ch_create_grid": [C.c_int, C.POINTER(C.c_int64), _D, C.c_int, C.c_int, _P, C.POINTER(_P)],
    "ch_create_grid_ex": [C.c_int, C.POINTER(C.c_int64), _D, C.c_int, C.c_int, C.POINTER(ch_grid_options),
                          _P, C.POINTER(_P)],
    "ch_set_mobility": [_P, _P],
    "ch_destroy_grid": [_P],
    "ch_rhs": [_P, _P, _P, C.c_int, _DP, _DP],
    "ch_jacvec": [_P, _P, _P, _P, C.c_int],
    "ch_lambda_max": [_P, _P, C.c_int, _DP],
    "ch_lambda_max_bound": [C.c_int, C.POINTER(C.c_int64), _D, C.c_int, _D, _D, _DP],
    "ch_lim_schedule": [_D, _D, C.c_int, _IP, _IP, _DP],
    "ch_estimate": [_P, _P, _P, _D, _DP],
    "ch_phi_krylov": [_P, _P, _D, _D, C.c_int, C.c_int, C.c_int, _P, _DP, C.POINTER(ch_stats)],
    "ch_ee_step": [_P, _P, _D, C.POINTER(ch_params), _P, _DP, _DP],
    "ch_lim_step": [_P, _P, _D, C.c_int, _P, _IP, _DP],
    "ch_integrate": [_P, C.POINTER(ch_params), _P, C.POINTER(ch_stats)],
    "ch_set_record_capacity": [_P, C.c_int64],
    "ch_get_records": [_P, C.c_int64, _DP, _IP, _IP, _IP, _IP, _DP, C.POINTER(C.c_int64)],
    "ch_get_state": [_P, _DP, _DP],
    "ch_set_state": [_P, _D, _D],
    "ch_energy_mass": [_P, _P, _DP, _DP],
    "ch_timing_start": [_P, C.c_int],
    "ch_timing_read": [_P, _DP, C.POINTER(C.c_int64), C.POINTER(C.c_int64)],
    "ch_timing_work": [_P, _DP, _DP],
    "ch_bench_kernel": [_P, C.c_int, C.c_int, _DP, _DP, _DP, _DP],
    "ch_create_batch": [C.c_int, C.c_int, C.POINTER(C.c_int64), _DP, C.c_int, C.c_int, _P, C.POINTER(_P)],
    "ch_destroy_batch": [_P],
    "ch_batch_layout": [_P, C.POINTER(C.c_int64), _IP],
    "ch_integrate_batch": [_P, C.POINTER(ch_params), _P, C.POINTER(ch_stats)],
    "ch_energy_mass_noalloc": [C.c_int, C.POINTER(C.c_int64), _D, _P, _P, _P],
    "ch_probe_fp64_peak": [_P, _DP],
}

KERNEL_CLASSES = ["prep", "tstage", "wstage", "mgs", "phi", "combine", "rhs1", "rhs2",
                  "resid1", "resid2", "lim2", "energy", "arm", "arnoldi"]


def lib_path() -> str:
    return _build.LIB


def load():
    """Load libch.so (raises if it has not been built)."""
    global _LIB
    if _LIB is None:
        path = _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"libch.so is not built ({path}); call paper_2502_14589_gb300.build.build()")
        L = C.CDLL(path)
        for name, args in _SIGS.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = C.c_int
        L.ch_last_error.restype = C.c_char_p
        L.ch_last_error.argtypes = []
        L.ch_kernel_launches.restype = C.c_int64
        L.ch_kernel_launches.argtypes = [_P]
        L.ch_batch_kernel_launches.restype = C.c_int64
        L.ch_batch_kernel_launches.argtypes = [_P]
        L.ch_batch_groups.restype = C.c_int
        L.ch_batch_groups.argtypes = [_P]
        _LIB = L
    return _LIB


def _check(st):
    if st != CH_OK:
        raise CHError(st, load().ch_last_error().decode())


def _ptr(t):
    import torch
    if t is None:
        return None
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError("vector arguments must be contiguous float64 CUDA tensors")
    return C.c_void_p(t.data_ptr())


# Points a vector argument of each live grid or batch handle must hold, and the CUDA
# device the handle's workspace lives on.  The C functions cannot check the length or the
# device of a caller's buffer, so the binding does before passing the pointer on.
_EXTENT = {}


def _register(h, points):
    import torch
    _EXTENT[h.value] = (int(points), torch.cuda.current_device())


def _vec(h, t):
    p = _ptr(t)
    ext = _EXTENT.get(getattr(h, "value", h))
    if t is not None and ext is not None:
        points, device = ext
        if t.numel() < points:
            raise ValueError(f"vector of {t.numel()} values; this handle needs {points}")
        if t.device.index != device:
            raise ValueError(f"vector on cuda:{t.device.index}; this handle lives on cuda:{device}")
    return p


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


# ---- C-named wrappers ---------------------------------------------------------------
def ch_create_grid(dim, n, eps, precision=CH_FP64, mmax_capacity=30, stream=None):
    nn = list(n) + [1] * (3 - len(n))
    arr = (C.c_int64 * 3)(*nn)
    h = C.c_void_p()
    _check(load().ch_create_grid(dim, arr, eps, precision, mmax_capacity, _stream(stream), C.byref(h)))
    _register(h, nn[0] * nn[1] * nn[2])
    return h


def ch_create_grid_ex(dim, n, eps, precision=CH_FP64, mmax_capacity=30, stream=None, bc="periodic",
                      variable_mobility=False):
    nn = list(n) + [1] * (3 - len(n))
    arr = (C.c_int64 * 3)(*nn)
    opts = ch_grid_options(BCS[bc] if isinstance(bc, str) else int(bc), int(bool(variable_mobility)))
    h = C.c_void_p()
    _check(load().ch_create_grid_ex(dim, arr, eps, precision, mmax_capacity, C.byref(opts), _stream(stream),
                                    C.byref(h)))
    _register(h, nn[0] * nn[1] * nn[2])
    return h


def ch_set_mobility(h, M):
    """Nodal mobility M (device float64 tensor of N values, or None for unit mobility)."""
    _check(load().ch_set_mobility(h, _vec(h, M)))


def ch_destroy_grid(h):
    _EXTENT.pop(getattr(h, "value", h), None)
    _check(load().ch_destroy_grid(h))


def ch_rhs(h, y, f, eyre=0, want_norms=False):
    nf, ng = C.c_double(), C.c_double()
    _check(load().ch_rhs(h, _vec(h, y), _vec(h, f), int(eyre), C.byref(nf) if want_norms else None,
                         C.byref(ng) if want_norms else None))
    return (nf.value, ng.value) if want_norms else None


def ch_jacvec(h, y_lin, v, w, eyre=0):
    _check(load().ch_jacvec(h, _vec(h, y_lin), _vec(h, v), _vec(h, w), int(eyre)))


def ch_lambda_max(h, y, eyre=0):
    out = C.c_double()
    _check(load().ch_lambda_max(h, _vec(h, y), int(eyre), C.byref(out)))
    return out.value


def ch_lambda_max_bound(dim, n, eps, y2min, y2max, eyre=0):
    """Host-only closed form of the spectral bound of Fig. 1 from the extremes of y^2 (no GPU needed)."""
    nn = (C.c_int64 * 3)(*(list(n) + [1] * (3 - len(n))))
    out = C.c_double()
    _check(load().ch_lambda_max_bound(dim, nn, eps, int(eyre), y2min, y2max, C.byref(out)))
    return out.value


def ch_lim_schedule(tau, lambda_max):
    """Host-only LIM schedule of Fig. 1 (no GPU needed): (p, order (1-based m), a_m)."""
    import numpy as np
    p = C.c_int()
    _check(load().ch_lim_schedule(tau, lambda_max, 0, C.byref(p), None, None))
    order = np.zeros(p.value, np.int32)
    a = np.zeros(p.value)
    _check(load().ch_lim_schedule(tau, lambda_max, p.value, C.byref(p), order.ctypes.data_as(_IP),
                                  a.ctypes.data_as(_DP)))
    return p.value, order, a


def ch_estimate(h, y0, y1, tau):
    out = C.c_double()
    _check(load().ch_estimate(h, _vec(h, y0), _vec(h, y1), tau, C.byref(out)))
    return out.value


def ch_phi_krylov(h, y_n, tau0, tol_phi, mmax, linear_restart, y_next, eyre=0):
    tu = C.c_double()
    st = ch_stats()
    _check(load().ch_phi_krylov(h, _vec(h, y_n), tau0, tol_phi, mmax, int(linear_restart), int(eyre),
                                _vec(h, y_next), C.byref(tu), C.byref(st)))
    return tu.value, st.as_dict()


def make_params(scheme="ee2", adaptive=True, T=1e-3, tau0=1e-7, tol=1e-6, mmax=30,
                tol_phi=-1.0, eyre=False, max_steps=10 ** 9):
    return ch_params(CH_EE2 if scheme == "ee2" else CH_LIM, int(adaptive), T, tau0, tol, mmax,
                     tol_phi, int(eyre), max_steps)


def ch_ee_step(h, y_n, tau, prm, y_next):
    tu, est = C.c_double(), C.c_double()
    _check(load().ch_ee_step(h, _vec(h, y_n), tau, C.byref(prm), _vec(h, y_next), C.byref(tu), C.byref(est)))
    return tu.value, est.value


def ch_lim_step(h, y_n, tau, y_next, eyre=0):
    p, lm = C.c_int(), C.c_double()
    _check(load().ch_lim_step(h, _vec(h, y_n), tau, int(eyre), _vec(h, y_next), C.byref(p), C.byref(lm)))
    return p.value, lm.value


def ch_integrate(h, prm, y):
    st = ch_stats()
    _check(load().ch_integrate(h, C.byref(prm), _vec(h, y), C.byref(st)))
    return st.as_dict()


def ch_set_record_capacity(h, cap):
    _check(load().ch_set_record_capacity(h, cap))


def ch_get_records(h, max_rec):
    import numpy as np
    tau = np.zeros(max_rec); est = np.zeros(max_rec)
    jexit = np.zeros(max_rec, np.int32); rs = np.zeros(max_rec, np.int32)
    sh = np.zeros(max_rec, np.int32); p = np.zeros(max_rec, np.int32)
    cnt = C.c_int64()
    _check(load().ch_get_records(h, max_rec, tau.ctypes.data_as(_DP), jexit.ctypes.data_as(_IP),
                                 rs.ctypes.data_as(_IP), sh.ctypes.data_as(_IP), p.ctypes.data_as(_IP),
                                 est.ctypes.data_as(_DP), C.byref(cnt)))
    n = cnt.value
    return dict(tau=tau[:n], jexit=jexit[:n], restarts=rs[:n], shrunk=sh[:n], p=p[:n], est=est[:n])


def ch_get_state(h):
    t, tau = C.c_double(), C.c_double()
    _check(load().ch_get_state(h, C.byref(t), C.byref(tau)))
    return t.value, tau.value


def ch_set_state(h, t, tau):
    _check(load().ch_set_state(h, t, tau))


def ch_energy_mass(h, y):
    e, m = C.c_double(), C.c_double()
    _check(load().ch_energy_mass(h, _vec(h, y), C.byref(e), C.byref(m)))
    return e.value, m.value


def ch_kernel_launches(h):
    return load().ch_kernel_launches(h)


def ch_timing_start(h, kernel_class):
    """Time every launch of one kernel class (name or index; None stops timing)."""
    k = -1 if kernel_class is None else (KERNEL_CLASSES.index(kernel_class)
                                         if isinstance(kernel_class, str) else int(kernel_class))
    _check(load().ch_timing_start(h, k))


def ch_bench_kernel(h, kernel_class, reps=200):
    """Mean launch time (us) and algorithmic bytes / flops / FP64 instructions per launch."""
    k = KERNEL_CLASSES.index(kernel_class) if isinstance(kernel_class, str) else int(kernel_class)
    us, b, f, i = C.c_double(), C.c_double(), C.c_double(), C.c_double()
    _check(load().ch_bench_kernel(h, k, reps, C.byref(us), C.byref(b), C.byref(f), C.byref(i)))
    return {"avg_us": us.value, "bytes": b.value, "flops": f.value, "fp64_instr": i.value}


def ch_timing_read(h):
    ms = C.c_double(); n = C.c_int64(); counts = (C.c_int64 * len(KERNEL_CLASSES))()
    _check(load().ch_timing_read(h, C.byref(ms), C.byref(n), counts))
    return ms.value, n.value, {k: counts[i] for i, k in enumerate(KERNEL_CLASSES)}


def ch_timing_work(h):
    f, b = C.c_double(), C.c_double()
    _check(load().ch_timing_work(h, C.byref(f), C.byref(b)))
    return f.value, b.value


class Grid:
    """Owning handle around ch_create_grid / ch_destroy_grid."""

    def __init__(self, dim, n, eps, precision=CH_FP64, mmax_capacity=30, stream=None, bc="periodic",
                 variable_mobility=False):
        n = [int(n)] * dim if isinstance(n, int) else [int(v) for v in n]
        self.dim, self.n, self.eps, self.bc = dim, tuple(n), eps, bc
        self.N = 1
        for v in n:
            self.N *= v
        if bc == "periodic" and not variable_mobility:
            self.h = ch_create_grid(dim, n, eps, precision, mmax_capacity, stream)
        else:
            self.h = ch_create_grid_ex(dim, n, eps, precision, mmax_capacity, stream, bc, variable_mobility)

    def close(self):
        if self.h is not None:
            ch_destroy_grid(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


# ---- batches --------------------------------------------------------------------------
def ch_create_batch(dim, sizes, eps, precision=CH_FP64, mmax_capacity=30, stream=None):
    """sizes: list of per-instance point counts per axis (int for a cube/square)."""
    count = len(sizes)
    flat = []
    for sz in sizes:
        sz = [int(sz)] * dim if isinstance(sz, (int,)) or hasattr(sz, "__index__") else [int(v) for v in sz]
        flat += sz + [1] * (3 - dim)
    arr = (C.c_int64 * (3 * count))(*flat)
    ep = (C.c_double * count)(*[float(e) for e in eps])
    h = C.c_void_p()
    _check(load().ch_create_batch(dim, count, arr, ep, precision, mmax_capacity, _stream(stream), C.byref(h)))
    _register(h, ch_batch_layout(h, count)[0][count])
    return h


def ch_destroy_batch(h):
    _EXTENT.pop(getattr(h, "value", h), None)
    _check(load().ch_destroy_batch(h))


def ch_batch_layout(h, count):
    offs = (C.c_int64 * (count + 1))()
    cl = C.c_int()
    _check(load().ch_batch_layout(h, offs, C.byref(cl)))
    return list(offs), cl.value


def ch_integrate_batch(h, prm, y, count):
    st = (ch_stats * count)()
    _check(load().ch_integrate_batch(h, C.byref(prm), _vec(h, y), st))
    return [s.as_dict() for s in st]


def ch_batch_kernel_launches(h):
    return load().ch_batch_kernel_launches(h)


def ch_batch_groups(h):
    return load().ch_batch_groups(h)


def ch_energy_mass_noalloc(dim, n, eps, y, out, stream=None):
    """Energy and mass of y into the device tensor out[0:2] without any allocation (queued on
    the stream, not synchronised); see include/ch.h for whom this entry point is for."""
    import torch
    nn = (C.c_int64 * 3)(*(list(n) + [1] * (3 - len(n))))
    yp, op = _ptr(y), _ptr(out)
    if y.numel() < nn[0] * nn[1] * nn[2]:
        raise ValueError(f"vector of {y.numel()} values; the grid has {nn[0] * nn[1] * nn[2]} points")
    if out.numel() < 2:
        raise ValueError("out must hold 2 values")
    if out.device != y.device:
        raise ValueError(f"y on {y.device} and out on {out.device}: both must be on one GPU")
    if stream is not None and stream.device != y.device:
        raise ValueError(f"stream of {stream.device}; y and out live on {y.device}")
    # the C entry point works on the current device: make it the tensors' device
    with torch.cuda.device(y.device):
        _check(load().ch_energy_mass_noalloc(dim, nn, eps, yp, op, _stream(stream)))


def ch_probe_fp64_peak(stream=None):
    """Measured FP64 FMA rate of the current GPU (TFLOP/s, FMA = 2 flop)."""
    out = C.c_double()
    _check(load().ch_probe_fp64_peak(_stream(stream), C.byref(out)))
    return out.value
