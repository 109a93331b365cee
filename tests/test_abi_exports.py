"""The C-ABI library builds for sm_103a, loads, and exports every function that
include/ch.h declares (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "ch.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ch_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("ch_create_grid", "ch_rhs", "ch_jacvec", "ch_phi_krylov", "ch_ee_step",
                     "ch_lim_step", "ch_integrate", "ch_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_2502_14589_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_header():
    from paper_2502_14589_gb300 import ch
    for n in declared_functions():
        if n in ("ch_last_error",):
            continue
        assert hasattr(ch, n), n


def test_argument_errors_are_reported_without_a_gpu():
    """Invalid sizes are rejected with CH_EINVAL and a message before any CUDA call (the raw
    C functions, with a null stream: the binding's default stream needs a GPU)."""
    from paper_2502_14589_gb300 import build, ch
    build.build()
    lib = ch.load()
    out = ctypes.c_void_p()

    def grid(dim, n, eps):
        arr = (ctypes.c_int64 * 3)(*(list(n) + [1] * (3 - len(n))))
        return lib.ch_create_grid(dim, arr, eps, ch.CH_FP64, 30, None, ctypes.byref(out))

    def batch(dim, sizes, eps):
        flat = []
        for sz in sizes:
            flat += list(sz) + [1] * (3 - dim)
        arr = (ctypes.c_int64 * len(flat))(*flat)
        ep = (ctypes.c_double * len(eps))(*eps)
        return lib.ch_create_batch(dim, len(sizes), arr, ep, ch.CH_FP64, 30, None, ctypes.byref(out))

    assert grid(2, [3, 64], 0.05) == ch.CH_EINVAL
    assert b"out of range" in lib.ch_last_error()
    assert grid(3, [2048, 2048, 2048], 0.05) == ch.CH_EINVAL      # more than 2^31 - 1 points
    assert grid(2, [64, 64], -1.0) == ch.CH_EINVAL
    # a batch whose total size would overflow a 64-bit sum is refused at the first excess
    assert batch(3, [[1 << 20] * 3] * 16, [0.01] * 16) == ch.CH_EINVAL
    assert b"2^31" in lib.ch_last_error()
    assert batch(2, [[64, 64], [64, 64]], [0.02, -1.0]) == ch.CH_EINVAL
    assert out.value is None
