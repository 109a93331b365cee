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
