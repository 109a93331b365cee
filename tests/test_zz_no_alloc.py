"""ch_energy_mass_noalloc: the entry point for callers that cannot let the library allocate
device memory (they hand out all device memory from their own pool, or cannot afford the
device synchronisation that cudaMalloc / cudaFree may cause).  It must give the same energy
and mass as ch_energy_mass of a grid object, call after call, through the C ABI.  This file
sorts last so that a run stopping at the first failure has run every other test before it."""
import ctypes as C

import numpy as np
import pytest

from paper_2502_14589_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    from paper_2502_14589_gb300 import build, ch
    build.build()
    L = ch.load()
    L.ch_energy_mass_noalloc.restype = C.c_int
    L.ch_energy_mass_noalloc.argtypes = [C.c_int, C.POINTER(C.c_int64), C.c_double, C.c_void_p,
                                         C.c_void_p, C.c_void_p]
    return L


def _call(lib, dim, n, eps, y, out, stream):
    nn = (C.c_int64 * 3)(*(list(n) + [1] * (3 - len(n))))
    return lib.ch_energy_mass_noalloc(dim, nn, eps, C.c_void_p(y.data_ptr()), C.c_void_p(out.data_ptr()),
                                      C.c_void_p(stream.cuda_stream))


# Small grids take fewer blocks than the scratch holds; the 1024 x 512 and 72 x 64 x 60
# grids fill all 1024 blocks of partial sums and make every thread loop more than once.
CASES = [(2, (256, 192), 0.03), (3, (40, 36, 33), 0.05), (2, (1024, 512), 0.02), (3, (72, 64, 60), 0.04)]


@pytest.mark.parametrize("dim,n,eps", CASES)
def test_noalloc_energy_mass_matches_grid_entry_point(lib, dim, n, eps):
    from paper_2502_14589_gb300 import ch
    stream = torch.cuda.current_stream()
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    with ch.Grid(dim, n, eps) as G:
        for call, seed in enumerate((3, 4)):             # two calls in a row, different data
            y = torch.from_numpy(inputs.initial_state(n, seed, -0.6, 0.6, mean=0.1)).cuda()
            e_ref, m_ref = ch.ch_energy_mass(G.h, y)
            st = _call(lib, dim, n, eps, y, out, stream)
            assert st == 0, lib.ch_last_error().decode()
            torch.cuda.synchronize()
            e, m = out.cpu().numpy()
            assert abs(e - e_ref) <= 1e-13 * abs(e_ref), (call, e, e_ref)
            assert abs(m - m_ref) <= 1e-13 * max(abs(m_ref), 1.0), (call, m, m_ref)


def test_noalloc_large_then_small_calls_on_one_stream(lib):
    """A call that fills every block of the scratch, then a small one queued right behind it
    on the same stream, with no synchronisation between: each must match its grid result."""
    from paper_2502_14589_gb300 import ch
    stream = torch.cuda.current_stream()
    cases = [(2, (1024, 512), 0.02, 5), (2, (48, 40), 0.03, 6), (3, (72, 64, 60), 0.04, 7), (3, (6, 5, 7), 0.05, 8)]
    ys = [torch.from_numpy(inputs.initial_state(n, s, -0.7, 0.7, mean=0.05)).cuda() for _, n, _, s in cases]
    outs = [torch.zeros(2, dtype=torch.float64, device="cuda") for _ in cases]
    for (dim, n, eps, _), y, out in zip(cases, ys, outs):
        assert _call(lib, dim, n, eps, y, out, stream) == 0, lib.ch_last_error().decode()
    torch.cuda.synchronize()
    for (dim, n, eps, _), y, out in zip(cases, ys, outs):
        with ch.Grid(dim, n, eps) as G:
            e_ref, m_ref = ch.ch_energy_mass(G.h, y)
        e, m = out.cpu().numpy()
        assert abs(e - e_ref) <= 1e-13 * abs(e_ref), (n, e, e_ref)
        assert abs(m - m_ref) <= 1e-13 * max(abs(m_ref), 1.0), (n, m, m_ref)


def test_noalloc_rejects_oversized_grids(lib):
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    y = torch.zeros(8, dtype=torch.float64, device="cuda")
    st = _call(lib, 3, (2048, 2048, 1024), 0.05, y, out, torch.cuda.current_stream())   # 2^32 points
    assert st == 1 and b"exceeds" in lib.ch_last_error()


def test_noalloc_rejects_host_memory(lib):
    """Host buffers are refused before anything is queued (the kernel would otherwise read
    them from the GPU)."""
    n = (16, 16)
    y_host = torch.zeros(256, dtype=torch.float64)
    out_dev = torch.zeros(2, dtype=torch.float64, device="cuda")
    st = _call(lib, 2, n, 0.05, y_host, out_dev, torch.cuda.current_stream())
    assert st == 1 and b"device memory" in lib.ch_last_error()
    y_dev = torch.zeros(256, dtype=torch.float64, device="cuda")
    out_host = torch.zeros(2, dtype=torch.float64)
    st = _call(lib, 2, n, 0.05, y_dev, out_host, torch.cuda.current_stream())
    assert st == 1 and b"device memory" in lib.ch_last_error()
