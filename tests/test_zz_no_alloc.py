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


@pytest.mark.parametrize("dim,n,eps", [(2, (256, 192), 0.03), (3, (40, 36, 33), 0.05)])
def test_noalloc_energy_mass_matches_grid_entry_point(lib, dim, n, eps):
    from paper_2502_14589_gb300 import ch
    stream = torch.cuda.current_stream()
    nn = (C.c_int64 * 3)(*(list(n) + [1] * (3 - len(n))))
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    with ch.Grid(dim, n, eps) as G:
        for call, seed in enumerate((3, 4)):             # two calls in a row, different data
            y = torch.from_numpy(inputs.initial_state(n, seed, -0.6, 0.6, mean=0.1)).cuda()
            e_ref, m_ref = ch.ch_energy_mass(G.h, y)
            st = lib.ch_energy_mass_noalloc(dim, nn, eps, C.c_void_p(y.data_ptr()),
                                            C.c_void_p(out.data_ptr()), C.c_void_p(stream.cuda_stream))
            assert st == 0, lib.ch_last_error().decode()
            torch.cuda.synchronize()
            e, m = out.cpu().numpy()
            assert abs(e - e_ref) <= 1e-13 * abs(e_ref), (call, e, e_ref)
            assert abs(m - m_ref) <= 1e-13 * max(abs(m_ref), 1.0), (call, m, m_ref)


def test_noalloc_rejects_oversized_grids(lib):
    nn = (C.c_int64 * 3)(2048, 2048, 1024)               # 2^32 points > 2^31 - 1
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    y = torch.zeros(8, dtype=torch.float64, device="cuda")
    st = lib.ch_energy_mass_noalloc(3, nn, 0.05, C.c_void_p(y.data_ptr()), C.c_void_p(out.data_ptr()),
                                    C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 1 and b"exceeds" in lib.ch_last_error()
