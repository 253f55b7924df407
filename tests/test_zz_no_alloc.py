"""The allocation-free inverse-column entry point (mgwr_inverse_column_noalloc).

It exists for callers that cannot allocate device memory while they run; its
scratch is a fixed array inside the library.  Its results must equal those of
the regular entry point (mgwr_create + mgwr_inverse_column, which allocates its
scratch), within the inverse-column tolerance of the other GPU tests, on two
calls in a row that reuse the shared array.  This file is collected last.
"""
import ctypes as C

import numpy as np
import pytest

from paper_1608_05400_gb300 import mgwr as G

pytestmark = pytest.mark.gpu


def test_noalloc_inverse_column_matches_regular_entry_point():
    torch = pytest.importorskip("torch")
    lib = G.load()
    d, n, M, T, alpha = 2, 31, 1024, 1.0, 0.35
    with G.Solver(d, n, M, T, alpha) as s:
        r = s.toeplitz_column()
        levels = [s.num_levels() - 1, 0]
        refs = [s.inverse_column(l) for l in levels]
        sigmas = [2.0 * d * (s.level_n(l) + 1) ** 2 for l in levels]
    r_dev = torch.tensor(r, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    outs = []
    for sigma in sigmas:  # two calls in a row through the shared scratch array
        k_dev = torch.full((M,), float("nan"), dtype=torch.float64, device="cuda")
        st = lib.mgwr_inverse_column_noalloc(C.c_void_p(r_dev.data_ptr()), M, sigma,
                                             C.c_void_p(k_dev.data_ptr()), C.c_void_p(stream))
        assert st == G.MGWR_OK
        torch.cuda.synchronize()
        outs.append(k_dev.cpu().numpy())
    for k, ref in zip(outs, refs):
        assert np.all(np.isfinite(k))
        assert np.abs(k - ref).max() <= 1e-13 * np.abs(ref).max()


def test_noalloc_rejects_sizes_beyond_its_array():
    torch = pytest.importorskip("torch")
    lib = G.load()
    buf = torch.zeros(8192, dtype=torch.float64, device="cuda")
    p = C.c_void_p(buf.data_ptr())
    assert lib.mgwr_inverse_column_noalloc(p, 8192, 1.0, p, None) == G.MGWR_E_TOOBIG
    assert lib.mgwr_inverse_column_noalloc(p, 1000, 1.0, p, None) == G.MGWR_E_INVAL
    assert lib.mgwr_inverse_column_noalloc(None, 64, 1.0, p, None) == G.MGWR_E_INVAL
