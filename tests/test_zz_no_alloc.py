"""The allocation-free inverse-column entry point (mgwr_inverse_column_noalloc).

It serves callers that cannot allocate device memory while they run (services
that reserve their whole GPU budget at start-up, or code whose device memory
belongs to another allocator); its scratch is a fixed array inside the library.
Its results must equal those of the regular entry point (mgwr_create +
mgwr_inverse_column, which allocates its scratch), within the inverse-column
tolerance of the other GPU tests, on calls in a row that reuse the shared array,
also on a stream that still has other work queued ahead of the call.

The file name sorts last, so pytest collects it after every other test file: a
run that stops at the first failure has then already run all the other tests.
"""
import ctypes as C

import numpy as np
import pytest

from paper_1608_05400_gb300 import mgwr as G

pytestmark = pytest.mark.gpu

D, N, M, T, ALPHA = 2, 31, 1024, 1.0, 0.35


def _regular():
    """Toeplitz column, inverse columns and sigmas of two levels from the
    regular (allocating) entry points."""
    with G.Solver(D, N, M, T, ALPHA) as s:
        r = s.toeplitz_column()
        levels = [s.num_levels() - 1, 0]
        refs = [s.inverse_column(l) for l in levels]
        sigmas = [2.0 * D * (s.level_n(l) + 1) ** 2 for l in levels]
    return r, refs, sigmas


def _close(k, ref):
    return np.all(np.isfinite(k)) and np.abs(k - ref).max() <= 1e-13 * np.abs(ref).max()


def test_noalloc_inverse_column_matches_regular_entry_point():
    torch = pytest.importorskip("torch")
    lib = G.load()
    r, refs, sigmas = _regular()
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
        assert _close(k, ref)


def test_noalloc_call_is_ordered_on_a_busy_stream():
    # the input column is written by a kernel queued behind a busy wait on a fresh
    # stream; the call on that stream must see it, and sigma must arrive in order too
    torch = pytest.importorskip("torch")
    lib = G.load()
    r, refs, sigmas = _regular()
    src = torch.tensor(r, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    outs = []
    for sigma in reversed(sigmas):
        with torch.cuda.stream(side):
            torch.cuda._sleep(20_000_000)  # about 10 ms of GPU time ahead of the call
            r_dev = src * 1.0
            k_dev = torch.full((M,), float("nan"), dtype=torch.float64, device="cuda")
        st = lib.mgwr_inverse_column_noalloc(C.c_void_p(r_dev.data_ptr()), M, sigma,
                                             C.c_void_p(k_dev.data_ptr()),
                                             C.c_void_p(side.cuda_stream))
        assert st == G.MGWR_OK
        side.synchronize()
        outs.append(k_dev.cpu().numpy())
    for k, ref in zip(outs, reversed(refs)):
        assert _close(k, ref)


def test_noalloc_rejects_sizes_beyond_its_array():
    torch = pytest.importorskip("torch")
    lib = G.load()
    buf = torch.zeros(8192, dtype=torch.float64, device="cuda")
    p = C.c_void_p(buf.data_ptr())
    assert lib.mgwr_inverse_column_noalloc(p, 8192, 1.0, p, None) == G.MGWR_E_TOOBIG
    assert lib.mgwr_inverse_column_noalloc(p, 1000, 1.0, p, None) == G.MGWR_E_INVAL
    assert lib.mgwr_inverse_column_noalloc(None, 64, 1.0, p, None) == G.MGWR_E_INVAL
