"""FFT-engine launch shapes and the tuner: every split E (radix-8 butterflies per
thread) computes the same butterflies in the same order, so sweeps and defects
are bitwise identical for all E, and agree with the oracle; the tuner picks a
valid split per kernel class, leaves the handle's state alone and records its
choice for later handles of the same shape."""
import numpy as np
import pytest

from oracle import mgwr as omg
from paper_1608_05400_gb300 import inputs
from paper_1608_05400_gb300 import mgwr as G

pytestmark = pytest.mark.gpu

K = {name: i for i, name in enumerate(G.KERNEL_CLASSES)}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    G.load()


def rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def _run(d, n, M, hier, E, op):
    s = G.Solver(d, n, M, 1.0, 0.45)
    with s:
        if hier == G.MGWR_H32:
            s.set_precision(G.MGWR_MIXED)
        word = "32" if hier == G.MGWR_H32 else "64"
        s.set_engine_split(K["sweep" + word], E)
        s.set_engine_split(K["defect" + word], E)
        l = s.num_levels() - 1
        N = n ** d
        u = inputs.random_field(N, M, seed=1)
        f = inputs.random_field(N, M, seed=2, scale=2.0 * d * (n + 1) ** 2)
        s.field_set(hier, l, G.MGWR_U, u)
        s.field_set(hier, l, G.MGWR_F, f)
        if op == "sweep":
            s.smooth(hier, l, G.MGWR_RED)
            s.smooth(hier, l, G.MGWR_BLACK)
            out = s.field_get(hier, l, G.MGWR_U)
        else:
            s.defect(hier, l)
            out = s.field_get(hier, l, G.MGWR_R)
        used = s.engine_split(K[op + word])
    return out, used, u, f


@pytest.mark.parametrize("hier", [G.MGWR_H64, G.MGWR_H32])
@pytest.mark.parametrize("op", ["sweep", "defect"])
@pytest.mark.parametrize("d,n,M", [(1, 15, 4), (1, 31, 16), (2, 15, 64), (1, 63, 128), (2, 31, 1024),
                                   (1, 15, 2048), (2, 7, 4096), (1, 7, 8192)])
def test_every_split_gives_identical_results(hier, op, d, n, M):
    ref, used1, u, f = _run(d, n, M, hier, 1, op)
    assert used1 == 1
    for E in (2, 4):
        out, used, _, _ = _run(d, n, M, hier, E, op)
        assert used in (1, 2, 4) and used <= E
        np.testing.assert_array_equal(out, ref)
    # and against the oracle's direct sums
    W = omg.WRMG(d, n, M, 1.0, 0.45) if M <= 4096 else None
    if W is not None:
        l = W.finest
        if op == "sweep":
            r = u.copy()
            W.sweep(l, r, f, 0)
            W.sweep(l, r, f, 1)
        else:
            r = W.defect(l, u, f)
        tol = 1e-12 if hier == G.MGWR_H64 else 2e-5
        if op == "sweep":
            assert rel(ref, r) <= tol
        else:
            scale = np.abs(f).max() + W.levels[l].sigma * 2 * np.abs(u).max()
            assert np.abs(ref - r).max() <= tol * scale


def test_split_requests_fall_back_to_what_a_length_takes():
    with G.Solver(1, 7, 4, 1.0, 0.5) as s:      # L = 8: one butterfly per stage
        s.set_engine_split(K["sweep64"], 4)
        assert s.engine_split(K["sweep64"]) == 1
    with G.Solver(1, 7, 8192, 1.0, 0.5) as s:   # partitioned lines: E = 1 or 2
        s.set_engine_split(K["defect64"], 4)
        assert s.engine_split(K["defect64"]) == 1
        s.set_engine_split(K["defect64"], 2)
        assert s.engine_split(K["defect64"]) == 2
        with pytest.raises(G.MGWRError):
            s.set_engine_split(K["restrict"], 2)
        with pytest.raises(G.MGWRError):
            s.set_engine_split(K["sweep64"], 3)
        with pytest.raises(G.MGWRError):
            s.set_engine_split(K["sweep64"], 2, level=s.num_levels())
        s.set_engine_split(K["sweep64"], 2, level=1)
        assert s.engine_split(K["sweep64"], 1) == 2 and s.engine_split(K["sweep64"], 0) == 1


@pytest.mark.parametrize("precision", [G.MGWR_FP64, G.MGWR_MIXED, G.MGWR_MIXED_DD, G.MGWR_DD])
def test_autotune_keeps_state_and_results(precision):
    d, n, M = 2, 63, 256
    f = inputs.Problem(d, n, M, 1.0, 0.4, "t2").rhs()
    with G.Solver(d, n, M, 1.0, 0.4) as s0:
        s0.set_precision(precision)
        s0.set_rhs(f)
        st0 = s0.solve(1, 1, 1, tol=1e-10, max_cycles=40)
        u0 = s0.solution()
    with G.Solver(d, n, M, 1.0, 0.4) as s:
        s.set_precision(precision)
        s.set_rhs(f)
        s.solve(1, 1, 1, tol=1e-10, max_cycles=1, allow_noconv=True)
        before = s.solution()
        chosen = s.autotune()
        flags = G.MGWR_SPLIT_STAGED | G.MGWR_SPLIT_TENSOR | G.MGWR_SPLIT_RADIX
        assert all(e & ~flags in (1, 2, 4) for v in chosen.values() for e in v)
        np.testing.assert_array_equal(s.solution(), before)  # tuning touches no state
        s.set_rhs(f)
        st = s.solve(1, 1, 1, tol=1e-10, max_cycles=40)
        rounding = G.MGWR_SPLIT_TENSOR | G.MGWR_SPLIT_RADIX
        if any(e & rounding for e in chosen.get("sweep32", [])):
            # tensor-core and register-pass sweeps round differently from the FFT engine
            assert rel(s.solution(), u0) <= 1e-9 and abs(st.cycles - st0.cycles) <= 2
        else:
            np.testing.assert_array_equal(s.solution(), u0)
            assert (st.cycles, st.relres) == (st0.cycles, st0.relres)
    # a later handle of the same shape starts with the recorded choices
    with G.Solver(d, n, M, 1.0, 0.9) as s2:
        s2.set_precision(precision)
        for name, v in chosen.items():
            assert [s2.engine_split(K[name], l) for l in range(s2.num_levels())] == v


def _sweep32(d, n, M, split, batch=1, delta=False):
    # one FP32 smoothing step on the finest level (red, then black), split forced
    alphas = [0.45] if batch == 1 else list(np.linspace(0.2, 0.8, batch))
    s = G.Solver(d, n, M, 1.0, alphas if batch > 1 else 0.45)
    with s:
        s.set_precision(G.MGWR_MIXED)
        s.set_engine_split(K["sweep32"], split)
        l = s.num_levels() - 1
        N = n ** d
        shape = (N, M) if batch == 1 else (batch, N, M)
        u = inputs.random_field(N * batch, M, seed=3).reshape(shape)
        f = inputs.random_field(N * batch, M, seed=4, scale=2.0 * d * (n + 1) ** 2).reshape(shape)
        s.field_set(G.MGWR_H32, l, G.MGWR_U, u)
        s.field_set(G.MGWR_H32, l, G.MGWR_F, f)
        if delta:
            out = s.smooth_defect(G.MGWR_H32, l)
            res = (s.field_get(G.MGWR_H32, l, G.MGWR_U), s.field_get(G.MGWR_H32, l, G.MGWR_R), out)
        else:
            s.smooth(G.MGWR_H32, l, G.MGWR_RED)
            s.smooth(G.MGWR_H32, l, G.MGWR_BLACK)
            res = (s.field_get(G.MGWR_H32, l, G.MGWR_U),)
        used = s.engine_split(K["sweep32"])
    return res, used


@pytest.mark.parametrize("d,n,M,batch", [(1, 15, 64, 1), (1, 63, 128, 1), (2, 15, 64, 1), (2, 31, 256, 1),
                                         (2, 63, 1024, 1), (1, 15, 2048, 1), (2, 7, 4096, 1),
                                         (2, 3, 64, 1), (2, 15, 256, 3), (1, 31, 512, 5)])
@pytest.mark.parametrize("E", [1, 2, 4])
def test_staged_sweep_is_bitwise_the_direct_sweep(d, n, M, batch, E):
    # input lines through bulk copies into shared memory: the same values summed
    # in the same order, on every grid shape (boundary lines, the row-wrapping
    # pairs, an odd last pair) and for batches
    ref, used = _sweep32(d, n, M, E, batch)
    got, used_s = _sweep32(d, n, M, E | G.MGWR_SPLIT_STAGED, batch)
    assert used_s == used | G.MGWR_SPLIT_STAGED
    for a, b in zip(got, ref):
        np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("d,n,M", [(2, 31, 256), (1, 127, 1024)])
def test_staged_sweep_records_the_same_changes(d, n, M):
    ref, _ = _sweep32(d, n, M, 1, delta=True)
    got, _ = _sweep32(d, n, M, 1 | G.MGWR_SPLIT_STAGED, delta=True)
    for a, b in zip(got, ref):
        np.testing.assert_array_equal(a, b)


def test_staged_split_falls_back_and_is_checked():
    with G.Solver(1, 7, 32, 1.0, 0.5) as s:  # M < 64: direct loads
        s.set_precision(G.MGWR_MIXED)
        s.set_engine_split(K["sweep32"], 1 | G.MGWR_SPLIT_STAGED)
        assert s.engine_split(K["sweep32"]) == 1
    with G.Solver(1, 7, 8192, 1.0, 0.5) as s:  # partitioned lines: direct loads
        s.set_engine_split(K["sweep32"], 2 | G.MGWR_SPLIT_STAGED)
        assert s.engine_split(K["sweep32"]) == 2
        with pytest.raises(G.MGWRError):
            s.set_engine_split(K["sweep64"], 1 | G.MGWR_SPLIT_STAGED)
        with pytest.raises(G.MGWRError):
            s.set_engine_split(K["defect32"], 1 | G.MGWR_SPLIT_STAGED)
        with pytest.raises(G.MGWRError):
            s.set_engine_split(K["sweep32"], 3 | G.MGWR_SPLIT_STAGED)


@pytest.mark.parametrize("precision", [G.MGWR_MIXED, G.MGWR_MIXED_DD])
def test_staged_solve_equals_direct_solve(precision):
    d, n, M = 2, 63, 512
    f = inputs.Problem(d, n, M, 1.0, 0.6, "t2").rhs()
    out = []
    for split in (1, 1 | G.MGWR_SPLIT_STAGED):
        with G.Solver(d, n, M, 1.0, 0.6) as s:
            s.set_precision(precision)
            s.set_engine_split(K["sweep32"], split)
            s.set_rhs(f)
            st = s.solve(1, 1, 1, tol=1e-10, max_cycles=40)
            out.append((s.solution(), st.cycles, st.relres))
    np.testing.assert_array_equal(out[0][0], out[1][0])
    assert out[0][1:] == out[1][1:]


TENSOR_SHAPES = [(1, 63, 64, 1), (2, 15, 128, 1), (2, 31, 256, 1), (1, 255, 256, 1), (2, 63, 256, 3),
                 (2, 3, 64, 1), (1, 7, 128, 2), (2, 127, 64, 1)]


@pytest.mark.parametrize("d,n,M,batch", TENSOR_SHAPES)
def test_tensor_sweep_agrees_with_the_fft_sweep(d, n, M, batch):
    # the dense Toeplitz product on the tensor cores (bf16 x 3 pieces, FP32
    # accumulation) against the FFT engine: both FP32-accurate, not bitwise
    ref, _ = _sweep32(d, n, M, 1, batch)
    got, used = _sweep32(d, n, M, 1 | G.MGWR_SPLIT_TENSOR, batch)
    assert used == 1 | G.MGWR_SPLIT_TENSOR
    for a, b in zip(got, ref):
        assert rel(a, b) <= 2e-6, rel(a, b)


@pytest.mark.parametrize("d,n,M", [(1, 63, 64), (2, 15, 128), (2, 31, 256)])
def test_tensor_sweep_matches_the_oracle(d, n, M):
    W = omg.WRMG(d, n, M, 1.0, 0.45)
    got, _ = _sweep32(d, n, M, 1 | G.MGWR_SPLIT_TENSOR)
    N = n ** d
    u = inputs.random_field(N, M, seed=3)
    f = inputs.random_field(N, M, seed=4, scale=2.0 * d * (n + 1) ** 2)
    W.sweep(W.finest, u, f, 0)
    W.sweep(W.finest, u, f, 1)
    assert rel(got[0], u) <= 2e-5


@pytest.mark.parametrize("d,n,M", [(2, 31, 256), (1, 127, 128)])
def test_tensor_sweep_records_its_changes(d, n, M):
    ref, _ = _sweep32(d, n, M, 1, delta=True)
    got, _ = _sweep32(d, n, M, 1 | G.MGWR_SPLIT_TENSOR, delta=True)
    assert rel(got[0], ref[0]) <= 2e-6
    assert rel(got[1], ref[1]) <= 1e-4  # the defect: differences of nearly equal values


def test_tensor_split_falls_back_and_is_checked():
    with G.Solver(2, 7, 512, 1.0, 0.5) as s:  # beyond 256 steps: the FFT engine
        s.set_precision(G.MGWR_MIXED)
        s.set_engine_split(K["sweep32"], 1 | G.MGWR_SPLIT_TENSOR)
        assert s.engine_split(K["sweep32"]) == 1
        with pytest.raises(G.MGWRError):
            s.set_engine_split(K["sweep64"], 1 | G.MGWR_SPLIT_TENSOR)
        with pytest.raises(G.MGWRError):
            s.set_engine_split(K["sweep32"], 1 | G.MGWR_SPLIT_TENSOR | G.MGWR_SPLIT_STAGED)


@pytest.mark.parametrize("precision", [G.MGWR_MIXED, G.MGWR_MIXED_DD])
@pytest.mark.parametrize("d,n,M,batch", [(2, 63, 256, 1), (1, 255, 128, 1), (2, 31, 64, 4)])
def test_tensor_solve_converges_like_the_fft_solve(precision, d, n, M, batch):
    alphas = 0.6 if batch == 1 else list(np.linspace(0.2, 0.8, batch))
    if batch == 1:
        f = inputs.Problem(d, n, M, 1.0, 0.6, "t2").rhs()
    else:
        f = np.stack([inputs.Problem(d, n, M, 1.0, float(a), "t2").rhs() for a in alphas])
    out = []
    for split in (1, 1 | G.MGWR_SPLIT_TENSOR):
        with G.Solver(d, n, M, 1.0, alphas) as s:
            s.set_precision(precision)
            s.set_engine_split(K["sweep32"], split)
            s.set_rhs(f)
            st = s.solve(1, 1, 1, tol=1e-10, max_cycles=40)
            out.append((s.solution(), st.outer))
    assert abs(out[1][1] - out[0][1]) <= 1  # outer steps: different FP32 rounding may need one more
    assert rel(out[1][0], out[0][0]) <= 1e-9


# register-pass engine: every transform length it serves (L = 2M = 128 .. 8192),
# 1-D and 2-D, batches, grids with fewer line pairs than one block holds
RADIX_SHAPES = [(1, 63, 64, 1), (2, 15, 128, 1), (2, 31, 256, 1), (1, 255, 512, 1), (2, 63, 1024, 1),
                (1, 31, 2048, 1), (2, 15, 4096, 1), (2, 3, 64, 1), (1, 7, 4096, 2), (2, 63, 256, 3),
                (2, 127, 64, 1), (1, 1023, 128, 1)]


@pytest.mark.parametrize("d,n,M,batch", RADIX_SHAPES)
def test_radix_sweep_agrees_with_the_fft_sweep(d, n, M, batch):
    # radix-32 register passes against the radix-8 shared-memory cascade: both
    # FP32 transforms of the same convolution, not bitwise
    ref, _ = _sweep32(d, n, M, 1, batch)
    got, used = _sweep32(d, n, M, 1 | G.MGWR_SPLIT_RADIX, batch)
    assert used == 1 | G.MGWR_SPLIT_RADIX
    for a, b in zip(got, ref):
        assert rel(a, b) <= 2e-6, rel(a, b)


@pytest.mark.parametrize("form", [1, 4])
@pytest.mark.parametrize("d,n,M", [(1, 63, 64), (2, 15, 512), (2, 31, 2048), (2, 7, 4096)])
def test_radix_sweep_matches_the_oracle(d, n, M, form):
    W = omg.WRMG(d, n, M, 1.0, 0.45)
    got, _ = _sweep32(d, n, M, form | G.MGWR_SPLIT_RADIX)
    N = n ** d
    u = inputs.random_field(N, M, seed=3)
    f = inputs.random_field(N, M, seed=4, scale=2.0 * d * (n + 1) ** 2)
    W.sweep(W.finest, u, f, 0)
    W.sweep(W.finest, u, f, 1)
    assert rel(got[0], u) <= 2e-5


@pytest.mark.parametrize("d,n,M", [(2, 31, 256), (1, 127, 1024), (2, 15, 4096)])
def test_radix_sweep_records_its_changes(d, n, M):
    ref, _ = _sweep32(d, n, M, 1, delta=True)
    got, _ = _sweep32(d, n, M, 1 | G.MGWR_SPLIT_RADIX, delta=True)
    assert rel(got[0], ref[0]) <= 2e-6
    assert rel(got[1], ref[1]) <= 1e-4  # the defect: differences of nearly equal values


def test_radix_split_falls_back_and_is_checked():
    with G.Solver(2, 7, 32, 1.0, 0.5) as s:  # below 64 steps: the shared-memory engine
        s.set_precision(G.MGWR_MIXED)
        s.set_engine_split(K["sweep32"], 1 | G.MGWR_SPLIT_RADIX)
        assert s.engine_split(K["sweep32"]) == 1
        with pytest.raises(G.MGWRError):
            s.set_engine_split(K["sweep64"], 1 | G.MGWR_SPLIT_RADIX)
        with pytest.raises(G.MGWRError):
            s.set_engine_split(K["sweep32"], 1 | G.MGWR_SPLIT_RADIX | G.MGWR_SPLIT_TENSOR)


@pytest.mark.parametrize("precision", [G.MGWR_MIXED, G.MGWR_MIXED_DD])
@pytest.mark.parametrize("d,n,M,batch", [(2, 63, 256, 1), (1, 255, 2048, 1), (2, 31, 64, 4),
                                         (2, 31, 4096, 1)])
def test_radix_solve_converges_like_the_fft_solve(precision, d, n, M, batch):
    alphas = 0.6 if batch == 1 else list(np.linspace(0.2, 0.8, batch))
    if batch == 1:
        f = inputs.Problem(d, n, M, 1.0, 0.6, "t2").rhs()
    else:
        f = np.stack([inputs.Problem(d, n, M, 1.0, float(a), "t2").rhs() for a in alphas])
    out = []
    for split in (1, 1 | G.MGWR_SPLIT_RADIX):
        with G.Solver(d, n, M, 1.0, alphas) as s:
            s.set_precision(precision)
            s.set_engine_split(K["sweep32"], split)
            s.set_rhs(f)
            st = s.solve(1, 1, 1, tol=1e-10, max_cycles=40)
            out.append((s.solution(), st.outer))
    assert abs(out[1][1] - out[0][1]) <= 1  # outer steps: different FP32 rounding may need one more
    assert rel(out[1][0], out[0][0]) <= 1e-9


@pytest.mark.parametrize("d,n,M,batch", [(2, 63, 1024, 1), (1, 255, 512, 1), (2, 15, 4096, 1),
                                         (2, 31, 64, 2), (1, 127, 128, 1), (2, 63, 256, 3)])
def test_radix_paired_first_pass_matches_the_single_one(d, n, M, batch):
    # 2 | MGWR_SPLIT_RADIX: the same butterflies with 8-byte gathers and stores;
    # the compiler may fuse multiply-adds differently in the two code shapes, so
    # the fields agree to a few FP32 roundings of their scale, not bitwise
    a, used_a = _sweep32(d, n, M, 1 | G.MGWR_SPLIT_RADIX, batch, delta=True)
    b, used_b = _sweep32(d, n, M, 2 | G.MGWR_SPLIT_RADIX, batch, delta=True)
    assert (used_a, used_b) == (1 | G.MGWR_SPLIT_RADIX, 2 | G.MGWR_SPLIT_RADIX)
    for x, y in zip(a[:2], b[:2]):
        assert np.abs(x - y).max() <= 16 * 2.0 ** -24 * np.abs(x).max()


# resident blocks: grids whose pairs take several rounds of the blocks (2-D
# 63 x 63 at M = 2048 and 4096, 1-D 4095 at M = 256) and batches of more
# instances than SMs (one block per instance)
RESIDENT_SHAPES = RADIX_SHAPES + [(2, 63, 2048, 1), (2, 63, 4096, 1), (1, 4095, 256, 1),
                                  (2, 15, 512, 200), (2, 7, 4096, 3)]


@pytest.mark.parametrize("d,n,M,batch", RESIDENT_SHAPES)
def test_radix_resident_sweep_is_the_paired_sweep(d, n, M, batch):
    # 4 | MGWR_SPLIT_RADIX: the paired arithmetic, with the spectrum and the
    # twiddle bases read from shared memory by blocks that loop over the line
    # pairs: the same values in the same order, so the same bits, changes included
    a, used_a = _sweep32(d, n, M, 2 | G.MGWR_SPLIT_RADIX, batch, delta=True)
    b, used_b = _sweep32(d, n, M, 4 | G.MGWR_SPLIT_RADIX, batch, delta=True)
    assert (used_a, used_b) == (2 | G.MGWR_SPLIT_RADIX, 4 | G.MGWR_SPLIT_RADIX)
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)


def test_peak_probe_measures_both_pipes():
    # the FP64 / FP32 FMA-chain peaks: positive, FP32 far above FP64 on this part
    # (GB300: 1/64 of the rate), neither above the nominal per-clock rates at the
    # highest SM clock (152 SMs: 2 FP64 and 128 FP32 FMA per clock, 2.2 GHz bound)
    p = G.peak_probe()
    assert 0.05 < p["fp64_tflops"] <= 152 * 2 * 2 * 2.2e9 / 1e12
    assert 1.0 < p["fp32_tflops"] <= 152 * 128 * 2 * 2.2e9 / 1e12
    assert p["fp32_tflops"] > 8 * p["fp64_tflops"]
