"""GPU parity of the inner cycles of the refinement modes, through the C ABI.

The mixed modes (MGWR_MIXED, MGWR_MIXED_DD) run their WRMG cycles (Algorithm 1)
on the FP32 hierarchy and MGWR_DD on the double-float hierarchy.  An outer FP64
refinement converges to the right answer even when an inner cycle is wrong
(only more slowly), so these tests compare the inner cycles themselves, iterate
by iterate, with the oracle's FP64 cycle on the same inputs: V(1,1), V(0,1) and
W(1,0), 1-D and 2-D, M up to 4096, every FP32 smoother variant the tuner can pick
(bulk-copy staged input lines, tensor-core dense Toeplitz product, register-pass
FFT engine, single and paired first pass) besides the shared-memory FFT engine.  They also compare the fused FP32 defect-restriction kernel, which
only a cycle reaches, with the oracle's restriction of the defect after one
smoothing step, and with the unfused kernels bit for bit.

Tolerances.  FP32: every half-sweep and defect rounds each value to about
eps32 * log2(2M) of its line's scale (the 2e-5 bound of the FP32 component
tests).  A cycle then turns the defect's rounding into an iterate error through
the coarse-grid correction: the defect after a smoothing step is h^-2 times sums
of the changes u_new - u_old, each carrying an absolute error of eps32 |u|, and
the correction solves A e = r with it, so the iterate deviates from the exact
cycle's by up to about eps32 kappa(A_h) |u|, kappa(A_h) = (4d/h^2) / (d pi^2) =
4 / (pi h)^2 (the same limit bounds one step of the mixed refinement).  The
tests allow twice that, and at least the component bound: 2e-5 on the 2-D
15 x 15 grid, 1e-4 on 31 x 31, 4e-4 on 1-D 63, 1.6e-3 on 1-D 127, all of the
field's maximum (a wrong stencil, weight, colour or boundary tap is an O(1)
error).  Double-float carries about 48 bits (2^-48 = 3.6e-15) times the same
kappa: 1e-10 of the field's maximum per iterate bounds it on these grids.
"""
import math

import numpy as np
import pytest

from oracle import mgwr as omg
from paper_1608_05400_gb300 import inputs
from paper_1608_05400_gb300 import mgwr as G

pytestmark = pytest.mark.gpu

TOL32 = 2e-5
TOLDD = 1e-10


def rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def tol32(n):
    """FP32 cycle iterates: twice eps32 * kappa(A_h), kappa = 4 / (pi h)^2, h = 1/(n+1),
    and at least the FP32 component bound."""
    return max(TOL32, 2.0 * 2.0 ** -24 * 4.0 * (n + 1) ** 2 / math.pi ** 2)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    G.load()


# (d, n, M, (nu1, nu2, gamma), cycles compared)
CASES = [
    (2, 31, 64, (1, 1, 1), 3),
    (2, 15, 256, (0, 1, 1), 3),
    (2, 31, 128, (1, 0, 2), 3),
    (1, 63, 64, (1, 1, 1), 3),
    (1, 127, 512, (0, 1, 1), 3),
    (2, 15, 1024, (1, 1, 1), 2),
    (2, 15, 4096, (1, 1, 1), 2),
]

# launch shape of the FP32 sweep: the FFT engine, its bulk-copy staged form, the
# tensor-core form (M = 64, 128, 256 only) or the register-pass engine (single
# or paired first pass)
VARIANTS = {"fft": 1, "staged": 1 | G.MGWR_SPLIT_STAGED, "tensor": 1 | G.MGWR_SPLIT_TENSOR,
            "radix": 1 | G.MGWR_SPLIT_RADIX, "radix2": 2 | G.MGWR_SPLIT_RADIX}


def _run(precision, hier, tol, d, n, M, cyc, count, order, split=None):
    nu1, nu2, gamma = cyc
    name = "text" if order == G.MGWR_ORDER_TEXT else "table"
    W = omg.WRMG(d, n, M, 1.0, 0.6, order=name)
    with G.Solver(d, n, M, 1.0, 0.6) as s:
        s.set_precision(precision)
        s.set_order(order)
        if split is not None:
            s.set_engine_split(G.KERNEL_CLASSES.index("sweep32"), split)
        L = s.num_levels() - 1
        f = inputs.random_field(n ** d, M, seed=5)
        if hier == G.MGWR_H32:
            f = f.astype(np.float32).astype(np.float64)  # the values the FP32 fields hold
        u = np.zeros_like(f)
        s.field_set(hier, L, G.MGWR_F, f)
        s.field_set(hier, L, G.MGWR_U, u)
        for k in range(count):
            s.cycle(hier, gamma, nu1, nu2)
            u = W.cycle(L, u, f, nu1, nu2, gamma)
            got = s.field_get(hier, L, G.MGWR_U)
            assert rel(got, u) <= tol, (k, rel(got, u))


@pytest.mark.parametrize("variant", sorted(VARIANTS))
@pytest.mark.parametrize("d,n,M,cyc,count", CASES)
def test_fp32_cycles_match_oracle_iterates(variant, d, n, M, cyc, count):
    if variant == "tensor" and M not in (64, 128, 256):
        pytest.skip("the tensor-core sweep serves M = 64, 128, 256")
    _run(G.MGWR_MIXED, G.MGWR_H32, tol32(n), d, n, M, cyc, count, G.MGWR_ORDER_TEXT,
         VARIANTS[variant])


@pytest.mark.parametrize("d,n,M,cyc,count", CASES)
def test_double_float_cycles_match_oracle_iterates(d, n, M, cyc, count):
    _run(G.MGWR_DD, G.MGWR_HDD, TOLDD, d, n, M, cyc, count, G.MGWR_ORDER_TEXT)


@pytest.mark.parametrize("hier", [G.MGWR_H32, G.MGWR_HDD])
def test_inner_cycles_in_table_order(hier):
    precision, tol = (G.MGWR_MIXED, tol32(63)) if hier == G.MGWR_H32 else (G.MGWR_DD, TOLDD)
    _run(precision, hier, tol, 1, 63, 128, (1, 1, 1), 3, G.MGWR_ORDER_TABLE)


@pytest.mark.parametrize("d,n,M", [(2, 31, 64), (2, 15, 256), (2, 63, 128), (1, 63, 64),
                                   (1, 31, 1024), (2, 7, 4096)])
@pytest.mark.parametrize("order", [G.MGWR_ORDER_TEXT, G.MGWR_ORDER_TABLE])
def test_fused_restriction_matches_oracle(d, n, M, order):
    # one smoothing step, then the full weighting of its defect straight from the
    # black half-sweep's changes (the FP32 cycle's fused kernel): against the
    # oracle's restriction of its direct-sum defect, and bitwise against the
    # unfused pair (defect from the changes written out, then restricted)
    name = "text" if order == G.MGWR_ORDER_TEXT else "table"
    W = omg.WRMG(d, n, M, 1.0, 0.45, order=name)
    with G.Solver(d, n, M, 1.0, 0.45) as s:
        s.set_precision(G.MGWR_MIXED)
        s.set_order(order)
        for l in range(1, s.num_levels()):
            nl = s.level_n(l)
            u = inputs.random_field(nl ** d, M, seed=100 + l).astype(np.float32).astype(np.float64)
            f = inputs.random_field(nl ** d, M, seed=200 + l, scale=W.levels[l].sigma)
            f = f.astype(np.float32).astype(np.float64)
            s.field_set(G.MGWR_H32, l - 1, G.MGWR_U, np.ones(((nl - 1) // 2) ** d * M).reshape(-1, M))
            s.field_set(G.MGWR_H32, l, G.MGWR_U, u)
            s.field_set(G.MGWR_H32, l, G.MGWR_F, f)
            s.smooth_restrict(G.MGWR_H32, l)
            fused = s.field_get(G.MGWR_H32, l - 1, G.MGWR_F)
            assert not s.field_get(G.MGWR_H32, l - 1, G.MGWR_U).any()  # the correction is cleared
            ref_u = u.copy()
            W.smooth(l, ref_u, f, 1)
            ref = omg.restrict_fw(W.defect(l, ref_u, f), d, nl)
            scale = np.abs(f).max() + W.levels[l].sigma * 2 * np.abs(ref_u).max()
            assert np.abs(fused - ref).max() <= TOL32 * scale, (l, np.abs(fused - ref).max() / scale)
            s.field_set(G.MGWR_H32, l, G.MGWR_U, u)
            s.field_set(G.MGWR_H32, l, G.MGWR_F, f)
            s.smooth_defect(G.MGWR_H32, l)
            s.restrict(G.MGWR_H32, l)
            np.testing.assert_array_equal(fused, s.field_get(G.MGWR_H32, l - 1, G.MGWR_F))


@pytest.mark.parametrize("hier", [G.MGWR_H64, G.MGWR_HDD])
def test_smooth_restrict_on_the_wide_hierarchies(hier):
    # the same component on the FP64 and double-float hierarchies (defect written,
    # then restricted) against the oracle
    d, n, M = 2, 31, 128
    W = omg.WRMG(d, n, M, 1.0, 0.45)
    tol = 1e-12 if hier == G.MGWR_H64 else 1e-11
    with G.Solver(d, n, M, 1.0, 0.45) as s:
        if hier == G.MGWR_HDD:
            s.set_precision(G.MGWR_DD)
        l = s.num_levels() - 1
        u = inputs.random_field(n ** d, M, seed=7)
        f = inputs.random_field(n ** d, M, seed=8, scale=W.levels[l].sigma)
        s.field_set(hier, l, G.MGWR_U, u)
        s.field_set(hier, l, G.MGWR_F, f)
        s.smooth_restrict(hier, l)
        ref_u = u.copy()
        W.smooth(l, ref_u, f, 1)
        ref = omg.restrict_fw(W.defect(l, ref_u, f), d, n)
        scale = np.abs(f).max() + W.levels[l].sigma * 2 * np.abs(ref_u).max()
        assert np.abs(s.field_get(hier, l - 1, G.MGWR_F) - ref).max() <= tol * scale


@pytest.mark.parametrize("precision", [G.MGWR_MIXED, G.MGWR_MIXED_DD])
@pytest.mark.parametrize("d,n,M", [(2, 31, 1024), (1, 255, 64), (2, 15, 4096), (1, 63, 512)])
def test_outer_defect_of_a_refinement_step_matches_oracle(precision, d, n, M):
    # One outer step of the refinement, then its outer defect, which becomes the
    # FP32 right-hand side of the next step's inner cycles: with the switch at 0
    # every outer defect takes the FP32-convolution form (T_M u by one FP32
    # convolution of the rounded iterate, f - A_h u in the outer precision), whose
    # error is about 1e-6 of |T_M u|; with the switch at +inf the defect is exact
    # before its rounding to FP32.  Both against the oracle's direct-sum defect.
    W = omg.WRMG(d, n, M, 1.0, 0.55)
    f = inputs.random_field(n ** d, M, seed=21)
    L = W.finest
    for switch in (0.0, math.inf):
        with G.Solver(d, n, M, 1.0, 0.55) as s:
            s.set_precision(precision)
            s.set_outer_switch(switch)
            s.set_rhs(f)
            s.solve(1, 1, 1, tol=1e-300, max_cycles=1, allow_noconv=True)
            u = s.solution()
            r32 = s.field_get(G.MGWR_H32, L, G.MGWR_F)
        ref = W.defect(L, u, f)
        tu = np.abs(u @ W.Tm.T).max()
        err = np.abs(r32 - ref).max()
        rounding = 2.0 ** -23 * np.abs(ref).max()
        bound = (2e-6 * tu if switch == 0.0 else 0.0) + rounding
        assert err <= bound, (switch, err, bound, tu)


@pytest.mark.parametrize("precision", [G.MGWR_MIXED, G.MGWR_MIXED_DD])
@pytest.mark.parametrize("d,n,M", [(2, 31, 1024), (1, 127, 64), (2, 15, 4096), (1, 63, 16)])
def test_carried_defect_from_a_full_anchor_matches_oracle(precision, d, n, M):
    # One outer step with a full defect (switch +inf) leaves u_old; the next solve
    # computes the full defect of u_old (the anchor, kept in double-float) and,
    # with the switch at 0, carries it through one more step:
    # r = r_old - (T_M (x) I + A_h) e, e = u_new - u_old.  Against the oracle's
    # direct-sum defect of u_new, the FP32 right-hand side it leaves errs by the
    # FP32 convolution of e (about 1e-6 of |T_M e|), its rounding to FP32, and
    # the anchor's own rounding (a few FP64 or double-float units of the defect's
    # terms); carrying from the wrong defect (f, or the anchor's FP32 rounding)
    # misses by |A u_old| or eps32 |r_old|.
    W = omg.WRMG(d, n, M, 1.0, 0.55)
    f = inputs.random_field(n ** d, M, seed=23)
    L = W.finest
    with G.Solver(d, n, M, 1.0, 0.55) as s:
        s.set_precision(precision)
        s.set_inner_cycles(1)
        s.set_outer_switch(math.inf)
        s.set_rhs(f)
        s.solve(1, 1, 1, tol=1e-300, max_cycles=1, allow_noconv=True)
        u_old = s.solution()
        s.set_outer_switch(0.0)
        s.solve(1, 1, 1, tol=1e-300, max_cycles=1, allow_noconv=True)
        u_new = s.solution()
        r32 = s.field_get(G.MGWR_H32, L, G.MGWR_F)
    ref = W.defect(L, u_new, f)
    e = u_new - u_old
    te = np.abs(e @ W.Tm.T).max()
    err = np.abs(r32 - ref).max()
    terms = np.abs(f).max() + np.abs(u_old @ W.Tm.T).max() + 4 * d * (n + 1) ** 2 * np.abs(u_old).max()
    anchor = (2.0 ** -44 if precision == G.MGWR_MIXED_DD else 2.0 ** -50) * terms
    bound = 2e-6 * te + 2.0 ** -23 * np.abs(ref).max() + anchor
    assert err <= bound, (err, bound, te, anchor)
    # the step made progress from the anchor, so the check is not vacuous
    assert np.abs(ref).max() < 0.5 * np.abs(W.defect(L, u_old, f)).max()


@pytest.mark.parametrize("precision", [G.MGWR_MIXED, G.MGWR_MIXED_DD])
def test_carried_defects_save_full_defects_and_solve_the_same(precision):
    # default switch (carry while the defect is >= 1e-2 of the anchor's) against
    # +inf (every outer defect in full): the same solution to the tolerance, about
    # the same outer steps, fewer full outer defects, and the reported relative
    # defect is the full one of the returned iterate
    d, n, M, tol = 2, 63, 256, 1e-10
    prob = inputs.Problem(d, n, M, 1.0, 0.6, "t2")
    full_class = "defect64" if precision == G.MGWR_MIXED else "defect_dd"
    out = {}
    for switch in (None, math.inf):
        with G.Solver(d, n, M, 1.0, 0.6) as s:
            s.set_precision(precision)
            if switch is not None:
                s.set_outer_switch(switch)
            s.set_rhs(prob.rhs())
            s.profile(True)
            st = s.solve(1, 1, 1, tol=tol, max_cycles=40)
            prof = s.profile_read()
            u = s.solution()
            W = omg.WRMG(d, n, M, 1.0, 0.6)
            rel_o = np.abs(W.defect(W.finest, u, prob.rhs())).max() / np.abs(prob.rhs()).max()
            out[switch] = (st, prof[full_class]["launches"], prof["defect32"]["launches"], u, rel_o)
            if precision == G.MGWR_MIXED and switch is None:
                # to 1e-10 every full defect (anchors and the stop) takes the
                # double-float-convolution form; at +inf all are FP64
                assert prof["defect_dd"]["launches"] >= 1 and prof["defect64"]["launches"] == 0
            if precision == G.MGWR_MIXED and switch is not None:
                assert prof["defect_dd"]["launches"] == 0
    (st_c, full_c, carried_c, u_c, rel_c), (st_f, full_f, carried_f, u_f, rel_f) = out[None], out[math.inf]
    assert st_c.status == st_f.status == G.MGWR_OK
    assert carried_f == 0 and carried_c > 0
    assert full_c < full_f
    assert abs(st_c.outer - st_f.outer) <= 1
    # the reported defect against the oracle's: both in FP64 (or double-float),
    # summed in different orders, so they differ by a few units of the terms
    fmax = np.abs(prob.rhs()).max()
    terms = fmax + 4 * d * (n + 1) ** 2 * np.abs(u_c).max() + np.abs(u_c @ W.Tm.T).max()
    # (MGWR_MIXED's stop to 1e-10 uses its double-float-convolution defect:
    # about 2^-44 of |T_M u| besides the FP64 stencil's rounding)
    eps = 2.0 ** -40
    assert rel_c <= tol and abs(st_c.relres - rel_c) <= 1e-3 * rel_c + eps * terms / fmax
    assert rel(u_c, u_f) <= 1e-8


@pytest.mark.parametrize("d,n,M", [(2, 31, 1024), (1, 255, 64), (2, 15, 4096), (1, 63, 16)])
def test_double_float_anchor_and_the_step_carried_from_it(d, n, M):
    # MGWR_MIXED to a tolerance of at least 1e-10 renews its anchors with T_M u
    # by a double-float convolution of the split FP64 iterate (stencil and source
    # in FP64).  Driven step by step: the first step with the switch at 2 (no
    # carry: the defect is below twice its anchor) takes that form, the second
    # with the switch at 0 carries from its double-float result.  Each FP32
    # right-hand side against the oracle's direct-sum defect of the iterate: the
    # anchor errs by about 2^-44 |T_M u| besides its rounding to FP32, the
    # carried one by that plus the FP32 convolution of the step's correction.
    W = omg.WRMG(d, n, M, 1.0, 0.45)
    f = inputs.random_field(n ** d, M, seed=29)
    L = W.finest
    with G.Solver(d, n, M, 1.0, 0.45) as s:
        s.set_precision(G.MGWR_MIXED)
        s.set_rhs(f)
        s.set_outer_switch(2.0)
        with G.Group() as g:
            g.add(s, 1, 1, 1, tol=1e-9, max_cycles=4)
            g.step()
            u1 = s.solution()
            r1 = s.field_get(G.MGWR_H32, L, G.MGWR_F)
            s.set_outer_switch(0.0)
            g.step()
            u2 = s.solution()
            r2 = s.field_get(G.MGWR_H32, L, G.MGWR_F)
            g.run()
    fmax = np.abs(f).max()
    tu1 = np.abs(u1 @ W.Tm.T).max()
    ref1 = W.defect(L, u1, f)
    fp64 = 2.0 ** -50 * (fmax + tu1 + 4 * d * (n + 1) ** 2 * np.abs(u1).max())
    anchor_err = 2.0 ** -40 * tu1 + fp64
    err1 = np.abs(r1 - ref1).max()
    assert err1 <= anchor_err + 2.0 ** -23 * np.abs(ref1).max(), (err1, anchor_err)
    ref2 = W.defect(L, u2, f)
    te = np.abs((u2 - u1) @ W.Tm.T).max()
    err2 = np.abs(r2 - ref2).max()
    bound2 = anchor_err + 2e-6 * te + 2.0 ** -23 * np.abs(ref2).max() + fp64
    assert err2 <= bound2, (err2, bound2, te)
    assert np.abs(ref2).max() < 0.5 * np.abs(ref1).max()
