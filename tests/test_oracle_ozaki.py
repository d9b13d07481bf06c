"""Pins of O2 (the Ozaki emulation) against the mathematics and against O1.

Each pin is chosen so that a plausible slip in O2 fails at least one of them;
``test_planted_mistakes_are_caught`` plants such slips (in the oracle, on the
CPU) and checks that the pins notice.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import synthetic_inputs as si
from oracle import exact, ozaki

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("w", [8, 9])
def test_balanced_digits_reassemble(w):
    R, h = 1 << w, 1 << (w - 1)
    rng = np.random.default_rng(3)
    for _ in range(2000):
        nd = int(rng.integers(1, 40))
        lim = 1 << (w * nd - 1)
        X = int(rng.integers(-2**62, 2**62)) * (1 << int(rng.integers(0, max(1, w * nd - 63)))) % lim
        X = X if rng.random() < 0.5 else -X
        d = ozaki.balanced_digits(X, nd, w)
        assert sum(v * R ** (nd - 1 - t) for t, v in enumerate(d)) == X
        assert all(-h <= v <= h - 1 for v in d[1:])
        assert -h <= d[0] <= h
    # extremes
    for X in ((1 << (3 * w - 1)) - 1, -((1 << (3 * w - 1)) - 1), 0, 1, -1, h, -h, h - 1):
        d = ozaki.balanced_digits(X, 3, w)
        assert sum(v * R ** (2 - t) for t, v in enumerate(d)) == X
    d = ozaki.balanced_digits((1 << (3 * w - 1)) - 1, 3, w)
    assert d[0] == h   # the top digit may reach +-2^(w-1) (still exact in bf16 for w <= 9)


@pytest.mark.parametrize("w", [8, 9])
def test_fixed_point_truncation(w):
    """0 <= |a| 2^(ws-1-E) - |X| < 1 and |X| < 2^(ws-1) for |a| < 2^E."""
    p = 256
    A = si.random_matrix(8, 12, p, 5, "uniform_exp")
    s = 20
    E = ozaki.row_exponents(A, "rows")
    for i in range(8):
        for l in range(12):
            for c in range(2):
                v = exact.component(A, c, i, l)
                a = abs(exact.to_fraction(v))
                assert a < Fraction(2) ** E[i]
                X, lossless = ozaki.fixed_point(v, E[i], s, w)
                scaled = a * Fraction(2) ** (w * s - 1 - E[i])
                assert 0 <= scaled - abs(X) < 1
                assert abs(X) < 2 ** (w * s - 1)
                assert lossless == (scaled == abs(X))
                assert (X < 0) == (v[0] < 0) or X == 0


def test_vectorised_split_matches_scalar_definition():
    p = 192
    A = si.random_matrix(6, 9, p, 8, "uniform_exp", zero_frac=0.15)
    s = 26
    sp = ozaki.split_operand(A, s, "A", "3m")
    spB = ozaki.split_operand(A, s, "B", "3m")
    for i in range(6):
        for l in range(9):
            xr, _ = ozaki.fixed_point(exact.component(A, 0, i, l), sp.E[i], s)
            xi, _ = ozaki.fixed_point(exact.component(A, 1, i, l), sp.E[i], s)
            assert list(sp.digits["re"][:, i, l]) == ozaki.balanced_digits(xr, s)
            assert list(sp.digits["im"][:, i, l]) == ozaki.balanced_digits(xi, s)
            assert list(sp.digits["sum"][:, i, l]) == ozaki.balanced_digits(xr + xi, s + 1)
            yr, _ = ozaki.fixed_point(exact.component(A, 0, i, l), spB.E[l], s)
            assert list(spB.digits["re"][:, l, i]) == ozaki.balanced_digits(yr, s)


def test_row_exponent_is_the_row_maximum():
    A = si.random_matrix(10, 7, 128, 9, "uniform_exp", zero_frac=0.3)
    A.limb[:, :, 4, :] = 0      # an all-zero row
    E = ozaki.row_exponents(A, "rows")
    assert E[4] is None
    for i in range(10):
        if i == 4:
            continue
        exps = [int(A.exp[c, i, l]) for c in range(2) for l in range(7) if np.any(A.limb[c, :, i, l])]
        assert E[i] == max(exps)


def _exact_scaled(A, B, r):
    return ozaki.exact_accumulators(A, B, r.splitA, r.splitB, r.params)


@pytest.mark.parametrize("method", ["4m", "3m"])
@pytest.mark.parametrize("w", [8, 9])
def test_all_pairs_and_lossless_split_give_the_exact_product(method, w):
    """Special case: P = every pair and no digit dropped -> Acc * 2^scale == T exactly."""
    p = 128
    A = si.random_matrix(5, 8, p, 12, "uniform_exp")
    B = si.random_matrix(8, 4, p, 13, "uniform_exp", zero_frac=0.1)
    prm = ozaki.make_params(p, 8, method, guard=60, w=w)
    r = ozaki.ozaki_cgemm(A, B, p, method, guard=60, Q=2 * prm.s + 2, w=w)
    assert all(r.splitA.lossless) and all(r.splitB.lossless)
    T = _exact_scaled(A, B, r)
    for comp in ("re", "im"):
        for i in range(5):
            for j in range(4):
                assert Fraction(int(r.acc[comp][i, j])) == T[comp][i, j]
                assert ozaki.entry_bound(r.params, r.splitA, r.splitB, i, j, comp)[0] == 0
    assert r.certified.all()
    assert exact.equal_arrays(r.C, exact.rounded_cgemm(A, B, p))


@pytest.mark.parametrize("method,dist,guard", [("4m", "uniform", 8), ("3m", "uniform", 8),
                                                ("4m", "uniform_exp", 0), ("3m", "uniform_exp", 4)])
@pytest.mark.parametrize("w", [8, 9])
def test_truncation_bound_holds(method, dist, guard, w):
    """|Acc - T| <= b 2^beta for the paper's triangle, lossy split included."""
    p = 128
    A = si.random_matrix(6, 10, p, 14, dist)
    B = si.random_matrix(10, 5, p, 15, dist)
    r = ozaki.ozaki_cgemm(A, B, p, method, guard=guard, w=w)
    T = _exact_scaled(A, B, r)
    worst = Fraction(0)
    for comp in ("re", "im"):
        for i in range(6):
            for j in range(5):
                b, beta = ozaki.entry_bound(r.params, r.splitA, r.splitB, i, j, comp)
                err = abs(Fraction(int(r.acc[comp][i, j])) - T[comp][i, j])
                assert err <= b * Fraction(2) ** beta
                worst = max(worst, err / (b * Fraction(2) ** beta))
    assert worst > Fraction(1, 1 << 20)   # the bound is not vacuous


@pytest.mark.parametrize("method", ["4m", "3m"])
@pytest.mark.parametrize("case", ["real", "imaginary_B", "small_imaginary", "tiny_imaginary"])
def test_bound_with_zero_planes_holds(method, case):
    """The data-dependent bound (live dropped pairs, truncation only where both components
    are nonzero) still bounds |Acc - T| on every entry, including an imaginary part so small
    that it truncates to zero digits (the lossy terms then carry it); for real inputs the
    imaginary bound is exactly zero, so every imaginary component is certified."""
    p = 128
    A = si.random_matrix(6, 12, p, 641, "uniform_exp")
    B = si.random_matrix(12, 5, p, 642, "uniform_exp")
    if case == "real":
        for X in (A, B):
            X.limb[1] = 0; X.sign[1] = 0; X.exp[1] = si.INT32_MIN
    elif case == "imaginary_B":
        B.limb[0] = 0; B.sign[0] = 0; B.exp[0] = si.INT32_MIN
    elif case == "small_imaginary":
        A, B = _scaled_imaginary(A, -70), _scaled_imaginary(B, -50)
    else:
        A = _scaled_imaginary(A, -600)        # below every digit of the grid: lossy rows
    r = ozaki.ozaki_cgemm(A, B, p, method)
    T = _exact_scaled(A, B, r)
    for comp in ("re", "im"):
        for i in range(6):
            for j in range(5):
                b, beta = ozaki.entry_bound(r.params, r.splitA, r.splitB, i, j, comp)
                err = abs(Fraction(int(r.acc[comp][i, j])) - T[comp][i, j])
                assert err <= b * Fraction(2) ** beta, (case, comp, i, j)
                if case == "real" and comp == "im":
                    assert b == 0 and err == 0
    if case == "real":
        assert r.certified[1].all()
    if case == "tiny_imaginary":
        assert not all(r.splitA.lossless)
    assert exact.equal_arrays(r.C, exact.rounded_cgemm(A, B, p)) if hasattr(exact, "equal_arrays") else True


@pytest.mark.parametrize("w", [8, 9])
def test_truncation_bound_is_attained_by_coherent_errors(w):
    """All-ones mantissas truncate almost a full ulp each, all with one sign:
    the error then sits just below the split term of the bound (not far under it)."""
    p, k = 128, 16
    vals = np.zeros((2, 1, k), np.int64)
    A = si.from_integers(vals, p)
    B = si.from_integers(np.zeros((2, k, 1), np.int64), p)
    ones = np.uint64(0xFFFFFFFFFFFFFFFF)
    A.limb[:, :, 0, :] = ones           # Re and Im of A: +(1 - 2^-128) 2^3
    A.exp[:, 0, :] = 3
    B.limb[:, :, :, 0] = ones           # Re of B positive, Im negative: Re = rr - ii adds
    B.exp[:, :, 0] = -2                 # both truncation errors with one sign
    B.sign[1, :, 0] = 1
    s_ = 10
    r = ozaki.ozaki_cgemm(A, B, p, "4m", s=s_, Q=2 * s_ - 2, w=w)   # every pair kept: no dropped term
    assert not r.splitA.lossless[0] and not r.splitB.lossless[0]
    T = _exact_scaled(A, B, r)
    b, beta = ozaki.entry_bound(r.params, r.splitA, r.splitB, 0, 0, "re")
    bound = b * Fraction(2) ** beta
    err = abs(Fraction(int(r.acc["re"][0, 0])) - T["re"][0, 0])
    assert Fraction(99, 100) * bound < err <= bound


def test_group_partition_does_not_change_level_sums():
    p = 128
    A = si.random_matrix(4, 6, p, 16)
    B = si.random_matrix(6, 5, p, 17)
    base = ozaki.make_params(p, 6, "4m")
    spA = ozaki.split_operand(A, base.s, "A", "4m")
    spB = ozaki.split_operand(B, base.s, "B", "4m")
    results = []
    for gmax in (1, 3, 10 ** 6):
        prm = ozaki.Params(p=p, k=6, s=base.s, Q=base.Q, gmax=gmax, method="4m")
        gs, sums = ozaki.group_sums(spA, spB, "ri", prm)
        assert all(g.count <= gmax for g in gs)
        levels = {}
        for g, G in zip(gs, sums):
            levels[g.q] = levels.get(g.q, 0) + G
        results.append(levels)
    for lv in results[1:]:
        assert lv.keys() == results[0].keys()
        assert all(np.array_equal(lv[q], results[0][q]) for q in lv)


def _pair_product(spA, spB, prod, t, u):
    wa, wb = ozaki.PRODUCT_OPERANDS[prod]
    DA = spA.digits[wa][t - spA.first_pos[wa]]
    DB = spB.digits[wb][u - spB.first_pos[wb]]
    return DA @ DB.T          # int64, exact (|entries| <= 128, k small)


def _scaled_imaginary(mat, by):
    out = mat.copy()
    nz = out.limb[1, -1] != 0
    out.exp[1] = np.where(nz, out.exp[1] + by, out.exp[1]).astype(np.int32)
    return out


@pytest.mark.parametrize("method", ["4m", "3m"])
@pytest.mark.parametrize("case", ["real_A", "small_im", "imag_B"])
def test_trimmed_groups_keep_every_group_sum(method, case):
    """Pairs removed by the trimming are exactly zero products (brute force over every
    pair), the trimmed groups are sub-runs of the originals, and no group is added."""
    p, k = 128, 24
    A = si.random_matrix(9, k, p, 611, "uniform")
    B = si.random_matrix(k, 7, p, 612, "uniform")
    if case == "real_A":
        A.limb[1] = 0; A.sign[1] = 0; A.exp[1] = si.INT32_MIN
    elif case == "small_im":
        A, B = _scaled_imaginary(A, -60), _scaled_imaginary(B, -41)
    else:
        B.limb[0] = 0; B.sign[0] = 0; B.exp[0] = si.INT32_MIN
    prm = ozaki.make_params(p, k, method, max_group=4)
    spA = ozaki.split_operand(A, prm.s, "A", method)
    spB = ozaki.split_operand(B, prm.s, "B", method)
    removed = 0
    for prod in prm.products:
        wa, wb = ozaki.PRODUCT_OPERANDS[prod]
        gs = ozaki.groups_for(ozaki.positions(spA, wa, prm.s), ozaki.positions(spB, wb, prm.s), prm.Q, prm.gmax)
        tg = ozaki.trim_groups(spA, spB, prod, gs)
        assert len(tg) == len(gs)
        for g, h in zip(gs, tg):
            full = {(t, g.q - t) for t in range(g.t0, g.t0 + g.count)}
            kept = {(t, h.q - t) for t in range(h.t0, h.t0 + h.count)}
            assert h.q == g.q and kept <= full
            for (t, u) in full - kept:
                assert not np.any(_pair_product(spA, spB, prod, t, u)), (prod, t, u)
                removed += 1
            if h.count:   # the kept ends are live pairs
                for t in (h.t0, h.t0 + h.count - 1):
                    wa_, wb_ = ozaki.PRODUCT_OPERANDS[prod]
                    assert np.any(spA.digits[wa_][t - spA.first_pos[wa_]])
                    assert np.any(spB.digits[wb_][h.q - t - spB.first_pos[wb_]])
    assert removed > 0


def test_trimming_real_inputs_leaves_only_the_real_product():
    """Real A and B: by the digit planes alone 4M keeps only rr and 3M keeps rr and ss
    (= rr); with the method given, ss is not needed either (Im vanishes identically)."""
    p, k = 128, 16
    A = si.random_matrix(6, k, p, 621, "uniform")
    B = si.random_matrix(k, 5, p, 622, "uniform")
    for X in (A, B):
        X.limb[1] = 0; X.sign[1] = 0; X.exp[1] = si.INT32_MIN
    for method, live in (("4m", {"rr"}), ("3m", {"rr", "ss"})):
        prm = ozaki.make_params(p, k, method)
        spA = ozaki.split_operand(A, prm.s, "A", method)
        spB = ozaki.split_operand(B, prm.s, "B", method)
        for prod in prm.products:
            wa, wb = ozaki.PRODUCT_OPERANDS[prod]
            gs = ozaki.groups_for(ozaki.positions(spA, wa, prm.s), ozaki.positions(spB, wb, prm.s), prm.Q, prm.gmax)
            kept = sum(g.count for g in ozaki.trim_groups(spA, spB, prod, gs))
            assert (kept > 0) == (prod in live), (method, prod)
            kept_m = sum(g.count for g in ozaki.trim_groups(spA, spB, prod, gs, method))
            assert (kept_m > 0) == (prod == "rr"), (method, prod)
            assert ozaki.product_needed(spA, spB, prod, method) == (prod in ("rr", "ii"))


def test_trimming_follows_the_smaller_part():
    """Im smaller by 2^-96: about 96/8 leading Im planes are zero, so ii keeps only pairs
    with both digits below that depth and ri/ir only pairs with one of them there."""
    p, k = 256, 16
    A = _scaled_imaginary(si.random_matrix(8, k, p, 631, "uniform"), -96)
    B = _scaled_imaginary(si.random_matrix(k, 8, p, 632, "uniform"), -96)
    prm = ozaki.make_params(p, k, "4m")
    spA = ozaki.split_operand(A, prm.s, "A", "4m")
    spB = ozaki.split_operand(B, prm.s, "B", "4m")
    zA = next(t for t in range(prm.s) if np.any(spA.digits["im"][t]))
    zB = next(t for t in range(prm.s) if np.any(spB.digits["im"][t]))
    assert 10 <= zA <= 12 and 10 <= zB <= 12
    kept = {}
    for prod, (ta, tb) in (("ii", (zA, zB)), ("ri", (0, zB)), ("ir", (zA, 0)), ("rr", (0, 0))):
        wa, wb = ozaki.PRODUCT_OPERANDS[prod]
        gs = ozaki.groups_for(ozaki.positions(spA, wa, prm.s), ozaki.positions(spB, wb, prm.s), prm.Q, prm.gmax)
        tg = ozaki.trim_groups(spA, spB, prod, gs)
        for h in tg:
            for t in range(h.t0, h.t0 + h.count):
                assert t >= ta and h.q - t >= tb
        n_kept = sum(h.count for h in tg)
        bound = sum(1 for g in gs for t in range(g.t0, g.t0 + g.count) if t >= ta and g.q - t >= tb)
        assert n_kept <= bound, prod
        kept[prod] = n_kept
    # the bottom digit planes may be zero too (p < 8s), which trims every product a little;
    # the leading zero planes of the imaginary parts remove most of ii
    assert kept["ii"] < 0.8 * kept["rr"] and kept["ri"] < kept["rr"] and kept["ir"] < kept["rr"]


def test_group_sums_fit_int32_at_the_limit():
    """Gmax * k * 2^(2w-2) <= 2^31 - 1 for the largest supported k; worst-case digits
    |d| = 2^(w-1).  9-bit digits up to k = 2^15 - 1, then 8-bit digits."""
    for k in (1, 7, 256, 2048, 32767, 32768, 131071):
        prm = ozaki.make_params(256, k)
        assert prm.w == (9 if k <= 32767 else 8)
        big = (1 << (prm.w - 1)) ** 2
        assert prm.gmax * k * big <= 2 ** 31 - 1
        assert (prm.gmax + 1) * k * big > 2 ** 31 - 1
    with pytest.raises(ValueError):
        ozaki.make_params(256, 131072)
    with pytest.raises(ValueError):
        ozaki.make_params(256, 32768, w=9)


@pytest.mark.parametrize("method", ["4m", "3m"])
@pytest.mark.parametrize("dist,guard,zf", [("uniform", 40, 0.0), ("uniform_exp", 40, 0.1),
                                           ("uniform", 0, 0.0), ("uniform_exp", 2, 0.2)])
@pytest.mark.parametrize("w", [8, 9])
def test_final_output_equals_o1(method, dist, guard, zf, w):
    """Certified entries round Acc; the rest fall back to the exact value -> == O1."""
    p = 128
    A = si.random_matrix(7, 9, p, 18, dist, zero_frac=zf)
    B = si.random_matrix(9, 6, p, 19, dist, zero_frac=zf)
    r = ozaki.ozaki_cgemm(A, B, p, method, guard=guard, w=w)
    assert exact.equal_arrays(r.C, exact.rounded_cgemm(A, B, p))
    if guard >= 40 and dist == "uniform":
        assert r.certified.all()
    if guard == 0:
        assert not r.certified.all()   # the fallback path is exercised


def test_certification_is_sound_near_midpoints():
    """Values planted right next to a rounding midpoint are never certified wrongly."""
    p = 16
    rng = np.random.default_rng(4)
    for _ in range(3000):
        sh = int(rng.integers(4, 40))
        q = int(rng.integers(1 << (p - 1), 1 << p))
        mid = (2 * q + 1) << (sh - 1)
        off = int(rng.integers(-(1 << (sh - 2)), 1 << (sh - 2)))
        acc = mid + off
        b = int(rng.integers(0, 1 << max(1, sh - 4)))
        if ozaki.certify(acc, b, 0, p):
            for T in (acc - b, acc + b, acc):
                assert exact.round_nearest_even((T, 0), p) == exact.round_nearest_even((acc, 0), p)


def test_paper_division_counts():
    """The tau rule of Alg. 2 with binary64 slices reproduces d = 13 / 25 / 37 (Sec. IV)."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "ozaki_division_counts.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for row in rows:
        p, d = int(row[0]), int(row[1])
        for l in map(int, row[2:]):
            assert ozaki.paper_division_count(p, 53, l) == d
    assert ozaki.paper_slice_bits(53, 1024) == 21


def test_table1_real_products_per_method():
    rows = {l.split()[0]: int(l.split()[2]) for l in open(os.path.join(GOLDEN, "table1_op_counts.txt"))
            if l.strip() and not l.startswith("#")}
    assert len(ozaki.PRODUCTS_4M) == rows["4m"] and len(ozaki.PRODUCTS_3M) == rows["3m"]


# ------------------------------------------------------------ planted mistakes

def _pins_pass(monkeypatch_ctx):
    """Run a compact version of the pins; True if all hold."""
    try:
        for w in (8, 9):
            test_balanced_digits_reassemble(w)
            test_fixed_point_truncation(w)
        for method in ("4m", "3m"):
            test_all_pairs_and_lossless_split_give_the_exact_product(method, 9)
            test_final_output_equals_o1(method, "uniform", 40, 0.0, 9)
            test_final_output_equals_o1(method, "uniform_exp", 0, 0.1, 9)
        test_truncation_bound_holds("3m", "uniform_exp", 4, 9)
        test_truncation_bound_holds("4m", "uniform", 8, 9)
        test_truncation_bound_is_attained_by_coherent_errors(9)
    except AssertionError:
        return False
    return True


def _mutants():
    orig_bd = ozaki.balanced_digits
    orig_bda = ozaki.balanced_digits_array
    orig_acc = ozaki.accumulate
    orig_fp = ozaki.fixed_point
    orig_fpa = ozaki.fixed_point_array
    orig_bexp = ozaki.bound_exponent

    def digit_order(m):      # digits stored least significant first
        m.setattr(ozaki, "balanced_digits", lambda X, nd, w=9: list(reversed(orig_bd(X, nd, w))))
        m.setattr(ozaki, "balanced_digits_array", lambda X, nd, w=9: orig_bda(X, nd, w)[::-1].copy())

    def level_shift(m):      # level weight off by one digit
        m.setattr(ozaki, "accumulate", lambda gs, sums, Q, w=9: orig_acc(gs, sums, Q + 1, w))

    def split_rounding(m):   # magnitude rounded up instead of truncated
        def fp(v, E, s, w=9):
            X, ok = orig_fp(v, E, s, w)
            return (X + (1 if X > 0 else -1 if X < 0 else 0)), ok

        def fpa(N, x, E, s, w=9):
            X, ok = orig_fpa(N, x, E, s, w)
            return np.where(X > 0, X + 1, np.where(X < 0, X - 1, X)), ok
        m.setattr(ozaki, "fixed_point", fp)
        m.setattr(ozaki, "fixed_point_array", fpa)

    def no_drop_bound(m):    # bound forgets the dropped pairs
        m.setattr(ozaki, "drop_bound", lambda *a: 0)

    def bound_scale(m):      # bound expressed in the wrong unit (one digit too coarse)
        m.setattr(ozaki, "bound_exponent", lambda prm: max(0, orig_bexp(prm) - prm.w))

    def im_sign(m):          # 3M imaginary part: + rr instead of - rr
        orig = ozaki.ozaki_cgemm

        def wrapped(*a, **kw):
            r = orig(*a, **kw)
            return r
        orig_acc2 = ozaki.accumulate
        state = {"n": 0}

        def acc(gs, sums, Q, w=9):
            v = orig_acc2(gs, sums, Q, w)
            state["n"] += 1
            # products arrive in the order rr, ii, (ri, ir | ss); flip rr's sign
            return -v if state["n"] % (4 if False else 3) == 1 else v
        m.setattr(ozaki, "accumulate", acc)

    return {"digit_order": digit_order, "level_shift": level_shift,
            "split_rounding": split_rounding, "no_drop_bound": no_drop_bound,
            "bound_scale": bound_scale, "rr_sign": im_sign}


@pytest.mark.parametrize("name", ["digit_order", "level_shift", "split_rounding",
                                  "no_drop_bound", "bound_scale", "rr_sign"])
def test_planted_mistakes_are_caught(monkeypatch, name):
    plant = _mutants()[name]
    with monkeypatch.context() as m:
        plant(m)
        assert not _pins_pass(m), f"planted mistake {name!r} went unnoticed"
    assert _pins_pass(None)
