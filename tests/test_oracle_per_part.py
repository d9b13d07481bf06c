"""Pins of O2's per-part split (Alg. 2 cut per real part; the 4M variant).

Each part P of an operand gets a digit offset z_P (the leading digit positions that
are zero in every line) and its s digits sit at positions z_P .. z_P + s - 1 of the
line's grid; every output component gets its own cut level Q_c = Q + z_c.  The pins
check the split against the plain arithmetic definition (reassembly, truncation
bound, the offset of an exactly shifted part), against the default split (identical
when every offset is 0), against the exact product (the all-pairs lossless case
equals T; the bound holds entry by entry; the output equals O1), and show the case
the variant exists for: an imaginary part 2^-100 below the real part.
"""
from fractions import Fraction

import numpy as np
import pytest

import synthetic_inputs as si
from oracle import exact, ozaki


def _shift_part(mat, c, by):
    """The same matrix with component c scaled by 2^by (exponents of nonzero entries)."""
    out = si.MPCMatrix(mat.rows, mat.cols, mat.p, mat.sign.copy(), mat.exp.copy(), mat.limb.copy())
    nz = mat.limb[c, -1] != 0
    out.exp[c] = np.where(nz, mat.exp[c] + by, mat.exp[c])
    return out


def _pair(m, k, n, p, seed, shift_im=0, dist="uniform"):
    A = _shift_part(si.random_matrix(m, k, p, seed, dist), 1, shift_im)
    B = _shift_part(si.random_matrix(k, n, p, seed + 1, dist), 1, shift_im)
    return A, B


@pytest.mark.parametrize("w", [8, 9])
def test_offset_of_an_exactly_shifted_part(w):
    """Im = Re 2^-100 entry by entry: every line has E^im = E - 100, so z_im = floor(100/w)
    and z_re = 0; an all-zero part gets Z_CAP."""
    p, s = 128, 20
    A = si.random_matrix(6, 9, p, 41, "uniform_exp")
    A.sign[1], A.limb[1] = A.sign[0].copy(), A.limb[1] * 0 + A.limb[0]
    A.exp[1] = A.exp[0] - 100
    sp = ozaki.split_operand(A, s, "A", "4m", w, "per_part")
    assert sp.first_pos == {"re": 0, "im": 100 // w}
    R = _shift_part(A, 1, 0)
    R.limb[1] = 0
    sp = ozaki.split_operand(R, s, "A", "4m", w, "per_part")
    assert sp.first_pos["im"] == ozaki.Z_CAP and sp.first_pos["re"] == 0
    with pytest.raises(ValueError):
        ozaki.split_operand(A, s, "A", "3m", w, "per_part")


@pytest.mark.parametrize("shift", [0, -37, -100, 64])
def test_part_digits_reassemble_on_their_own_grid(shift):
    """sum_t d_t 2^(w(s-1-t)) = X_P = sign floor(|v| 2^(w(s+z_P)-1-E)) exactly, with
    0 <= |v| 2^(w(s+z_P)-1-E) - |X_P| < 1 and |X_P| < 2^(ws-1); the digits are balanced."""
    p, s, w = 192, 26, 9
    A = _shift_part(si.random_matrix(5, 7, p, 43, "uniform_exp"), 1, shift)
    sp = ozaki.split_operand(A, s, "A", "4m", w, "per_part")
    E = ozaki.row_exponents(A, "rows")
    R = 1 << w
    for c, which in enumerate(("re", "im")):
        z = sp.first_pos[which]
        D = sp.digits[which]
        assert np.all(np.abs(D[1:]) <= R // 2) and np.all(np.abs(D[0]) <= R // 2)
        for i in range(A.rows):
            for l in range(A.cols):
                X = sum(int(D[t, i, l]) * R ** (s - 1 - t) for t in range(s))
                v = exact.to_fraction(exact.component(A, c, i, l))
                scaled = abs(v) * Fraction(2) ** (w * (s + z) - 1 - E[i])
                assert 0 <= scaled - abs(X) < 1 and abs(X) < 2 ** (w * s - 1)
                assert X == 0 or (X < 0) == (v < 0)


@pytest.mark.parametrize("w", [8, 9])
def test_equals_the_default_split_when_no_part_is_smaller(w):
    """Comparable parts: every offset is 0, so digits, groups, accumulators and outputs are
    those of the default split bit for bit."""
    p = 160
    A, B = _pair(12, 20, 10, p, 45)
    a = ozaki.ozaki_cgemm(A, B, p, "4m", w=w)
    b = ozaki.ozaki_cgemm(A, B, p, "4m", w=w, split="per_part")
    assert b.splitA.first_pos == {"re": 0, "im": 0} and b.params.Qc == {"re": a.params.Q, "im": a.params.Q}
    for which in ("re", "im"):
        assert np.array_equal(a.splitA.digits[which], b.splitA.digits[which])
        assert np.array_equal(a.splitB.digits[which], b.splitB.digits[which])
    for pr in a.params.products:
        assert [(g.q, g.t0, g.count) for g in a.groups[pr]] == [(g.q, g.t0, g.count) for g in b.groups[pr]]
    for comp in ("re", "im"):
        assert np.array_equal(a.acc[comp], b.acc[comp])
    assert np.array_equal(a.C.limb, b.C.limb) and np.array_equal(a.C.exp, b.C.exp)


@pytest.mark.parametrize("shift", [-100, -23])
def test_all_pairs_lossless_is_the_exact_product(shift):
    """With every pair kept and a lossless split, Acc_c 2^(E+F-(2w-2)-wQ_c) is T_c exactly for
    both components.  Every pair of every product is kept once Q_c >= 2s - 2 + z_a + z_b for
    all its products, i.e. base Q >= 2s - 2 + 2 max z (the subdominant product of a
    component reaches deeper levels)."""
    p, w = 64, 9
    A, B = _pair(4, 6, 5, p, 47, shift)
    prm = ozaki.make_params(p, 6, "4m", guard=60, w=w)
    zmax = -shift // w + 1
    r = ozaki.ozaki_cgemm(A, B, p, "4m", guard=60, Q=2 * prm.s - 2 + 2 * zmax, w=w, split="per_part")
    assert all(r.splitA.lossless) and all(r.splitB.lossless)
    T = ozaki.exact_accumulators(A, B, r.splitA, r.splitB, r.params)
    for comp in ("re", "im"):
        for i in range(A.rows):
            for j in range(B.cols):
                assert r.acc[comp][i, j] == T[comp][i, j]
                assert ozaki.entry_bound(r.params, r.splitA, r.splitB, i, j, comp)[0] == 0


@pytest.mark.parametrize("shift,dist", [(-100, "uniform"), (-100, "uniform_exp"), (-9, "uniform_exp"), (30, "uniform")])
def test_bound_holds_and_output_is_o1(shift, dist):
    """|Acc_c - T_c| <= b 2^beta on every entry (T in Acc units), and the rounded output
    (certified or recomputed) equals O1."""
    p, w = 128, 9
    A, B = _pair(7, 40, 6, p, 49, shift, dist)
    r = ozaki.ozaki_cgemm(A, B, p, "4m", w=w, split="per_part")
    T = ozaki.exact_accumulators(A, B, r.splitA, r.splitB, r.params)
    for comp in ("re", "im"):
        for i in range(A.rows):
            for j in range(B.cols):
                b, beta = ozaki.entry_bound(r.params, r.splitA, r.splitB, i, j, comp)
                assert abs(Fraction(int(r.acc[comp][i, j])) - T[comp][i, j]) <= b * 2 ** beta
    ref = exact.rounded_cgemm(A, B, p)
    assert np.array_equal(r.C.limb, ref.limb) and np.array_equal(r.C.exp, ref.exp) and \
        np.array_equal(r.C.sign, ref.sign)


def test_small_imaginary_parts_keep_their_precision():
    """Im = 2^-100 Re (scale): the default split leaves Im with about p + guard - 100 bits, so
    no imaginary component is certified and every one needs the exact recomputation; the
    per-part split gives Im its own s digits and certifies them."""
    p, w = 128, 9
    A, B = _pair(6, 48, 5, p, 51, -100)
    common = ozaki.ozaki_cgemm(A, B, p, "4m", w=w)
    part = ozaki.ozaki_cgemm(A, B, p, "4m", w=w, split="per_part")
    assert part.splitA.first_pos["im"] == part.splitB.first_pos["im"] >= 100 // w - 1
    assert not common.certified[1].any()            # imaginary parts: all to the fallback
    assert part.certified[1].all() and part.certified[0].all()
    assert np.array_equal(common.C.limb, part.C.limb)   # both end at RN_p(T)


def test_planted_mistakes_are_caught(monkeypatch):
    """Slips in the variant fail the pins above: scaling a component by the base Q instead
    of its own Q_c, or an offset one position too large (digits no longer fit s places)."""
    p, w = 128, 9
    A, B = _pair(5, 30, 4, p, 53, -100)
    ref = exact.rounded_cgemm(A, B, p)
    with monkeypatch.context() as m:
        m.setattr(ozaki.Params, "q_comp", lambda self, comp: self.Q)
        r = ozaki.ozaki_cgemm(A, B, p, "4m", w=w, split="per_part")
        assert not np.array_equal(r.C.exp, ref.exp)
    orig = ozaki.part_offset
    with monkeypatch.context() as m:
        m.setattr(ozaki, "part_offset", lambda E, EP, w_: orig(E, EP, w_) + 1)
        sp = ozaki.split_operand(A, 20, "A", "4m", w, "per_part")
        # the digits no longer fit s places: the top digit leaves the balanced range
        assert np.abs(sp.digits["im"]).max() > (1 << (w - 1))
