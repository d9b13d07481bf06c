"""O2 -- step-by-step emulation of the Ozaki complex GEMM (TEST INFRASTRUCTURE).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU legs may
use this module.  It shares no code with the CUDA path; it exists so that
every integer stage of that path (digits, slice-pair sums, accumulators,
certification flags, rounded outputs) can be compared bit for bit.

Algorithm 2 of the paper (Kouya, Sec. III-C) in this library's reading:

1. Row maxima (Alg. 2, mu_A / mu_B).  Per row i of A one exponent
   E_i = max exponent over the row, over BOTH real and imaginary planes (a
   common split for Re and Im, Sec. III-C last paragraph); per column j of B
   likewise F_j.  Every |a_il| < 2**E_i.
2. Split (Alg. 2, tau / A_alpha := (A + S_A) - S_A).  The paper cuts each
   row on a grid set by tau into short S-bit floats so that the slice products
   are exact.  Here the grid is fixed per row: X = sign * floor(|a| 2**(ws-1-E))
   (truncation of the magnitude) and X is written in s balanced base-2**w
   digits d_0 (most significant) .. d_{s-1}, every |d| <= 2**(w-1), so that
   a ~= sum_t d_t 2**(E-(w-1)-wt).  Digit t plays the role of slice A_{t+1}.
   w = 9 by default (8 selectable): every integer |d| <= 256 is exact in bf16
   and products (|.| <= 2**(2w-2)) are exact.
3. Products (Alg. 2, C_ab := A_a B_b for a + b <= d + 1).  Kept pair set
   P = {(t, u): t + u <= Q} (0-based; the paper's triangle is Q = s - 1).
   Pairs of one level q = t + u have one weight 2**(E+F-(2w-2)-wq); their
   products are summed in groups of at most Gmax pairs,
   Gmax*k*2**(2w-2) < 2**31, so every group sum fits an int32.
4. Accumulation (Alg. 2, "L-bit FP arithmetic").  Here exact: the integer
   Acc = sum_q H_q 2**(w(Q-q)), value = Acc * 2**(E_i+F_j-(2w-2)-wQ).
5. 4M / 3M assembly (Eqs. 4m_way, 3m_way) on the exact accumulators:
   4M: Re = rr - ii, Im = ri + ir;  3M: Re = rr - ii, Im = ss - rr - ii, where
   ss is the product of the digit expansions of X_re + X_im (row) and
   Y_re + Y_im (column), s + 1 digits each (positions -1 .. s-1).
6. Rounding.  Acc differs from the exact T by at most B (a bound from the
   dropped pairs and the split truncation).  If no rounding midpoint of the
   p-bit grid lies within B of Acc, RN_p(Acc) == RN_p(T) ("certified");
   otherwise the entry is recomputed exactly (O1) -- so the final output is
   always RN_p(T).

Per-part split (``split="per_part"``, 4M).  Alg. 2 splits every real matrix
(Re A, Im A, Re B, Im B) on its own: mu, the row maximum of that part, is taken
again before every slice, and tau follows it.  On the fixed per-row grid of
step 2 a re-measured maximum only decides at which grid position the next
nonzero digit of that part starts.  The variant therefore gives part P a digit
offset z_P: the number of leading digit positions that are zero in every line
of P, z_P = min over lines of floor((E_line - E^P_line) / w) (E^P_line the
largest exponent of part P in the line; an all-zero part gets Z_CAP).  Part P
is cut on the grid 2^(E - (w-1) - w(z_P + t)), t < s: X_P = sign floor(|v|
2^(w(s + z_P) - 1 - E)) in s digits at positions z_P .. z_P + s - 1.  Every
output component c takes its own cut level Q_c = Q + z_c, z_c the smallest
z_a + z_b over the products entering c, so a part that is smaller by 2^-D
everywhere keeps its full s digits instead of losing about D/w of them to
leading zeros, and the products of a component far below its magnitude keep
only the pairs that reach its precision (the paper's future-work remark that
the number of divisions should follow the magnitudes of the real and imaginary
parts, Sec. V, item 3).  Accumulation, bounds and certification are those of
the default path with the component's own Q_c.
"""
from __future__ import annotations

import functools
import math
from dataclasses import dataclass, field

import numpy as np

from . import exact as o1

DIGIT_BITS = 9                  # default digit width w (8 is the other supported width)
Z_CAP = 2048                    # per-part split: offset of an all-zero part, and the cap of z
INT32_MAX = 2 ** 31 - 1


def digit_max(w: int = DIGIT_BITS) -> int:
    """Largest |d| of a balanced base-2**w digit (the top digit may reach it)."""
    return 1 << (w - 1)


def prod_log2(w: int = DIGIT_BITS) -> int:
    """|d_a * d_b| <= 2**prod_log2(w)."""
    return 2 * w - 2


def auto_digit_bits(k: int) -> int:
    """9-bit digits when one pair's sum fits an int32 (k 2**16 < 2**31), else 8."""
    return 9 if k * (1 << prod_log2(9)) <= INT32_MAX else 8
DEFAULT_GUARD = 40

PRODUCTS_4M = ("rr", "ii", "ri", "ir")
PRODUCTS_3M = ("rr", "ii", "ss")
# (A digit set, B digit set) of each real product
PRODUCT_OPERANDS = {"rr": ("re", "re"), "ii": ("im", "im"), "ri": ("re", "im"),
                    "ir": ("im", "re"), "ss": ("sum", "sum")}


def ceil_log2(k: int) -> int:
    return (k - 1).bit_length() if k > 1 else 0


@dataclass
class Params:
    p: int
    k: int
    s: int
    Q: int
    gmax: int
    method: str
    guard: int = DEFAULT_GUARD
    w: int = DIGIT_BITS          # bits per digit
    split: str = "common"        # "common" (one exponent per line) or "per_part"
    Qc: dict = None              # per-part split: cut level per component ('re', 'im')

    @property
    def products(self):
        return PRODUCTS_4M if self.method == "4m" else PRODUCTS_3M

    def q_comp(self, comp: str) -> int:
        """Cut level of output component `comp`."""
        return self.Qc[comp] if self.Qc else self.Q

    def q_prod(self, prod: str) -> int:
        """Cut level of the component a real product enters (4M: one component each;
        3M: the common Q)."""
        if not self.Qc:
            return self.Q
        return self.Qc["re" if prod in ("rr", "ii") else "im"]


def make_params(p: int, k: int, method: str = "4m", guard: int = DEFAULT_GUARD,
                s: int | None = None, Q: int | None = None, max_group: int = 0,
                w: int | None = None) -> Params:
    """Slice count s, cut level Q and group size.

    w = auto_digit_bits(k) unless given (9, or 8 when k >= 2**15);
    s = ceil((p + ceil(log2 k) + guard) / w) digits; Q = s - 1 (the paper's
    triangle alpha + beta <= d + 1).  Both may be overridden.  Groups hold at
    most Gmax pairs (the int32 limit), or ``max_group`` if smaller; the level
    sums do not depend on the grouping.
    """
    if w is None:
        w = auto_digit_bits(k)
    if s is None:
        s = -(-(p + ceil_log2(k) + guard) // w)
    if Q is None:
        Q = s - 1
    gmax = INT32_MAX // (k << prod_log2(w)) if k > 0 else 1
    if gmax < 1:
        raise ValueError("k too large for int32 group sums")
    if max_group > 0:
        gmax = min(gmax, max_group)
    return Params(p=p, k=k, s=s, Q=Q, gmax=gmax, method=method, guard=guard, w=w)


# ------------------------------------------------------------- step 1

def mantissas(mat, c: int):
    """Object array of the signed integers N with component value N * 2**(exp - 64L).

    A component whose top limb is 0 is zero (format definition).
    """
    L = mat.limb.shape[1]
    M = np.zeros((mat.rows, mat.cols), dtype=object)
    for j in range(L - 1, -1, -1):
        M = (M * (1 << 64)) + mat.limb[c, j].astype(object)
    M = np.where(mat.limb[c, L - 1] == 0, 0, M)
    return np.where(mat.sign[c] != 0, -M, M)


def row_exponents(mat, by: str):
    """E per row ('rows') or per column ('cols') over both planes; None if all zero."""
    nonzero = np.stack([mantissas(mat, c) != 0 for c in range(2)])
    e = np.where(nonzero, mat.exp.astype(np.int64), np.iinfo(np.int64).min)
    axis = (0, 2) if by == "rows" else (0, 1)
    emax = e.max(axis=axis)
    return [None if v == np.iinfo(np.int64).min else int(v) for v in emax]


# ------------------------------------------------------------- step 2

def fixed_point(v, E: int, s: int, w: int = DIGIT_BITS):
    """X = sign * floor(|v| * 2**(ws-1-E)) for v = (N, x); returns (X, lossless)."""
    N, x = v
    if N == 0:
        return 0, True
    sh = x + w * s - 1 - E
    a = abs(N)
    if sh >= 0:
        X, lossless = a << sh, True
    else:
        X = a >> (-sh)
        lossless = (X << (-sh)) == a
    return (-X if N < 0 else X), lossless


def balanced_digits(X: int, nd: int, w: int = DIGIT_BITS):
    """Digits d_0 .. d_{nd-1} (most significant first) with X = sum d_t R**(nd-1-t), R = 2**w.

    The nd-1 low digits are the residues of X mod R taken in [-R/2, R/2 - 1];
    the top digit is what remains.
    """
    R, h = 1 << w, 1 << (w - 1)
    out = []
    for _ in range(nd - 1):
        d = ((X + h) % R) - h
        out.append(d)
        X = (X - d) // R
    out.append(X)
    out.reverse()
    return out


@dataclass
class Split:
    """Digits of one operand (A by rows, or B by columns; B stored transposed)."""
    E: list                    # per row (A) / column (B); None for an all-zero line
    lossless: list             # per line: every element exact on the grid
    digits: dict = field(default_factory=dict)  # 're'/'im'/'sum' -> int array [nd][lines][k]
    first_pos: dict = field(default_factory=dict)  # digit position of plane 0
    live: dict = field(default_factory=dict)    # per digit set: plane has a nonzero digit
    values: tuple = (True, True)                 # some element has a nonzero real / imaginary part


def fixed_point_array(N, x, E_line, s: int, w: int = DIGIT_BITS):
    """Vectorised ``fixed_point`` over an object array N (exponent x per element)."""
    sh = x + w * s - 1 - E_line                   # int64 array
    a = np.abs(N)
    up = a * np.vectorize(lambda t: 1 << int(t) if t >= 0 else 1, otypes=[object])(sh)
    down = np.vectorize(lambda v, t: v >> int(-t) if t < 0 else v, otypes=[object])(a, sh)
    X = np.where(sh >= 0, up, down)
    back = np.vectorize(lambda v, t: v << int(-t) if t < 0 else v, otypes=[object])(X, sh)
    lossless = (sh >= 0) | (back == a)
    return np.where(N < 0, -X, X), lossless


def balanced_digits_array(X, nd: int, w: int = DIGIT_BITS):
    """Vectorised ``balanced_digits``: int64 array [nd, ...], most significant first."""
    R, h = 1 << w, 1 << (w - 1)
    out = np.zeros((nd,) + X.shape, np.int64)
    for t in range(nd - 1, 0, -1):
        d = ((X + h) % R) - h
        out[t] = d.astype(np.int64)
        X = (X - d) // R
    out[0] = X.astype(np.int64)
    return out


def part_exponents(mat, c: int, by: str):
    """Largest exponent of component c per row ('rows') or column ('cols'); None if zero."""
    nz = mantissas(mat, c) != 0
    e = np.where(nz, mat.exp[c].astype(np.int64), np.iinfo(np.int64).min)
    emax = e.max(axis=1 if by == "rows" else 0)
    return [None if v == np.iinfo(np.int64).min else int(v) for v in emax]


def part_offset(E: list, EP: list, w: int) -> int:
    """z_P: leading digit positions of part P that are zero in every line (Z_CAP if P is zero)."""
    zs = [(e - ep) // w for e, ep in zip(E, EP) if ep is not None]
    return min(min(zs), Z_CAP) if zs else Z_CAP


def split_operand(mat, s: int, side: str, method: str, w: int = DIGIT_BITS, split: str = "common") -> Split:
    """Alg. 2's split for A (side='A', lines = rows) or B (side='B', lines = columns).

    For B the digit planes are stored K-major: digits[.][u][j][l].  With
    split="per_part" (4M only) each part has its own digit offset (module notes).
    """
    by = "rows" if side == "A" else "cols"
    E = row_exponents(mat, by)
    L = mat.limb.shape[1]
    Nre, Nim = mantissas(mat, 0), mantissas(mat, 1)
    xre = mat.exp[0].astype(np.int64) - 64 * L
    xim = mat.exp[1].astype(np.int64) - 64 * L
    if side == "B":                       # lines = columns: work on the transpose
        Nre, Nim, xre, xim = Nre.T, Nim.T, xre.T, xim.T
    Eline = np.array([0 if e is None else e for e in E], np.int64)[:, None]
    zero_line = np.array([e is None for e in E])[:, None]
    z = {"re": 0, "im": 0}
    if split == "per_part":
        if method != "4m":
            raise ValueError("the per-part split is defined for the 4M method")
        for c, which in enumerate(("re", "im")):
            z[which] = part_offset(E, part_exponents(mat, c, by), w)
    # part P: s digits at positions z_P .. z_P + s - 1, i.e. the grid of s + z_P digits
    Xr, okr = fixed_point_array(Nre, xre, Eline, s + z["re"], w)
    Xi, oki = fixed_point_array(Nim, xim, Eline, s + z["im"], w)
    Xr = np.where(zero_line, 0, Xr)
    Xi = np.where(zero_line, 0, Xi)
    ok = (okr & oki) | zero_line
    sp = Split(E=E, lossless=[bool(v) for v in ok.all(axis=1)])
    sp.digits["re"] = balanced_digits_array(Xr, s, w)
    sp.digits["im"] = balanced_digits_array(Xi, s, w)
    sp.first_pos["re"], sp.first_pos["im"] = z["re"], z["im"]
    if method == "3m":
        sp.digits["sum"] = balanced_digits_array(Xr + Xi, s + 1, w)
        sp.first_pos["sum"] = -1
    for which, D in sp.digits.items():
        sp.live[which] = [bool(np.any(D[x])) for x in range(D.shape[0])]
    sp.values = (bool(np.any(Nre != 0)), bool(np.any(Nim != 0)))
    return sp


def value_nonzero(sp: Split, which: str) -> bool:
    """The operand component behind a digit set has a nonzero value somewhere."""
    return {"re": sp.values[0], "im": sp.values[1], "sum": sp.values[0] or sp.values[1]}[which]


# ------------------------------------------------------------- step 3

@dataclass
class Group:
    q: int          # level t + u
    t0: int         # first digit position t of A in the group (pairs t0 .. t0+count-1)
    count: int


def level_pairs(tA: tuple, tB: tuple, Q: int):
    """Levels q and their pairs (t, q - t), t ascending, of {t+u <= Q}."""
    (a0, a1), (b0, b1) = tA, tB
    out = []
    for q in range(a0 + b0, min(Q, a1 + b1) + 1):
        lo, hi = max(a0, q - b1), min(a1, q - b0)
        if lo <= hi:
            out.append((q, lo, hi - lo + 1))
    return out


def groups_for(tA: tuple, tB: tuple, Q: int, gmax: int):
    """Canonical group list: levels ascending, pairs of a level cut in runs of <= gmax."""
    gs = []
    for q, lo, n in level_pairs(tA, tB, Q):
        t = lo
        while n > 0:
            c = min(n, gmax)
            gs.append(Group(q, t, c))
            t += c
            n -= c
    return gs


PRODUCT_COMPONENTS = {"4m": {"rr": ("re",), "ii": ("re",), "ri": ("im",), "ir": ("im",)},
                      "3m": {"rr": ("re", "im"), "ii": ("re", "im"), "ss": ("im",)}}


def product_needed(spA: Split, spB: Split, prod: str, method: str) -> bool:
    """False when every component the product enters vanishes identically (e.g. the 3M
    sums for real inputs): then all of its groups are emptied."""
    return any(not component_identically_zero(spA.values, spB.values, c)
               for c in PRODUCT_COMPONENTS[method][prod])


def trim_groups(spA: Split, spB: Split, prod: str, gs: list, method: str = None) -> list:
    """The groups with the pairs at their two ends removed whose A or B digit plane is zero
    everywhere (their products are exactly zero, so every group sum is unchanged).

    This is the reading of the paper's remark that the number of divisions should follow
    the magnitudes of the real and imaginary parts (end of Sec. III-C; conclusion, item 3):
    with one exponent per row for both parts, a part that is smaller by 2^-D has about D/8
    leading digit planes of zeros, and the pairs that use them are skipped.  Trimming only
    at the ends keeps a group one run of consecutive pairs; a group may become empty
    (count 0).  Whole planes are tested, so the result depends on the matrices only.
    With the method given, a product whose components all vanish identically
    (``product_needed``) loses every pair.
    """
    wa, wb = PRODUCT_OPERANDS[prod]
    fa, fb = spA.first_pos[wa], spB.first_pos[wb]
    liveA = [bool(np.any(spA.digits[wa][x])) for x in range(spA.digits[wa].shape[0])]
    liveB = [bool(np.any(spB.digits[wb][x])) for x in range(spB.digits[wb].shape[0])]

    needed = method is None or product_needed(spA, spB, prod, method)

    def live(t, u):
        return needed and liveA[t - fa] and liveB[u - fb]
    out = []
    for g in gs:
        t0, c = g.t0, g.count
        while c > 0 and not live(t0, g.q - t0):
            t0, c = t0 + 1, c - 1
        while c > 0 and not live(t0 + c - 1, g.q - (t0 + c - 1)):
            c -= 1
        out.append(Group(g.q, t0, c))
    return out


def positions(sp: Split, which: str, s: int):
    first = sp.first_pos[which]
    nd = sp.digits[which].shape[0]
    return (first, first + nd - 1)


def group_sums(spA: Split, spB: Split, prod: str, prm: Params):
    """Exact int64 group sums G_g = sum_{(t,u) in g} D^A_t (D^B_u)^T for one real product.

    The contraction uses a float64 matmul; it is exact because every entry
    and partial sum is an integer below 2**31 < 2**53.
    """
    wa, wb = PRODUCT_OPERANDS[prod]
    DA, DB = spA.digits[wa], spB.digits[wb]
    fa, fb = spA.first_pos[wa], spB.first_pos[wb]
    tA, tB = positions(spA, wa, prm.s), positions(spB, wb, prm.s)
    gs = groups_for(tA, tB, prm.q_prod(prod), prm.gmax)
    out = []
    for g in gs:
        ts = range(g.t0, g.t0 + g.count)
        a = np.concatenate([DA[t - fa] for t in ts], axis=1).astype(np.float64)
        b = np.concatenate([DB[g.q - t - fb] for t in ts], axis=1).astype(np.float64)
        out.append(np.rint(a @ b.T).astype(np.int64))
    return gs, out


# ------------------------------------------------------------- step 4

def accumulate(gs, sums, Q: int, w: int = DIGIT_BITS):
    """Acc = sum_g G_g * 2**(w(Q - q_g)) as Python ints (object array)."""
    shape = sums[0].shape if sums else (0, 0)
    acc = np.zeros(shape, dtype=object)
    for g, G in zip(gs, sums):
        acc = acc + G.astype(object) * (1 << (w * (Q - g.q)))
    return acc


# ------------------------------------------------------------- step 6 (bound)

@functools.lru_cache(maxsize=None)
def drop_bound(tA: tuple, tB: tuple, Q: int, k: int, liveA=None, liveB=None, w: int = DIGIT_BITS) -> int:
    """Integer bound on the dropped pairs of one product, in Acc units.

    Dropped level Q+j contributes at most n_{Q+j} k 2**(2w-2) 2**(-wj).  The
    j = 1 term is k 2**(w-2) n; the rest is below k*max_n/3 (geometric tail:
    2**(-2) / (1 - 2**-w) < 1/3).  With
    liveA / liveB (per digit plane, from position tA[0] / tB[0]) only the pairs
    whose two planes both have a nonzero digit are counted: the others are
    exactly zero.
    """
    if liveA is not None:
        levels = {}
        for q, lo, n in level_pairs(tA, tB, 10 ** 9):
            levels[q] = sum(1 for t in range(lo, lo + n) if liveA[t - tA[0]] and liveB[q - t - tB[0]])
    else:
        levels = {q: n for q, _, n in level_pairs(tA, tB, 10 ** 9)}
    n1 = levels.get(Q + 1, 0)
    rest = [n for q, n in levels.items() if q >= Q + 2]
    nmax = max(rest) if rest else 0
    return k * ((1 << (w - 2)) * n1 + (-(-nmax // 3)))


def split_coeffs(prod: str):
    """(c_a, f_a, c_b, f_b): truncation ulps and magnitude factors per operand."""
    if prod == "ss":
        return 2, 2, 2, 2
    return 1, 1, 1, 1


def bound_exponent(prm: Params) -> int:
    """beta: the bound is b * 2**beta with beta = max(0, 2w - 1 + w(Q - s)).

    One unit of the split grid, 2**(E-(ws-1)), times |b| < 2**F, in Acc units
    2**(E+F-(2w-2)-wQ), is 2**(2w-1+w(Q-s)).  Per-part split: a part with offset z_a
    has the unit 2**(E-(w(s+z_a)-1)) and the other factor |b| < 2**(F-w z_b), so in the
    units 2**(E+F-(2w-2)-w Q_c) of its component (Q_c = Q + z_c, z_c <= z_a + z_b) the
    same term is at most 2**(2w-1+w(Q-s)): beta is unchanged."""
    return max(0, 2 * prm.w - 1 + prm.w * (prm.Q - prm.s))


def entry_bound(prm: Params, spA: Split, spB: Split, i: int, j: int, comp: str):
    """(b, beta) with |Acc_comp - T_comp * 2**-(scale)| <= b 2**beta."""
    if spA.E[i] is None or spB.E[j] is None:
        return 0, 0
    beta = bound_exponent(prm)
    if component_identically_zero(spA.values, spB.values, comp):
        return 0, beta
    if prm.method == "4m":
        prods = ("rr", "ii") if comp == "re" else ("ri", "ir")
    else:
        prods = ("rr", "ii") if comp == "re" else ("ss", "rr", "ii")
    b = 0
    for pr in prods:
        bd, gate = product_bound(prm, spA, spB, pr)
        b += -(-bd >> beta) if beta < 4096 else (1 if bd else 0)
        if gate:
            ca, fa, cb, fb = split_coeffs(pr)
            # truncation of A (row i lossy) times |b| <= fb 2^F; |a^| <= fa 2^E times truncation of B
            b += prm.k * ((0 if spA.lossless[i] else ca * fb) + (0 if spB.lossless[j] else fa * cb))
    return b, beta


def component_identically_zero(vA: tuple, vB: tuple, comp: str) -> bool:
    """Component `comp` of A B vanishes for every entry, given which components of A and B
    (re, im) have a nonzero value somewhere.  Then every product entering it, and the
    3M sums (which equal one part digit for digit), cancel exactly in Acc."""
    (ar, ai), (br, bi) = vA, vB
    if comp == "re":
        return (not ar or not br) and (not ai or not bi)
    return (not ar or not bi) and (not ai or not br)


def product_bound(prm: Params, spA: Split, spB: Split, pr: str):
    """(dropped-pair bound over live pairs, truncation counts) of one real product.

    The truncation terms apply only when both operand components of the product
    have a nonzero value somewhere: otherwise the product and its digit product
    are both exactly zero.  Cached on the splits (it depends on them only).
    """
    key = ("bound", pr, prm.q_prod(pr), prm.k, prm.s, prm.w)
    cache = spA.__dict__.setdefault("_bound_cache", {})
    hit = cache.get(key)
    if hit is None or hit[0] is not spB:        # keyed on the very B split (kept alive here)
        wa, wb = PRODUCT_OPERANDS[pr]
        tA, tB = positions(spA, wa, prm.s), positions(spB, wb, prm.s)
        bd = drop_bound(tA, tB, prm.q_prod(pr), prm.k, tuple(spA.live[wa]), tuple(spB.live[wb]), prm.w)
        hit = (spB, (bd, value_nonzero(spA, wa) and value_nonzero(spB, wb)))
        cache[key] = hit
    return hit[1]


def certify(acc: int, b: int, beta: int, p: int) -> bool:
    """True iff no midpoint of the p-bit grid lies within b*2**beta of acc."""
    if b == 0:
        return True
    a = abs(acc)
    n = a.bit_length()
    if n <= p:
        return False
    sh = n - p
    if b.bit_length() + beta > sh - 3:
        return False
    r = a & ((1 << sh) - 1)
    h = 1 << (sh - 1)
    return abs(r - h) > (b << beta)


# ------------------------------------------------------------- full pipeline

@dataclass
class OzakiResult:
    params: Params
    splitA: Split
    splitB: Split
    groups: dict          # product -> list[Group]
    group_sums: dict      # product -> list[int64 array m x n]
    acc: dict             # 're'/'im' -> object array of exact combined accumulators
    scale: np.ndarray     # E_i + F_j - (2w-2) - wQ (object array)
    certified: np.ndarray  # bool [2, m, n]
    C: object             # MPCMatrix, final rounded output (== O1)


def component_offsets(spA: Split, spB: Split) -> dict:
    """Per-part split: z_c = min over the 4M products of component c of z_a + z_b."""
    za, zb = spA.first_pos, spB.first_pos
    return {"re": min(za["re"] + zb["re"], za["im"] + zb["im"]),
            "im": min(za["re"] + zb["im"], za["im"] + zb["re"])}


def ozaki_cgemm(A, B, p: int, method: str = "4m", guard: int = DEFAULT_GUARD,
                s: int | None = None, Q: int | None = None, fallback=None, max_group: int = 0,
                w: int | None = None, split: str = "common") -> OzakiResult:
    """Emulate the whole Ozaki complex GEMM; ``fallback(i, j) -> (re, im)`` exact values.

    Without ``fallback`` the exact O1 triple loop is used for uncertified entries.
    ``split``: "common" (one exponent per line for both parts) or "per_part" (4M).
    """
    m, k, n = A.rows, A.cols, B.cols
    prm = make_params(p, k, method, guard, s, Q, max_group, w)
    w = prm.w
    spA = split_operand(A, prm.s, "A", method, w, split)
    spB = split_operand(B, prm.s, "B", method, w, split)
    if split == "per_part":
        prm.split = split
        prm.Qc = {c: prm.Q + z for c, z in component_offsets(spA, spB).items()}
    groups, sums, acc_p = {}, {}, {}
    for pr in prm.products:
        gs, gsum = group_sums(spA, spB, pr, prm)
        groups[pr], sums[pr] = gs, gsum
        acc_p[pr] = accumulate(gs, gsum, prm.q_prod(pr), w) if gs else np.zeros((m, n), dtype=object)
    acc_re = acc_p["rr"] - acc_p["ii"]
    acc_im = (acc_p["ri"] + acc_p["ir"]) if method == "4m" else (acc_p["ss"] - acc_p["rr"] - acc_p["ii"])
    scale = np.zeros((m, n), dtype=object)
    cert = np.zeros((2, m, n), bool)
    vals = [[[None] * n for _ in range(m)] for _ in range(2)]
    pending = []
    for i in range(m):
        for j in range(n):
            Ei = spA.E[i] if spA.E[i] is not None else 0
            Fj = spB.E[j] if spB.E[j] is not None else 0
            scale[i, j] = Ei + Fj - prod_log2(prm.w) - prm.w * prm.Q
            for c, (comp, acc) in enumerate((("re", acc_re), ("im", acc_im))):
                x = Ei + Fj - prod_log2(prm.w) - prm.w * prm.q_comp(comp)
                b, beta = entry_bound(prm, spA, spB, i, j, comp)
                a = int(acc[i, j])
                if certify(a, b, beta, p):
                    cert[c, i, j] = True
                    vals[c][i][j] = o1.round_nearest_even((a, x), p)
                else:
                    pending.append((c, i, j))
    if pending:
        need = sorted({(i, j) for _, i, j in pending})
        exact_vals = {}
        for (i, j) in need:
            exact_vals[(i, j)] = fallback(i, j) if fallback else _exact_entry(A, B, i, j)
        for c, i, j in pending:
            vals[c][i][j] = o1.round_nearest_even(exact_vals[(i, j)][c], p)
    C = o1.pack(vals[0], vals[1], p)
    return OzakiResult(prm, spA, spB, groups, sums, {"re": acc_re, "im": acc_im}, scale, cert, C)


def _exact_entry(A, B, i, j):
    Ar = A.submatrix(i, i + 1, 0, A.cols)
    Bc = B.submatrix(0, B.rows, j, j + 1)
    re, im = o1.exact_cgemm(Ar, Bc, "4m")
    return re[0][0], im[0][0]


def exact_accumulators(A, B, spA: Split, spB: Split, prm: Params):
    """Exact T scaled to Acc units, as rationals: T * 2**-(E+F-(2w-2)-wQ)."""
    from fractions import Fraction
    re, im = o1.exact_cgemm(A, B, "4m")
    m, n = A.rows, B.cols
    out = {"re": np.zeros((m, n), dtype=object), "im": np.zeros((m, n), dtype=object)}
    for i in range(m):
        for j in range(n):
            Ei = spA.E[i] if spA.E[i] is not None else 0
            Fj = spB.E[j] if spB.E[j] is not None else 0
            for comp, T in (("re", re), ("im", im)):
                x = Ei + Fj - prod_log2(prm.w) - prm.w * prm.q_comp(comp)
                out[comp][i, j] = o1.to_fraction(T[i][j]) / (Fraction(2) ** x)
    return out


# ------------------------------------------------------------- paper pin

def paper_slice_bits(S: int, l: int) -> int:
    """Bits per slice of Alg. 2 with S-bit slice arithmetic and inner size l.

    tau puts the split point ceil((S + log2 l)/2) bits above the row maximum,
    so a slice keeps S - ceil((S + log2 l)/2) bits.
    """
    return S - math.ceil((S + math.log2(l)) / 2)


def paper_division_count(p: int, S: int, l: int) -> int:
    """Smallest d whose d slices of ``paper_slice_bits`` bits cover p bits."""
    return math.ceil(p / paper_slice_bits(S, l))
