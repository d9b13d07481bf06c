"""O2r -- Alg. 2's residual split, emulated in exact integers (TEST INFRASTRUCTURE).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU legs may use this
module.  It shares no code with the CUDA path.  It is the oracle of the library's
``MPC_SPLIT_RESIDUAL`` variant (4M), stage by stage: slice units, digits, slice-pair
products, exact accumulators, bounds, certification and the rounded output (== O1).

Alg. 2 (Kouya, Sec. III-C) cuts every real matrix row by row (columns for B), and
before EVERY slice it measures again mu, the largest magnitude left in the row, sets
tau = 2^(ceil(log2 mu) + beta) and takes the slice (A + tau) - tau in S-bit
arithmetic; the slice is then subtracted from A in L-bit arithmetic.  An S-bit
round-to-nearest-even addition rounds the residual to the grid of unit
ulp(tau) = 2^(ceil(log2 mu) + beta - S + 1), so each slice is the residual rounded to
nearest (ties to even) at a unit that follows the residual's own magnitude.

Reading used here (the paper's S - beta bits per slice become w bits per digit):

1. Each real part P of a line (row of A, column of B) is cut on its own (Alg. 2 runs on
   real matrices; the 4M form multiplies the four real parts, Eq. 4m_way).
2. Slice t of the line: c_t = ceil(log2 max_l |R_l|) over the current residuals R,
   unit exponent b_t = c_t - (w - 1), digit d = RNE(R / 2^b_t) (so |d| <= 2^(w-1),
   exact in bf16), R := R - d 2^b_t (exact).  Because |R| <= 2^(b_t - 1) afterwards,
   c_(t+1) <= b_t - 1, so units fall by at least w per slice; they fall by more exactly
   when the residual of the whole line is unusually small (the line "skips" grid
   positions, e.g. a run of zero bits shared by all its elements).
3. s slices are cut.  The remainder after the last one, |R| <= 2^(b_(s-1) - 1) <=
   2^(b_floor - 1) with b_floor = c_0 - (w - 1) - w (s - 1) (the unit of the last of s
   regular slices), is dropped (the paper keeps it as a final rounded slice A_d, which
   makes its product inexact).  A line whose residual vanishes earlier has zero slices
   from there on.
4. Products: every kept pair (t, u), t + u <= Q (Q = s - 1: the paper's triangle),
   gives its own exact product G_tu = D^A_t (D^B_u)^T (int32: k 2^(2w-2) < 2^31).  The
   table lists, per real product (rr, ii, ri, ir), the pairs level by level (q = t + u
   ascending, t ascending); a pair whose A or B digit plane is zero in every line is
   skipped, as is every pair of a product that enters only components of A B that
   vanish identically.  Consecutive live pairs of a level whose offsets agree at every
   entry may share one exact group sum: pair (t + 1, u - 1) joins the group of (t, u)
   when slice t + 1 of A and slice u of B each lie exactly w below their previous slice
   in every line where they are nonzero (``merged_table``; at most gmax pairs, the int32
   limit).  A group's sum is the sum of its pairs' products, so no accumulator changes.
5. Accumulation ("C := C + C_ab in L-bit arithmetic"), exact: component c of entry
   (i, j) has its own window, anchored at M = max over its products of
   b^A_(i,0) + b^B_(j,0) (lines where either part is zero do not count); its unit is
   2^lo, lo = M - w Q.  A pair's term sits at offset o = b^A_(i,t) + b^B_(j,u) - lo.
   Within one (product, level), consecutive pairs (t ascending) with equal offset are
   summed exactly (with their sign in c) and each sum is added at its offset; a sum
   whose offset is negative is added as floor(sum 2^o) and counted as one truncation.
   No offset exceeds w Q (units fall by w per slice from the anchors and M is the largest
   anchor sum), so a fixed-width accumulator of the default split's size holds the sum.
6. Bound: the default split's bound (dropped pairs over live planes, one truncation term
   per lossy line, in units 2^beta) holds here too -- slice t's unit is at most
   b_0 - w t, the default grid's, every window is anchored at the largest b^A_0 + b^B_0
   of its products, and the remainder is at most half a floor unit -- plus
   ceil(truncations / 2^beta).  Certification and the exact fallback as in ``ozaki``.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import exact as o1
from . import ozaki as oz

PRODUCTS = ("rr", "ii", "ri", "ir")
# (A part, B part) of each 4M real product, and the component it enters with its sign
OPERANDS = {"rr": ("re", "re"), "ii": ("im", "im"), "ri": ("re", "im"), "ir": ("im", "re")}
ENTERS = {"rr": ("re", 1), "ii": ("re", -1), "ri": ("im", 1), "ir": ("im", 1)}


def ceil_log2_int(v: int) -> int:
    """ceil(log2 v) for an integer v >= 1: bitlen(v - 1)."""
    return (v - 1).bit_length()


def ceil_log2_abs(N: int, x: int) -> int:
    """ceil(log2 |N 2^x|) for N != 0."""
    return x + ceil_log2_int(abs(N))


def rne_quotient(r: int, sh: int) -> int:
    """RNE(r / 2^sh) for a signed integer r and sh >= 0 (ties to the even quotient)."""
    if sh == 0:
        return r
    q, rem = divmod(r, 1 << sh)          # floor division: 0 <= rem < 2^sh
    twice, unit = 2 * rem, 1 << sh
    if twice > unit or (twice == unit and (q & 1)):
        q += 1
    return q


@dataclass
class LineSplit:
    units: list          # s entries: unit exponent b_t of slice t, None for a zero slice
    digits: list         # s lists of k ints
    remainder: list      # k ints, in units of 2^Z
    Z: int               # exponent of the remainder's unit
    c0: int | None       # ceil(log2 max |a|), None for an all-zero line
    floor: int | None    # b_floor: the unit of the last of s regular slices


def split_line(vals, s: int, w: int) -> LineSplit:
    """Steps 2-3 of the module notes for one line of one part; vals = [(N, x)] exact."""
    k = len(vals)
    nz = [(N, x) for N, x in vals if N != 0]
    if not nz:
        return LineSplit([None] * s, [[0] * k for _ in range(s)], [0] * k, 0, None, None)
    c0 = max(ceil_log2_abs(N, x) for N, x in nz)
    b_floor = c0 - (w - 1) - w * (s - 1)
    Z = min(min(x for _, x in nz), b_floor)
    R = [N << (x - Z) if N != 0 else 0 for N, x in vals]
    units, digits = [], []
    c = c0
    for _ in range(s):
        if c is None:
            units.append(None)
            digits.append([0] * k)
            continue
        b = c - (w - 1)
        if b < Z:                          # finer than every input bit: rescale (exact)
            R = [r << (Z - b) for r in R]
            Z = b
        sh = b - Z
        d = [rne_quotient(r, sh) for r in R]
        R = [r - (dd << sh) for r, dd in zip(R, d)]
        units.append(b)
        digits.append(d)
        mx = max(abs(r) for r in R)
        c = None if mx == 0 else Z + ceil_log2_int(mx)
    return LineSplit(units, digits, R, Z, c0, b_floor)


@dataclass
class ResidualSplit:
    """One operand cut by ``split_line``: per part, per line.  B is stored by columns."""
    units: dict = field(default_factory=dict)    # part -> list[s] of lists[lines] (None: zero slice)
    digits: dict = field(default_factory=dict)   # part -> int64 array [s][lines][k]
    lines: dict = field(default_factory=dict)    # part -> list[LineSplit]
    lossless: list = None                        # per line: both parts' remainders are 0
    live: dict = field(default_factory=dict)     # part -> per slice: a nonzero digit in some line
    values: tuple = (True, True)                 # some element has a nonzero re / im part
    E: list = None                               # per line: None iff both parts are zero
    first_pos: dict = field(default_factory=lambda: {"re": 0, "im": 0})

    def anchor(self, part: str, line: int):
        """b_0 of the line's part (None if the part is zero in the line)."""
        return self.units[part][0][line]


def split_operand(mat, s: int, side: str, w: int) -> ResidualSplit:
    """Cut A by rows (side 'A') or B by columns (side 'B')."""
    vals = o1.matrix_values(mat)          # [c][r][col] -> (N, x)
    if side == "A":
        lines = [[[vals[c][i][l] for l in range(mat.cols)] for i in range(mat.rows)] for c in range(2)]
    else:
        lines = [[[vals[c][l][j] for l in range(mat.rows)] for j in range(mat.cols)] for c in range(2)]
    sp = ResidualSplit()
    nlines = len(lines[0])
    for c, part in enumerate(("re", "im")):
        ls = [split_line(v, s, w) for v in lines[c]]
        sp.lines[part] = ls
        sp.units[part] = [[ls[i].units[t] for i in range(nlines)] for t in range(s)]
        k = len(lines[c][0]) if nlines else 0
        D = np.zeros((s, nlines, k), np.int64)
        for i, L in enumerate(ls):
            for t in range(s):
                D[t, i] = L.digits[t]
        sp.digits[part] = D
        sp.live[part] = [bool(np.any(D[t])) for t in range(s)]
    sp.lossless = [all(r == 0 for r in sp.lines["re"][i].remainder) and
                   all(r == 0 for r in sp.lines["im"][i].remainder) for i in range(nlines)]
    sp.values = tuple(any(L.c0 is not None for L in sp.lines[part]) for part in ("re", "im"))
    sp.E = [None if sp.lines["re"][i].c0 is None and sp.lines["im"][i].c0 is None else 0
            for i in range(nlines)]
    return sp


def pair_table(spA: ResidualSplit, spB: ResidualSplit, prm: oz.Params):
    """Step 4: [(product, q, t, live)] in table order (per product, q then t ascending)."""
    out = []
    for pr in PRODUCTS:
        pa, pb = OPERANDS[pr]
        needed = oz.product_needed(spA, spB, pr, "4m")
        for q, lo, n in oz.level_pairs((0, prm.s - 1), (0, prm.s - 1), prm.Q):
            for t in range(lo, lo + n):
                live = needed and spA.live[pa][t] and spB.live[pb][q - t]
                out.append((pr, q, t, live))
    return out


def irregular_steps(sp: ResidualSplit, part: str, s: int, w: int) -> list:
    """Per slice t: some line where slice t is nonzero has a unit other than its previous one - w."""
    out = [False] * s
    for t in range(1, s):
        out[t] = any(u is not None and u != u_prev - w
                     for u_prev, u in zip(sp.units[part][t - 1], sp.units[part][t]))
    return out


def merged_table(spA: ResidualSplit, spB: ResidualSplit, table, prm: oz.Params, gmax: int):
    """The table with runs of consecutive live pairs of one level merged (module notes, step
    4): entries (product, q, t0, count); a merged pair's own entry gets count 0."""
    irr = {("A", p): irregular_steps(spA, p, prm.s, prm.w) for p in ("re", "im")}
    irr.update({("B", p): irregular_steps(spB, p, prm.s, prm.w) for p in ("re", "im")})
    out = [[pr, q, t, 1 if live else 0] for pr, q, t, live in table]
    head = None
    for e, (pr, q, t, live) in enumerate(table):
        if e == 0 or (table[e - 1][0], table[e - 1][1]) != (pr, q):
            head = None
        if not live:
            head = None
            continue
        pa, pb = OPERANDS[pr]
        if head is not None and out[head][3] < gmax and not irr[("A", pa)][t] and not irr[("B", pb)][q - t + 1]:
            out[head][3] += 1
            out[e][3] = 0
            continue
        head = e
    return [tuple(x) for x in out]


def pair_products(spA: ResidualSplit, spB: ResidualSplit, table):
    """G_tu = D^A_t (D^B_u)^T per live table entry (exact: every value < 2^31 < 2^53)."""
    out = []
    for pr, q, t, live in table:
        if not live:
            out.append(None)
            continue
        pa, pb = OPERANDS[pr]
        a = spA.digits[pa][t].astype(np.float64)
        b = spB.digits[pb][q - t].astype(np.float64)
        out.append(np.rint(a @ b.T).astype(np.int64))
    return out


def window_low(spA, spB, i: int, j: int, comp: str, prm: oz.Params):
    """lo of component comp at (i, j), or None when every product of comp vanishes there."""
    best = None
    for pr in PRODUCTS:
        if ENTERS[pr][0] != comp:
            continue
        pa, pb = OPERANDS[pr]
        ba, bb = spA.anchor(pa, i), spB.anchor(pb, j)
        if ba is None or bb is None:
            continue
        best = ba + bb if best is None else max(best, ba + bb)
    return None if best is None else best - prm.w * prm.Q


def _floor_shift(v: np.ndarray, sh: np.ndarray) -> np.ndarray:
    """floor(v / 2^sh) for int64 v and shifts sh >= 0 (any size)."""
    big = sh >= 63
    out = v >> np.minimum(sh, 63)
    return np.where(big, np.where(v < 0, -1, 0), out)


def accumulate(spA, spB, table, products, prm: oz.Params, m: int, n: int):
    """Step 5: exact accumulators, window exponents and truncation counts per component.

    Vectorised over the entries (i, j); the runs are formed exactly as the module notes
    say (consecutive pairs of one (product, level) with equal offset, per entry).
    """
    NONE = np.iinfo(np.int64).min
    acc, lo, trunc = {}, {}, {}
    top = None                           # largest offset of any run (the window's top: <= w Q)
    for comp in ("re", "im"):
        low = np.array([[window_low(spA, spB, i, j, comp, prm) for j in range(n)] for i in range(m)],
                       dtype=object).reshape(m, n)
        has = np.vectorize(lambda v: v is not None, otypes=[bool])(low) if m * n else np.zeros((m, n), bool)
        low_i = np.where(has, low, 0).astype(np.int64)
        total = np.zeros((m, n), dtype=object)
        cnt = np.zeros((m, n), np.int64)
        run_sum = np.zeros((m, n), np.int64)
        run_off = np.full((m, n), NONE, np.int64)

        def flush(mask):
            nonlocal total
            sel = mask & (run_off != NONE)
            pos = sel & (run_off >= 0)
            neg = sel & (run_off < 0)
            if pos.any():
                sh = np.where(pos, run_off, 0).astype(object)
                total = total + np.where(pos, run_sum.astype(object) << sh, 0)
            if neg.any():
                sh = np.where(neg, -run_off, 0)
                f = _floor_shift(run_sum, sh)
                dropped = neg & (np.where(sh >= 63, run_sum != 0, (f << np.minimum(sh, 62)) != run_sum))
                cnt[...] += dropped
                total = total + np.where(neg, f, 0).astype(object)
            run_sum[sel] = 0
            run_off[sel] = NONE

        key = None
        for (pr, q, t, live), G in zip(table, products):
            c, sign = ENTERS[pr]
            if c != comp or not live:
                continue
            if (pr, q) != key:
                flush(np.ones((m, n), bool))
                key = (pr, q)
            pa, pb = OPERANDS[pr]
            ua = np.array([NONE if u is None else u for u in spA.units[pa][t]], np.int64)
            ub = np.array([NONE if u is None else u for u in spB.units[pb][q - t]], np.int64)
            valid = has & (ua[:, None] != NONE) & (ub[None, :] != NONE)
            off = np.where(valid, ua[:, None] + ub[None, :] - low_i, NONE)
            if valid.any():
                hi = int(off[valid].max())
                top = hi if top is None else max(top, hi)
            flush(valid & (off != run_off))
            run_off[valid] = off[valid]
            run_sum[valid] += sign * G[valid]
        flush(np.ones((m, n), bool))
        acc[comp], lo[comp], trunc[comp] = total, low, cnt
    return acc, lo, trunc, top


@dataclass
class ResidualResult:
    params: oz.Params
    splitA: ResidualSplit
    splitB: ResidualSplit
    table: list           # one entry per kept pair: (product, q, t, live)
    groups: list          # the merged table: (product, q, t0, count)
    products: list
    acc: dict
    lo: dict
    trunc: dict
    max_offset: int | None    # largest term offset: at most w Q, so a fixed-width accumulator holds it
    certified: np.ndarray
    C: object


def ozaki_cgemm_residual(A, B, p: int, guard: int = oz.DEFAULT_GUARD, s: int | None = None,
                         Q: int | None = None, w: int | None = None, fallback=None,
                         max_group: int = 0) -> ResidualResult:
    """The whole 4M Ozaki complex GEMM with the residual split; output == O1."""
    m, k, n = A.rows, A.cols, B.cols
    prm = oz.make_params(p, k, "4m", guard, s, Q, max_group, w)
    spA = split_operand(A, prm.s, "A", prm.w)
    spB = split_operand(B, prm.s, "B", prm.w)
    table = pair_table(spA, spB, prm)
    groups = merged_table(spA, spB, table, prm, prm.gmax)
    prods = pair_products(spA, spB, table)
    acc, lo, trunc, top = accumulate(spA, spB, table, prods, prm, m, n)
    beta = oz.bound_exponent(prm)
    cert = np.zeros((2, m, n), bool)
    vals = [[[None] * n for _ in range(m)] for _ in range(2)]
    pending = []
    for i in range(m):
        for j in range(n):
            for c, comp in enumerate(("re", "im")):
                low = lo[comp][i, j]
                if low is None:
                    cert[c, i, j] = True
                    vals[c][i][j] = (0, 0)
                    continue
                b = entry_bound(prm, spA, spB, i, j, comp, int(trunc[comp][i, j]))
                a = int(acc[comp][i, j])
                if oz.certify(a, b, beta, p):
                    cert[c, i, j] = True
                    vals[c][i][j] = o1.round_nearest_even((a, low), p)
                else:
                    pending.append((c, i, j))
    if pending:
        exact_vals = {}
        for (i, j) in sorted({(i, j) for _, i, j in pending}):
            exact_vals[(i, j)] = fallback(i, j) if fallback else oz._exact_entry(A, B, i, j)
        for c, i, j in pending:
            vals[c][i][j] = o1.round_nearest_even(exact_vals[(i, j)][c], p)
    C = o1.pack(vals[0], vals[1], p)
    return ResidualResult(prm, spA, spB, table, groups, prods, acc, lo, trunc, top, cert, C)


def entry_bound(prm: oz.Params, spA, spB, i: int, j: int, comp: str, trunc: int) -> int:
    """Step 6: b with |Acc - T 2^-lo| <= b 2^beta."""
    b, beta = oz.entry_bound(prm, spA, spB, i, j, comp)
    return b + (-(-trunc >> beta))


def bound_exponent(prm: oz.Params) -> int:
    return oz.bound_exponent(prm)
