"""O1 -- exact complex matrix product, rounded once to p bits (TEST INFRASTRUCTURE).

This is the truth the CUDA path is checked against.  It is test
infrastructure: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline``/reference leg of ``bench.py`` may import it.  It shares no
code with the CUDA path.

What it computes (Kouya, Sec. III-A):

* Eq. (cmatmul) / (simple_triple_loop):  (C)_ij = sum_k (A)_ik (B)_kj.
* Eq. (4m_way_base): each scalar complex product as
  Re = ReA ReB - ImA ImB,  Im = ReA ImB + ImA ReB.
* Eq. (3m_way_base): the 3M form t1 = ReA ReB, t2 = ImA ImB,
  Re = t1 - t2, Im = (ReA + ImA)(ReB + ImB) - t1 - t2.  In exact arithmetic
  it equals the 4M form; both are offered so a test can check that.

All sums are exact (Python integers with a binary scale).  The only rounding
is the final one to a p-bit significand, round-to-nearest, ties-to-even
(the paper never names a rounding mode; MPFR's default is nearest-even).

Exact values are carried as pairs (N, x) meaning N * 2**x with N a signed
Python int.
"""
from __future__ import annotations

import numpy as np

INT32_MIN = -(2 ** 31)
INT32_MAX = 2 ** 31 - 1


class ExponentRangeError(ArithmeticError):
    """The rounded exponent does not fit the format's int32 exponent."""


# ---------------------------------------------------------------- decoding

def component(mat, c: int, r: int, col: int):
    """Exact value of component c (0 = Re, 1 = Im) of element (r, col).

    Format: value = (-1)**sign * M * 2**(exp - 64L), M = sum limb_j 2**(64 j);
    the component is zero iff its top limb is 0.
    Returns (N, x) with value = N * 2**x; zero is (0, 0).
    """
    L = mat.limb.shape[1]
    if int(mat.limb[c, L - 1, r, col]) == 0:
        return (0, 0)
    M = 0
    for j in range(L - 1, -1, -1):
        M = (M << 64) | int(mat.limb[c, j, r, col])
    if M == 0:
        return (0, 0)
    N = -M if int(mat.sign[c, r, col]) else M
    return (N, int(mat.exp[c, r, col]) - 64 * L)


def matrix_values(mat):
    """All components as (N, x) pairs: out[c][r][col]."""
    return [[[component(mat, c, r, col) for col in range(mat.cols)]
             for r in range(mat.rows)] for c in range(2)]


# ------------------------------------------------------------ exact sums

def add(a, b):
    """Exact sum of two scaled integers."""
    (na, xa), (nb, xb) = a, b
    if na == 0:
        return b
    if nb == 0:
        return a
    if xa <= xb:
        return (na + (nb << (xb - xa)), xa)
    return ((na << (xa - xb)) + nb, xb)


def neg(a):
    return (-a[0], a[1])


def mul(a, b):
    return (a[0] * b[0], a[1] + b[1])


def exact_cgemm(A, B, method: str = "4m"):
    """Exact T = A B as ([[Re (N,x)]], [[Im (N,x)]]) per Eqs. (4m_way_base)/(3m_way_base).

    The triple loop is the definition (Eq. simple_triple_loop) written out.
    """
    if A.cols != B.rows:
        raise ValueError("inner dimensions differ")
    a = matrix_values(A)
    b = matrix_values(B)
    m, k, n = A.rows, A.cols, B.cols
    re = [[(0, 0)] * n for _ in range(m)]
    im = [[(0, 0)] * n for _ in range(m)]
    for i in range(m):
        for j in range(n):
            sr, si = (0, 0), (0, 0)
            for l in range(k):
                ar, ai = a[0][i][l], a[1][i][l]
                br, bi = b[0][l][j], b[1][l][j]
                if method == "4m":
                    pr = add(mul(ar, br), neg(mul(ai, bi)))
                    pi = add(mul(ar, bi), mul(ai, br))
                elif method == "3m":
                    t1 = mul(ar, br)
                    t2 = mul(ai, bi)
                    pr = add(t1, neg(t2))
                    pi = add(add(mul(add(ar, ai), add(br, bi)), neg(t1)), neg(t2))
                else:
                    raise ValueError(method)
                sr = add(sr, pr)
                si = add(si, pi)
            re[i][j] = sr
            im[i][j] = si
    return re, im


# --------------------------------------------------------------- rounding

def round_nearest_even(v, p: int):
    """RN_p of an exact value v = (N, x): returns (N', x') with |N'| < 2**p.

    Round to nearest with ties to even, on a p-bit significand.  Unbounded
    exponent (the range check is done by ``encode``).
    """
    N, x = v
    if N == 0:
        return (0, 0)
    s = -1 if N < 0 else 1
    a = abs(N)
    n = a.bit_length()
    if n <= p:
        return (N, x)
    sh = n - p
    q = a >> sh
    r = a - (q << sh)
    half = 1 << (sh - 1)
    if r > half or (r == half and (q & 1)):
        q += 1
        if q >> p:            # carried into a new leading bit: 2**p
            q >>= 1
            sh += 1
    return (s * q, x + sh)


def encode(v, p: int):
    """Format fields (sign, exp, M) of a p-bit value v = (N, x) (|N| < 2**p).

    M is normalised to L = ceil(p/64) limbs; exp is checked against int32.
    """
    N, x = v
    L = (p + 63) // 64
    if N == 0:
        return (0, INT32_MIN, 0)
    a = abs(N)
    n = a.bit_length()
    assert n <= p
    M = a << (64 * L - n)
    e = x + n
    if e < INT32_MIN + 1 or e > INT32_MAX:
        raise ExponentRangeError(e)
    return (1 if N < 0 else 0, e, M)


def pack(values_re, values_im, p: int):
    """Pack rounded values into an ``MPCMatrix``-shaped set of arrays."""
    from synthetic_inputs import MPCMatrix  # container only, no arithmetic
    m = len(values_re)
    n = len(values_re[0]) if m else 0
    out = MPCMatrix.zeros(m, n, p)
    L = out.L
    for c, vals in enumerate((values_re, values_im)):
        for i in range(m):
            for j in range(n):
                s, e, M = encode(vals[i][j], p)
                out.sign[c, i, j] = s
                out.exp[c, i, j] = e
                for t in range(L):
                    out.limb[c, t, i, j] = (M >> (64 * t)) & 0xFFFFFFFFFFFFFFFF
    return out


def rounded_cgemm(A, B, p: int, method: str = "4m"):
    """O1: RN_p(A B), packed in the device format."""
    re, im = exact_cgemm(A, B, method)
    rre = [[round_nearest_even(v, p) for v in row] for row in re]
    rim = [[round_nearest_even(v, p) for v in row] for row in im]
    return pack(rre, rim, p)


def to_fraction(v):
    from fractions import Fraction
    N, x = v
    return Fraction(N) * (Fraction(2) ** x)


def relative_error_ulps(got, exact, p: int) -> float:
    """|got - exact| / |exact| in units of 2**-p (inf if exact == 0 != got)."""
    from fractions import Fraction
    g, e = to_fraction(got), to_fraction(exact)
    if e == 0:
        return 0.0 if g == 0 else float("inf")
    return float(abs(g - e) / abs(e) * (Fraction(2) ** p))


def equal_arrays(X, Y) -> bool:
    return (np.array_equal(X.sign, Y.sign) and np.array_equal(X.exp, Y.exp)
            and np.array_equal(X.limb, Y.limb))
