"""Oracle for the blocked complex LU solve (TEST INFRASTRUCTURE).

Only tests/ and bench.py's CPU legs use this module; it shares no code with
the CUDA path.  It follows the paper's LU (Kouya, Sec. IV-C, Fig. 3): the
matrix is factored K columns at a time, and after each panel the rectangle
A22 - L21 U12 is updated by one complex matrix product; K = 1 is "Normal
LU".  The solve is forward then backward substitution (Sec. IV-C).  The
paper does not fix the pivoting, the loop orders or where results are
rounded; this library's reading, which the GPU path implements, is:

* pivot of column j: the first row i >= j maximising RN_p(|Re a_ij| + |Im a_ij|);
  rows are swapped across the whole matrix;
* l_ij = RN_p(a_ij / a_jj) componentwise from the exact complex quotient;
* a_ic = RN_p(a_ic - l_ij a_jc) componentwise from the exact complex value,
  column by column (j), for the rest of the panel; after the panel (all its
  row interchanges done) the same update, j = kb..kend-1, gives U12;
* trailing update: P = RN_p(L21 U12) (the exact product, rounded once, as the
  complex GEMM returns it), then A22 = RN_p(A22 - P) componentwise;
* solve: b permuted by the swaps in order; y_i = RN_p(y_i - l_ij y_j) for
  j = 0..n-1, i > j; then x_j = RN_p(y_j / u_jj) and y_i = RN_p(y_i - u_ij x_j)
  for j = n-1..0, i < j.

Values are exact pairs (N, x) = N * 2**x as in ``oracle.exact``.
"""
from __future__ import annotations

from . import exact as o1


class SingularMatrix(ArithmeticError):
    pass


def rn(v, p):
    return o1.round_nearest_even(v, p)


def absval(v):
    return (abs(v[0]), v[1])


def round_rational(num, den, p):
    """RN_p(num / den) for exact values num = (Nn, xn), den = (Nd, xd), den != 0.

    Correct rounding of a rational: an integer quotient with at least p + 3
    bits plus a sticky bit for a nonzero remainder, rounded once.
    """
    (Nn, xn), (Nd, xd) = num, den
    if Nd == 0:
        raise ZeroDivisionError
    if Nn == 0:
        return (0, 0)
    neg = (Nn < 0) != (Nd < 0)
    a, d = abs(Nn), abs(Nd)
    k = p + 3 + d.bit_length() - a.bit_length()
    if k >= 0:
        q, r = divmod(a << k, d)
    else:
        q, r = divmod(a, d << (-k))
    v = (2 * q + (1 if r else 0)) * (-1 if neg else 1)
    return rn((v, xn - xd - k - 1), p)


def cdiv(a, d, p):
    """Componentwise RN_p of the exact complex quotient a / d."""
    (ar, ai), (dr, di) = a, d
    den = o1.add(o1.mul(dr, dr), o1.mul(di, di))
    nre = o1.add(o1.mul(ar, dr), o1.mul(ai, di))
    nim = o1.add(o1.mul(ai, dr), o1.neg(o1.mul(ar, di)))
    return (round_rational(nre, den, p), round_rational(nim, den, p))


def cfma(a, l, u, p):
    """Componentwise RN_p of the exact a - l u."""
    (ar, ai), (lr, li), (ur, ui) = a, l, u
    re = o1.add(ar, o1.add(o1.neg(o1.mul(lr, ur)), o1.mul(li, ui)))
    im = o1.add(ai, o1.neg(o1.add(o1.mul(lr, ui), o1.mul(li, ur))))
    return (rn(re, p), rn(im, p))


def key(a, p):
    return o1.to_fraction(rn(o1.add(absval(a[0]), absval(a[1])), p))


def lu_solve(A, Bm, p: int, K: int):
    """Factor A (MPCMatrix n x n) and solve A X = B (n x nrhs).

    Returns (LU as [[(re, im)]], ipiv list, X as [[(re, im)]]); raises
    SingularMatrix if a pivot is zero.
    """
    n = A.rows
    vals = o1.matrix_values(A)
    a = [[(vals[0][i][j], vals[1][i][j]) for j in range(n)] for i in range(n)]
    bv = o1.matrix_values(Bm)
    nrhs = Bm.cols
    b = [[(bv[0][i][c], bv[1][i][c]) for c in range(nrhs)] for i in range(n)]
    ipiv = []
    for kb in range(0, n, K):
        kend = min(kb + K, n)
        for j in range(kb, kend):
            piv, best = j, key(a[j][j], p)
            for i in range(j + 1, n):
                kv = key(a[i][j], p)
                if kv > best:
                    piv, best = i, kv
            if best == 0:
                raise SingularMatrix(j)
            ipiv.append(piv)
            a[j], a[piv] = a[piv], a[j]
            for i in range(j + 1, n):
                a[i][j] = cdiv(a[i][j], a[j][j], p)
            for i in range(j + 1, n):
                for c in range(j + 1, kend):
                    a[i][c] = cfma(a[i][c], a[i][j], a[j][c], p)
        # U12 = L11^-1 A12 once the panel's row interchanges are all applied
        for j in range(kb, kend):
            for i in range(j + 1, kend):
                for c in range(kend, n):
                    a[i][c] = cfma(a[i][c], a[i][j], a[j][c], p)
        if kend < n:
            for i in range(kend, n):
                for c in range(kend, n):
                    sr, si = (0, 0), (0, 0)
                    for t in range(kb, kend):
                        (lr, li), (ur, ui) = a[i][t], a[t][c]
                        sr = o1.add(sr, o1.add(o1.mul(lr, ur), o1.neg(o1.mul(li, ui))))
                        si = o1.add(si, o1.add(o1.mul(lr, ui), o1.mul(li, ur)))
                    pr, pi = rn(sr, p), rn(si, p)
                    ar, ai = a[i][c]
                    a[i][c] = (rn(o1.add(ar, o1.neg(pr)), p), rn(o1.add(ai, o1.neg(pi)), p))
    return a, ipiv, substitute(a, ipiv, b, p)


def substitute(a, ipiv, b, p: int):
    """The solve with given factors (Sec. IV-C): b := P b by the interchanges in order,
    forward substitution with the unit lower triangle of `a`, backward substitution
    with its upper triangle; every operation rounded once (RN_p), column-oriented.
    `a` is n x n and `b` n x nrhs, both lists of rows of (re, im) exact values; `b`
    is overwritten and returned."""
    n, nrhs = len(a), (len(b[0]) if b else 0)
    for j in range(n):
        r = ipiv[j]
        b[j], b[r] = b[r], b[j]
    for c in range(nrhs):
        for j in range(n):
            for i in range(j + 1, n):
                b[i][c] = cfma(b[i][c], a[i][j], b[j][c], p)
        for j in range(n - 1, -1, -1):
            b[j][c] = cdiv(b[j][c], a[j][j], p)
            for i in range(j):
                b[i][c] = cfma(b[i][c], a[i][j], b[j][c], p)
    return b


def pack_values(rows, p):
    """[[(re, im)]] -> MPCMatrix (format arrays).

    Entries the factorisation never changed keep the input's mantissa, whose integer
    carries the 64L - p zero bits below the p-bit grid; rounding a p-bit value to p bits
    returns the same value with a mantissa of at most p bits, as the format wants."""
    re = [[rn(v[0], p) for v in row] for row in rows]
    im = [[rn(v[1], p) for v in row] for row in rows]
    return o1.pack(re, im, p)
