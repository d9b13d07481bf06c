"""Pins of the LU oracle against things other than itself."""
import random
from fractions import Fraction

import mpmath
import numpy as np
import pytest

import synthetic_inputs as si
from oracle import exact, lu


def test_round_rational_matches_float_division_p53():
    rng = random.Random(5)
    for _ in range(2000):
        n = (rng.getrandbits(rng.randint(1, 160)) - (1 << 40), rng.randint(-50, 50))
        d = (rng.getrandbits(rng.randint(1, 160)) + 1, rng.randint(-50, 50))
        if n[0] == 0:
            continue
        got = exact.to_fraction(lu.round_rational(n, d, 53))
        assert got == Fraction(float(exact.to_fraction(n) / exact.to_fraction(d)))


@pytest.mark.parametrize("p", [64, 128, 333])
def test_round_rational_matches_mpmath(p):
    rng = random.Random(p)
    for _ in range(300):
        n = (rng.getrandbits(rng.randint(1, 400)) * rng.choice((-1, 1)), rng.randint(-80, 80))
        d = (rng.getrandbits(rng.randint(1, 400)) + 1, rng.randint(-80, 80))
        if n[0] == 0:
            continue
        got = exact.to_fraction(lu.round_rational(n, d, p))
        with mpmath.workprec(1200):   # operands exact
            xa = mpmath.ldexp(mpmath.mpf(n[0]), n[1])
            xb = mpmath.ldexp(mpmath.mpf(d[0]), d[1])
        q = mpmath.fdiv(xa, xb, prec=p, rounding="n")
        s, man, ex, _ = q._mpf_
        assert got == (-1) ** s * Fraction(int(man)) * Fraction(2) ** int(ex)


def _to_complex(M):
    out = np.zeros((M.rows, M.cols), np.complex128)
    for r in range(M.rows):
        for c in range(M.cols):
            out[r, c] = complex(float(exact.to_fraction(exact.component(M, 0, r, c))),
                                float(exact.to_fraction(exact.component(M, 1, r, c))))
    return out


@pytest.mark.parametrize("K", [1, 4, 12])
def test_pivots_match_lapack_zgetrf(K):
    """|.|_1 partial pivoting: the same row interchanges as LAPACK on the float64 copy."""
    scipy_linalg = pytest.importorskip("scipy.linalg")
    n, p = 12, 192
    A = si.random_matrix(n, n, p, 41 + K)
    b = si.random_matrix(n, 1, p, 42)
    _, ipiv, _ = lu.lu_solve(A, b, p, K)
    _, piv = scipy_linalg.lu_factor(_to_complex(A))
    assert ipiv == list(piv)


def test_factors_reconstruct_the_permuted_matrix():
    n, p, K = 10, 160, 4
    A = si.random_matrix(n, n, p, 51)
    b = si.random_matrix(n, 1, p, 52)
    a, ipiv, _ = lu.lu_solve(A, b, p, K)
    PA = [[(exact.component(A, 0, i, j), exact.component(A, 1, i, j)) for j in range(n)] for i in range(n)]
    for j, r in enumerate(ipiv):
        PA[j], PA[r] = PA[r], PA[j]
    F = lambda v: complex(0) if v is None else v
    worst = 0.0
    for i in range(n):
        for j in range(n):
            acc_r, acc_i = Fraction(0), Fraction(0)
            for t in range(min(i, j) + 1):
                lr, li = ((Fraction(1), Fraction(0)) if t == i else
                          (exact.to_fraction(a[i][t][0]), exact.to_fraction(a[i][t][1])))
                ur, ui = exact.to_fraction(a[t][j][0]), exact.to_fraction(a[t][j][1])
                acc_r += lr * ur - li * ui
                acc_i += lr * ui + li * ur
            er = abs(acc_r - exact.to_fraction(PA[i][j][0]))
            ei = abs(acc_i - exact.to_fraction(PA[i][j][1]))
            worst = max(worst, float(max(er, ei)) * 2.0 ** p)
    assert worst < 64 * n          # |PA - LU| <= O(n) ulps of entries of size <= 1


def test_solution_error_and_mpmath_agreement():
    """Diagonally dominant A, x = 1 + i: x is recovered to ~2^-p; mpmath's lu_solve agrees."""
    n, p, K = 8, 128, 3
    rng = np.random.default_rng(3)
    vals = rng.integers(-9, 10, size=(2, n, n))
    vals[0] += np.eye(n, dtype=np.int64) * 100
    A = si.from_integers(vals, p)
    x_true = np.zeros((2, n, 1), np.int64)
    x_true[:] = 1
    # b = A x exactly (small integers)
    Ac = vals[0] + 1j * vals[1]
    bc = Ac @ (np.ones(n) * (1 + 1j))
    bv = np.stack([bc.real.astype(np.int64)[:, None], bc.imag.astype(np.int64)[:, None]])
    b = si.from_integers(bv, p)
    _, _, x = lu.lu_solve(A, b, p, K)
    for i in range(n):
        for c in range(2):
            err = abs(exact.to_fraction(x[i][0][c]) - 1)
            assert err < Fraction(1, 2 ** (p - 8))
    with mpmath.workprec(p):
        M = mpmath.matrix([[mpmath.mpc(int(vals[0, i, j]), int(vals[1, i, j])) for j in range(n)] for i in range(n)])
        rhs = mpmath.matrix([mpmath.mpc(float(bc[i].real), float(bc[i].imag)) for i in range(n)])
        xm = mpmath.lu_solve(M, rhs)
        for i in range(n):
            assert abs(complex(xm[i]) - complex(float(exact.to_fraction(x[i][0][0])),
                                                float(exact.to_fraction(x[i][0][1])))) < 1e-30


def test_identity_and_singular():
    n, p = 6, 128
    I = si.identity_matrix(n, p)
    b = si.random_matrix(n, 2, p, 61)
    a, ipiv, x = lu.lu_solve(I, b, p, 4)
    assert ipiv == list(range(n))
    X = lu.pack_values(x, p)
    assert exact.equal_arrays(X, b)
    S = si.random_matrix(n, n, p, 62)
    S.limb[:, :, :, 2] = 0          # a zero column
    with pytest.raises(lu.SingularMatrix):
        lu.lu_solve(S, b, p, 2)


def test_substitution_solves_an_exact_triangular_system():
    """The solve with given factors, pinned by the residual: L and U hold small complex
    integers with unit or power-of-two diagonals, so at p = 64 no operation rounds and
    the returned x must satisfy (L U) x = P b exactly (checked in Fractions, by matrix
    products rather than by substitution)."""
    rnd = random.Random(11)
    n, p = 7, 64

    def cval(re, im):
        return ((re, 0), (im, 0))

    a = [[None] * n for _ in range(n)]
    for i in range(n):
        for j in range(n):
            if i == j:
                a[i][j] = rnd.choice([cval(1, 0), cval(-2, 0), cval(0, 1), cval(4, 0), cval(0, -2)])
            else:
                a[i][j] = cval(rnd.randint(-3, 3), rnd.randint(-3, 3))
    ipiv = [rnd.randint(j, n - 1) for j in range(n)]
    b = [[cval(rnd.randint(-5, 5), rnd.randint(-5, 5))] for _ in range(n)]
    x = lu.substitute(a, ipiv, [row[:] for row in b], p)

    def cf(v):
        return complex_frac(exact.to_fraction(v[0]), exact.to_fraction(v[1]))

    def complex_frac(re, im):
        return (re, im)

    def cmul(u, v):
        return (u[0] * v[0] - u[1] * v[1], u[0] * v[1] + u[1] * v[0])

    def cadd(u, v):
        return (u[0] + v[0], u[1] + v[1])

    zero = (Fraction(0), Fraction(0))
    Lm = [[cf(a[i][j]) if i > j else ((Fraction(1), Fraction(0)) if i == j else zero) for j in range(n)]
          for i in range(n)]
    Um = [[cf(a[i][j]) if i <= j else zero for j in range(n)] for i in range(n)]
    LU = [[zero] * n for _ in range(n)]
    for i in range(n):
        for j in range(n):
            s = zero
            for t in range(n):
                s = cadd(s, cmul(Lm[i][t], Um[t][j]))
            LU[i][j] = s
    pb = [cf(row[0]) for row in b]
    for j in range(n):                     # P b: the interchanges in order
        r = ipiv[j]
        pb[j], pb[r] = pb[r], pb[j]
    xs = [cf(row[0]) for row in x]
    for i in range(n):
        s = zero
        for j in range(n):
            s = cadd(s, cmul(LU[i][j], xs[j]))
        assert s == pb[i], i
