"""Pins of O1 (exact product + one RNE rounding) against things other than itself."""
import random
from fractions import Fraction

import mpmath
import numpy as np
import pytest

import synthetic_inputs as si
from oracle import c_oracle, exact


def test_generator_format_and_distribution():
    p = 192
    A = si.random_matrix(64, 64, p, 7)
    L = si.limbs_for(p)
    nz = np.any(A.limb != 0, axis=1)
    # normalised: top bit set; at most p significant bits
    assert np.all((A.limb[:, L - 1] >> np.uint64(63))[nz] == 1)
    low_bits = 64 * L - p
    assert np.all((A.limb[:, 0] & np.uint64((1 << low_bits) - 1)) == 0)
    # uniform on [-1, 1): exponents <= 0, P(exp = 0) ~ 1/2, mean ~ 0
    assert np.all(A.exp[nz] <= 0)
    frac0 = np.mean(A.exp[nz] == 0)
    assert 0.45 < frac0 < 0.55
    vals = [float(exact.to_fraction(exact.component(A, 0, r, c))) for r in range(64) for c in range(64)]
    assert all(-1.0 <= v < 1.0 for v in vals)
    assert abs(np.mean(vals)) < 0.05 and abs(np.mean(np.abs(vals)) - 0.5) < 0.03


def _rand_exact(rng, nbits):
    N = rng.getrandbits(nbits) - (1 << (nbits - 1))
    return (N, rng.randint(-300, 300))


def test_rne_matches_python_float_p53():
    """Python's Fraction -> float conversion is correctly rounded (nearest-even)."""
    rng = random.Random(1)
    cases = [_rand_exact(rng, rng.randint(54, 200)) for _ in range(3000)]
    # explicit ties: odd 54-bit integers are exactly halfway between 53-bit neighbours
    cases += [((rng.getrandbits(52) | (1 << 53)) * 2 + 1, -60) for _ in range(500)]
    cases += [((rng.getrandbits(52) | (1 << 53)) * 2 + 1, 10) for _ in range(500)]
    for v in cases:
        N, x = exact.round_nearest_even(v, 53)
        assert float(exact.to_fraction((N, x))) == float(exact.to_fraction(v))


@pytest.mark.parametrize("p", [24, 100, 128, 256, 1024])
def test_rne_matches_mpmath(p):
    rng = random.Random(p)
    for _ in range(400):
        nbits = rng.randint(p + 1, p + 200)
        v = _rand_exact(rng, nbits)
        if rng.random() < 0.3:   # a tie: exactly one bit beyond p
            a = (rng.getrandbits(p) | (1 << p)) * 2 + 1
            v = (a if rng.random() < 0.5 else -a, rng.randint(-50, 50))
        N, x = exact.round_nearest_even(v, p)
        with mpmath.workprec(p):
            ref = mpmath.ldexp(mpmath.mpf(v[0]), v[1])   # rounds to p bits, nearest-even
        sgn, man, ex, _ = ref._mpf_       # value = (-1)**sgn * man * 2**ex
        assert Fraction(N) * Fraction(2) ** x == (-1) ** sgn * Fraction(int(man)) * Fraction(2) ** int(ex)


def _fraction_cgemm(A, B):
    """Eq. (simple_triple_loop) with Fractions: a different arithmetic route."""
    m, k, n = A.rows, A.cols, B.cols
    f = lambda M, c, r, col: exact.to_fraction(exact.component(M, c, r, col))
    re = [[sum((f(A, 0, i, l) * f(B, 0, l, j) - f(A, 1, i, l) * f(B, 1, l, j) for l in range(k)), Fraction(0))
           for j in range(n)] for i in range(m)]
    im = [[sum((f(A, 0, i, l) * f(B, 1, l, j) + f(A, 1, i, l) * f(B, 0, l, j) for l in range(k)), Fraction(0))
           for j in range(n)] for i in range(m)]
    return re, im


@pytest.mark.parametrize("seed", range(4))
def test_exact_matches_fraction_brute_force(seed):
    rng = np.random.default_rng(seed)
    m, k, n = (int(v) for v in rng.integers(1, 5, size=3))
    dist = "uniform_exp" if seed % 2 else "uniform"
    A = si.random_matrix(m, k, 128, 100 + seed, dist)
    B = si.random_matrix(k, n, 128, 200 + seed, dist, zero_frac=0.2)
    re, im = exact.exact_cgemm(A, B)
    fre, fim = _fraction_cgemm(A, B)
    for i in range(m):
        for j in range(n):
            assert exact.to_fraction(re[i][j]) == fre[i][j]
            assert exact.to_fraction(im[i][j]) == fim[i][j]


def test_small_integers_match_numpy_complex_matmul():
    """Small-integer operands: the exact product is numpy's complex128 matmul (exact here)."""
    A = si.small_integer_matrix(9, 13, 128, 5)
    B = si.small_integer_matrix(13, 7, 128, 6)

    def as_complex(M):
        vals = np.zeros((M.rows, M.cols), np.complex128)
        for r in range(M.rows):
            for c in range(M.cols):
                vals[r, c] = complex(float(exact.to_fraction(exact.component(M, 0, r, c))),
                                     float(exact.to_fraction(exact.component(M, 1, r, c))))
        return vals
    ref = as_complex(A) @ as_complex(B)
    C = exact.rounded_cgemm(A, B, 128)
    assert np.array_equal(as_complex(C), ref)
    C2 = c_oracle.rounded_cgemm_matrix(A, B, 128)
    assert exact.equal_arrays(C, C2)


@pytest.mark.parametrize("p", [64, 128, 200])
def test_identity_is_exact(p):
    A = si.random_matrix(6, 6, p, 9, "uniform_exp", zero_frac=0.1)
    eye = si.identity_matrix(6, p)
    assert exact.equal_arrays(exact.rounded_cgemm(A, eye, p), A)
    assert exact.equal_arrays(exact.rounded_cgemm(eye, A, p), A)


def test_3m_equals_4m_exactly():
    A = si.random_matrix(5, 6, 192, 21, "uniform_exp")
    B = si.random_matrix(6, 4, 192, 22, "uniform_exp", zero_frac=0.2)
    T4 = exact.exact_cgemm(A, B, "4m")
    T3 = exact.exact_cgemm(A, B, "3m")
    for c in range(2):
        for i in range(5):
            for j in range(4):
                assert exact.to_fraction(T4[c][i][j]) == exact.to_fraction(T3[c][i][j])


def test_block_linearity():
    """[A1 A2][B1; B2] = A1 B1 + A2 B2 exactly (the sum over l)."""
    p = 128
    A = si.random_matrix(4, 10, p, 31, "uniform_exp")
    B = si.random_matrix(10, 3, p, 32, "uniform_exp")
    full = exact.exact_cgemm(A, B)
    left = exact.exact_cgemm(A.submatrix(0, 4, 0, 6), B.submatrix(0, 6, 0, 3))
    right = exact.exact_cgemm(A.submatrix(0, 4, 6, 10), B.submatrix(6, 10, 0, 3))
    for c in range(2):
        for i in range(4):
            for j in range(3):
                assert exact.to_fraction(full[c][i][j]) == (exact.to_fraction(left[c][i][j])
                                                            + exact.to_fraction(right[c][i][j]))


def test_power_of_two_scaling():
    p = 256
    A = si.random_matrix(5, 7, p, 41)
    B = si.random_matrix(7, 6, p, 42, "uniform_exp")
    C = exact.rounded_cgemm(A, B, p)
    A2 = A.copy()
    nz = np.any(A2.limb != 0, axis=1)
    A2.exp = np.where(nz, A2.exp + 37, A2.exp).astype(np.int32)
    C2 = exact.rounded_cgemm(A2, B, p)
    nzc = np.any(C.limb != 0, axis=1)
    assert np.array_equal(C.limb, C2.limb) and np.array_equal(C.sign, C2.sign)
    assert np.array_equal(C2.exp[nzc], C.exp[nzc] + 37)


@pytest.mark.parametrize("p,dist,zf", [(64, "uniform", 0.0), (128, "uniform_exp", 0.1),
                                       (320, "uniform", 0.3), (1024, "uniform_exp", 0.0)])
def test_c_oracle_matches_python(p, dist, zf):
    A = si.random_matrix(7, 9, p, 51, dist, zero_frac=zf)
    B = si.random_matrix(9, 5, p, 52, dist, zero_frac=zf)
    assert exact.equal_arrays(exact.rounded_cgemm(A, B, p), c_oracle.rounded_cgemm_matrix(A, B, p))


def test_c_oracle_sampled_entries_match_full():
    p = 256
    A = si.random_matrix(20, 30, p, 61, "uniform_exp")
    B = si.random_matrix(30, 25, p, 62, "uniform_exp")
    full = c_oracle.rounded_cgemm_matrix(A, B, p)
    ent = np.array([(i, j) for i in range(0, 20, 3) for j in range(0, 25, 4)])
    sg, ex, li = c_oracle.rounded_cgemm(A, B, p, ent)
    for e, (i, j) in enumerate(ent):
        assert np.array_equal(sg[:, e], full.sign[:, i, j])
        assert np.array_equal(ex[:, e], full.exp[:, i, j])
        assert np.array_equal(li[:, :, e], full.limb[:, :, i, j])


def test_exponent_overflow_is_reported():
    p = 128
    A = si.random_matrix(2, 2, p, 71)
    B = si.random_matrix(2, 2, p, 72)
    A.exp[:] = np.where(np.any(A.limb != 0, axis=1), 2 ** 30 + 5, A.exp)
    B.exp[:] = np.where(np.any(B.limb != 0, axis=1), 2 ** 30 + 5, B.exp)
    with pytest.raises(exact.ExponentRangeError):
        exact.rounded_cgemm(A, B, p)
    with pytest.raises(exact.ExponentRangeError):
        c_oracle.rounded_cgemm_matrix(A, B, p)


def test_table1_operation_counts():
    """Table 1: 4M = 2 add/sub + 4 mul, 3M = 5 add/sub + 3 mul per complex product."""
    import ast
    import inspect
    import textwrap
    rows = {}
    for line in open(__file__.replace("test_oracle_exact.py", "golden/table1_op_counts.txt")):
        if line.strip() and not line.startswith("#"):
            meth, a, m_ = line.split()
            rows[meth] = (int(a), int(m_))
    # count the exact adds / products of each formula in O1's scalar step
    src = inspect.getsource(exact.exact_cgemm)
    tree = ast.parse(textwrap.dedent(src))
    counts = {}
    for node in ast.walk(tree):
        if isinstance(node, ast.If) and isinstance(node.test, ast.Compare):
            lit = getattr(node.test.comparators[0], "value", None)
            if lit in ("4m", "3m"):
                calls = [n.func.id for b in node.body for n in ast.walk(b)
                         if isinstance(n, ast.Call) and isinstance(n.func, ast.Name)]
                counts[lit] = (calls.count("add"), calls.count("mul"))
    assert counts == rows
