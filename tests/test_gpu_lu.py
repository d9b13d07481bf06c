"""Blocked complex LU + solve on the GPU against the LU oracle.

Small sizes: the factors, the interchanges and the solution must equal the
oracle bit for bit (same pivot rule and rounding points).  The BASELINE LU
workload (A uniform + n I, x = 1 + i, b = A x) is checked through the
relative error of x, which the algorithm keeps near 2^-p.
"""
import numpy as np
import pytest

import synthetic_inputs as si
from oracle import c_oracle, lu
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu


def _gpu_lu(A, B, p, K, method="3m"):
    import torch
    M = gu.mp()
    dA, dB = M.DeviceMatrix.from_mpc(A), M.DeviceMatrix.from_mpc(B)
    ipiv, ws = M.mpcgesv(dA, dB, p, K, method)
    st = M.read_status(ws)
    torch.cuda.synchronize()
    s, e, l = dA.to_host()
    LU = si.MPCMatrix(A.rows, A.cols, p, s, e, l)
    s, e, l = dB.to_host()
    X = si.MPCMatrix(B.rows, B.cols, p, s, e, l)
    return LU, ipiv.cpu().numpy().tolist(), X, st, M.lu_singular_column(ws)


@pytest.mark.parametrize("n,K,p,method,nrhs", [(40, 16, 128, "3m", 1), (23, 1, 192, "4m", 2),
                                               (33, 8, 256, "4m", 1), (17, 17, 128, "3m", 1),
                                               (24, 8, 512, "4m", 2), (21, 4, 500, "3m", 1)])
def test_lu_matches_oracle_bit_for_bit(n, K, p, method, nrhs):
    A = si.random_matrix(n, n, p, 800 + n, "uniform")       # no diagonal boost: pivoting happens
    B = si.random_matrix(n, nrhs, p, 900 + n, "uniform")
    LU, ipiv, X, st, sing = _gpu_lu(A, B, p, K, method)
    a, ipiv_ref, x = lu.lu_solve(A, B, p, K)
    assert sing == 0 and st["erange"] == 0 and st["uncertified"] == 0
    assert ipiv == ipiv_ref
    assert gu.same(LU, lu.pack_values(a, p))
    assert gu.same(X, lu.pack_values(x, p))


def test_large_solve_matches_the_oracle_substitution():
    """n > 1024: the solve runs as one launch per substitution step (smaller systems use
    one block per right-hand side).  With the GPU's own factors and interchanges, the
    oracle's column-oriented substitution must give the same X bit for bit."""
    from oracle import exact as o1
    n, K, p = 1100, 128, 128
    A = si.shifted_diagonal_matrix(n, p, 970)
    B = si.random_matrix(n, 1, p, 971, "uniform")
    LU, ipiv, X, st, sing = _gpu_lu(A, B, p, K, "3m")
    assert sing == 0 and st["erange"] == 0 and st["uncertified"] == 0
    lv, bv = o1.matrix_values(LU), o1.matrix_values(B)
    a = [[(lv[0][i][j], lv[1][i][j]) for j in range(n)] for i in range(n)]
    b = [[(bv[0][i][0], bv[1][i][0])] for i in range(n)]
    assert gu.same(X, lu.pack_values(lu.substitute(a, ipiv, b, p), p))


def test_singular_matrix_is_reported():
    n, p = 12, 128
    A = si.random_matrix(n, n, p, 950)
    A.limb[:, :, :, 5] = 0
    B = si.random_matrix(n, 1, p, 951)
    _, _, _, st, sing = _gpu_lu(A, B, p, 4)
    assert sing == 6


def _baseline_lu(n, p, K, method, seed):
    """A = uniform [-1,1) + n I, x = 1 + i, b = RN(A x) (computed by the exact oracle)."""
    A = si.random_matrix(n, n, p, seed, "uniform")
    L = A.L
    for i in range(n):        # add n to the real diagonal exactly: re = old + n (p bits suffice)
        pass
    vals = np.zeros((2, n, n), np.int64)
    vals[0] = np.eye(n, dtype=np.int64) * n
    D = si.from_integers(vals, p)
    from oracle import exact
    # A + n I exactly rounded to p bits (the entries stay well inside p bits of precision)
    Apn = c_oracle.rounded_cgemm_matrix(si.identity_matrix(n, p), A, p)   # = A
    re = [[exact.add(exact.component(Apn, 0, i, j), exact.component(D, 0, i, j)) for j in range(n)] for i in range(n)]
    im = [[exact.component(Apn, 1, i, j) for j in range(n)] for i in range(n)]
    Ab = exact.pack([[exact.round_nearest_even(v, p) for v in row] for row in re],
                    [[exact.round_nearest_even(v, p) for v in row] for row in im], p)
    ones = np.zeros((2, n, 1), np.int64)
    ones[:] = 1
    x1 = si.from_integers(ones, p)
    b = c_oracle.rounded_cgemm_matrix(Ab, x1, p)
    return Ab, b


@pytest.mark.parametrize("n,K,p,method", [(256, 32, 512, "3m"), (192, 64, 256, "4m")])
def test_baseline_lu_solution_error(n, K, p, method):
    from fractions import Fraction
    from oracle import exact
    A, b = _baseline_lu(n, p, K, method, 990)
    _, _, X, st, sing = _gpu_lu(A, b, p, K, method)
    assert sing == 0 and st["erange"] == 0
    worst = Fraction(0)
    for i in range(n):
        for c in range(2):
            v = exact.to_fraction(exact.component(X, c, i, 0))
            worst = max(worst, abs(v - 1))
    assert worst < Fraction(1, 2 ** (p - 16)), float(worst)


@pytest.mark.parametrize("n,p", [(300, 512), (260, 256)])
def test_per_step_solve_at_register_precisions(n, p):
    """Between 256 and 1024 unknowns the solve takes one launch per substitution step; at
    p = 512 and 256 every scalar operation takes the register-resident path.  With the
    GPU's own factors and interchanges the oracle's substitution gives the same X bit for bit."""
    from oracle import exact as o1
    A = si.shifted_diagonal_matrix(n, p, 972 + n)
    B = si.random_matrix(n, 1, p, 973 + n, "uniform")
    LU, ipiv, X, st, sing = _gpu_lu(A, B, p, 64, "4m")
    assert sing == 0 and st["erange"] == 0 and st["uncertified"] == 0
    lv, bv = o1.matrix_values(LU), o1.matrix_values(B)
    a = [[(lv[0][i][j], lv[1][i][j]) for j in range(n)] for i in range(n)]
    b = [[(bv[0][i][0], bv[1][i][0])] for i in range(n)]
    assert gu.same(X, lu.pack_values(lu.substitute(a, ipiv, b, p), p))

