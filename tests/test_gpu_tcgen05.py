"""The tcgen05 slice-GEMM kernel against the mma.sync kernel and the oracle.

Both kernels compute the same exact int32 group sums; every group plane must
agree bit for bit, the outputs must equal O1, and no bounded wait may time out.
Shapes cover single and many tiles, ragged M / N / K edges, 3M sum digits,
units of one pair and of 15 pairs (9-bit digits: 120 chunks of 256 elements) or
63 pairs (8-bit digits: 960-element chunks), both TMEM buffers, and more units
than SMs (persistent loop).  Kernels: single CTAs with 128 x 256 tiles (two TMEM
accumulators) and with 128 x 128 tiles (four), and CTA pairs running one 256-row
cta_group::2 MMA.  The single-CTA kernels tile C^T = B^T A^T (stored transposed) where
that pads less; the cases below include such shapes.
"""
import numpy as np
import pytest

import synthetic_inputs as si
from oracle import c_oracle
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu

CASES = [
    # m, k, n, p, method, dist, digit bits
    (128, 64, 256, 128, "4m", "uniform", 9),        # exactly one tile, one k-block per pair
    (200, 150, 300, 128, "4m", "uniform_exp", 9),   # ragged tiles and k tail
    (37, 70, 29, 192, "3m", "uniform_exp", 9),      # smaller than one tile
    (260, 2048, 520, 128, "3m", "uniform", 9),      # 15-pair groups: 120 chunks per unit
    (260, 2048, 520, 128, "3m", "uniform", 8),      # 63-pair groups of 8-bit digits: 135 chunks
    (512, 320, 768, 256, "4m", "uniform", 9),       # many units per CTA
    # shapes the single-CTA 128 x 256 tiles cover with less padding as C^T = B^T A^T
    # (the 200 x 300 case above is one too)
    (300, 130, 90, 192, "4m", "uniform_exp", 9),
    (520, 2048, 260, 128, "3m", "uniform", 9),
    (1000, 64, 40, 128, "4m", "uniform", 8),
]


def _planes(A, B, p, method, kernel, w):
    prm = dict(kernel=kernel, digit_bits=w)
    C, ws, st = gu.run(A, B, p, method, "ozaki", params=prm)
    pl = gu.plan(A, B, p, method, params=prm)
    return C, gu.ws_groups(ws, pl, A.rows, B.cols), st


@pytest.mark.parametrize("kernel", ["tcgen05", "tcgen05_2sm", "tcgen05_n128", "tcgen05_2sm_n128"])
@pytest.mark.parametrize("m,k,n,p,method,dist,w", CASES)
def test_tcgen05_matches_mma_sync_and_oracle(m, k, n, p, method, dist, w, kernel):
    """(260 rows = 3 row tiles: the 2-SM kernel's second CTA of the last pair has no rows.)"""
    A = si.random_matrix(m, k, p, 500 + m, dist)
    B = si.random_matrix(k, n, p, 600 + n, dist)
    Ct, Gt, st_t = _planes(A, B, p, method, kernel, w)
    Cm, Gm, st_m = _planes(A, B, p, method, "mma_sync", w)
    assert st_t["device_timeout"] == 0
    bad = np.argwhere(Gt != Gm)
    assert len(bad) == 0, f"{len(bad)} group-sum mismatches, first {bad[:4].tolist()}"
    assert gu.same(Ct, Cm)
    ref = c_oracle.rounded_cgemm_matrix(A, B, p)
    assert gu.same(Ct, ref)
