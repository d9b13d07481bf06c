"""The bench's roofline numerators on the CPU: the slice-pair count that sets the slice
GEMM's algorithmic FLOPs, against the oracle's own group tables and the closed forms."""
import os
import sys

import pytest

from oracle import ozaki

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


@pytest.mark.parametrize("p,k,method", [(128, 32, "4m"), (256, 256, "3m"), (512, 1024, "4m"),
                                        (1024, 2048, "3m"), (256, 40000, "3m"), (1024, 2048, "4m")])
def test_pair_count_equals_the_oracle_groups_and_the_closed_form(p, k, method):
    prm = ozaki.make_params(p, k, method)
    first = {"re": 0, "im": 0, "sum": -1}
    npos = {"re": prm.s, "im": prm.s, "sum": prm.s + 1}
    total = 0
    for pr in prm.products:
        wa, wb = ozaki.PRODUCT_OPERANDS[pr]
        gs = ozaki.groups_for((first[wa], first[wa] + npos[wa] - 1), (first[wb], first[wb] + npos[wb] - 1),
                              prm.Q, prm.gmax)
        total += sum(g.count for g in gs)
    assert bench.pair_count(prm.s, prm.Q, method) == total
    s = prm.s
    assert prm.Q == s - 1
    tri = s * (s + 1) // 2                        # t + u <= s - 1 on an s x s grid
    sums = (s + 1) ** 2 - s * (s - 1) // 2        # positions -1 .. s-1 for the 3M sums
    assert total == (4 * tri if method == "4m" else 2 * tri + sums)


def test_bench_workload_flops():
    """The headline figure: 22 021 kept pairs at m = n = k = 2048, p = 1024, 3M."""
    prm = ozaki.make_params(1024, 2048, "3m")
    assert (prm.s, prm.Q, prm.w) == (120, 119, 9)
    pairs = bench.pair_count(prm.s, prm.Q, "3m")
    assert pairs == 22021
    assert pairs * 2.0 * 2048 ** 3 == pytest.approx(3.78317899300864e14)
