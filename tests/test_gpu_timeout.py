"""A bounded device wait of the tcgen05 slice GEMM that runs out.

Every mbarrier wait of the tcgen05 kernels is bounded.  With a per-call limit
of 1000 SM cycles (mpc_oz_params.wait_limit_cycles; the waits then poll, so
the limit is exact) the epilogue's first wait must run out: the first chunk
alone is 4 k-blocks of 128 x 256 x 64 bf16 MMAs, about 2048 tensor-core
cycles, after the TMA loads that feed it.  The kernel must then set
mpc_status.device_timeout, let its copies and MMAs land, free its tensor
memory and return, so that the next call with the default limit is exact
again.  Nothing here faults, traps or hangs the GPU: every wait is bounded
and the abort path waits only with bounded waits.
"""
import pytest

import synthetic_inputs as si
from oracle import c_oracle
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kernel", ["tcgen05", "tcgen05_2sm", "tcgen05_n128", "tcgen05_2sm_n128"])
def test_wait_limit_runs_out_then_next_call_is_exact(kernel):
    p = 256
    A = si.random_matrix(256, 512, p, 71, "uniform")
    B = si.random_matrix(512, 256, p, 72, "uniform")
    ref = c_oracle.rounded_cgemm_matrix(A, B, p)
    _, _, st = gu.run(A, B, p, "4m", "ozaki", params=dict(kernel=kernel, wait_limit_cycles=1000))
    assert st["device_timeout"] != 0
    for _ in range(2):
        C, _, st = gu.run(A, B, p, "4m", "ozaki", params=dict(kernel=kernel))
        assert st["device_timeout"] == 0
        assert gu.same(C, ref)
