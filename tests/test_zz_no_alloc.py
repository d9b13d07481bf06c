"""mpcgemm_noalloc: the entry point for callers that cannot allocate device memory.

It runs the same complex GEMM as mpcgemm() but keeps its scratch in a static
device array of the library instead of a caller workspace.  The test calls it
through the C ABI twice in a row (different inputs, so a stale scratch would
show) and compares each result with mpcgemm()'s on the same inputs -- the
tolerance of every other parity test here, i.e. bit for bit --, reads the
device status of each call back through mpcgemm_noalloc_read_status (which
must show no error), and checks that a problem larger than the array is
refused with MPC_ENOSPC.  The file is named
to be collected last; it passes alone in a fresh process and after the rest.
"""
import ctypes

import numpy as np
import pytest

import synthetic_inputs as si
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu


def _noalloc(A, B, p, method, algo):
    import torch
    M = gu.mp()
    m, k, n = A.rows, A.cols, B.cols
    dA, dB = M.DeviceMatrix.from_mpc(A), M.DeviceMatrix.from_mpc(B)
    dC = M.DeviceMatrix.empty(m, n, p)
    sa, sb, sc = dA.struct(), dB.struct(), dC.struct()
    stream = torch.cuda.current_stream()
    rc = M.lib().mpcgemm_noalloc(m, n, k, p, ctypes.byref(sa), ctypes.byref(sb), ctypes.byref(sc),
                                 M._native.METHODS[method], M._native.ALGOS[algo], int(stream.cuda_stream))
    assert rc == 0, M.strerror(rc)
    st = M._native.Status()
    rc = M.lib().mpcgemm_noalloc_read_status(ctypes.byref(st), int(stream.cuda_stream))
    assert rc == 0, M.strerror(rc)
    assert (st.erange, st.fallback_overflow, st.uncertified, st.device_timeout) == (0, 0, 0, 0)
    torch.cuda.synchronize()
    s, e, l = dC.to_host()
    return si.MPCMatrix(m, n, p, s, e, l)


@pytest.mark.parametrize("method,algo,p", [("3m", "ozaki", 256), ("4m", "ozaki", 192), ("4m", "plain", 320)])
def test_noalloc_matches_mpcgemm_twice(method, algo, p):
    for call, seed in enumerate((901, 917)):
        A = si.random_matrix(150 + 7 * call, 130, p, seed, "uniform_exp", zero_frac=0.05)
        B = si.random_matrix(130, 140 - 5 * call, p, seed + 1, "uniform_exp")
        got = _noalloc(A, B, p, method, algo)
        ref, _, _ = gu.run(A, B, p, method, algo)
        bad = gu.mismatches(got, ref)
        assert len(bad) == 0, f"call {call}: {len(bad)} components differ, first {bad[:4].tolist()}"


def test_noalloc_refuses_problems_larger_than_its_array():
    M = gu.mp()
    d = M._native.MpcMat()
    big = 1024
    d.rows = d.cols = d.ld = big
    for c in range(2):
        d.sign[c] = d.exp[c] = d.limb[c] = 0x1000
    assert M.plan(big, big, big, 1024, "3m", "ozaki")["ws_bytes"] > M._native.NOALLOC_SCRATCH_BYTES
    rc = M.lib().mpcgemm_noalloc(big, big, big, 1024, ctypes.byref(d), ctypes.byref(d), ctypes.byref(d), 1, 1, None)
    assert rc == -28
