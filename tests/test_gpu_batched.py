"""Batched complex GEMM: one persistent tcgen05 launch over many uneven problems.

Every problem of a batch must give exactly what a single mpcgemm call gives
(bit for bit), which equals the exact oracle; the batch may mix sizes,
precisions, methods, algorithms and empty problems, exceed one launch's 48
problems, and be captured in a CUDA graph and replayed.
"""
import numpy as np
import pytest

import synthetic_inputs as si
from oracle import c_oracle
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu


def _make(specs, seed):
    M = gu.mp()
    probs, host = [], []
    for x, (m, k, n, p, method, algo) in enumerate(specs):
        A = si.random_matrix(m, k, p, seed + 2 * x, "uniform_exp")
        B = si.random_matrix(k, n, p, seed + 2 * x + 1, "uniform_exp")
        dA, dB = M.DeviceMatrix.from_mpc(A), M.DeviceMatrix.from_mpc(B)
        dC = M.DeviceMatrix.empty(m, n, p)
        probs.append((dA, dB, dC, p, method, algo))
        host.append((A, B))
    return probs, host


def _result(dC, p):
    s, e, l = dC.to_host()
    return si.MPCMatrix(dC.rows, dC.cols, p, s, e, l)


SPECS = [(200, 150, 300, 256, "3m", "ozaki"), (64, 64, 64, 1024, "4m", "ozaki"), (37, 70, 29, 512, "3m", "ozaki"),
         (130, 33, 260, 128, "4m", "ozaki"), (96, 80, 112, 320, "4m", "plain"), (5, 0, 7, 128, "4m", "ozaki"),
         (0, 10, 4, 128, "3m", "ozaki"), (257, 129, 65, 192, "3m", "ozaki")]


@pytest.mark.parametrize("kernel", ["auto", "tcgen05", "mma_sync"])
def test_batched_equals_single_calls_and_oracle(kernel):
    import torch
    M = gu.mp()
    probs, host = _make(SPECS, 700)
    ws = M.mpcgemm_batched(probs, params=dict(kernel=kernel))
    torch.cuda.synchronize()
    total, offs = M.batched_workspace(probs, dict(kernel=kernel))
    for x, ((dA, dB, dC, p, method, algo), (A, B)) in enumerate(zip(probs, host)):
        got = _result(dC, p)
        single, _, _ = gu.run(A, B, p, method, algo)
        assert gu.same(got, single), (x, SPECS[x])
        if A.rows * B.cols and A.cols:
            assert gu.same(got, c_oracle.rounded_cgemm_matrix(A, B, p)), (x, SPECS[x])
        st = M.read_status(ws, offset=offs[x])
        assert st["device_timeout"] == 0 and st["erange"] == 0


def test_batch_larger_than_one_launch():
    import torch
    M = gu.mp()
    specs = [(16 + x % 40, 24, 20 + 2 * (x % 40), 128 + 64 * (x % 3), "3m" if x % 2 else "4m", "ozaki") for x in range(70)]   # more than the 64 problems of one launch
    probs, host = _make(specs, 1700)
    M.mpcgemm_batched(probs)
    torch.cuda.synchronize()
    for (dA, dB, dC, p, method, algo), (A, B) in zip(probs, host):
        assert gu.same(_result(dC, p), c_oracle.rounded_cgemm_matrix(A, B, p))


def test_batched_call_replays_from_a_cuda_graph():
    import torch
    M = gu.mp()
    probs, host = _make(SPECS[:4], 2700)
    ws = M.mpcgemm_batched(probs)          # warm-up outside capture (workspace, attributes)
    torch.cuda.synchronize()
    for (_, _, dC, _, _, _) in probs:
        dC.limb.zero_()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            M.mpcgemm_batched(probs, workspace=ws, stream=s)
    for _ in range(2):
        for (_, _, dC, _, _, _) in probs:
            dC.limb.zero_()
        g.replay()
        torch.cuda.synchronize()
        for (dA, dB, dC, p, method, algo), (A, B) in zip(probs, host):
            assert gu.same(_result(dC, p), c_oracle.rounded_cgemm_matrix(A, B, p))


def test_large_batch_graph_with_and_without_side_streams():
    """16 problems or more run their per-problem kernels on side streams of the caller's
    stream (graph branches under capture) once that stream has made a batched call
    outside capture; a stream that never did runs everything itself.  Both graphs must
    replay to the exact products."""
    import torch
    M = gu.mp()
    specs = [(20 + 3 * x, 40, 18 + x, 128 + 64 * (x % 3), "3m" if x % 2 else "4m", "ozaki") for x in range(20)]
    probs, host = _make(specs, 4700)
    warm, fresh = torch.cuda.Stream(), torch.cuda.Stream()
    ws = M.mpcgemm_batched(probs, stream=warm)          # creates the side streams of `warm`
    torch.cuda.synchronize()
    for s in (warm, fresh):
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(s):
            with torch.cuda.graph(g, stream=s):
                M.mpcgemm_batched(probs, workspace=ws, stream=s)
        for (_, _, dC, _, _, _) in probs:
            dC.limb.zero_()
        g.replay()
        torch.cuda.synchronize()
        for (dA, dB, dC, p, method, algo), (A, B) in zip(probs, host):
            assert gu.same(_result(dC, p), c_oracle.rounded_cgemm_matrix(A, B, p))


def test_autotuner_picks_a_working_configuration():
    import torch
    M = gu.mp()
    from paper_2307_06072_gb300.autotune import Autotuner
    probs, host = _make(SPECS[:3], 3700)
    tuner = Autotuner()
    best = tuner.choose(probs)
    assert best in tuner.candidates and len(tuner.last_timings) >= 3
    assert tuner.choose(probs) is best          # cached by signature
    M.mpcgemm_batched(probs, params=best)
    torch.cuda.synchronize()
    for (dA, dB, dC, p, method, algo), (A, B) in zip(probs, host):
        assert gu.same(_result(dC, p), c_oracle.rounded_cgemm_matrix(A, B, p))


def test_batched_workload_of_64_problems_sampled():
    """The benchmark's batched workload itself (64 Ozaki-3M problems, m, n, k log-uniform
    in [64, 1024], p in {256, 512, 1024}) under every configuration the autotuner may
    pick: sampled entries of every problem equal the exact C oracle bit for bit."""
    import torch
    from paper_2307_06072_gb300.autotune import CANDIDATES
    M = gu.mp()
    host = si.batch_problems(si.batch_specs())
    probs, ref, ents = [], [], []
    for x, (A, B, p) in enumerate(host):
        probs.append((M.DeviceMatrix.from_mpc(A), M.DeviceMatrix.from_mpc(B),
                      M.DeviceMatrix.empty(A.rows, B.cols, p), p, "3m", "ozaki"))
        ent = gu.sampled_entries(A.rows, B.cols, 8, 900 + x)
        ents.append(ent)
        ref.append(c_oracle.rounded_cgemm(A, B, p, ent))
    for cand in CANDIDATES:
        for (_, _, dC, _, _, _) in probs:
            dC.sign.fill_(0xFF)   # stale values must not survive
        ws = M.mpcgemm_batched(probs, params=cand)
        torch.cuda.synchronize()
        total, offs = M.batched_workspace(probs, cand)
        for x, (dA, dB, dC, p, method, algo) in enumerate(probs):
            gs, ge, gl = gu.take_entries(_result(dC, p), ents[x])
            sg, ex, li = ref[x]
            assert np.array_equal(gs, sg) and np.array_equal(ge, ex) and np.array_equal(gl, li), (cand, x)
            st = M.read_status(ws, offset=offs[x])
            assert st["device_timeout"] == 0 and st["uncertified"] == 0, (cand, x)
