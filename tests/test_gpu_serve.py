"""Serving loop: mixed GEMM / LU requests, continuous batching, per-slot workspaces.

Every request's result must be bit for bit the same served in the mix as run
alone, the loop must overlap work (several requests in flight), batch GEMMs
that wait together, allocate no device memory after it starts beyond the
results' pivot vectors, and keep each batch within its slot's workspace.
"""
import numpy as np
import pytest

import synthetic_inputs as si
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu


def _requests(M, seed):
    from paper_2307_06072_gb300.serve import Request
    rng = np.random.default_rng(seed)
    reqs, host = [], []
    for x in range(14):
        if x % 5 == 4:   # an LU solve
            n, p = int(rng.integers(24, 64)), int(rng.choice([128, 256]))
            A = si.random_matrix(n, n, p, seed + 10 * x, "uniform")
            B = si.random_matrix(n, 1, p, seed + 10 * x + 1, "uniform")
            host.append(("lu", A, B, p))
            reqs.append(Request(x, "lu", arrival=0.003 * (x // 4), A=M.DeviceMatrix.from_mpc(A),
                                B=M.DeviceMatrix.from_mpc(B), p=p, block=16, work=8 * n ** 3 / 3))
        else:
            m, k, n = (int(v) for v in rng.integers(32, 300, size=3))
            p = int(rng.choice([128, 256, 512]))
            A = si.random_matrix(m, k, p, seed + 10 * x, "uniform_exp")
            B = si.random_matrix(k, n, p, seed + 10 * x + 1, "uniform_exp")
            host.append(("gemm", A, B, p))
            reqs.append(Request(x, "gemm", arrival=0.003 * (x // 4), A=M.DeviceMatrix.from_mpc(A),
                                B=M.DeviceMatrix.from_mpc(B), p=p, C=M.DeviceMatrix.empty(m, n, p),
                                method="3m" if x % 2 else "4m", work=8.0 * m * n * k))
    return reqs, host


def _out(d, p):
    s, e, l = d.to_host()
    return si.MPCMatrix(d.rows, d.cols, p, s, e, l)


def test_results_are_the_same_alone_and_in_the_mix():
    import torch
    M = gu.mp()
    from paper_2307_06072_gb300.serve import Server
    reqs, host = _requests(M, 4000)
    srv = Server(slots=3, hbm_budget=3 << 30)
    stats = srv.run(reqs)
    torch.cuda.synchronize()
    assert stats["requests"] == len(reqs) and all(r.t_done is not None for r in reqs)
    assert stats["max_in_flight"] >= 2               # work overlapped on the device
    assert stats["max_gemm_batch"] >= 2              # waiting GEMMs were batched
    assert stats["rejected"] == 0
    assert stats["p99_ms"] >= stats["p50_ms"] > 0
    for r, (kind, A, B, p) in zip(reqs, host):
        if kind == "gemm":
            alone, _, _ = gu.run(A, B, p, r.method, "ozaki")
            assert gu.same(_out(r.C, p), alone), r.rid
        else:
            dA, dB = M.DeviceMatrix.from_mpc(A), M.DeviceMatrix.from_mpc(B)
            ipiv, _ = M.mpcgesv(dA, dB, p, r.block, r.method)
            torch.cuda.synchronize()
            assert gu.same(_out(r.A, p), _out(dA, p)), r.rid
            assert gu.same(_out(r.B, p), _out(dB, p)), r.rid
            assert np.array_equal(r.ipiv.cpu().numpy(), ipiv.cpu().numpy())


def test_admission_respects_the_slot_workspaces():
    import torch
    M = gu.mp()
    from paper_2307_06072_gb300.serve import Server
    reqs, _ = _requests(M, 5000)
    probe = Server(slots=1, hbm_budget=1 << 20)
    sizes = sorted(probe.footprint(r) for r in reqs)
    slot = sizes[-2] + 256                       # every request fits but the largest
    srv = Server(slots=3, hbm_budget=3 * slot)
    ptrs = [w.ptr for w in srv.workspaces]
    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated()
    stats = srv.run(reqs)
    torch.cuda.synchronize()
    assert stats["rejected"] == (1 if sizes[-1] > srv.slot_bytes else 0)
    assert stats["requests"] + stats["rejected"] == len(reqs)
    assert [w.ptr for w in srv.workspaces] == ptrs and all(w.nbytes == srv.slot_bytes for w in srv.workspaces)
    assert srv.peak_in_use <= srv.budget
    lu_pivots = sum(4 * max(r.A.rows, 1) for r in reqs if r.kind == "lu" and r.ipiv is not None)
    assert torch.cuda.memory_allocated() - before <= lu_pivots + (1 << 16)   # only the pivot vectors
