"""Host logic of the serving loop, on the CPU: admission by memory footprint,
continuous batching of GEMMs, LU solves alone in their slot.  The GPU launches are
replaced by fakes that complete a fixed time after they start (the GPU tests run the
real loop and check that results do not depend on the mix)."""
import time

from paper_2307_06072_gb300 import serve


class _FakeEvent:
    def __init__(self, done_at):
        self.done_at = done_at

    def query(self):
        return time.perf_counter() >= self.done_at


def _server(slots, budget, max_batch=48, duration=0.01):
    srv = serve.Server.__new__(serve.Server)   # no CUDA streams: only their number is used
    srv.streams = [None] * slots
    srv.budget, srv.max_batch = budget, max_batch
    srv.in_use = srv.peak_in_use = srv.max_inflight = 0
    srv.batches = []
    launched = []

    def footprint(req):
        return req.nbytes

    def launch(slot, reqs, t):
        if reqs[0].kind == "gemm":
            srv.batches.append(len(reqs))
        for r in reqs:
            r.t_admit = t
        launched.append([r.kind for r in reqs])
        return serve._Flight(slot, reqs, _FakeEvent(time.perf_counter() + duration), sum(r.nbytes for r in reqs))

    srv.footprint, srv._launch = footprint, launch
    return srv, launched


def _requests(kinds, gap=0.002, nbytes=1):
    out = []
    for x, kind in enumerate(kinds):
        r = serve.Request(x, kind, x * gap, None, None, 256)
        r.nbytes = nbytes
        out.append(r)
    return out


def test_every_request_completes_gemms_batch_and_lu_runs_alone():
    reqs = _requests(["gemm"] * 5 + ["lu"] + ["gemm"] * 6 + ["lu"] + ["gemm"] * 4)
    srv, launched = _server(slots=2, budget=100)
    out = srv.run(reqs)
    assert out["requests"] == len(reqs) and all(r.t_done is not None and r.t_done >= r.arrival for r in reqs)
    assert all(len(g) == 1 for g in launched if "lu" in g)              # an LU solve takes a slot alone
    assert any(len(g) > 1 for g in launched)                            # waiting GEMMs joined one batch
    assert sum(len(g) for g in launched) == len(reqs)
    assert out["max_in_flight"] <= 2


def test_memory_in_use_stays_within_the_budget():
    reqs = _requests(["gemm"] * 20, gap=0.0005)
    srv, launched = _server(slots=4, budget=3)
    out = srv.run(reqs)
    assert srv.peak_in_use <= 3 and out["peak_in_use_gb"] <= out["budget_gb"]
    assert srv.in_use == 0                                              # everything released


def test_batches_respect_max_batch():
    reqs = _requests(["gemm"] * 15, gap=0.0)
    srv, launched = _server(slots=1, budget=100, max_batch=4)
    srv.run(reqs)
    assert max(srv.batches) == 4 and sum(srv.batches) == 15


def test_a_request_larger_than_the_budget_runs_when_nothing_else_does():
    reqs = _requests(["gemm", "lu", "gemm"], gap=0.0, nbytes=10)
    srv, launched = _server(slots=2, budget=5)
    out = srv.run(reqs)
    assert out["requests"] == 3 and all(r.t_done is not None for r in reqs)
    assert out["max_in_flight"] == 1                                     # admitted one at a time
