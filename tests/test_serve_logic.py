"""Host logic of the serving loop, on the CPU: admission against each slot's
pre-sized workspace, continuous batching of GEMMs, LU solves alone in their slot,
rejection of requests larger than a slot.  The GPU launches are
replaced by fakes that complete a fixed time after they start (the GPU tests run the
real loop and check that results do not depend on the mix)."""
import time

from paper_2307_06072_gb300 import serve


class _FakeEvent:
    def __init__(self, done_at):
        self.done_at = done_at

    def query(self):
        return time.perf_counter() >= self.done_at


def _server(slots, slot_bytes, max_batch=48, duration=0.01):
    srv = serve.Server.__new__(serve.Server)   # no CUDA streams or workspaces: only their sizes are used
    srv.streams = [None] * slots
    srv.slot_bytes, srv.budget, srv.max_batch = slot_bytes, slots * slot_bytes, max_batch
    srv.in_use = srv.peak_in_use = srv.max_inflight = 0
    srv.batches, srv.rejected = [], []
    launched = []

    def footprint(req):
        return req.nbytes

    def launch(slot, reqs, t, nbytes):
        assert nbytes == sum(r.nbytes for r in reqs)
        if reqs[0].kind == "gemm":
            srv.batches.append(len(reqs))
        for r in reqs:
            r.t_admit = t
        launched.append([(r.kind, r.nbytes) for r in reqs])
        return serve._Flight(slot, reqs, _FakeEvent(time.perf_counter() + duration), sum(r.nbytes for r in reqs))

    srv.footprint, srv._launch = footprint, launch
    return srv, launched


def _requests(kinds, gap=0.002, nbytes=1):
    out = []
    for x, kind in enumerate(kinds):
        r = serve.Request(x, kind, x * gap, None, None, 256)
        r.nbytes = nbytes[x] if isinstance(nbytes, list) else nbytes
        out.append(r)
    return out


def test_every_request_completes_gemms_batch_and_lu_runs_alone():
    reqs = _requests(["gemm"] * 5 + ["lu"] + ["gemm"] * 6 + ["lu"] + ["gemm"] * 4)
    srv, launched = _server(slots=2, slot_bytes=50)
    out = srv.run(reqs)
    assert out["requests"] == len(reqs) and out["rejected"] == 0
    assert all(r.t_done is not None and r.t_done >= r.arrival for r in reqs)
    assert all(len(g) == 1 for g in launched if any(k == "lu" for k, _ in g))   # an LU solve takes a slot alone
    assert any(len(g) > 1 for g in launched)                                    # waiting GEMMs joined one batch
    assert sum(len(g) for g in launched) == len(reqs)
    assert out["max_in_flight"] <= 2


def test_every_batch_fits_its_slot_and_memory_stays_within_the_budget():
    sizes = [1, 2, 3, 1, 1, 2, 3, 3, 1, 2] * 3
    reqs = _requests(["gemm"] * len(sizes), gap=0.0005, nbytes=sizes)
    srv, launched = _server(slots=4, slot_bytes=4)
    out = srv.run(reqs)
    assert out["requests"] == len(reqs) and out["rejected"] == 0
    assert all(sum(b for _, b in g) <= 4 for g in launched)              # a batch fits the slot's workspace
    assert srv.peak_in_use <= srv.budget == 16
    assert srv.in_use == 0                                              # everything released


def test_batches_respect_max_batch():
    reqs = _requests(["gemm"] * 15, gap=0.0)
    srv, launched = _server(slots=1, slot_bytes=100, max_batch=4)
    srv.run(reqs)
    assert max(srv.batches) == 4 and sum(srv.batches) == 15


def test_a_request_larger_than_a_slot_is_rejected_and_the_rest_are_served():
    reqs = _requests(["gemm", "lu", "gemm", "lu", "gemm"], gap=0.0, nbytes=[2, 9, 6, 5, 5])
    srv, launched = _server(slots=2, slot_bytes=5)
    out = srv.run(reqs)
    assert out["rejected"] == 2 and sorted(r.rid for r in srv.rejected) == [1, 2]
    assert out["requests"] == 3
    assert all(r.t_done is not None for r in reqs if r.rid not in (1, 2))
    assert all(r.t_done is None for r in srv.rejected)
    assert sum(len(g) for g in launched) == 3
