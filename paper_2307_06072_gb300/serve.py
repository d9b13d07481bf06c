"""Request loop for mixed complex GEMM and LU-solve requests on one GPU.

Requests arrive over time (their ``arrival`` offsets); operands already live
on the device.  The loop keeps a few CUDA streams ("slots"), each with a
workspace of budget / slots bytes allocated once when the server starts, so
the memory the loop uses is fixed and bounded by the budget.  Whenever a slot
is free it admits waiting requests in arrival order as long as their
workspace footprint fits that slot's workspace: waiting GEMMs are admitted
together and run as one batched call (continuous batching: requests that
arrived while others were running join the next batch), an LU solve runs
alone in its slot.  A request whose footprint exceeds a slot's workspace can
never run and is rejected (counted in the statistics).  Work in different
slots overlaps on the device.  A request's latency runs from its arrival to
the completion of its work on the GPU.

Every operation is deterministic (exact arithmetic, one rounding per result),
so a request's result does not depend on what it ran with.
"""
from __future__ import annotations

import time
from dataclasses import dataclass

import numpy as np

from . import Workspace, _native, batched_workspace, mpcgemm_batched, mpcgesv


@dataclass
class Request:
    rid: int
    kind: str                 # "gemm" or "lu"
    arrival: float            # seconds after the loop starts
    A: object
    B: object
    p: int
    method: str = "3m"
    C: object = None          # GEMM output
    block: int = 64           # LU panel width
    t_admit: float | None = None
    t_done: float | None = None
    ipiv: object = None
    work: float = 0.0         # 8 m n k (GEMM) or 8 n^3 / 3 (LU)

    @property
    def latency(self) -> float:
        return self.t_done - self.arrival


@dataclass
class _Flight:
    slot: int
    reqs: list
    event: object
    nbytes: int


class Server:
    def __init__(self, slots: int = 4, hbm_budget: int = 32 << 30, max_batch: int = 64, device="cuda"):
        import torch
        self.torch = torch
        self.device = torch.device(device)
        self.streams = [torch.cuda.Stream(self.device) for _ in range(slots)]
        self.budget = int(hbm_budget)
        self.slot_bytes = (self.budget // slots) & ~255
        self.workspaces = []
        for _ in range(slots):                       # the loop's whole device memory, reserved once
            ws = Workspace(self.device)
            ws.get(self.slot_bytes)
            self.workspaces.append(ws)
        self.max_batch = max_batch
        self.in_use = 0
        self.peak_in_use = 0
        self.batches = []         # sizes of the GEMM batches launched
        self.max_inflight = 0
        self.rejected = []        # requests larger than a slot's workspace

    def footprint(self, req: Request) -> int:
        if req.kind == "gemm":
            return batched_workspace([(req.A, req.B, req.C, req.p, req.method, "ozaki")])[0]
        return int(_native.lib().mpcgesv_workspace_size(req.A.rows, req.p, req.block,
                                                        _native.METHODS[req.method])) + 4 * req.A.rows

    def _launch(self, slot: int, reqs: list, t: float, nbytes: int) -> _Flight:
        torch = self.torch
        st = self.streams[slot]
        ws = self.workspaces[slot]   # admission kept nbytes within it: nothing is allocated here
        with torch.cuda.stream(st):
            if reqs[0].kind == "gemm":
                problems = [(r.A, r.B, r.C, r.p, r.method, "ozaki") for r in reqs]
                mpcgemm_batched(problems, workspace=ws, stream=st)
                self.batches.append(len(reqs))
            else:
                r = reqs[0]
                r.ipiv, _ = mpcgesv(r.A, r.B, r.p, r.block, r.method, workspace=ws, stream=st)
            ev = torch.cuda.Event()
            ev.record(st)
        for r in reqs:
            r.t_admit = t
        return _Flight(slot, reqs, ev, nbytes)

    def run(self, requests: list) -> dict:
        """Serve all requests; returns latency / throughput statistics."""
        size = {id(r): self.footprint(r) for r in requests}   # planned once per request
        served = [r for r in requests if size[id(r)] <= self.slot_bytes]
        self.rejected = [r for r in requests if size[id(r)] > self.slot_bytes]
        pending = sorted(served, key=lambda r: r.arrival)
        queue: list = []
        flights: list = []
        free = list(range(len(self.streams)))
        t0 = time.perf_counter()
        while pending or queue or flights:
            now = time.perf_counter() - t0
            while pending and pending[0].arrival <= now:
                queue.append(pending.pop(0))
            for f in list(flights):
                if f.event.query():
                    done = time.perf_counter() - t0
                    for r in f.reqs:
                        r.t_done = done
                    self.in_use -= f.nbytes
                    free.append(f.slot)
                    flights.remove(f)
            progressed = False
            while free and queue:
                head = queue[0]
                if head.kind == "lu":
                    batch, need = [queue.pop(0)], size[id(head)]
                else:   # waiting GEMMs in arrival order, as many as fit the slot's workspace
                    batch, need = [], 0
                    for r in list(queue):
                        if r.kind != "gemm" or len(batch) >= self.max_batch:
                            continue
                        b = size[id(r)]
                        if need + b > self.slot_bytes:
                            continue
                        batch.append(r)
                        need += b
                        queue.remove(r)
                slot = free.pop(0)
                self.in_use += need
                self.peak_in_use = max(self.peak_in_use, self.in_use)
                flights.append(self._launch(slot, batch, time.perf_counter() - t0, need))
                self.max_inflight = max(self.max_inflight, len(flights))
                progressed = True
            if not progressed:
                time.sleep(0.0002)
        total = time.perf_counter() - t0
        lat = np.array([r.latency for r in served]) if served else np.zeros(1)
        work = sum(r.work for r in served)
        return {"requests": len(served), "rejected": len(self.rejected), "seconds": total,
                "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
                "p999_ms": float(np.percentile(lat, 99.9) * 1e3), "mean_ms": float(lat.mean() * 1e3),
                "throughput_req_s": len(served) / total, "work_8mnk_s": work / total,
                "gemm_batches": len(self.batches), "mean_gemm_batch": float(np.mean(self.batches)) if self.batches else 0.0,
                "max_gemm_batch": max(self.batches) if self.batches else 0, "max_in_flight": self.max_inflight,
                "peak_in_use_gb": round(self.peak_in_use / 1e9, 3),
                "reserved_gb": round(len(self.streams) * self.slot_bytes / 1e9, 3),
                "budget_gb": round(self.budget / 1e9, 3)}
