"""Autotuner for the slice-GEMM configuration of a (batched) complex GEMM.

The tunable parts are the work-unit shape and size: the tcgen05 kernel in
single CTAs with 128 x 256 output tiles (two TMEM accumulators) or 128 x 128
tiles (four TMEM accumulators: the MMAs run further ahead of the drain), or in
CTA pairs running one cta_group::2 MMA (256 x 256 tiles, each SM loading half
of B),
the digit width, and the cap on slice pairs per group (smaller groups give
more, shorter units, which balances small problems better; the int32 limit
is the largest).  The k-block (64 bf16 = one 128-byte swizzled row) is
fixed by the kernel.  Every candidate computes the same exact result, so the
tuner simply times each one on the caller's data once and caches the winner
per problem signature.
"""
from __future__ import annotations

import math

from . import _native

CANDIDATES = (
    {"kernel": "tcgen05"},
    {"kernel": "tcgen05", "max_group": 8},
    {"kernel": "tcgen05", "max_group": 16},
    {"kernel": "tcgen05_n128"},
    {"kernel": "tcgen05_n128", "max_group": 8},
    {"kernel": "tcgen05_2sm"},
    {"kernel": "tcgen05_2sm", "max_group": 8},
    {"kernel": "tcgen05_2sm", "digit_bits": 8},
)


def _bucket(v: int) -> int:
    return 0 if v <= 0 else int(round(math.log2(v) * 2))


def signature(problems) -> tuple:
    """Shape classes of a batch: (m, n, k) on a half-octave grid, p and method."""
    return tuple(sorted((_bucket(A.rows), _bucket(B.cols), _bucket(A.cols), p, method, algo)
                        for (A, B, C, p, method, algo) in problems))


class Autotuner:
    def __init__(self, candidates=CANDIDATES):
        self.candidates = list(candidates)
        self.cache: dict[tuple, dict] = {}
        self.last_timings: list[tuple[dict, float]] = []

    def choose(self, problems, workspace=None, stream=None, repeats: int = 3) -> dict:
        """Best parameters for this batch (timed on first sight of its signature)."""
        import torch
        from . import mpcgemm_batched
        key = signature(problems)
        if key in self.cache:
            return self.cache[key]
        stream = stream if stream is not None else torch.cuda.current_stream()
        timings = []
        for cand in self.candidates:
            try:
                ws = mpcgemm_batched(problems, cand, workspace, stream)   # warm-up (and workspace growth)
                workspace = ws
                start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                start.record(stream)
                for _ in range(repeats):
                    mpcgemm_batched(problems, cand, workspace, stream)
                end.record(stream)
                end.synchronize()
                timings.append((cand, start.elapsed_time(end) / repeats))
            except _native.MPCError:
                continue
        if not timings:
            raise RuntimeError("no candidate configuration ran")
        best = min(timings, key=lambda t: t[1])[0]
        self.last_timings = timings
        self.cache[key] = best
        return best
