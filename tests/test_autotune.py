"""Host logic of the autotuner, on the CPU: the GPU calls and CUDA events are replaced
by fakes with scripted costs (the GPU tests run the real thing)."""
from types import SimpleNamespace

import pytest

import paper_2307_06072_gb300 as pkg
from paper_2307_06072_gb300 import _native, autotune


class _Clock:
    t = 0.0


class _FakeEvent:
    def __init__(self, enable_timing=False):
        self.t = None

    def record(self, stream=None):
        self.t = _Clock.t

    def synchronize(self):
        pass

    def elapsed_time(self, end):
        return end.t - self.t


def _problem(m, n, k, p=256, method="3m", algo="ozaki"):
    A = SimpleNamespace(rows=m, cols=k)
    B = SimpleNamespace(rows=k, cols=n)
    return (A, B, None, p, method, algo)


@pytest.fixture
def fake_gpu(monkeypatch):
    import torch
    calls = []
    cost = {"auto": 5.0, "tcgen05": 3.0, "tcgen05_n128": 4.0, "tcgen05_2sm": 1.0}

    def fake_batched(problems, params=None, workspace=None, stream=None):
        calls.append(dict(params))
        if params.get("digit_bits") == 8:
            raise _native.MPCError(_native.MPC_EINVAL)
        _Clock.t += cost[params["kernel"]] + (0.5 if params.get("max_group") else 0.0)
        return workspace if workspace is not None else object()

    monkeypatch.setattr(pkg, "mpcgemm_batched", fake_batched)
    monkeypatch.setattr(torch.cuda, "Event", _FakeEvent)
    return calls


def test_picks_the_fastest_candidate_and_skips_failures(fake_gpu):
    tuner = autotune.Autotuner()
    probs = [_problem(100, 200, 300), _problem(64, 64, 64)]
    best = tuner.choose(probs, stream=object(), repeats=2)
    assert best == {"kernel": "tcgen05_2sm"}
    timed = [c for c, _ in tuner.last_timings]
    assert {"kernel": "tcgen05_2sm", "digit_bits": 8} not in timed          # raised: skipped
    assert len(timed) == len(autotune.CANDIDATES) - 1
    ms = {str(c): t for c, t in tuner.last_timings}
    assert ms[str({"kernel": "tcgen05"})] == pytest.approx(3.0)           # per repeat
    assert ms[str({"kernel": "tcgen05", "max_group": 16})] == pytest.approx(3.5)


def test_cached_per_signature(fake_gpu):
    tuner = autotune.Autotuner()
    probs = [_problem(100, 200, 300)]
    best = tuner.choose(probs, stream=object())
    n = len(fake_gpu)
    same_class = [_problem(104, 196, 290)]                                 # same half-octave buckets
    assert autotune.signature(same_class) == autotune.signature(probs)
    assert tuner.choose(same_class, stream=object()) is best
    assert len(fake_gpu) == n                                              # nothing ran again
    other = [_problem(100, 200, 300, p=512)]
    assert autotune.signature(other) != autotune.signature(probs)
    tuner.choose(other, stream=object())
    assert len(fake_gpu) > n


def test_signature_ignores_problem_order():
    a, b = _problem(100, 200, 300), _problem(64, 64, 64, p=1024, method="4m")
    assert autotune.signature([a, b]) == autotune.signature([b, a])


def test_no_runnable_candidate_is_an_error(fake_gpu):
    tuner = autotune.Autotuner(candidates=[{"kernel": "tcgen05_2sm", "digit_bits": 8}])
    with pytest.raises(RuntimeError):
        tuner.choose([_problem(10, 10, 10)], stream=object())
