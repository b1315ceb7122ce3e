"""Host-side serving logic that needs no GPU: window counts, memory
estimates and refusal of jobs that can never fit."""
import pytest

import readsim
from paper_2305_07545_gb300 import serve


def test_window_count_and_estimate():
    b, o = readsim.from_strings(["ACGTACGTAC", "AC", "", "A" * 30])
    assert serve.window_count(o, 5) == 6 + 0 + 0 + 26
    j = serve.Job(b, o, K=5, m=1 << 10)
    j.windows = serve.window_count(o, 5)
    small = serve.estimate_bytes(j)
    j2 = serve.Job(b, o, K=40, m=1 << 10)
    j2.windows = j.windows
    assert serve.estimate_bytes(j2) > small > (1 << 10) // 16 * 8
    # the library's own bound: more reads never need less memory
    b3, o3 = readsim.random_reads(2000, 50, 150, seed=5)
    j3 = serve.Job(b3, o3, K=21, m=1 << 20)
    j3.windows = serve.window_count(o3, 21)
    b4, o4 = readsim.random_reads(4000, 50, 150, seed=5)
    j4 = serve.Job(b4, o4, K=21, m=1 << 20)
    j4.windows = serve.window_count(o4, 21)
    assert serve.estimate_bytes(j4) > serve.estimate_bytes(j3) > (1 << 20) // 2


def test_over_budget_job_is_refused():
    b, o = readsim.random_reads(100, 100, 100, seed=1)
    with serve.Server(hbm_budget=1 << 20, slots=1) as s:
        with pytest.raises(ValueError):
            s.submit(serve.Job(b, o, K=21, m=1 << 22))   # a 2 MiB countBF alone


class _FakeHandle:
    """Stands in for a countBF handle: records the jobs it ran and can hold
    a job until released."""

    def __init__(self, log, gate):
        self.log, self.gate = log, gate

    def reset(self):
        pass

    def insert(self, bases, offsets):
        self.log.append(len(offsets) - 1)
        assert self.gate.wait(10)

    def classify(self):
        pass

    def stats(self):
        return dict(inserted=1, distinct=1, trustworthy=0, erroneous=1, device_bytes=1 << 10)

    def digest(self):
        return "0" * 32

    def close(self):
        pass


def test_cancelled_job_never_runs():
    import threading
    log, gate = [], threading.Event()
    make = lambda job, budget: _FakeHandle(log, gate)  # noqa: E731
    b1, o1 = readsim.random_reads(3, 50, 50, seed=1)
    b2, o2 = readsim.random_reads(5, 50, 50, seed=2)
    b3, o3 = readsim.random_reads(7, 50, 50, seed=3)
    with serve.Server(hbm_budget=1 << 30, slots=1, make_handle=make) as s:
        f1 = s.submit(serve.Job(b1, o1, K=21, m=1 << 12))
        f2 = s.submit(serve.Job(b2, o2, K=21, m=1 << 12))
        f3 = s.submit(serve.Job(b3, o3, K=21, m=1 << 12))
        assert f2.cancel()            # still waiting behind the first job
        gate.set()
        assert f1.result(10).inserted == 1 and f3.result(10).inserted == 1
    assert f2.cancelled()
    assert log == [3, 7]              # the cancelled job's reads were never inserted
