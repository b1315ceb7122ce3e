"""Host-side serving logic that needs no GPU: window counts, memory
estimates and refusal of jobs that can never fit."""
import numpy as np
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


def test_over_budget_job_is_refused():
    b, o = readsim.random_reads(100, 100, 100, seed=1)
    with serve.Server(hbm_budget=1 << 20, slots=1) as s:
        with pytest.raises(ValueError):
            s.submit(serve.Job(b, o, K=21, m=1 << 20))
