"""Serving: continuous batching of counting jobs over the countBF library.

Each job's results must be the same alone and in the mix, and the HBM
budget must bound what runs at once.
"""
import numpy as np
import pytest

import oracle
import readsim

torch = pytest.importorskip("torch")
import paper_2305_07545_gb300 as kc  # noqa: E402
from paper_2305_07545_gb300 import serve  # noqa: E402

pytestmark = pytest.mark.gpu


def _jobs(n=10, keep=True):
    jobs = []
    for i in range(n):
        if i % 3 == 0:
            b, o = readsim.scaled("tiny", 200 + 300 * i, seed_offset=40 + i).generate()
        else:
            b, o = readsim.random_reads(100 + 150 * i, 40, 250, seed=60 + i,
                                        alphabet=b"ACGTN", weights=[25, 25, 25, 25, 0.2])
        m = [1 << 14, 1 << 16, 5000, 1 << 18][i % 4]
        jobs.append(serve.Job(b, o, K=21 if i % 2 else 25, m=m, counter_bits=4,
                              nhash=3 + i % 2, tau=2, name=f"job{i}", keep_lists=keep))
    return jobs


def _key(r):
    return (r.inserted, r.distinct, r.trustworthy, r.erroneous, r.counters_digest,
            r.trusted.tobytes(), r.erroneous_keys.tobytes())


def test_each_result_is_the_same_alone_and_in_the_mix():
    jobs = _jobs()
    with serve.Server(slots=1) as alone:
        a = [alone.submit(j).result() for j in jobs]          # one at a time
    with serve.Server(slots=4) as mixed:
        futs = [mixed.submit(j) for j in jobs]                  # all at once
        b = [f.result() for f in futs]
        assert mixed.max_running > 1                            # they did overlap
    for ra, rb in zip(a, b):
        assert _key(ra) == _key(rb), ra.name
    # and against the oracle for two of them
    for j, r in list(zip(jobs, a))[:2]:
        eta = 64 // j.counter_bits
        m_act = (j.m + eta - 1) // eta * eta
        ref = oracle.run(j.bases, j.offsets, j.K, m_act, j.counter_bits, j.nhash, j.tau)
        assert r.distinct == len(ref.distinct_lo)
        assert np.array_equal(r.trusted, ref.distinct_lo[ref.trusted_mask])


def test_budget_bounds_what_runs_at_once():
    # every job's handle holds at most what the server reserved for it (the
    # library enforces it: the handle's hbm_budget is that reservation), and
    # the reservations of jobs running together stay within the budget
    jobs = _jobs(8, keep=False)
    for j in jobs:
        j.windows = serve.window_count(j.offsets, j.K)
    biggest = max(serve.estimate_bytes(j) for j in jobs)
    budget = int(2.2 * biggest)
    with serve.Server(hbm_budget=budget, slots=8) as s:
        res = [f.result() for f in [s.submit(j) for j in jobs]]
        assert s.max_in_use <= budget
        again = [f.result() for f in [s.submit(j) for j in jobs]]   # pooled handles
    for r in res + again:
        assert 0 < r.device_bytes <= r.reserved <= budget, r.name
    assert len(res) == len(jobs) and all(r.inserted > 0 for r in res)
    assert [x.counters_digest for x in res] == [x.counters_digest for x in again]


def test_estimate_bounds_the_library():
    # the library's own bound holds for one insert + classify, host or
    # device inputs, both update designs, one- and two-word keys
    for i, (K, m, host) in enumerate([(21, 1 << 16, True), (25, 1 << 22, False),
                                      (31, 1 << 24, True), (55, 1 << 20, True)]):
        b, o = readsim.scaled("tiny", 1500 + 500 * i, seed_offset=70 + i).generate()
        job = serve.Job(b, o, K=K, m=m)
        job.windows = serve.window_count(o, K)
        need = kc.kmerco_estimate_bytes(K, m, 4, 4, 3, len(o) - 1, int(o[-1]), job.windows, host)
        with kc.CountBF(K, m, 4, 4, 3, hbm_budget=need) as bf:
            if host:
                bf.insert(b, o)
            else:
                db, do = torch.from_numpy(b).cuda(), torch.from_numpy(o.view(np.int64)).cuda()
                torch.cuda.synchronize()   # the library runs on its own stream
                bf.insert(db, do)
            bf.classify()
            assert bf.stats()["device_bytes"] <= need


def test_a_failing_job_does_not_stop_the_server():
    jobs = _jobs(4, keep=False)
    bad = serve.Job(*readsim.from_strings(["ACGTACGTACGTACGTACGTACGTA"] * 3), K=21, m=1 << 12,
                    name="bad")
    bad.offsets = bad.offsets.copy()
    bad.offsets[1], bad.offsets[2] = bad.offsets[2], bad.offsets[1]
    with serve.Server(slots=2) as s:
        futs = [s.submit(j) for j in jobs[:2]] + [s.submit(bad)] + [s.submit(j) for j in jobs[2:]]
        with pytest.raises(kc.KmercoError):
            futs[2].result()
        assert all(f.result().inserted > 0 for i, f in enumerate(futs) if i != 2)
