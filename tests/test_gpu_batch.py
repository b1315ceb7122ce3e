"""Batched insertion: many samples, each with its own countBF, in one launch.

Each sample's results must equal the oracle's for that sample alone.
"""
import numpy as np
import pytest

import oracle
import readsim

torch = pytest.importorskip("torch")
import paper_2305_07545_gb300 as kc  # noqa: E402
from test_gpu_parity import check  # noqa: E402

pytestmark = pytest.mark.gpu


def _samples():
    """Uneven samples: sizes, geometries and content differ; one is empty."""
    out = []
    for i in range(10):
        n = [0, 1, 7, 50, 300, 900, 2000, 120, 4000, 33][i]
        if n == 0:
            b, o = readsim.from_strings([])
        elif i == 2:
            b, o = readsim.from_strings(["ACGTACGTAC", "AC", "ACGTNACGTACGTACGTACGTACGTACG"] * 3)
            o = o[:n + 1] if len(o) > n + 1 else o
        else:
            b, o = readsim.random_reads(n, 0, 200, seed=900 + i, alphabet=b"ACGTacgtN",
                                        weights=[24, 24, 24, 24, 1, 1, 1, 1, 0.2])
        m = [1 << 12, 1000, 1 << 16, 4099, 1 << 20, 1 << 18, 1 << 22, 777, 1 << 24, 1 << 14][i]
        alpha = [4, 4, 8, 5, 4, 4, 4, 16, 4, 2][i]
        nhash = [3, 4, 1, 2, 4, 3, 4, 2, 4, 6][i]
        out.append((b, o, m, alpha, nhash, 2 if alpha > 2 else 1))
    return out


def _dev(a):
    if a.dtype == np.uint64:
        a = a.view(np.int64)
    t = torch.from_numpy(np.ascontiguousarray(a)).cuda() if len(a) else \
        torch.zeros(1, dtype=torch.uint8 if a.dtype == np.uint8 else torch.int64, device="cuda")
    return t


def _run_batch(samples, K, stream, reset_twice=False, accumulate=False, schedule=None):
    filters = [kc.CountBF(K, m, alpha, nhash, tau, stream=stream.cuda_stream)
               for (_, _, m, alpha, nhash, tau) in samples]
    dev = [(_dev(b), _dev(o)) for (b, o, *_rest) in samples]
    torch.cuda.synchronize()
    nreads = [len(o) - 1 for (_, o, *_r) in samples]
    with kc.Batch(filters) as batch:
        if schedule is not None:
            batch.schedule(*schedule)
        kc.kmerco_batch_insert(batch.b, [d[0] if n else None for d, n in zip(dev, nreads)],
                               [d[1] for d in dev], nreads, reset=not accumulate)
        if reset_twice or accumulate:
            kc.kmerco_batch_insert(batch.b, [d[0] if n else None for d, n in zip(dev, nreads)],
                                   [d[1] for d in dev], nreads, reset=not accumulate)
        batch.classify()
        info = batch.info()
    results = []
    for f in filters:
        keys, est = f.distinct()
        results.append(dict(stats=f.stats(), counters=f.counters(), keys=keys, est=est,
                            trusted=f.trusted(), erroneous=f.erroneous()))
        f.close()
    return results, info


@pytest.mark.parametrize("K", [21, 40])
def test_batch_matches_oracle_per_sample(K):
    samples = _samples()
    stream = torch.cuda.Stream()
    results, info = _run_batch(samples, K, stream)
    assert info["samples"] == len(samples) and info["tuned"] == 1
    assert info["schedule"] in (0, 1)
    if info["schedule"] == 0:
        assert info["chunk"] in (1024, 2048) and info["blocks_per_sm"] >= 2
    else:
        assert info["streams"] in (1, 2, 4, 8)
    for (b, o, m, alpha, nhash, tau), g in zip(samples, results):
        check(g, b, o, K, alpha, nhash, tau)


@pytest.mark.parametrize("schedule", [(0, 0), (1, 1), (1, 4), (1, 8)])
def test_every_batch_schedule_matches_oracle(schedule):
    samples = _samples()
    stream = torch.cuda.Stream()
    results, info = _run_batch(samples, 31, stream, reset_twice=True, schedule=schedule)
    assert (info["schedule"], info["streams"]) == schedule and info["graph"] == 1
    for (b, o, m, alpha, nhash, tau), g in zip(samples, results):
        check(g, b, o, 31, alpha, nhash, tau)


def test_batch_graph_replay_gives_the_same_results():
    samples = _samples()
    stream = torch.cuda.Stream()
    once, _ = _run_batch(samples, 21, stream)
    twice, info = _run_batch(samples, 21, stream, reset_twice=True)
    assert info["graph"] == 1
    for a, b in zip(once, twice):
        for k in ("counters", "keys", "est", "trusted", "erroneous"):
            assert np.array_equal(a[k], b[k]), k


def test_batch_without_reset_accumulates():
    samples = _samples()[3:7]
    stream = torch.cuda.Stream()
    results, _ = _run_batch(samples, 21, stream, accumulate=True)
    for (b, o, m, alpha, nhash, tau), g in zip(samples, results):
        b2 = np.concatenate([b, b])
        o2 = np.concatenate([o, o[1:] + o[-1]])
        check(g, b2, o2, 21, alpha, nhash, tau)


def test_batch_rejects_bad_arguments():
    stream = torch.cuda.Stream()
    a = kc.CountBF(21, 1 << 12, 4, 3, 2, stream=stream.cuda_stream)
    b = kc.CountBF(31, 1 << 12, 4, 3, 2, stream=stream.cuda_stream)
    c = kc.CountBF(21, 1 << 12, 4, 3, 2)   # its own stream
    for hs in ([a, b], [a, c], [a, a]):
        with pytest.raises(kc.KmercoError) as e:
            kc.Batch(hs)
        assert e.value.status == kc.EINVAL
    with kc.Batch([a]) as batch:
        for bad in ((2, 0), (1, 0), (1, 3), (1, 16), (-2, 0)):
            with pytest.raises(kc.KmercoError) as e:
                batch.schedule(*bad)
            assert e.value.status == kc.EINVAL
    bases, offs = readsim.random_reads(10, 50, 60, seed=1)
    with kc.Batch([a]) as batch, pytest.raises(kc.KmercoError) as e:
        batch.insert([bases], [offs])   # host pointers
    assert e.value.status == kc.EINVAL
    for f in (a, b, c):
        f.close()


def test_batch_classify_graph_replay():
    # the second classification of the same input replays the captured graph
    samples = _samples()[2:8]
    stream = torch.cuda.Stream()
    filters = [kc.CountBF(25, m, alpha, nhash, tau, stream=stream.cuda_stream)
               for (_, _, m, alpha, nhash, tau) in samples]
    dev = [(_dev(b), _dev(o)) for (b, o, *_rest) in samples]
    torch.cuda.synchronize()
    nreads = [len(o) - 1 for (_, o, *_r) in samples]
    with kc.Batch(filters) as batch:
        for rep in range(3):
            kc.kmerco_batch_insert(batch.b, [d[0] if n else None for d, n in zip(dev, nreads)],
                                   [d[1] for d in dev], nreads, reset=True)
            l0 = batch.info()["launches"]
            batch.classify()
            assert batch.info()["launches"] > l0
            for (b, o, m, alpha, nhash, tau), f in zip(samples, filters):
                keys, est = f.distinct()
                g = dict(stats=f.stats(), counters=f.counters(), keys=keys, est=est,
                         trusted=f.trusted(), erroneous=f.erroneous())
                check(g, b, o, 25, alpha, nhash, tau)
    for f in filters:
        f.close()


def test_batch_sample_with_a_run_longer_than_one_block():
    # one sample whose 4.3e6 distinct 31-mers all begin with twelve A's: they
    # share the top 24 key bits, a run of equal top bits beyond what one
    # block sorts (2^22 keys), so the batch sorts that run after the graph and
    # splits the sample again; a small sample rides along
    st = readsim.Stream(2222)
    n = (1 << 22) + 100_000
    tails = readsim.ASCII[st.integers(n * 19, 4).astype(np.uint8)].reshape(n, 19)
    heads = np.full((n, 12), ord("A"), np.uint8)
    b1 = np.concatenate([heads, tails], axis=1).reshape(-1)
    o1 = np.arange(n + 1, dtype=np.uint64) * np.uint64(31)
    b2, o2 = readsim.random_reads(300, 40, 160, seed=2223)
    samples = [(b1, o1, 1 << 26, 4, 3, 2), (b2, o2, 1 << 16, 4, 3, 2)]
    stream = torch.cuda.Stream()
    results, info = _run_batch(samples, 31, stream)
    for (b, o, m, alpha, nhash, tau), g in zip(samples, results):
        check(g, b, o, 31, alpha, nhash, tau, cross_check=False)
    assert results[0]["stats"]["distinct"] > (1 << 22)
