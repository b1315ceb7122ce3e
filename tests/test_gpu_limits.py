"""Error paths that need no GPU fault, and the caller's device allocator.

- A tiny retry limit makes the bounded device loops (compare-and-swap
  retries of a counter update, Algorithm 3; probes of a distinct-set insert)
  give up on contended input: classify reports KMERCO_ETIMEOUT, and after a
  reset the handle counts exactly again.  Nothing spins: every loop returns
  once it reaches the limit.
- A cap on the distinct list: more distinct keys than the cap give
  KMERCO_ENOMEM at classify; after a reset the handle counts exactly again.
- A handle whose device memory comes from torch's caching allocator gives
  the same results bit for bit, and torch accounts for its memory.
"""
import numpy as np
import pytest

import oracle
import readsim

torch = pytest.importorskip("torch")
import paper_2305_07545_gb300 as kc  # noqa: E402

pytestmark = pytest.mark.gpu


def _dev(a: np.ndarray):
    if a.dtype == np.uint64:
        a = a.view(np.int64)
    t = torch.from_numpy(np.ascontiguousarray(a)).cuda()
    torch.cuda.synchronize()
    return t


def _exact(bf, b, o, K, m, alpha, nhash, tau):
    bf.classify()
    keys, est = bf.distinct()
    ref = oracle.run(b, o, K, bf.stats()["m_actual"], alpha, nhash, tau)
    assert np.array_equal(bf.counters(), ref.filter)
    assert np.array_equal(keys, ref.distinct_lo)
    assert np.array_equal(est.astype(np.uint64), ref.est)
    assert np.array_equal(bf.trusted(), ref.distinct_lo[ref.trusted_mask])


# one read holding a single 21-mer window: one key, nothing contended
ONE = readsim.from_strings(["ACGTTGCATTGACCAGTAGGA"])


@pytest.mark.parametrize("mode,alpha", [(kc.UPDATE_ATOMIC, 4), (kc.UPDATE_PARTITIONED, 4),
                                        (kc.UPDATE_PARTITIONED, 16)])
def test_retry_limit_reports_timeout_and_reset_recovers(mode, alpha):
    # 20,000 windows of random bases: the distinct set is sized for them at
    # load factor 1/2, so many inserts need more than one probe past their
    # home slot; with a limit of one the probe loop gives up.  (16-bit
    # counters take the compare-and-swap apply with the handle's bound.)
    b, o = readsim.random_reads(200, 120, 120, seed=91)
    with kc.CountBF(21, 1 << 20, alpha, 4, 2, update_mode=mode, retry_limit=1) as bf:
        bf.insert(_dev(b), _dev(o))
        with pytest.raises(kc.KmercoError) as e:
            bf.classify()
        assert e.value.status == kc.ETIMEOUT
        with pytest.raises(kc.KmercoError) as e:
            bf.stats()
        assert e.value.status == kc.ETIMEOUT
        bf.reset()
        ob, oo = ONE
        bf.insert(_dev(ob), _dev(oo))
        _exact(bf, ob, oo, 21, 1 << 20, alpha, 4, 2)


def test_counter_retry_limit_on_one_hot_counter():
    # the same read 3000 times into a single-cell countBF under the atomic
    # design: thousands of threads race on one 64-bit cell, so compare-and-
    # swap retries run out at a limit of one (the reads hold 18 distinct
    # keys, so the distinct set is uncontended beyond its home slots)
    b, o = readsim.from_strings(["ACGTTGCATTGACCAGTAGGACCATTAGCAGGATTACA"] * 3000)
    with kc.CountBF(21, 16, 16, 4, 3, update_mode=kc.UPDATE_ATOMIC, retry_limit=1) as bf:
        bf.insert(_dev(b), _dev(o))
        with pytest.raises(kc.KmercoError) as e:
            bf.classify()
        assert e.value.status == kc.ETIMEOUT
        bf.reset()
        ob, oo = ONE
        bf.insert(_dev(ob), _dev(oo))
        _exact(bf, ob, oo, 21, 16, 16, 4, 3)


def test_distinct_cap_reports_enomem_and_reset_recovers():
    b, o = readsim.random_reads(50, 60, 60, seed=92)          # about 2,000 distinct 21-mers
    with kc.CountBF(21, 1 << 16, 4, 3, 2, max_distinct=100) as bf:
        bf.insert(_dev(b), _dev(o))
        with pytest.raises(kc.KmercoError) as e:
            bf.classify()
        assert e.value.status == kc.ENOMEM
        bf.reset()
        sb, so = readsim.random_reads(2, 60, 60, seed=93)      # 80 windows
        bf.insert(_dev(sb), _dev(so))
        _exact(bf, sb, so, 21, 1 << 16, 4, 3, 2)
        assert bf.stats()["distinct"] <= 100


@pytest.mark.parametrize("K,m,mode", [(21, 1 << 20, kc.UPDATE_ATOMIC),
                                      (31, 1 << 24, kc.UPDATE_PARTITIONED),
                                      (55, 1 << 22, kc.UPDATE_AUTO)])
def test_torch_allocator_gives_the_same_results(K, m, mode):
    b, o = readsim.scaled("tiny", 1500, seed_offset=K).generate()
    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated()
    with kc.CountBF(K, m, 4, 4, 2, update_mode=mode, allocator="torch") as bf:
        after_create = torch.cuda.memory_allocated()
        assert after_create - before >= bf.stats()["device_bytes"] >= m // 2
        bf.insert(b, o)      # host inputs: the staging buffers come from torch too
        bf.classify()
        st = bf.stats()
        grown = torch.cuda.memory_allocated() - before
        # torch rounds each block up to 512 bytes
        assert st["device_bytes"] <= grown <= st["device_bytes"] + 64 * 512 + st["device_bytes"] // 100
        keys, est = bf.distinct()
        cells = bf.counters()
        trusted = bf.trusted()
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == before     # every block went back to torch
    ref = oracle.run(b, o, K, m, 4, 4, 2)
    assert np.array_equal(cells, ref.filter)
    hi = keys[:, 1] if K > 32 else np.zeros(len(keys), np.uint64)
    lo = keys[:, 0] if K > 32 else keys
    assert np.array_equal(lo, ref.distinct_lo) and np.array_equal(hi, ref.distinct_hi)
    assert np.array_equal(est.astype(np.uint64), ref.est)
    tlo = trusted[:, 0] if K > 32 else trusted
    assert np.array_equal(tlo, ref.distinct_lo[ref.trusted_mask])


def test_torch_allocator_out_of_budget_is_enomem():
    with pytest.raises(kc.KmercoError) as e:
        kc.CountBF(21, 1 << 30, 4, 3, 2, allocator="torch", hbm_budget=1 << 20)
    assert e.value.status == kc.ENOMEM


def test_torch_allocator_with_a_batch():
    bs, os_ = [], []
    filters = []
    stream = torch.cuda.Stream()
    for i in range(3):
        b, o = readsim.scaled("tiny", 300 + 200 * i, seed_offset=50 + i).generate()
        bs.append(b)
        os_.append(o)
        filters.append(kc.CountBF(21, 1 << 18, 4, 3, 2, allocator="torch",
                                  stream=stream.cuda_stream))
    d = [(_dev(b), _dev(o)) for b, o in zip(bs, os_)]
    with kc.Batch(filters) as batch:
        for sched, streams in ((0, 0), (1, 2)):
            batch.schedule(sched, streams)
            batch.insert([x[0] for x in d], [x[1] for x in d])
            batch.classify()
            for f, b, o in zip(filters, bs, os_):
                ref = oracle.run(b, o, 21, 1 << 18, 4, 3, 2)
                assert np.array_equal(f.counters(), ref.filter)
                assert np.array_equal(f.distinct()[0], ref.distinct_lo)
    for f in filters:
        f.close()



def test_pass_size_bounds():
    # at most 2^31 increments per partitioned pass
    with pytest.raises(kc.KmercoError) as e:
        kc.CountBF(21, 1 << 20, 4, 3, 2, update_mode=kc.UPDATE_PARTITIONED,
                   pass_codes=(1 << 31) + 1)
    assert e.value.status == kc.EINVAL
    b, o = readsim.scaled("tiny", 800, seed_offset=123).generate()
    for alpha in (4, 16):   # counting and compare-and-swap apply, one full-size pass
        with kc.CountBF(21, 1 << 22, alpha, 3, 2, update_mode=kc.UPDATE_PARTITIONED,
                        pass_codes=1 << 31) as bf:
            bf.insert(_dev(b), _dev(o))
            _exact(bf, b, o, 21, 1 << 22, alpha, 3, 2)
