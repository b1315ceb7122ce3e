"""The sharded count of one sample on one GPU: P ranks as threads of one
process (LocalComm), each with its own library handles and stream, through
the same exchange code that torch.distributed drives across GPUs
(kmerco_merge_cells for the chunked saturating countBF merge, kmerco_rank_of
for the key-range routing).  The owners' lists in rank order and every
rank's merged countBF must equal the oracle's result for the whole sample,
bit for bit.  No kernel waits on another rank: all waiting is on the host.
"""
import threading

import numpy as np
import pytest

import oracle
import readsim

torch = pytest.importorskip("torch")
import paper_2305_07545_gb300 as kc  # noqa: E402
from paper_2305_07545_gb300 import shard  # noqa: E402

pytestmark = pytest.mark.gpu


def _rows(hi, lo, K):
    return lo if K <= 32 else np.stack([lo, hi], axis=1)


def _sharded(bases, offsets, world, K, m, alpha, nhash, tau, **opts):
    kc.load()   # built and loaded once, before the rank threads start
    hub = shard.LocalComm(world)
    res, engines, err = [None] * world, [None] * world, []

    def run(r):
        try:
            engines[r] = shard.LibraryEngine(K, m, alpha, nhash, tau, device=0, **opts)
            res[r] = shard.count_sharded(engines[r], hub.view(r), bases, offsets,
                                         samples_per_rank=256)
        except BaseException as e:   # reported by the test thread
            err.append(e)
            hub._barrier.abort()

    threads = [threading.Thread(target=run, args=(r,)) for r in range(world)]
    for t in threads:
        t.start()
    for t in threads:
        t.join(600)
    if err:
        raise err[0]
    return res, engines


@pytest.mark.parametrize("K,m,world,mode", [(21, 1 << 20, 2, kc.UPDATE_AUTO),
                                            (31, 1 << 24, 3, kc.UPDATE_PARTITIONED),
                                            (55, 1 << 22, 2, kc.UPDATE_ATOMIC)])
def test_sharded_count_equals_whole_sample(K, m, world, mode):
    bases, offsets = readsim.scaled("tiny", 3000, seed_offset=90 + K).generate()
    alpha, nhash, tau = 4, 4, 2
    res, engines = _sharded(bases, offsets, world, K, m, alpha, nhash, tau, update_mode=mode)
    ref = oracle.run(bases, offsets, K, m, alpha, nhash, tau)
    tr = np.concatenate([r.owner.trusted() for r in res])
    er = np.concatenate([r.owner.erroneous() for r in res])
    m_tr, m_er = ref.trusted_mask, ~ref.trusted_mask
    assert np.array_equal(tr, _rows(ref.distinct_hi[m_tr], ref.distinct_lo[m_tr], K))
    assert np.array_equal(er, _rows(ref.distinct_hi[m_er], ref.distinct_lo[m_er], K))
    for r in res:   # every rank holds the whole sample's countBF
        assert np.array_equal(r.owner.counters(), ref.filter)
        assert (r.windows, r.inserted, r.distinct) == (ref.n_windows, ref.n_inserted,
                                                       len(ref.distinct_lo))
        assert r.trustworthy == int(m_tr.sum())
    assert len({r.owner.digest() for r in res}) == 1
    # each owner's estimates are Algorithm 5 on the merged countBF
    for r in res:
        keys, est = r.owner.distinct()
        hi = keys[:, 1] if K > 32 else np.zeros(len(keys), np.uint64)
        lo = keys[:, 0] if K > 32 else keys
        want, _ = oracle.classify(ref.filter, hi, lo, K, m, alpha, nhash, tau)
        assert np.array_equal(est.astype(np.uint64), want)
    assert all(len(r.owner.distinct()[0]) > 0 for r in res)   # every rank owned a range
    for r, e in zip(res, engines):
        r.owner.close()
        e.close()
