"""kmerco_get_lists_async: the classified lists (Algorithm 2) copied on the
handle's result stream while the next sample is inserted and classified.

Three samples go through one handle: the first sample's lists are queued
into pinned host memory and left in flight while the second, larger sample
is inserted and classified (its classification must grow the lists' buffer,
so it waits on the host); the second's lists go to device memory while a
third, smaller sample is classified (that one waits on the device only).
After kmerco_sync every buffer must equal the oracle's lists for its own
sample, bit for bit.
"""
import numpy as np
import pytest

import oracle
import readsim

torch = pytest.importorskip("torch")
import paper_2305_07545_gb300 as kc  # noqa: E402

pytestmark = pytest.mark.gpu


def _rows(hi, lo, K):
    return lo if K <= 32 else np.stack([lo, hi], axis=1)


def _np(t, n, kw):
    a = t[: n * kw].cpu().numpy().view(np.uint64)
    return a if kw == 1 else a.reshape(n, 2)


@pytest.mark.parametrize("K,m", [(31, 1 << 22), (55, 1 << 22)])
def test_async_lists_equal_the_oracle_across_samples(K, m):
    alpha, nhash, tau = 4, 4, 2
    kw = 1 if K <= 32 else 2
    samples = [readsim.scaled("tiny", n, seed_offset=300 + K + i).generate()
               for i, n in enumerate((600, 3000, 900))]
    refs = [oracle.run(b, o, K, m, alpha, nhash, tau) for b, o in samples]
    cap = max(len(r.distinct_lo) for r in refs)
    outs = []
    with kc.CountBF(K, m, alpha, nhash, tau) as bf:
        with pytest.raises(kc.KmercoError) as e:   # nothing classified yet
            kc.kmerco_get_lists_async(bf.h)
        assert e.value.status == kc.ESTATE
        for i, (b, o) in enumerate(samples):
            if i:
                bf.reset()
            bf.insert(b, o)
            bf.classify()
            if i == 1:   # device destination
                tr = torch.empty(cap * kw, dtype=torch.int64, device="cuda")
                er = torch.empty(cap * kw, dtype=torch.int64, device="cuda")
            else:        # pinned host destination
                tr = torch.empty(cap * kw, dtype=torch.int64).pin_memory()
                er = torch.empty(cap * kw, dtype=torch.int64).pin_memory()
            with pytest.raises(kc.KmercoError) as e:   # a cap below its list
                kc.kmerco_get_lists_async(bf.h, tr, 0, er, 0)
            assert e.value.status == kc.ESIZE
            nt, ne = kc.kmerco_get_lists_async(bf.h, tr, cap, er, cap)
            outs.append((tr, er, nt, ne))
        kc.kmerco_sync(bf.h)
        # the synchronous getters still agree with the last sample
        assert np.array_equal(bf.trusted(), _np(outs[-1][0], outs[-1][2], kw))
    for (tr, er, nt, ne), ref in zip(outs, refs):
        mask = ref.trusted_mask
        assert (nt, ne) == (int(mask.sum()), int((~mask).sum()))
        assert np.array_equal(_np(tr, nt, kw),
                              _rows(ref.distinct_hi[mask], ref.distinct_lo[mask], K))
        assert np.array_equal(_np(er, ne, kw),
                              _rows(ref.distinct_hi[~mask], ref.distinct_lo[~mask], K))


def test_async_lists_one_list_only():
    b, o = readsim.scaled("tiny", 1200, seed_offset=77).generate()
    ref = oracle.run(b, o, 21, 1 << 20, 4, 3, 2)
    with kc.CountBF(21, 1 << 20, 4, 3, 2) as bf:
        bf.insert(b, o)
        bf.classify()
        er = torch.empty(len(ref.distinct_lo), dtype=torch.int64).pin_memory()
        nt, ne = kc.kmerco_get_lists_async(bf.h, None, 0, er, len(ref.distinct_lo))
        kc.kmerco_sync(bf.h)
    assert nt == int(ref.trusted_mask.sum())
    assert np.array_equal(er[:ne].numpy().view(np.uint64), ref.distinct_lo[~ref.trusted_mask])


def test_async_lists_of_batch_handles():
    # handles classified together by a batch: each one's lists copied on its
    # own result stream, then a second batch classification (which must wait
    # for those copies before it rewrites the lists) of new inputs
    stream = torch.cuda.Stream()
    specs = [(readsim.scaled("tiny", 400 + 300 * i, seed_offset=500 + i).generate(), 1 << 18)
             for i in range(3)]
    filters = [kc.CountBF(21, m, 4, 3, 2, stream=stream.cuda_stream) for _, m in specs]

    def dev(a):
        return torch.from_numpy(a.view(np.int64) if a.dtype == np.uint64 else a).cuda()

    with kc.Batch(filters) as batch:
        for rnd in range(2):
            inputs = specs if rnd == 0 else specs[::-1]   # other samples in each handle
            d = [(dev(b), dev(o)) for (b, o), _ in inputs]
            torch.cuda.synchronize()
            batch.insert([x[0] for x in d], [x[1] for x in d])
            batch.classify()
            outs = []
            for f in filters:
                nt = kc.kmerco_get_trusted(f.h)
                ne = kc.kmerco_get_erroneous(f.h)
                tr = torch.empty(max(nt, 1), dtype=torch.int64).pin_memory()
                er = torch.empty(max(ne, 1), dtype=torch.int64).pin_memory()
                assert kc.kmerco_get_lists_async(f.h, tr, nt, er, ne) == (nt, ne)
                outs.append((tr, er, nt, ne))
            for f, ((b, o), _), (tr, er, nt, ne) in zip(filters, inputs, outs):
                kc.kmerco_sync(f.h)
                ref = oracle.run(b, o, 21, 1 << 18, 4, 3, 2)
                mask = ref.trusted_mask
                assert np.array_equal(tr[:nt].numpy().view(np.uint64), ref.distinct_lo[mask])
                assert np.array_equal(er[:ne].numpy().view(np.uint64), ref.distinct_lo[~mask])
    for f in filters:
        f.close()
