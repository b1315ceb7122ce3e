"""CUDA path vs the oracle, bit-exact, through the C ABI.

Everything here is integer work, so every comparison is exact: the packed
countBF cells, the sorted distinct keys, their estimates, the trustworthy
and erroneous lists and the totals.
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
    torch.cuda.synchronize()   # the library runs on its own stream
    return t


def gpu_run(bases, offsets, K, m, alpha, nhash, tau, device_inputs=True, forward_only=False,
            batches=None, update_mode=0, dims=None, pass_codes=0, canonical_hash=False,
            whole_file=False):
    with kc.CountBF(K, m, alpha, nhash, tau, forward_only=forward_only,
                    update_mode=update_mode, dims=dims, pass_codes=pass_codes,
                    canonical_hash=canonical_hash, whole_file=whole_file) as bf:
        parts = batches or [(bases, offsets)]
        for b, o in parts:
            if device_inputs:
                bf.insert(_dev(b), _dev(o))
            else:
                bf.insert(b, o)
        bf.classify()
        keys, est = bf.distinct()
        return dict(stats=bf.stats(), counters=bf.counters(), keys=keys, est=est,
                    trusted=bf.trusted(), erroneous=bf.erroneous())


def _split_keys(keys, K):
    if K <= 32:
        return np.zeros(len(keys), np.uint64), keys
    return keys[:, 1].copy(), keys[:, 0].copy()


def check(g, bases, offsets, K, alpha, nhash, tau, forward_only=False, cross_check=True,
          canonical_hash=False, whole_file=False, totals=True):
    st = g["stats"]
    m = st["m_actual"]
    dims = (st["dim_x"], st["dim_y"]) if st["dim_x"] else None
    ref = oracle.run(bases, offsets, K, m, alpha, nhash, tau, canonical=not forward_only,
                     dims=dims, cross_check=cross_check, canonical_hash=canonical_hash,
                     whole_file=whole_file)
    assert np.array_equal(g["counters"], ref.filter), "countBF cells"
    hi, lo = _split_keys(g["keys"], K)
    assert np.array_equal(lo, ref.distinct_lo) and np.array_equal(hi, ref.distinct_hi), "distinct"
    assert np.array_equal(g["est"].astype(np.uint64), ref.est), "estimates"
    thi, tlo = _split_keys(g["trusted"], K)
    ehi, elo = _split_keys(g["erroneous"], K)
    assert np.array_equal(tlo, ref.distinct_lo[ref.trusted_mask])
    assert np.array_equal(thi, ref.distinct_hi[ref.trusted_mask])
    assert np.array_equal(elo, ref.distinct_lo[~ref.trusted_mask])
    assert np.array_equal(ehi, ref.distinct_hi[~ref.trusted_mask])
    if totals:   # window totals of the handle (not restored by a load)
        assert st["windows"] == ref.n_windows
        assert st["n_skipped"] == ref.n_skipped
        assert st["inserted"] == ref.n_inserted
    assert st["distinct"] == len(ref.distinct_lo)
    assert st["trustworthy"] == int(ref.trusted_mask.sum())
    assert st["erroneous"] == len(ref.distinct_lo) - int(ref.trusted_mask.sum())
    maxc = (1 << alpha) - 1
    eta = 64 // alpha
    sat = sum(int(((int(w) >> (alpha * l)) & maxc) == maxc) for w in ref.filter for l in range(eta)) \
        if len(ref.filter) <= 4096 else None
    if sat is not None:
        assert st["saturated_counters"] == sat
    return ref


def test_tiny_workload_full_parity():
    w = readsim.WORKLOADS["tiny"]
    b, o = w.generate()
    g = gpu_run(b, o, w.K, w.m, w.alpha, w.nhash, w.tau)
    ref = check(g, b, o, w.K, w.alpha, w.nhash, w.tau)
    assert ref.n_skipped > 0 and ref.trusted_mask.any() and (~ref.trusted_mask).any()


SWEEP = [
    # K, m, alpha, nhash, tau
    (21, 1 << 12, 4, 3, 2),
    (31, 1000, 4, 4, 3),       # m rounded up to a multiple of eta
    (17, 999, 5, 2, 1),        # eta = 12, 4 wasted bits, non power-of-two m and eta
    (11, 4099, 7, 5, 2),
    (25, 512, 8, 1, 3),
    (40, 3000, 12, 3, 5),      # two-word keys
    (55, 1 << 14, 4, 4, 3),    # two-word keys, the long-K workload's K
    (9, 700, 16, 2, 2),
    (13, 300, 32, 3, 1),
    (7, 2048, 1, 3, 0),        # 1-bit counters
    (5, 64, 2, 6, 1),          # heavy collisions and saturation
    (1, 16, 4, 2, 1),          # K = 1
    (32, 1 << 10, 4, 4, 3),    # K = 32, widest one-word key
    (33, 1 << 10, 4, 4, 3),    # K = 33, narrowest two-word key
    (64, 1 << 10, 4, 4, 3),    # K = 64
    (31, 1 << 20, 4, 9, 3),    # k_h not a multiple of 4
]


@pytest.mark.parametrize("K,m,alpha,nhash,tau", SWEEP)
def test_parameter_sweep(K, m, alpha, nhash, tau):
    b, o = readsim.random_reads(300, 0, 200, seed=7 * K + m, alphabet=b"ACGTacgtNRY",
                                weights=[24, 24, 24, 24, 1, 1, 1, 1, 0.3, 0.05, 0.05])
    g = gpu_run(b, o, K, m, alpha, nhash, tau)
    check(g, b, o, K, alpha, nhash, tau)


@pytest.mark.parametrize("K", [21, 31, 55])
def test_long_reads_cross_many_chunks(K):
    b, o = readsim.random_reads(3, 9000, 20000, seed=K, alphabet=b"ACGTN",
                                weights=[25, 25, 25, 25, 0.02])
    g = gpu_run(b, o, K, 1 << 16, 4, 4, 3)
    check(g, b, o, K, 4, 4, 3)


def test_many_tiny_and_empty_reads():
    b, o = readsim.random_reads(20000, 0, 30, seed=3)
    g = gpu_run(b, o, 21, 1 << 14, 4, 3, 2)
    ref = check(g, b, o, 21, 4, 3, 2)
    assert ref.n_inserted > 0


UPDATE_CASES = [
    # K, m, alpha, nhash, tau
    (21, 1 << 12, 4, 4, 2),            # one coarse region per few cells
    (21, 1 << 20, 4, 3, 2),            # 2^16 cells: slices are the coarse regions
    (31, 1 << 24, 4, 4, 3),            # 2^20 cells: coarse region == one slice
    (31, 1 << 25, 4, 4, 3),            # 2^21 cells: coarse regions split into 2 slices
    (21, 3 * (1 << 23) + 48, 4, 4, 2), # non power-of-two m, partial last slice
    (17, 12 << 20, 5, 4, 3),           # eta = 12
    (25, 1 << 24, 8, 2, 3),            # eta = 8, k_h = 2
    (21, 1 << 27, 1, 3, 0),            # eta = 64: 2^21 cells, 16-bit lanes (counter << 7) | cell
    (15, 1 << 26, 2, 2, 1),            # eta = 32: lanes (counter << 8) | cell
    (19, 21 << 20, 3, 4, 2),           # eta = 21, not a power of two: lanes (counter << 9) | cell
]


@pytest.mark.parametrize("mode", [kc.UPDATE_ATOMIC, kc.UPDATE_PARTITIONED])
@pytest.mark.parametrize("K,m,alpha,nhash,tau", UPDATE_CASES)
def test_both_update_designs(mode, K, m, alpha, nhash, tau):
    b, o = readsim.scaled("tiny", 1500, seed_offset=K + alpha).generate()
    g = gpu_run(b, o, K, m, alpha, nhash, tau, update_mode=mode)
    check(g, b, o, K, alpha, nhash, tau)


def test_partitioned_overflow_falls_back_exactly():
    # one read repeated: its few cells receive almost every increment, so the
    # coarse and slice buffers overflow and the global fallback takes over
    b, o = readsim.from_strings(["ACGTTGCATTGACCAGTAGGACCATTAGCAGGATTACA"] * 4000)
    for m in (1 << 20, 1 << 25):
        g = gpu_run(b, o, 21, m, 8, 4, 3, update_mode=kc.UPDATE_PARTITIONED)
        check(g, b, o, 21, 8, 4, 3)


def test_sort_bucket_larger_than_shared_memory():
    # 20,000 distinct 31-mers that all begin with AAAAAAA share the top 14 key
    # bits: one histogram bin holds more keys than a block sorts in shared
    # memory, so the classification sort takes its radix-sort fallback (about
    # 1.1e6 more keys put the set in the bucket sort's range)
    st = readsim.Stream(77)
    n = 20000
    tails = readsim.ASCII[st.integers(n * 24, 4).astype(np.uint8)].reshape(n, 24)
    heads = np.full((n, 7), ord("A"), np.uint8)
    b1 = np.concatenate([heads, tails], axis=1).reshape(-1)
    o1 = np.arange(n + 1, dtype=np.uint64) * np.uint64(31)
    b2, o2 = readsim.random_reads(10000, 130, 150, seed=78)
    b = np.concatenate([b1, b2])
    o = np.concatenate([o1, o2[1:] + o1[-1]])
    g = gpu_run(b, o, 31, 1 << 22, 4, 4, 2)
    ref = check(g, b, o, 31, 4, 4, 2)
    assert int(np.count_nonzero((ref.distinct_lo >> np.uint64(48)) == 0)) > 16384
    assert len(ref.distinct_lo) > (1 << 20)


@pytest.mark.parametrize("K", [31, 55])
def test_nearly_all_windows_distinct(K):
    # about a million windows of i.i.d. bases are nearly all distinct: the
    # distinct set grows to the window count and the sort sees ~1e6 keys
    b, o = readsim.random_reads(8000 if K == 31 else 6000, 150, 150, seed=K)
    g = gpu_run(b, o, K, 1 << 24, 4, 4, 2)
    ref = check(g, b, o, K, 4, 4, 2)
    assert len(ref.distinct_lo) > 0.95 * ref.n_inserted


def test_repeated_read_contention():
    # the same read 3000 times: every window hits the same cells and the same
    # distinct-set slot from many threads at once
    b, o = readsim.from_strings(["ACGTTGCATTGACCAGTAGGACCATTAGCAGGATTACA"] * 3000)
    for alpha in (4, 16):
        g = gpu_run(b, o, 21, 1 << 12, alpha, 4, 3)
        check(g, b, o, 21, alpha, 4, 3)


def test_unaligned_device_slice_and_nonzero_first_offset():
    b, o = readsim.random_reads(500, 50, 150, seed=11)
    pad = np.frombuffer(b"NNNNN", np.uint8)
    b2 = np.concatenate([pad, b])
    o2 = o + np.uint64(5)
    tb = _dev(np.concatenate([np.zeros(3, np.uint8), b2]))[3:]   # device pointer not 16-aligned
    with kc.CountBF(21, 1 << 14, 4, 3, 2) as bf:
        bf.insert(tb, _dev(o2))
        bf.classify()
        keys, est = bf.distinct()
        g = dict(stats=bf.stats(), counters=bf.counters(), keys=keys, est=est,
                 trusted=bf.trusted(), erroneous=bf.erroneous())
    check(g, b2, o2, 21, 4, 3, 2)


def test_host_inputs_match_device_inputs():
    b, o = readsim.scaled("tiny", 800, seed_offset=2).generate()
    gd = gpu_run(b, o, 21, 1 << 18, 4, 3, 2, device_inputs=True)
    gh = gpu_run(b, o, 21, 1 << 18, 4, 3, 2, device_inputs=False)
    for k in ("counters", "keys", "est", "trusted", "erroneous"):
        assert np.array_equal(gd[k], gh[k]), k


def test_batches_accumulate_and_grow_the_distinct_set():
    b, o = readsim.scaled("tiny", 2000, seed_offset=3).generate()
    cuts = [0, 10, 300, 2000]   # a small first batch sizes a small set that must grow
    batches = []
    for c0, c1 in zip(cuts[:-1], cuts[1:]):
        ob = o[c0:c1 + 1] - o[c0]
        batches.append((b[int(o[c0]):int(o[c1])].copy(), ob.copy()))
    g = gpu_run(b, o, 21, 1 << 20, 4, 3, 2, batches=batches)
    check(g, b, o, 21, 4, 3, 2)
    g2 = gpu_run(b, o, 21, 1 << 20, 4, 3, 2, batches=batches, device_inputs=False)
    assert np.array_equal(g["counters"], g2["counters"])


def test_classify_between_inserts():
    # classify, insert more reads, classify again: the second result covers
    # all reads (classify keeps the distinct keys as the key list)
    b, o = readsim.scaled("tiny", 1200, seed_offset=6).generate()
    half = 500
    b1, o1 = b[:int(o[half])].copy(), o[:half + 1].copy()
    b2, o2 = b[int(o[half]):].copy(), (o[half:] - o[half]).copy()
    with kc.CountBF(21, 1 << 18, 4, 3, 2) as bf:
        bf.insert(_dev(b1), _dev(o1))
        bf.classify()
        first = bf.stats()["distinct"]
        bf.insert(_dev(b2), _dev(o2))
        bf.classify()
        keys, est = bf.distinct()
        g = dict(stats=bf.stats(), counters=bf.counters(), keys=keys, est=est,
                 trusted=bf.trusted(), erroneous=bf.erroneous())
    ref = check(g, b, o, 21, 4, 3, 2)
    assert 0 < first < len(ref.distinct_lo)


def test_forward_only_strand():
    b, o = readsim.scaled("tiny", 300).generate()
    g = gpu_run(b, o, 21, 1 << 16, 4, 3, 2, forward_only=True)
    check(g, b, o, 21, 4, 3, 2, forward_only=True)


def test_query_matches_algorithm_5():
    b, o = readsim.scaled("tiny", 400).generate()
    K, m, alpha, nhash = 21, 1 << 14, 4, 3
    ex = oracle.extract(b, o, K)
    filt = oracle.insert_sequential(ex.hi, ex.lo, K, m, alpha, nhash)
    probe = np.concatenate([ex.lo[:500], readsim.Stream(5).integers(500, 1 << 42).astype(np.uint64)])
    with kc.CountBF(K, m, alpha, nhash, 2) as bf:
        bf.insert(b, o)
        est = bf.query(probe)
        est_dev = torch.zeros(len(probe), dtype=torch.int32, device="cuda")
        torch.cuda.synchronize()
        kc.kmerco_query(bf.h, _dev(probe), len(probe), est_dev)
    want = [oracle.query(filt, K, 0, int(x), m, alpha, nhash) for x in probe]
    assert est.tolist() == want
    assert est_dev.cpu().numpy().view(np.uint32).tolist() == want
    assert any(v == 0 for v in want[500:])


def test_merge_equals_single_handle():
    b, o = readsim.scaled("tiny", 1200, seed_offset=4).generate()
    half = 500
    b1, o1 = b[:int(o[half])].copy(), o[:half + 1].copy()
    b2, o2 = b[int(o[half]):].copy(), (o[half:] - o[half]).copy()
    with kc.CountBF(21, 1 << 16, 4, 3, 2) as x, kc.CountBF(21, 1 << 16, 4, 3, 2) as y:
        x.insert(_dev(b1), _dev(o1))
        y.insert(_dev(b2), _dev(o2))
        x.merge(y)
        x.classify()
        keys, est = x.distinct()
        g = dict(stats=x.stats(), counters=x.counters(), keys=keys, est=est,
                 trusted=x.trusted(), erroneous=x.erroneous())
    check(g, b, o, 21, 4, 3, 2)
    with kc.CountBF(21, 1 << 16, 4, 3, 2) as x, kc.CountBF(31, 1 << 16, 4, 3, 2) as y:
        with pytest.raises(kc.KmercoError):
            x.merge(y)


def test_reset_reuse_and_states():
    b, o = readsim.scaled("tiny", 300).generate()
    with kc.CountBF(21, 1 << 16, 4, 3, 2) as bf:
        with pytest.raises(kc.KmercoError) as e:
            bf.distinct()
        assert e.value.status == kc.ESTATE
        bf.insert(_dev(b), _dev(o))
        bf.classify()
        first = bf.counters(), bf.distinct()[0]
        n = kc.kmerco_get_distinct(bf.h)
        small = np.zeros(max(n - 1, 1), np.uint64)
        with pytest.raises(kc.KmercoError) as e:
            kc.kmerco_get_distinct(bf.h, small, None, n - 1)
        assert e.value.status == kc.ESIZE
        bf.reset()
        assert not bf.counters().any()
        bf.insert(_dev(b), _dev(o))
        bf.classify()
        assert np.array_equal(bf.counters(), first[0])
        assert np.array_equal(bf.distinct()[0], first[1])


@pytest.mark.parametrize("K,mode", [(21, kc.UPDATE_AUTO), (31, kc.UPDATE_PARTITIONED),
                                    (32, kc.UPDATE_ATOMIC), (55, kc.UPDATE_PARTITIONED)])
def test_reset_generations(K, mode):
    # a reset moves the distinct set to its next generation tag instead of
    # clearing it (K = 31 has three tags, so the fourth reset clears the
    # table; K = 32 has no spare bits and clears every time): each sample
    # counted after a reset must see none of the earlier samples' keys
    with kc.CountBF(K, 1 << 22, 4, 3, 2, update_mode=mode) as bf:
        for i in range(6):
            b, o = readsim.scaled("tiny", 400 + 150 * (i % 3), seed_offset=300 + i).generate()
            if i:
                bf.reset()
            bf.insert(_dev(b), _dev(o))
            if i == 2:   # a second insert on top, then more keys added by hand
                b2, o2 = readsim.scaled("tiny", 200, seed_offset=399).generate()
                bf.insert(_dev(b2), _dev(o2))
                b = np.concatenate([b, b2])
                o = np.concatenate([o, o2[1:] + o[-1]])
            bf.classify()
            keys, est = bf.distinct()
            g = dict(stats=bf.stats(), counters=bf.counters(), keys=keys, est=est,
                     trusted=bf.trusted(), erroneous=bf.erroneous())
            check(g, b, o, K, 4, 3, 2)


def test_empty_and_too_short_inputs():
    for reads in ([], [""], ["ACGT", "AC", ""], ["N" * 50]):
        b, o = readsim.from_strings(reads)
        g = gpu_run(b, o, 21, 1 << 10, 4, 3, 2, device_inputs=False)
        ref = check(g, b, o, 21, 4, 3, 2)
        assert ref.n_inserted == 0


def test_decreasing_offsets_rejected():
    b, o = readsim.from_strings(["ACGTACGTACGTACGTACGTACGT"] * 3)
    bad = o.copy()
    bad[1], bad[2] = bad[2], bad[1]
    with kc.CountBF(5, 1 << 10, 4, 3, 2) as bf:
        for dev in (False, True):
            with pytest.raises(kc.KmercoError) as e:
                if dev:
                    bf.insert(_dev(b), _dev(bad))
                else:
                    bf.insert(b, bad)
            assert e.value.status == kc.EINVAL
        bf.insert(_dev(b), _dev(o))   # the handle stays usable
        bf.classify()
        assert bf.stats()["inserted"] == 3 * 20


@pytest.mark.slow
def test_single_sample_workload_full_size():
    """The 1M-read, 2^28-counter workload the benchmark times, bit-exact."""
    w = readsim.WORKLOADS["single"]
    b, o = w.generate()
    g = gpu_run(b, o, w.K, w.m, w.alpha, w.nhash, w.tau)
    st = g["stats"]
    ex = oracle.extract(b, o, w.K)
    assert st["windows"] == ex.n_windows and st["inserted"] == ex.n
    filt = oracle.counters_closed_form(ex.hi, ex.lo, w.K, w.m, w.alpha, w.nhash)
    assert np.array_equal(g["counters"], filt)
    dhi, dlo, _ = oracle.distinct(ex.hi, ex.lo)
    assert np.array_equal(g["keys"], dlo)
    est, tr = oracle.classify(filt, dhi, dlo, w.K, w.m, w.alpha, w.nhash, w.tau)
    assert np.array_equal(g["est"].astype(np.uint64), est)
    assert np.array_equal(g["trusted"], dlo[tr])
    assert np.array_equal(g["erroneous"], dlo[~tr])


@pytest.mark.parametrize("K,pass_codes,host", [(21, 20000, False), (40, 50000, False),
                                                (55, 7777, False), (31, 1, False),
                                                (21, 300000, True), (33, 1, True),
                                                (25, 0, True)])
def test_partitioned_in_several_passes(K, pass_codes, host):
    # a batch with more increments than one pass stages runs as consecutive
    # chunk ranges, each staged, repartitioned and applied on its own; host
    # reads are copied in pieces while earlier pieces are inserted
    b, o = readsim.scaled("tiny", 4000, seed_offset=21).generate()
    g = gpu_run(b, o, K, 1 << 22, 4, 3, 2, update_mode=kc.UPDATE_PARTITIONED,
                pass_codes=pass_codes, device_inputs=not host)
    check(g, b, o, K, 4, 3, 2)
    assert g["stats"]["launches"] > (8 if pass_codes == 0 else 20)


@pytest.mark.parametrize("K", [21, 55])
def test_partitioned_wide_countbf(K):
    # 2^31 4-bit counters = 2^27 cells (1 GiB): 128 slices per coarse region
    b, o = readsim.scaled("tiny", 3000, seed_offset=22).generate()
    g = gpu_run(b, o, K, 1 << 31, 4, 4, 2, update_mode=kc.UPDATE_PARTITIONED)
    assert g["stats"]["words"] == 1 << 27
    check(g, b, o, K, 4, 4, 2, cross_check=False)


def test_partitioned_wide_two_dimensional():
    # 8209 x 8219 cells (just over 2^26), uneven last slice
    b, o = readsim.scaled("tiny", 2500, seed_offset=23).generate()
    g = gpu_run(b, o, 25, 0, 8, 4, 2, update_mode=kc.UPDATE_PARTITIONED, dims=(8209, 8219),
                pass_codes=300000)
    check(g, b, o, 25, 8, 4, 2)


@pytest.mark.parametrize("K", [21, 31, 32, 40, 55, 64])
@pytest.mark.parametrize("mode", [kc.UPDATE_ATOMIC, kc.UPDATE_PARTITIONED])
def test_hash_canonical_and_whole_file(K, mode):
    # the paper-literal variants: canonical = strand with the smaller H_0,
    # windows across read boundaries; each alone and both together
    b, o = readsim.random_reads(900, 0, 160, seed=700 + K, alphabet=b"ACGTacgtN",
                                weights=[24, 24, 24, 24, 1, 1, 1, 1, 0.3])
    for ch, wf in ((True, False), (False, True), (True, True)):
        g = gpu_run(b, o, K, 1 << 20, 4, 4, 2, update_mode=mode, canonical_hash=ch,
                    whole_file=wf, device_inputs=(K % 2 == 0))
        check(g, b, o, K, 4, 4, 2, canonical_hash=ch, whole_file=wf)


def test_whole_file_short_reads():
    # every read shorter than K: no window inside a read, many across them
    b, o = readsim.random_reads(3000, 1, 15, seed=77)
    g = gpu_run(b, o, 21, 1 << 16, 4, 3, 2, whole_file=True)
    ref = check(g, b, o, 21, 4, 3, 2, whole_file=True)
    assert ref.n_windows == int(o[-1]) - 21 + 1
    assert gpu_run(b, o, 21, 1 << 16, 4, 3, 2)["stats"]["windows"] == 0


@pytest.mark.parametrize("K,prefix", [(40, 0), (55, 0), (40, 30), (64, 40)])
def test_segmented_sort_of_large_key_sets(K, prefix):
    # over 2^20 distinct two-word keys: radix passes over the top key bits,
    # then a rank sort inside each segment; with a long shared prefix many
    # keys share their top bits, so segments beyond 256 keys take their own
    # radix sort
    rng = readsim.Stream(900 + K + prefix)
    n_reads, length = 22000, 120
    codes = np.frombuffer(b"ACGT", np.uint8)[rng.integers(n_reads * length, 4)]
    reads = codes.reshape(n_reads, length)
    if prefix:
        reads[: n_reads // 2, :prefix] = ord("A")
    b = np.ascontiguousarray(reads).reshape(-1)
    o = np.arange(0, n_reads * length + 1, length, dtype=np.uint64)
    g = gpu_run(b, o, K, 1 << 24, 4, 3, 2)
    assert g["stats"]["distinct"] > (1 << 20)
    check(g, b, o, K, 4, 3, 2)


@pytest.mark.parametrize("K,prefix", [(33, 0), (55, 0), (64, 0), (40, 30)])
def test_top_bits_sort_of_large_two_word_key_sets(K, prefix):
    # over 2^21 distinct two-word keys take the top-bits sort: three radix
    # passes on the top 24 key bits (for K = 33 one digit straddles the two
    # key words), then segments sorted in shared memory; with a long shared
    # prefix one run of equal top bits outgrows a segment and is radix sorted
    # on its own
    rng = readsim.Stream(1900 + K + prefix)
    n_reads, length = 40000, 130
    codes = np.frombuffer(b"ACGT", np.uint8)[rng.integers(n_reads * length, 4)]
    reads = codes.reshape(n_reads, length)
    if prefix:
        reads[: n_reads // 2, :prefix] = ord("A")
    b = np.ascontiguousarray(reads).reshape(-1)
    o = np.arange(0, n_reads * length + 1, length, dtype=np.uint64)
    g = gpu_run(b, o, K, 1 << 24, 4, 3, 2)
    assert g["stats"]["distinct"] > (1 << 21)
    check(g, b, o, K, 4, 3, 2, cross_check=False)


@pytest.mark.parametrize("update_mode", [kc.UPDATE_ATOMIC, kc.UPDATE_PARTITIONED])
def test_host_inputs_in_pieces_and_back_to_back_calls(update_mode):
    # two host-input calls in a row reuse the staging buffer: the second
    # call's copies must wait for the first call's kernels
    b, o = readsim.scaled("tiny", 6000, seed_offset=24).generate()
    half = 2500
    b1, o1 = b[:int(o[half])].copy(), o[:half + 1].copy()
    b2, o2 = b[int(o[half]):].copy(), (o[half:] - o[half]).copy()
    g = gpu_run(b, o, 27, 1 << 22, 4, 4, 2, update_mode=update_mode, device_inputs=False,
                batches=[(b1, o1), (b2, o2)])
    check(g, b, o, 27, 4, 4, 2)


def test_hbm_budget_is_enforced():
    # the countBF alone is over the budget
    with pytest.raises(kc.KmercoError) as e:
        kc.CountBF(21, 1 << 30, 4, 3, 2, hbm_budget=1 << 20)
    assert e.value.status == kc.ENOMEM
    # the distinct set for this input is over the budget: the call fails
    # before any device work and the handle stays usable
    b, o = readsim.scaled("tiny", 2000, seed_offset=41).generate()
    with kc.CountBF(21, 1 << 20, 4, 3, 2, hbm_budget=(1 << 19) + (1 << 20)) as bf:
        with pytest.raises(kc.KmercoError) as e:
            bf.insert(_dev(b), _dev(o))
        assert e.value.status == kc.ENOMEM
        bs, os_ = readsim.scaled("tiny", 40, seed_offset=42).generate()
        bf.insert(_dev(bs), _dev(os_))
        bf.classify()
        keys, est = bf.distinct()
        g = dict(stats=bf.stats(), counters=bf.counters(), keys=keys, est=est,
                 trusted=bf.trusted(), erroneous=bf.erroneous())
        assert g["stats"]["device_bytes"] <= (1 << 19) + (1 << 20)
    check(g, bs, os_, 21, 4, 3, 2)


@pytest.mark.parametrize("K,m,alpha,tau", [(21, 1 << 15, 4, 12), (31, 1 << 20, 4, 3),
                                           (55, 1 << 18, 8, 2)])
def test_split_then_estimates_on_request(K, m, alpha, tau):
    _split_then_estimates(K, m, alpha, 4, tau, both_kinds=True)


@pytest.mark.parametrize("K,m,alpha,nhash,tau", [(21, 1 << 16, 1, 1, 0), (33, 1 << 18, 2, 5, 1),
                                                 (64, 1 << 18, 3, 7, 2), (45, 1 << 12, 3, 7, 6)])
def test_split_only_query_edge_parameters(K, m, alpha, nhash, tau):
    # one hash and one-bit counters with tau = 0 (every inserted key is
    # trustworthy); five and seven hashes with a mix of both kinds; tau at the
    # largest value alpha allows on a saturated countBF
    _split_then_estimates(K, m, alpha, nhash, tau, both_kinds=False)


def _split_then_estimates(K, m, alpha, nhash, tau, both_kinds):
    # classify reads a key's counters only until one is at or below tau (that
    # decides "erroneous"); the lists must be exact at once, and the full
    # Algorithm 5 estimates of every key when they are asked for afterwards
    b, o = readsim.scaled("tiny", 1500, seed_offset=400 + K).generate()
    mode = kc.UPDATE_PARTITIONED if nhash <= 4 else kc.UPDATE_ATOMIC
    with kc.CountBF(K, m, alpha, nhash, tau, update_mode=mode) as bf:
        bf.insert(_dev(b), _dev(o))
        bf.classify()
        st = bf.stats()
        trusted, erroneous = bf.trusted(), bf.erroneous()
        keys, est = bf.distinct()
        keys2, est2 = bf.distinct()
    ref = oracle.run(b, o, K, st["m_actual"], alpha, nhash, tau)
    thi, tlo = _split_keys(trusted, K)
    ehi, elo = _split_keys(erroneous, K)
    assert np.array_equal(tlo, ref.distinct_lo[ref.trusted_mask])
    assert np.array_equal(thi, ref.distinct_hi[ref.trusted_mask])
    assert np.array_equal(elo, ref.distinct_lo[~ref.trusted_mask])
    assert np.array_equal(ehi, ref.distinct_hi[~ref.trusted_mask])
    assert np.array_equal(est.astype(np.uint64), ref.est)
    assert np.array_equal(est2, est) and np.array_equal(keys2, keys)
    if both_kinds:   # both kinds of keys occur, and erroneous keys with estimates below tau
        assert ref.trusted_mask.any() and (~ref.trusted_mask).any()
        assert (ref.est[~ref.trusted_mask] < tau).any()
