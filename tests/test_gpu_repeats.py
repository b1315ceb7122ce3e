"""The large repetitive workload (2^33 4-bit counters = 4 GiB, 31- and
55-mers) against the oracle.

- A prefix of the workload's own reads at the workload's full countBF
  geometry (2^29 cells: 64 coarse regions of 2^23 cells, 512 slices each),
  with a pass size small enough to force several insert passes, compared
  element by element with the oracle: every cell, the distinct keys, their
  estimates, both lists and the totals.
- More than 2^28 distinct keys through the classification sort and split,
  against a numpy sort + unique and the oracle's Algorithm 5 / Algorithm 2.
- The whole workload (20,000,000 reads), checked through properties that
  hold at any size and through sampled outputs the oracle computes one by
  one from the GPU's own countBF.
"""
import numpy as np
import pytest

import oracle
import readsim

torch = pytest.importorskip("torch")
import paper_2305_07545_gb300 as kc  # noqa: E402

pytestmark = pytest.mark.gpu

W = readsim.WORKLOADS["repeats"]


def _dev(a: np.ndarray):
    if a.dtype == np.uint64:
        a = a.view(np.int64)
    t = torch.from_numpy(np.ascontiguousarray(a)).cuda()
    torch.cuda.synchronize()
    return t


def _split(keys, K):
    if K <= 32:
        return np.zeros(len(keys), np.uint64), keys
    return keys[:, 1].copy(), keys[:, 0].copy()


@pytest.mark.parametrize("K", [31, 55])
def test_prefix_at_full_geometry_in_several_passes(K):
    n_reads = 150_000
    b, o = readsim.scaled("repeats", n_reads).generate()
    windows = n_reads * (150 - K + 1)
    pass_codes = (windows * W.nhash) // 5 + 1     # five passes
    with kc.CountBF(K, W.m, W.alpha, W.nhash, W.tau, pass_codes=pass_codes) as bf:
        bf.insert(_dev(b), _dev(o))
        bf.classify()
        st = bf.stats()
        assert st["words"] == 1 << 29
        cells = bf.counters()
        keys, est = bf.distinct()
        trusted, erroneous = bf.trusted(), bf.erroneous()
    ref = oracle.run(b, o, K, W.m, W.alpha, W.nhash, W.tau, cross_check=False)
    assert st["windows"] == ref.n_windows == windows and st["inserted"] == ref.n_inserted
    assert np.array_equal(cells, ref.filter), "countBF cells"
    hi, lo = _split(keys, K)
    assert np.array_equal(lo, ref.distinct_lo) and np.array_equal(hi, ref.distinct_hi)
    assert np.array_equal(est.astype(np.uint64), ref.est), "estimates"
    for got, mask in ((trusted, ref.trusted_mask), (erroneous, ~ref.trusted_mask)):
        ghi, glo = _split(got, K)
        assert np.array_equal(glo, ref.distinct_lo[mask]) and np.array_equal(ghi, ref.distinct_hi[mask])
    assert st["distinct"] == len(ref.distinct_lo)
    assert st["trustworthy"] == int(ref.trusted_mask.sum())
    # the repeat families give estimates well above tau and saturated counters
    assert ref.trusted_mask.any() and (~ref.trusted_mask).any()
    assert int(ref.est.max()) == (1 << W.alpha) - 1


def test_more_than_2_to_the_28_distinct_keys():
    # 2^28 + 2^22 distinct one-word keys (31-mers) built ascending from
    # random gaps, so the sorted distinct list is known without a sort: one
    # block of 2^20 keys has gaps of 1..16 (keys sharing their top bits), the
    # rest gaps below 2^33.  They go in through kmerco_add_distinct in a
    # strided order with a quarter of them a second time (dropped by the
    # distinct set), then are classified against a countBF of random cells.
    K, m, alpha, nhash, tau = 31, 1 << 30, 4, 4, 3
    n = (1 << 28) + (1 << 22)
    st = readsim.Stream(2828)
    gaps = (st.raw(n) >> np.uint64(31)) + np.uint64(1)           # 1 .. 2^33
    gaps[1000:1000 + (1 << 20)] = (gaps[1000:1000 + (1 << 20)] & np.uint64(15)) + np.uint64(1)
    for c in range(40):   # clusters of 300..900 consecutive values: one shared-memory
        at = (c + 1) * (n // 41)   # sub-bin of their segment holds them all
        gaps[at:at + 300 + 15 * c] = 1
    want = np.cumsum(gaps, dtype=np.uint64)
    assert int(want[-1]) < (1 << 62) and len(want) > (1 << 28)
    stride = 1_000_003                                             # prime, coprime to n
    order = (np.arange(n, dtype=np.uint64) * np.uint64(stride)) % np.uint64(n)
    keys = np.concatenate([want[order], want[: n // 4][::-1]])
    del order
    eta = 64 // alpha
    words = m // eta
    cells = st.raw(words) & np.uint64(0x3333333333333333)          # counters 0..3 ...
    cells |= (st.raw(words) & np.uint64(0x4444444444444444))     # ... and 4..7
    with kc.CountBF(K, m, alpha, nhash, tau) as bf:
        kc.kmerco_set_counters(bf.h, cells, words)
        d_keys = _dev(keys)
        kc.kmerco_add_distinct(bf.h, d_keys, len(keys))
        del d_keys, keys
        bf.classify()
        got, est = bf.distinct()
        trusted = bf.trusted()
        n_err = kc.kmerco_get_erroneous(bf.h)
    assert np.array_equal(got, want), "sorted distinct keys"
    del got
    # the split is the estimates' (Algorithm 2) ...
    assert np.array_equal(trusted, want[est > tau]), "trustworthy list"
    assert n_err == n - len(trusted)
    # ... and the estimates are the oracle's Algorithm 5 on the same countBF
    # (every key of 2^20 sampled positions, the dense block among them)
    pick = np.unique(np.concatenate([st.integers(1 << 20, n), np.arange(1000, 1000 + 4096)]))
    o_est, _ = oracle.classify(cells, np.zeros(len(pick), np.uint64), want[pick], K, m, alpha,
                               nhash, tau)
    assert np.array_equal(est[pick].astype(np.uint64), o_est), "estimates"
    assert (o_est == 0).any() and (o_est > tau).any()


@pytest.mark.parametrize("K", [40, 55, 64])
def test_two_word_top_bits_sort_with_clusters(K):
    # 2^21 + 2^18 random two-word keys of K bases (past the size where two-word
    # keys take the top-bits sort) with 60 planted clusters of 260..1,400 keys
    # that differ only in their last bases, so that one shared-memory sub-bin
    # of a segment holds a whole cluster; plus one run of 20,000 keys sharing
    # their top 24 bits (a segment too large for shared memory)
    bits = 2 * K
    n = (1 << 21) + (1 << 18)
    st = readsim.Stream(5500 + K)
    hi = st.raw(n) & np.uint64((1 << (bits - 64)) - 1)
    lo = st.raw(n)
    for c in range(60):
        at = c * (n // 61) + 7
        m = 260 + 19 * c
        hi[at:at + m] = hi[at]
        lo[at:at + m] = (lo[at] & ~np.uint64(0xFFFFF)) | st.raw(m) & np.uint64(0xFFFFF)
    run = slice(n - 30_000, n - 10_000)   # the same top 24 key bits
    if bits - 64 >= 24:
        hi[run] = (hi[run] & np.uint64((1 << (bits - 88)) - 1)) | np.uint64(0x5A5A5A << (bits - 88))
    else:
        below = 24 - (bits - 64)          # top bits that live in the low word
        hi[run] = hi[n - 30_000]
        lo[run] = (lo[run] & np.uint64((1 << (64 - below)) - 1)) | (lo[n - 30_000] >> np.uint64(64 - below) << np.uint64(64 - below))
    keys = np.stack([lo, hi], axis=1)
    order = np.lexsort((lo, hi))
    want = keys[order]
    keep = np.ones(n, bool)
    keep[1:] = (want[1:, 0] != want[:-1, 0]) | (want[1:, 1] != want[:-1, 1])
    want = want[keep]
    m_cnt, alpha, nhash, tau = 1 << 24, 4, 4, 3
    words = m_cnt // 16
    cells = st.raw(words) & np.uint64(0x7777777777777777)
    with kc.CountBF(K, m_cnt, alpha, nhash, tau) as bf:
        kc.kmerco_set_counters(bf.h, cells, words)
        kc.kmerco_add_distinct(bf.h, keys, n)
        bf.classify()
        got, est = bf.distinct()
        trusted = bf.trusted()
    assert len(want) > (1 << 21)
    assert np.array_equal(got, want), "sorted distinct keys"
    assert np.array_equal(trusted, want[est > tau])
    pick = np.unique(st.integers(20_000, len(want)))
    o_est, _ = oracle.classify(cells, want[pick, 1].copy(), want[pick, 0].copy(), K, m_cnt, alpha,
                               nhash, tau)
    assert np.array_equal(est[pick].astype(np.uint64), o_est)


@pytest.mark.slow
@pytest.mark.parametrize("K", [31, 55])
def test_whole_workload_properties_and_samples(K):
    b, o = W.generate()
    n_reads = len(o) - 1
    with kc.CountBF(K, W.m, W.alpha, W.nhash, W.tau) as bf:
        bf.insert(_dev(b), _dev(o))
        bf.classify()
        st = bf.stats()
        cells = bf.counters()
        keys, est = bf.distinct()
        n_tr = kc.kmerco_get_trusted(bf.h)
        n_er = kc.kmerco_get_erroneous(bf.h)
        kw = 1 if K <= 32 else 2
        tr_dev = torch.empty(max(n_tr, 1) * kw, dtype=torch.int64, device="cuda")
        er_dev = torch.empty(max(n_er, 1) * kw, dtype=torch.int64, device="cuda")
        torch.cuda.synchronize()
        kc.kmerco_get_trusted(bf.h, tr_dev, n_tr)
        kc.kmerco_get_erroneous(bf.h, er_dev, n_er)
        torch.cuda.synchronize()
    # totals: no read holds an N, so every window is inserted
    assert st["windows"] == st["inserted"] == n_reads * (150 - K + 1)
    assert st["distinct"] == len(keys) == n_tr + n_er
    hi, lo = _split(keys, K)
    # distinct keys strictly ascending (as (hi, lo) pairs)
    asc = (hi[1:] > hi[:-1]) | ((hi[1:] == hi[:-1]) & (lo[1:] > lo[:-1]))
    assert bool(asc.all())
    # the lists are the split of the distinct keys at tau, in key order
    mask = est > W.tau
    assert int(mask.sum()) == n_tr
    trusted = tr_dev[: n_tr * kw].cpu().numpy().view(np.uint64)
    erroneous = er_dev[: n_er * kw].cpu().numpy().view(np.uint64)
    if kw == 1:
        assert np.array_equal(trusted, keys[mask]) and np.array_equal(erroneous, keys[~mask])
    else:
        assert np.array_equal(trusted.reshape(-1, 2), keys[mask])
        assert np.array_equal(erroneous.reshape(-1, 2), keys[~mask])
    # sampled estimates: Algorithm 5 by the oracle on the GPU's countBF
    pick = readsim.Stream(55 + K).integers(20_000, len(keys))
    for i in pick.tolist():
        assert int(est[i]) == oracle.query(cells, K, int(hi[i]), int(lo[i]), W.m, W.alpha,
                                           W.nhash), i
    # sampled reads: every canonical K-mer of 2,000 reads is among the
    # distinct keys, and no estimate is below the K-mer's count in the sample
    # (saturated at 2^alpha - 1)
    rows = np.unique(readsim.Stream(66 + K).integers(2000, n_reads))   # distinct reads
    sb = np.concatenate([b[int(o[r]):int(o[r + 1])] for r in rows])
    so = np.zeros(len(rows) + 1, np.uint64)
    so[1:] = np.cumsum([int(o[r + 1] - o[r]) for r in rows])
    ex = oracle.extract(sb, so, K)
    shi, slo, cnt = oracle.distinct(ex.hi, ex.lo)
    if kw == 1:
        pos = np.minimum(np.searchsorted(lo, slo), len(lo) - 1)
    else:   # keys ascend by hi, then lo: search lo within each run of equal hi
        left, right = np.searchsorted(hi, shi, "left"), np.searchsorted(hi, shi, "right")
        pos = np.array([a + int(np.searchsorted(lo[a:z], np.uint64(v))) for a, z, v in
                        zip(left.tolist(), right.tolist(), slo.tolist())], np.int64)
        pos = np.minimum(pos, len(lo) - 1)
    assert np.array_equal(lo[pos], slo) and np.array_equal(hi[pos], shi)
    maxc = (1 << W.alpha) - 1
    assert bool((est[pos].astype(np.int64) >= np.minimum(cnt.astype(np.int64), maxc)).all())
