"""Pins of the oracle's paper-literal variants.

- Hash-chosen canonical K-mer (Section 2.3's equation with h = H_0): the
  forward K-mer when H_0(forward) < H_0(reverse complement), else the reverse
  complement.  Pinned by brute force with the independent Python hash, and
  by strand invariance.
- Windows over the whole file (the reads taken as one sequence): pinned by
  the K-mer totals the paper prints for K = 28 and K = 55, and by brute force.
"""
import os

import numpy as np
import pytest

import brute
import oracle
import readsim

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_examples.txt")


def _reads(b, o):
    return [bytes(b[o[i]:o[i + 1]]).decode() for i in range(len(o) - 1)]


def _valid(w):
    return all(c in "ACGTacgt" for c in w)


def _hash_canonical(w):
    w = w.upper()
    K = len(w)
    f, r = brute.pack(w), brute.pack(brute.reverse_complement(w))
    hf, hr = brute.kmer_hash(K, *f, 0), brute.kmer_hash(K, *r, 0)
    return f if hf < hr else r


@pytest.mark.parametrize("K", [1, 2, 5, 16, 21, 31, 32, 33, 40, 55, 64])
def test_hash_canonical_vs_bruteforce(K):
    b, o = readsim.random_reads(25, 0, 90, seed=500 + K, alphabet=b"ACGTacgtN",
                                weights=[24, 24, 24, 24, 1, 1, 1, 1, 0.3])
    want = [_hash_canonical(w) for s in _reads(b, o) for w in brute.kmers(s, K) if _valid(w)]
    ex = oracle.extract(b, o, K, canonical_hash=True)
    assert [(int(h), int(l)) for h, l in zip(ex.hi, ex.lo)] == want
    # it differs from the lexicographic choice on a good share of windows
    lex = oracle.extract(b, o, K)
    if K >= 5:
        differ = np.count_nonzero((lex.lo != ex.lo) | (lex.hi != ex.hi))
        assert 0.2 * ex.n < differ < 0.8 * ex.n


@pytest.mark.parametrize("K", [7, 31, 55])
def test_hash_canonical_is_strand_invariant(K):
    b, o = readsim.random_reads(40, 60, 120, seed=K)
    rc = [brute.reverse_complement(s) for s in _reads(b, o)]
    b2, o2 = readsim.from_strings(rc)
    a = oracle.extract(b, o, K, canonical_hash=True)
    c = oracle.extract(b2, o2, K, canonical_hash=True)
    key = lambda e: sorted(zip(e.hi.tolist(), e.lo.tolist()))  # noqa: E731
    assert key(a) == key(c)


def test_whole_file_windows_vs_bruteforce():
    b, o = readsim.random_reads(30, 0, 40, seed=8, alphabet=b"ACGTN",
                                weights=[25, 25, 25, 25, 0.5])
    seq = "".join(_reads(b, o))
    for K in (3, 21, 33):
        ws = brute.kmers(seq, K)
        ex = oracle.extract(b, o, K, whole_file=True)
        assert ex.n_windows == max(0, len(seq) - K + 1)
        assert ex.n_skipped == sum(not _valid(w) for w in ws)
        assert [(int(h), int(l)) for h, l in zip(ex.hi, ex.lo)] == \
            [brute.pack(brute.canonical(w)) for w in ws if _valid(w)]


def test_whole_file_totals_match_the_paper():
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            if line.startswith("totals |"):
                _, n28, n55, _ = [p.strip() for p in line.split("|")]
                rows.append((int(n28), int(n55)))
    assert len(rows) == 4
    b, o = readsim.random_reads(500, 80, 200, seed=3)   # no N: every window counts
    for n28, n55 in rows:
        d = n28 - n55
        w28 = oracle.extract(b, o, 28, whole_file=True).n_windows
        w55 = oracle.extract(b, o, 55, whole_file=True).n_windows
        assert w28 - w55 == d == 27
        # windows kept inside reads would differ by 27 per read
        assert oracle.extract(b, o, 28).n_windows - oracle.extract(b, o, 55).n_windows \
            == 27 * (len(o) - 1)


def test_variants_through_the_pipeline():
    b, o = readsim.random_reads(200, 20, 150, seed=12)
    for kw in (dict(canonical_hash=True), dict(whole_file=True),
               dict(canonical_hash=True, whole_file=True)):
        r = oracle.run(b, o, 21, 1 << 14, 4, 3, 2, **kw)    # closed form == sequential inside
        ex = oracle.extract(b, o, 21, **kw)
        assert r.n_inserted == ex.n
        assert np.array_equal(r.distinct_lo, np.unique(ex.lo))


# ------------------------------------------- Algorithm 1 as printed (diagnostic)
def test_literal_insertion_reduces_to_hash_canonical_with_one_hash():
    # with k_h = 1 QcountBF-I's strand choice is H_0(Read) < H_0(Read_RC),
    # state-independent, and with wide counters nothing overflows: the
    # printed insertion then builds exactly the hash-canonical filter, and its
    # first-seen windows are the sequential first-seen count of those keys
    b, o = readsim.random_reads(300, 30, 120, seed=41, alphabet=b"ACGTN",
                                weights=[25, 25, 25, 25, 0.3])
    for K, m in ((21, 1 << 12), (40, 777)):
        filt, dhi, dlo = oracle.literal_insertion(b, o, K, m, 16, 1)
        ref = oracle.run(b, o, K, m, 16, 1, 2, canonical_hash=True)
        assert np.array_equal(filt, ref.filter)
        ex = oracle.extract(b, o, K, canonical_hash=True)
        assert len(dlo) == oracle.seq_distinct(ex.hi, ex.lo, K, m, 16, 1)
        # every first-seen key is one of the distinct keys
        keys = set(zip(ref.distinct_hi.tolist(), ref.distinct_lo.tolist()))
        assert set(zip(dhi.tolist(), dlo.tolist())) <= keys


def test_literal_insertion_with_one_hash_saturates_like_the_reading():
    # with one hash per K-mer, "stop the insertion at the first full counter"
    # and "leave a full counter alone and go on" are the same rule, so the
    # printed loop equals the per-counter saturating reading even when
    # counters fill up (1- and 2-bit counters, a small filter)
    b, o = readsim.random_reads(200, 30, 80, seed=42)
    for alpha in (1, 2):
        filt, _, _ = oracle.literal_insertion(b, o, 15, 1 << 10, alpha, 1)
        ref = oracle.run(b, o, 15, 1 << 10, alpha, 1, 0, canonical_hash=True)
        assert np.array_equal(filt, ref.filter)
        assert int(ref.est.max()) == (1 << alpha) - 1      # saturation did happen
