"""Pins of the C oracle against the paper, published vectors and brute force.

Every test here runs on the CPU.  Together they are chosen so that a dropped
term, a wrong index, a swapped byte order or a transposed operand anywhere in
the oracle fails at least one of them.
"""
import os
import struct

import numpy as np
import pytest

import brute
import readsim

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.rstrip("\n")
            if not line or line.startswith("#"):
                continue
            rows.append(line)
    return rows


# --------------------------------------------------------------------------- hash
def _smhasher_verification(h):
    buf = b""
    for i in range(256):
        h1, h2 = h(bytes(range(i)), 256 - i)
        buf += struct.pack("<QQ", h1, h2)
    f1, _ = h(buf, 0)
    return f1 & 0xFFFFFFFF


def _kat():
    ver, vecs = None, []
    for row in _golden("murmur3_x64_128_kat.txt"):
        if row.startswith("smhasher_verification"):
            ver = int(row.split()[1], 16)
        elif row.startswith("vector"):
            parts = [p.strip() for p in row[len("vector"):].split("|")]
            vecs.append((parts[0].encode(), int(parts[1]), int(parts[2], 16), int(parts[3], 16)))
    return ver, vecs


def test_murmur_smhasher_verification(oracle_lib):
    ver, _ = _kat()
    assert _smhasher_verification(oracle_lib.murmur3_x64_128) == ver
    assert _smhasher_verification(brute.murmur3_x64_128) == ver


def test_murmur_published_vectors(oracle_lib):
    _, vecs = _kat()
    assert len(vecs) >= 3
    for key, seed, h1, h2 in vecs:
        assert oracle_lib.murmur3_x64_128(key, seed) == (h1, h2), key
        assert brute.murmur3_x64_128(key, seed) == (h1, h2), key


def test_murmur_c_vs_python_all_tail_lengths(oracle_lib):
    s = readsim.Stream(7)
    for n in range(0, 50):
        data = bytes(s.integers(n, 256).astype(np.uint8)) if n else b""
        seed = int(s.integers(1, 2 ** 32)[0])
        assert oracle_lib.murmur3_x64_128(data, seed) == brute.murmur3_x64_128(data, seed)


def test_kmer_hash_key_bytes(oracle_lib):
    # H_a(x) hashes the 8 little-endian bytes of a K<=32 key and the 16 bytes
    # lo-then-hi of a K>32 key, seed a.
    for K, s in ((21, "ACGTTGCAACGTACGTAAACC"), (32, "T" * 31 + "G"), (40, "ACGT" * 10)):
        hi, lo = brute.pack(s)
        for a in range(5):
            assert oracle_lib.kmer_hash(K, hi, lo, a) == brute.kmer_hash(K, hi, lo, a)


# ------------------------------------------------------------------ paper examples
def test_reverse_complement_example(oracle_lib):
    row = [r for r in _golden("paper_examples.txt") if r.startswith("rc |")][0]
    _, seq, comp, rc, _ = [p.strip() for p in row.split("|")]
    assert brute.complement(seq) == comp
    assert brute.reverse_complement(seq) == rc
    # the oracle's canonical key of the 8-mer is the packed reverse complement
    # (ATAGAGCC < GGCTCTAT); the forward key is the packed sequence
    b, o = readsim.from_strings([seq])
    fw = oracle_lib.extract(b, o, 8, canonical=False)
    cn = oracle_lib.extract(b, o, 8, canonical=True)
    assert (int(fw.hi[0]), int(fw.lo[0])) == brute.pack(seq)
    assert (int(cn.hi[0]), int(cn.lo[0])) == brute.pack(rc)
    b2, o2 = readsim.from_strings([rc])
    assert oracle_lib.extract(b2, o2, 8).lo[0] == cn.lo[0]


def test_kmer_example(oracle_lib):
    row = [r for r in _golden("paper_examples.txt") if r.startswith("kmers |")][0]
    _, seq, K, listed, _ = [p.strip() for p in row.split("|")]
    K = int(K)
    listed = listed.split()
    assert len(listed) == len(seq) - K + 1
    assert brute.kmers(seq, K) == listed
    b, o = readsim.from_strings([seq])
    ex = oracle_lib.extract(b, o, K, canonical=False)
    assert ex.n == ex.n_windows == len(listed)
    assert [int(v) for v in ex.lo] == [brute.pack(s)[1] for s in listed]
    cn = oracle_lib.extract(b, o, K, canonical=True)
    want = [brute.canonical(s) for s in listed]
    assert want == ["GCC", "AGC", "CTC", "AGA", "CTA", "ATA"]
    assert [int(v) for v in cn.lo] == [brute.pack(s)[1] for s in want]


def test_two_bit_packing_value(oracle_lib):
    b, o = readsim.from_strings(["ACGT", "acgt", "TTTT"])
    ex = oracle_lib.extract(b, o, 4, canonical=False)
    assert [int(v) for v in ex.lo] == [0b00011011, 0b00011011, 255]


def test_mask_example(oracle_lib):
    row = [r for r in _golden("paper_examples.txt") if r.startswith("mask |")][0]
    _, alpha, l1, me, mr, _ = [p.strip() for p in row.split("|")]
    alpha, l = int(alpha), int(l1) - 1  # paper counts counters from 1
    assert oracle_lib.extract_mask(alpha, l) == int(me, 16)
    assert oracle_lib.reset_mask(alpha, l) == int(mr, 16)
    assert oracle_lib.extract_mask(4, 15) == 0xF << 60


def test_eta_table(oracle_lib):
    rows = [r for r in _golden("paper_examples.txt") if r.startswith("eta |")]
    assert len(rows) == 9
    for r in rows:
        _, alpha, n, wasted, _ = [p.strip() for p in r.split("|")]
        alpha, n, wasted = int(alpha), int(n), int(wasted)
        assert oracle_lib.eta(alpha) == n
        assert 64 - oracle_lib.eta(alpha) * alpha == wasted


# ------------------------------------------------------------- window extraction
def test_window_counts_and_skips(oracle_lib):
    reads = ["ACG", "ACGTA", "ACNTACGT", "", "NNNNNNNN", "acgtRYacgt"]
    K = 4
    b, o = readsim.from_strings(reads)
    ex = oracle_lib.extract(b, o, K)
    ref = brute.run(reads, K, 64, 4, 1, 1)
    assert ex.n_windows == ref["windows"] == sum(max(0, len(r) - K + 1) for r in reads)
    assert ex.n_skipped == ref["skipped"]
    assert ex.n == len(ref["keys"])
    assert [int(v) for v in ex.lo] == [brute.pack(k)[1] for k in ref["keys"]]


@pytest.mark.parametrize("K", [1, 2, 5, 21, 31, 32, 33, 40, 55, 63, 64])
def test_extract_vs_bruteforce(oracle_lib, K):
    b, o = readsim.random_reads(40, 0, 90, seed=100 + K, alphabet=b"ACGTacgtNR",
                                weights=[24, 24, 24, 24, 1, 1, 1, 1, 0.3, 0.1])
    reads = [bytes(b[o[i]:o[i + 1]]).decode() for i in range(len(o) - 1)]
    ref = brute.run(reads, K, 1, 1, 1, 0)
    ex = oracle_lib.extract(b, o, K)
    assert ex.n_windows == ref["windows"] and ex.n_skipped == ref["skipped"]
    got = [(int(h), int(l)) for h, l in zip(ex.hi, ex.lo)]
    assert got == [brute.pack(k) for k in ref["keys"]]


# ---------------------------------------------------------------------- countBF
PARAMS = [
    # K, m, alpha, nhash, tau
    (21, 1 << 12, 4, 3, 2),
    (31, 1000, 4, 4, 3),      # m not a multiple of eta
    (17, 999, 5, 2, 1),       # eta = 12, 4 wasted bits
    (11, 4099, 7, 5, 2),      # eta = 9
    (25, 512, 8, 1, 3),
    (40, 3000, 12, 3, 5),     # two-word keys
    (9, 700, 16, 2, 2),
    (13, 300, 32, 3, 1),
    (7, 2048, 1, 3, 0),       # 1-bit counters: a plain Bloom filter
    (5, 64, 2, 6, 1),         # heavy collisions
]


@pytest.mark.parametrize("K,m,alpha,nhash,tau", PARAMS)
def test_pipeline_vs_bruteforce(oracle_lib, K, m, alpha, nhash, tau):
    b, o = readsim.random_reads(30, 0, 70, seed=K * 1000 + m, alphabet=b"ACGTacgN",
                                weights=[25, 25, 25, 25, 2, 2, 2, 0.5])
    reads = [bytes(b[o[i]:o[i + 1]]).decode() for i in range(len(o) - 1)]
    ref = brute.run(reads, K, m, alpha, nhash, tau)
    res = oracle_lib.run(b, o, K, m, alpha, nhash, tau, with_counts=True)
    assert [int(w) for w in res.filter] == ref["words"]
    assert [(int(h), int(l)) for h, l in zip(res.distinct_hi, res.distinct_lo)] == \
        [brute.pack(k) for k in ref["distinct"]]
    assert [int(e) for e in res.est] == ref["est"]
    trusted = [k for k, t in zip(ref["distinct"], res.trusted_mask) if t]
    assert trusted == ref["trusted"]
    assert [int(c) for c in res.exact_counts] == [ref["exact"][k] for k in ref["distinct"]]
    assert res.n_inserted == len(ref["keys"])


def _tiny_keys(oracle_lib, n_reads=300, seed=5, K=21):
    w = readsim.scaled("tiny", n_reads, seed_offset=seed)
    b, o = w.generate()
    return oracle_lib.extract(b, o, K)


@pytest.mark.parametrize("alpha", [1, 3, 4, 8, 16])
def test_closed_form_equals_sequential(oracle_lib, alpha):
    ex = _tiny_keys(oracle_lib)
    for m, nhash in ((1 << 14, 3), (777, 4), (64, 2)):
        a = oracle_lib.counters_closed_form(ex.hi, ex.lo, 21, m, alpha, nhash)
        b = oracle_lib.insert_sequential(ex.hi, ex.lo, 21, m, alpha, nhash)
        assert np.array_equal(a, b)


def test_wasted_bits_stay_zero(oracle_lib):
    ex = _tiny_keys(oracle_lib)
    for alpha in (5, 7, 14):
        eta = 64 // alpha
        f = oracle_lib.insert_sequential(ex.hi, ex.lo, 21, 50 * eta, alpha, 4)
        assert not np.any(f >> np.uint64(eta * alpha))


def test_order_does_not_matter(oracle_lib):
    ex = _tiny_keys(oracle_lib)
    perm = readsim.Stream(11).integers(ex.n, 1 << 62).argsort()
    a = oracle_lib.insert_sequential(ex.hi, ex.lo, 21, 4096, 4, 3)
    b = oracle_lib.insert_sequential(ex.hi[perm], ex.lo[perm], 21, 4096, 4, 3)
    assert np.array_equal(a, b)


def test_strand_does_not_matter(oracle_lib):
    reads = ["ACGTTGCATTGACCAGTAGGACCATTAGCAN", "GGCTCTATAAGCT", "TTTTTGGGGCCCAAA"]
    rcs = [brute.reverse_complement(r) for r in reads]
    b1, o1 = readsim.from_strings(reads)
    b2, o2 = readsim.from_strings(rcs[::-1])
    r1 = oracle_lib.run(b1, o1, 5, 128, 4, 3, 1)
    r2 = oracle_lib.run(b2, o2, 5, 128, 4, 3, 1)
    assert np.array_equal(r1.filter, r2.filter)
    assert np.array_equal(r1.distinct_lo, r2.distinct_lo)


def test_saturation(oracle_lib):
    # one 9-mer seen 20 times: 4-bit counters stop at 15, 8-bit ones reach 20
    b, o = readsim.from_strings(["ACGTTGCAA"] * 20)
    for alpha, want in ((4, 15), (8, 20), (2, 3), (1, 1)):
        r = oracle_lib.run(b, o, 9, 1 << 16, alpha, 2, 1)
        assert r.est.tolist() == [want]


def test_self_collision_counts_twice(oracle_lib):
    # with m = 1 every hash of every key lands in counter 0: each K-mer adds
    # k_h to it (Algorithm 3 loops over a and increments each time)
    b, o = readsim.from_strings(["ACGTA"])
    r = oracle_lib.run(b, o, 5, 1, 8, 3, 1)
    assert int(r.filter[0]) == 3 and r.est.tolist() == [3]


def test_tau_boundary(oracle_lib):
    # est == tau is erroneous ("less than or equal"); est == tau + 1 trusted
    key = "GATTACAGATTACAG"
    tau = 3
    for copies, trusted in ((tau, False), (tau + 1, True)):
        b, o = readsim.from_strings([key] * copies)
        r = oracle_lib.run(b, o, len(key), 1 << 20, 8, 4, tau)
        assert r.est.tolist() == [copies]
        assert r.trusted_mask.tolist() == [trusted]


def test_no_underestimate_and_exact_without_collisions(oracle_lib):
    w = readsim.WORKLOADS["tiny"]
    b, o = readsim.scaled("tiny", 600).generate()
    r = oracle_lib.run(b, o, w.K, w.m, w.alpha, w.nhash, w.tau, with_counts=True)
    maxc = (1 << w.alpha) - 1
    true = np.minimum(r.exact_counts, maxc)
    assert np.all(r.est >= true)
    # keys whose k_h counters are distinct and shared with no other key must
    # read back exactly min(count, 2^alpha - 1)
    gs = np.array([[oracle_lib.kmer_hash(w.K, int(h), int(l), a) % w.m for a in range(w.nhash)]
                   for h, l in zip(r.distinct_hi, r.distinct_lo)], dtype=np.int64)
    uniq, cnt = np.unique(gs, return_counts=True)
    shared = set(uniq[cnt > 1].tolist())
    clean = [i for i in range(len(gs)) if not (set(gs[i].tolist()) & shared)]
    assert len(clean) > 0.5 * len(gs)
    assert np.array_equal(r.est[clean], true[clean])


def test_seq_distinct_is_a_lower_bound(oracle_lib):
    ex = _tiny_keys(oracle_lib)
    d = len(oracle_lib.distinct(ex.hi, ex.lo)[0])
    s_small = oracle_lib.seq_distinct(ex.hi, ex.lo, 21, 256, 4, 3)
    s_big = oracle_lib.seq_distinct(ex.hi, ex.lo, 21, 1 << 22, 4, 3)
    assert s_small <= s_big <= d
    assert s_small < d  # a 256-counter filter must produce false positives


def test_merge_of_shards_equals_whole(oracle_lib):
    ex = _tiny_keys(oracle_lib)
    for alpha, m in ((4, 2048), (3, 1000), (8, 300)):
        whole = oracle_lib.insert_sequential(ex.hi, ex.lo, 21, m, alpha, 3)
        half = ex.n // 3
        a = oracle_lib.insert_sequential(ex.hi[:half], ex.lo[:half], 21, m, alpha, 3)
        b = oracle_lib.insert_sequential(ex.hi[half:], ex.lo[half:], 21, m, alpha, 3)
        assert np.array_equal(oracle_lib.merge(a, b, m, alpha), whole)


def test_classify_empty(oracle_lib):
    b, o = readsim.from_strings([])
    r = oracle_lib.run(b, o, 21, 1 << 10, 4, 3, 2)
    assert r.n_inserted == 0 and len(r.distinct_lo) == 0 and not np.any(r.filter)
