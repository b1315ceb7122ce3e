"""Brute-force KmerCo on ASCII strings, for tiny inputs only.

An independent restatement used to pin the C oracle: it works on Python
strings (reverse complement by letter substitution, canonical form by string
comparison, packing by positional arithmetic on Python ints, MurmurHash3
written again in Python) and shares nothing with ``oracle/`` or the CUDA
library.
"""
from __future__ import annotations

import struct

_COMP = {"A": "T", "C": "G", "G": "C", "T": "A", "N": "N"}
_CODE = {"A": 0, "C": 1, "G": 2, "T": 3}
M64 = (1 << 64) - 1


def complement(s: str) -> str:
    """Section 2.2: A<->T, C<->G, N unchanged."""
    return "".join(_COMP.get(c, c) for c in s)


def reverse_complement(s: str) -> str:
    return complement(s)[::-1]


def canonical(s: str) -> str:
    """Lexicographically smaller of s and its reverse complement (Section 2.3)."""
    r = reverse_complement(s)
    return r if r < s else s


def kmers(s: str, K: int) -> list[str]:
    """All L-K+1 windows of s (Section 1.1)."""
    return [s[i:i + K] for i in range(len(s) - K + 1)]


def pack(s: str) -> tuple[int, int]:
    """(hi, lo) words of sum code(s_i) * 4^(K-1-i)."""
    v = 0
    for c in s:
        v = v * 4 + _CODE[c]
    return v >> 64, v & M64


def _rotl(x: int, r: int) -> int:
    return ((x << r) | (x >> (64 - r))) & M64


def _fmix(k: int) -> int:
    k ^= k >> 33
    k = (k * 0xFF51AFD7ED558CCD) & M64
    k ^= k >> 33
    k = (k * 0xC4CEB9FE1A85EC53) & M64
    k ^= k >> 33
    return k


def murmur3_x64_128(data: bytes, seed: int = 0) -> tuple[int, int]:
    c1, c2 = 0x87C37B91114253D5, 0x4CF5AD432745937F
    h1 = h2 = seed & 0xFFFFFFFF
    n = len(data)
    nb = n // 16
    for b in range(nb):
        k1, k2 = struct.unpack_from("<QQ", data, 16 * b)
        k1 = (_rotl((k1 * c1) & M64, 31) * c2) & M64
        h1 ^= k1
        h1 = (_rotl(h1, 27) + h2) & M64
        h1 = (h1 * 5 + 0x52DCE729) & M64
        k2 = (_rotl((k2 * c2) & M64, 33) * c1) & M64
        h2 ^= k2
        h2 = (_rotl(h2, 31) + h1) & M64
        h2 = (h2 * 5 + 0x38495AB5) & M64
    tail = data[16 * nb:]
    t = int.from_bytes(tail, "little")
    t1, t2 = t & M64, t >> 64
    if len(tail) > 8:
        h2 ^= (_rotl((t2 * c2) & M64, 33) * c1) & M64
    if len(tail) > 0:
        h1 ^= (_rotl((t1 * c1) & M64, 31) * c2) & M64
    h1 ^= n
    h2 ^= n
    h1 = (h1 + h2) & M64
    h2 = (h2 + h1) & M64
    h1 = _fmix(h1)
    h2 = _fmix(h2)
    h1 = (h1 + h2) & M64
    h2 = (h2 + h1) & M64
    return h1, h2


def key_bytes(K: int, hi: int, lo: int) -> bytes:
    return struct.pack("<Q", lo) if K <= 32 else struct.pack("<QQ", lo, hi)


def kmer_hash(K: int, hi: int, lo: int, a: int) -> int:
    return murmur3_x64_128(key_bytes(K, hi, lo), a)[0]


def run(reads: list[str], K: int, m: int, alpha: int, nhash: int, tau: int,
        canonical_keys: bool = True) -> dict:
    """Whole path on strings; counters kept as a dict of Python ints."""
    keys = []
    skipped = 0
    windows = 0
    for r in reads:
        r = r.upper() if isinstance(r, str) else r.decode().upper()
        for w in kmers(r, K):
            windows += 1
            if any(c not in "ACGT" for c in w):
                skipped += 1
                continue
            keys.append(canonical(w) if canonical_keys else w)
    maxc = (1 << alpha) - 1
    eta = 64 // alpha
    count = {}
    for w in keys:
        hi, lo = pack(w)
        for a in range(nhash):
            g = kmer_hash(K, hi, lo, a) % m
            count[g] = count.get(g, 0) + 1
    W = (m + eta - 1) // eta
    words = [0] * W
    for g, c in count.items():
        words[g // eta] |= min(c, maxc) << (alpha * (g % eta))
    exact = {}
    for w in keys:
        exact[w] = exact.get(w, 0) + 1
    distinct = sorted(exact)  # strings sort like their packed values
    est = []
    for w in distinct:
        hi, lo = pack(w)
        vals = [min(count.get(kmer_hash(K, hi, lo, a) % m, 0), maxc) for a in range(nhash)]
        est.append(0 if min(vals) == 0 else min(vals))
    trusted = [w for w, e in zip(distinct, est) if e > tau]
    erroneous = [w for w, e in zip(distinct, est) if e <= tau]
    return dict(keys=keys, words=words, distinct=distinct, est=est, trusted=trusted,
                erroneous=erroneous, exact=exact, windows=windows, skipped=skipped)
