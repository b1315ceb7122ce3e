"""KmerCo oracle (arXiv 2305.07545): plain CPU countBF, written from the paper.

TEST INFRASTRUCTURE ONLY.  Only the test-suite, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import this package.  It shares
no code with the CUDA library (``paper_2305_07545_gb300``) and imports
nothing from it.

The arithmetic lives in ``kmerco_oracle.c`` (single-threaded C, compiled by
``build()``); this module only marshals numpy arrays into it and strings the
steps together in the paper's order:

1. extract every valid window of every read, canonicalise (Sections 1.1,
   2.2, 2.3; Algorithm 1);
2. build the countBF twice -- by its closed form and by the sequential
   Algorithm 3 loop -- and require the two to agree;
3. distinct K-mers = sort + unique of the keys (exact; replaces the
   order-dependent distinct file of Algorithm 1);
4. QcountBF-II (Algorithm 5) per distinct key, split at tau (Algorithm 2).

Parity pins: see the header of ``kmerco_oracle.c`` and ``tests/test_oracle_*``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kmerco_oracle.c")
_LIB = os.path.join(_HERE, "libkmerco_oracle.so")

_u8p = ctypes.POINTER(ctypes.c_uint8)
_u32p = ctypes.POINTER(ctypes.c_uint32)
_u64p = ctypes.POINTER(ctypes.c_uint64)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, -O2, no target-specific flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"],
                       check=True)
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        L.oracle_murmur3_x64_128.argtypes = [_u8p, ctypes.c_uint64, ctypes.c_uint32, _u64p]
        L.oracle_murmur3_x64_128.restype = None
        L.oracle_base_code.argtypes = [ctypes.c_uint8]
        L.oracle_base_code.restype = ctypes.c_int
        L.oracle_extract.argtypes = [_u8p, _u64p, ctypes.c_uint64, ctypes.c_int, ctypes.c_int,
                                     _u64p, _u64p, _u64p, _u64p]
        L.oracle_extract.restype = ctypes.c_uint64
        L.oracle_kmer_hash.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64,
                                       ctypes.c_uint32]
        L.oracle_kmer_hash.restype = ctypes.c_uint64
        L.oracle_eta.argtypes = [ctypes.c_int]
        L.oracle_eta.restype = ctypes.c_int
        L.oracle_words.argtypes = [ctypes.c_uint64, ctypes.c_int]
        L.oracle_words.restype = ctypes.c_uint64
        L.oracle_extract_mask.argtypes = [ctypes.c_int, ctypes.c_int]
        L.oracle_extract_mask.restype = ctypes.c_uint64
        L.oracle_reset_mask.argtypes = [ctypes.c_int, ctypes.c_int]
        L.oracle_reset_mask.restype = ctypes.c_uint64
        L.oracle_insert_sequential.argtypes = [_u64p, _u64p, ctypes.c_uint64, ctypes.c_int,
                                               ctypes.c_uint64, ctypes.c_int, ctypes.c_int, _u64p]
        L.oracle_insert_sequential.restype = None
        L.oracle_counters_closed_form.argtypes = [_u64p, _u64p, ctypes.c_uint64, ctypes.c_int,
                                                  ctypes.c_uint64, ctypes.c_int, ctypes.c_int,
                                                  _u32p, _u64p]
        L.oracle_counters_closed_form.restype = None
        L.oracle_query.argtypes = [_u64p, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64,
                                   ctypes.c_uint64, ctypes.c_int, ctypes.c_int]
        L.oracle_query.restype = ctypes.c_uint64
        L.oracle_seq_distinct.argtypes = [_u64p, _u64p, ctypes.c_uint64, ctypes.c_int,
                                          ctypes.c_uint64, ctypes.c_int, ctypes.c_int, _u64p]
        L.oracle_seq_distinct.restype = ctypes.c_uint64
        L.oracle_distinct.argtypes = [_u64p, _u64p, ctypes.c_uint64, _u64p, _u64p, _u64p]
        L.oracle_distinct.restype = ctypes.c_uint64
        L.oracle_classify.argtypes = [_u64p, _u64p, _u64p, ctypes.c_uint64, ctypes.c_int,
                                      ctypes.c_uint64, ctypes.c_int, ctypes.c_int,
                                      ctypes.c_uint64, _u64p, _u8p]
        L.oracle_classify.restype = ctypes.c_uint64
        L.oracle_merge.argtypes = [_u64p, _u64p, ctypes.c_uint64, ctypes.c_int]
        L.oracle_insert_sequential_2d.argtypes = [_u64p, _u64p, ctypes.c_uint64, ctypes.c_int,
                                                  ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int,
                                                  ctypes.c_int, _u64p]
        L.oracle_insert_sequential_2d.restype = None
        L.oracle_query_2d.argtypes = [_u64p, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64,
                                      ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int, ctypes.c_int]
        L.oracle_query_2d.restype = ctypes.c_uint64
        L.oracle_classify_2d.argtypes = [_u64p, _u64p, _u64p, ctypes.c_uint64, ctypes.c_int,
                                         ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int,
                                         ctypes.c_int, ctypes.c_uint64, _u64p, _u8p]
        L.oracle_classify_2d.restype = ctypes.c_uint64
        L.oracle_extract_ex.argtypes = [_u8p, _u64p, ctypes.c_uint64, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_int, _u64p, _u64p, _u64p, _u64p]
        L.oracle_extract_ex.restype = ctypes.c_uint64
        L.oracle_literal_insertion.argtypes = [_u8p, _u64p, ctypes.c_uint64, ctypes.c_int,
                                               ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                                               ctypes.c_int, ctypes.c_int, _u64p, _u64p, _u64p]
        L.oracle_literal_insertion.restype = ctypes.c_uint64
        L.oracle_paper_dims.argtypes = [ctypes.c_uint64, ctypes.c_double, _u64p, _u64p]
        L.oracle_paper_dims.restype = ctypes.c_int
        L.oracle_merge.restype = None
        _lib = L
    return _lib


def _p(a: np.ndarray, ty):
    return a.ctypes.data_as(ty)


def _check_params(K: int, m: int, alpha: int, nhash: int) -> None:
    if not (1 <= K <= 64):
        raise ValueError("K must be in [1, 64]")
    if not (1 <= alpha <= 32):
        raise ValueError("alpha must be in [1, 32]")
    if m < 1 or nhash < 1:
        raise ValueError("m and nhash must be >= 1")


# --------------------------------------------------------------------------- hash
def murmur3_x64_128(data: bytes, seed: int = 0) -> tuple[int, int]:
    """MurmurHash3_x64_128 of ``data`` -> (h1, h2) as unsigned 64-bit ints."""
    buf = np.frombuffer(bytes(data), dtype=np.uint8).copy() if data else np.zeros(1, np.uint8)
    out = np.zeros(2, np.uint64)
    lib().oracle_murmur3_x64_128(_p(buf, _u8p), len(data), seed & 0xFFFFFFFF, _p(out, _u64p))
    return int(out[0]), int(out[1])


def kmer_hash(K: int, hi: int, lo: int, a: int) -> int:
    """H_a of a packed K-mer (Section 3 'murmur', seed a, first output word)."""
    return int(lib().oracle_kmer_hash(K, hi, lo, a))


def base_code(c: str) -> int:
    return int(lib().oracle_base_code(ord(c)))


def eta(alpha: int) -> int:
    return int(lib().oracle_eta(alpha))


def words(m: int, alpha: int) -> int:
    return int(lib().oracle_words(m, alpha))


def extract_mask(alpha: int, l: int) -> int:
    return int(lib().oracle_extract_mask(alpha, l))


def reset_mask(alpha: int, l: int) -> int:
    return int(lib().oracle_reset_mask(alpha, l))


# --------------------------------------------------------------------------- steps
@dataclass
class Extracted:
    hi: np.ndarray
    lo: np.ndarray
    n_windows: int   # sum over reads of max(0, len - K + 1)
    n_skipped: int   # windows holding a non-ACGT byte

    @property
    def n(self) -> int:
        return len(self.lo)


def extract(bases: np.ndarray, offsets: np.ndarray, K: int, canonical: bool = True,
            canonical_hash: bool = False, whole_file: bool = False) -> Extracted:
    """All valid windows of all reads, in input order (Algorithm 1 loop).

    ``canonical_hash`` picks the strand with the smaller H_0 instead of the
    lexicographically smaller one; ``whole_file`` runs the windows across
    read boundaries (the reads as one sequence).
    """
    bases = np.ascontiguousarray(bases, dtype=np.uint8)
    offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
    nreads = len(offsets) - 1
    if nreads < 0:
        raise ValueError("offsets needs nreads + 1 entries")
    if canonical_hash and not canonical:
        raise ValueError("canonical_hash needs canonical K-mers")
    cap = int(sum(max(0, int(offsets[r + 1]) - int(offsets[r]) - K + 1) for r in range(nreads))) \
        if nreads < 4096 and not whole_file else int(max(0, int(offsets[-1]) - int(offsets[0])))
    hi = np.zeros(max(cap, 1), np.uint64)
    lo = np.zeros(max(cap, 1), np.uint64)
    nw = ctypes.c_uint64(0)
    ns = ctypes.c_uint64(0)
    bptr = bases if len(bases) else np.zeros(1, np.uint8)
    mode = 2 if canonical_hash else int(bool(canonical))
    n = lib().oracle_extract_ex(_p(bptr, _u8p), _p(offsets, _u64p), nreads, K, mode,
                                int(bool(whole_file)), _p(hi, _u64p), _p(lo, _u64p),
                                ctypes.byref(nw), ctypes.byref(ns))
    return Extracted(hi[:n].copy(), lo[:n].copy(), int(nw.value), int(ns.value))


def counters_closed_form(hi: np.ndarray, lo: np.ndarray, K: int, m: int, alpha: int,
                         nhash: int) -> np.ndarray:
    _check_params(K, m, alpha, nhash)
    hi = np.ascontiguousarray(hi, np.uint64)
    lo = np.ascontiguousarray(lo, np.uint64)
    counts = np.zeros(m, np.uint32)
    filt = np.zeros(words(m, alpha), np.uint64)
    lib().oracle_counters_closed_form(_p(hi, _u64p), _p(lo, _u64p), len(lo), K, m, alpha, nhash,
                                      _p(counts, _u32p), _p(filt, _u64p))
    return filt


def insert_sequential(hi: np.ndarray, lo: np.ndarray, K: int, m: int, alpha: int, nhash: int,
                      filt: np.ndarray | None = None) -> np.ndarray:
    _check_params(K, m, alpha, nhash)
    hi = np.ascontiguousarray(hi, np.uint64)
    lo = np.ascontiguousarray(lo, np.uint64)
    if filt is None:
        filt = np.zeros(words(m, alpha), np.uint64)
    lib().oracle_insert_sequential(_p(hi, _u64p), _p(lo, _u64p), len(lo), K, m, alpha, nhash,
                                   _p(filt, _u64p))
    return filt


def query(filt: np.ndarray, K: int, hi: int, lo: int, m: int, alpha: int, nhash: int) -> int:
    return int(lib().oracle_query(_p(filt, _u64p), K, hi, lo, m, alpha, nhash))


def seq_distinct(hi: np.ndarray, lo: np.ndarray, K: int, m: int, alpha: int, nhash: int) -> int:
    hi = np.ascontiguousarray(hi, np.uint64)
    lo = np.ascontiguousarray(lo, np.uint64)
    filt = np.zeros(words(m, alpha), np.uint64)
    return int(lib().oracle_seq_distinct(_p(hi, _u64p), _p(lo, _u64p), len(lo), K, m, alpha,
                                         nhash, _p(filt, _u64p)))


def distinct(hi: np.ndarray, lo: np.ndarray):
    """Sorted unique keys and their exact multiplicities."""
    hi = np.ascontiguousarray(hi, np.uint64)
    lo = np.ascontiguousarray(lo, np.uint64)
    n = len(lo)
    dhi = np.zeros(max(n, 1), np.uint64)
    dlo = np.zeros(max(n, 1), np.uint64)
    cnt = np.zeros(max(n, 1), np.uint64)
    if n == 0:
        return dhi[:0], dlo[:0], cnt[:0]
    d = int(lib().oracle_distinct(_p(hi, _u64p), _p(lo, _u64p), n, _p(dhi, _u64p),
                                  _p(dlo, _u64p), _p(cnt, _u64p)))
    if d == 2 ** 64 - 1:
        raise MemoryError("oracle_distinct: allocation failed")
    return dhi[:d].copy(), dlo[:d].copy(), cnt[:d].copy()


def classify(filt: np.ndarray, dhi: np.ndarray, dlo: np.ndarray, K: int, m: int, alpha: int,
             nhash: int, tau: int):
    """Algorithm 2: per-key estimates and the trusted flag (est > tau)."""
    dhi = np.ascontiguousarray(dhi, np.uint64)
    dlo = np.ascontiguousarray(dlo, np.uint64)
    d = len(dlo)
    est = np.zeros(max(d, 1), np.uint64)
    tr = np.zeros(max(d, 1), np.uint8)
    if d:
        lib().oracle_classify(_p(filt, _u64p), _p(dhi, _u64p), _p(dlo, _u64p), d, K, m, alpha,
                              nhash, tau, _p(est, _u64p), _p(tr, _u8p))
    return est[:d].copy(), tr[:d].astype(bool)


def paper_dims(n: int, fpp: float = 0.001) -> tuple[int, int]:
    """Eq. 1: the prime dimensions (X, Y) of a countBF sized for n items."""
    x = ctypes.c_uint64(0)
    y = ctypes.c_uint64(0)
    if lib().oracle_paper_dims(n, fpp, ctypes.byref(x), ctypes.byref(y)) != 0:
        raise ValueError("paper_dims: n must be >= 1 and 0 < fpp < 1")
    return int(x.value), int(y.value)


def insert_sequential_2d(hi: np.ndarray, lo: np.ndarray, K: int, dims: tuple[int, int],
                         alpha: int, nhash: int, filt: np.ndarray | None = None) -> np.ndarray:
    """Algorithm 3 on a two-dimensional countBF of X x Y cells (row-major)."""
    X, Y = dims
    _check_params(K, X * Y * eta(alpha), alpha, nhash)
    hi = np.ascontiguousarray(hi, np.uint64)
    lo = np.ascontiguousarray(lo, np.uint64)
    if filt is None:
        filt = np.zeros(X * Y, np.uint64)
    lib().oracle_insert_sequential_2d(_p(hi, _u64p), _p(lo, _u64p), len(lo), K, X, Y, alpha,
                                      nhash, _p(filt, _u64p))
    return filt


def query_2d(filt: np.ndarray, K: int, hi: int, lo: int, dims: tuple[int, int], alpha: int,
             nhash: int) -> int:
    return int(lib().oracle_query_2d(_p(filt, _u64p), K, hi, lo, dims[0], dims[1], alpha, nhash))


def classify_2d(filt: np.ndarray, dhi: np.ndarray, dlo: np.ndarray, K: int,
                dims: tuple[int, int], alpha: int, nhash: int, tau: int):
    dhi = np.ascontiguousarray(dhi, np.uint64)
    dlo = np.ascontiguousarray(dlo, np.uint64)
    d = len(dlo)
    est = np.zeros(max(d, 1), np.uint64)
    tr = np.zeros(max(d, 1), np.uint8)
    if d:
        lib().oracle_classify_2d(_p(filt, _u64p), _p(dhi, _u64p), _p(dlo, _u64p), d, K, dims[0],
                                 dims[1], alpha, nhash, tau, _p(est, _u64p), _p(tr, _u8p))
    return est[:d].copy(), tr[:d].astype(bool)


def literal_insertion(bases: np.ndarray, offsets: np.ndarray, K: int, m: int, alpha: int,
                      nhash: int, dims: tuple[int, int] | None = None):
    """Algorithms 1, 3 and 4 exactly as printed, in input order (diagnostic).

    Returns (filter, first-seen keys as (hi, lo) arrays).  Order dependent:
    the strand and the early overflow stop depend on the filter state.
    """
    bases = np.ascontiguousarray(bases, dtype=np.uint8)
    offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
    nreads = len(offsets) - 1
    dx, dy = dims if dims is not None else (0, 0)
    words_ = dx * dy if dims is not None else words(m, alpha)
    filt = np.zeros(max(words_, 1), np.uint64)
    cap = max(1, int(offsets[-1] - offsets[0]) if nreads > 0 else 1)
    dhi = np.zeros(cap, np.uint64)
    dlo = np.zeros(cap, np.uint64)
    bptr = bases if len(bases) else np.zeros(1, np.uint8)
    n = lib().oracle_literal_insertion(_p(bptr, _u8p), _p(offsets, _u64p), nreads, K, m, dx, dy,
                                       alpha, nhash, _p(filt, _u64p), _p(dhi, _u64p),
                                       _p(dlo, _u64p))
    return filt[:words_], dhi[:n].copy(), dlo[:n].copy()


def merge(dst: np.ndarray, src: np.ndarray, m: int, alpha: int) -> np.ndarray:
    """Counter-wise saturating sum of two filters, in place in ``dst``."""
    lib().oracle_merge(_p(dst, _u64p), _p(np.ascontiguousarray(src, np.uint64), _u64p), m, alpha)
    return dst


@dataclass
class Result:
    filter: np.ndarray       # W packed words
    distinct_hi: np.ndarray  # D keys, ascending
    distinct_lo: np.ndarray
    est: np.ndarray          # D estimates (QcountBF-II)
    trusted_mask: np.ndarray  # D booleans, est > tau
    n_windows: int
    n_skipped: int
    n_inserted: int
    exact_counts: np.ndarray | None = None


def run(bases: np.ndarray, offsets: np.ndarray, K: int, m: int, alpha: int, nhash: int,
        tau: int, canonical: bool = True, cross_check: bool = True,
        with_counts: bool = False, dims: tuple[int, int] | None = None,
        canonical_hash: bool = False, whole_file: bool = False) -> Result:
    """The whole path: extract -> countBF -> distinct -> classify.

    With ``cross_check`` the filter is built both by the closed form and by
    the sequential Algorithm 3 loop, and the two must be identical.  With
    ``dims = (X, Y)`` the countBF is two-dimensional (m is ignored; the
    closed form exists for the flat layout only, so there is no cross-check).
    """
    if dims is not None:
        ex = extract(bases, offsets, K, canonical, canonical_hash, whole_file)
        filt = insert_sequential_2d(ex.hi, ex.lo, K, dims, alpha, nhash)
        dhi, dlo, cnt = distinct(ex.hi, ex.lo)
        est, tr = classify_2d(filt, dhi, dlo, K, dims, alpha, nhash, tau)
        return Result(filt, dhi, dlo, est, tr, ex.n_windows, ex.n_skipped, ex.n,
                      cnt if with_counts else None)
    _check_params(K, m, alpha, nhash)
    ex = extract(bases, offsets, K, canonical, canonical_hash, whole_file)
    filt = insert_sequential(ex.hi, ex.lo, K, m, alpha, nhash)
    if cross_check:
        cf = counters_closed_form(ex.hi, ex.lo, K, m, alpha, nhash)
        if not np.array_equal(cf, filt):
            raise AssertionError("oracle: closed form and sequential Algorithm 3 disagree")
    dhi, dlo, cnt = distinct(ex.hi, ex.lo)
    est, tr = classify(filt, dhi, dlo, K, m, alpha, nhash, tau)
    return Result(filt, dhi, dlo, est, tr, ex.n_windows, ex.n_skipped, ex.n,
                  cnt if with_counts else None)
