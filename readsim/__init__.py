"""Seeded synthetic sequencing reads (inputs only; none of KmerCo's arithmetic).

Both the oracle and the CUDA library consume these reads; this module holds
no packing, hashing, canonicalisation or counting -- only a genome model and
a read sampler with sequencing errors.  Every random number comes from the
raw 64-bit output of numpy's PCG64 bit generator (whose raw stream is fixed
for a seed), mapped to uniforms and integers here, so a seed gives the same
reads on any machine and numpy version.

Reads are returned in CSR form: ``bases`` (uint8 ASCII, all reads back to
back) and ``offsets`` (uint64, nreads + 1 entries, ``offsets[0] == 0``);
read r is ``bases[offsets[r]:offsets[r+1]]``.

Named workloads (the paper measures on four SRA read sets that are not
available here; these stand in for them with the same shape -- short
Illumina-like reads, both strands, substitution/indel errors, N calls):

``tiny``      50 kb uniform genome, 2,000 reads x 100 bp, 1% substitutions,
              0.1% N; K=21, 2^20 4-bit counters, 3 hashes, tau=2.
``single``    5 Mb genome at 41% GC, 1,000,000 reads x 150 bp (30x), 0.5%
              substitutions + 0.025% insertions + 0.025% deletions; K=31,
              2^28 4-bit counters (128 MiB), 4 hashes, tau=3.
``repeats``   100 Mb uniform genome, 10% of it overwritten by repeat families
              (500-5,000 bp, 2-200 copies, 1% divergence per copy),
              20,000,000 reads x 150 bp, 1% substitutions; K=31, 2^33
              4-bit counters (4 GiB), 4 hashes, tau=3.
``repeats55`` the same reads counted as 55-mers (two-word keys).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
from dataclasses import dataclass, field

import numpy as np

ASCII = np.frombuffer(b"ACGT", dtype=np.uint8)
_TWO53 = float(2 ** 53)


class Stream:
    """Uniforms and integers from PCG64's raw 64-bit words."""

    def __init__(self, seed: int):
        self._bg = np.random.PCG64(seed)

    def raw(self, n: int) -> np.ndarray:
        return self._bg.random_raw(n).astype(np.uint64, copy=False)

    def fork(self, skip: int) -> "Stream":
        """A new stream positioned ``skip`` raw words after this one (which
        does not move): it yields what this stream would after ``skip`` draws."""
        s = Stream.__new__(Stream)
        s._bg = np.random.PCG64()
        s._bg.state = self._bg.state
        if skip:
            s._bg.advance(skip)
        return s

    def skip(self, n: int) -> None:
        """Move past n raw words without drawing them."""
        if n:
            self._bg.advance(n)

    def uniform(self, n: int) -> np.ndarray:
        """Doubles in [0, 1): top 53 bits of each raw word."""
        return (self.raw(n) >> np.uint64(11)).astype(np.float64) / _TWO53

    def integers(self, n: int, hi) -> np.ndarray:
        """Integers in [0, hi) (hi scalar or array), floor(u * hi)."""
        v = np.floor(self.uniform(n) * np.asarray(hi, dtype=np.float64)).astype(np.int64)
        return np.minimum(v, np.asarray(hi, dtype=np.int64) - 1)


def genome(length: int, gc: float, stream: Stream) -> np.ndarray:
    """Genome as base indices 0..3 (A, C, G, T); P(G) = P(C) = gc / 2."""
    u = stream.uniform(length)
    at = (1.0 - gc) / 2.0
    cuts = np.array([at, at + gc / 2.0, at + gc], dtype=np.float64)
    return np.searchsorted(cuts, u, side="right").astype(np.uint8)


def add_repeat_families(g: np.ndarray, fraction: float, len_lo: int, len_hi: int,
                        copies_lo: int, copies_hi: int, divergence: float,
                        stream: Stream) -> int:
    """Overwrite ``fraction`` of ``g`` with copies of random repeat families.

    Each family is a random sequence of length U[len_lo, len_hi]; it is copied
    U{copies_lo..copies_hi} times to uniform positions, each copy with
    ``divergence`` substitutions per base.  Returns the bases written.
    """
    G = len(g)
    target = int(fraction * G)
    written = 0
    while written < target:
        flen = int(len_lo + stream.integers(1, len_hi - len_lo + 1)[0])
        fam = stream.integers(flen, 4).astype(np.uint8)
        ncopy = int(copies_lo + stream.integers(1, copies_hi - copies_lo + 1)[0])
        for _ in range(ncopy):
            pos = int(stream.integers(1, G - flen)[0])
            cp = fam.copy()
            sub = stream.uniform(flen) < divergence
            shift = stream.integers(flen, 3).astype(np.uint8) + 1
            cp[sub] = (cp[sub] + shift[sub]) % 4
            g[pos:pos + flen] = cp
            written += flen
            if written >= target:
                break
    return written


@dataclass
class ReadModel:
    n_reads: int
    read_len: int | tuple[int, int]      # fixed, or uniform [lo, hi]
    sub: float = 0.0                     # substitution rate per emitted base
    ins: float = 0.0                     # insertion rate (random base, template waits)
    dele: float = 0.0                    # deletion rate (one template base skipped)
    n_rate: float = 0.0                  # rate of 'N' calls, applied last
    both_strands: bool = True            # reverse-complement half of the reads


def sample_reads(g: np.ndarray, model: ReadModel, stream: Stream,
                 chunk: int = 200_000, threads: int | None = None) -> tuple[np.ndarray, np.ndarray]:
    """Sample reads from a circular genome ``g`` (base indices).

    Reads are drawn in chunks of ``chunk`` reads.  Every chunk takes a fixed
    number of raw words from the stream, so chunk c starts at a known stream
    position and the chunks run on ``threads`` threads (default: the CPU
    count) with the same result as one after another; the stream ends where
    a sequential pass would leave it."""
    n = model.n_reads
    if isinstance(model.read_len, tuple):
        lo, hi = model.read_len
        lens = (lo + stream.integers(n, hi - lo + 1)).astype(np.uint64)
    else:
        lens = np.full(n, model.read_len, dtype=np.uint64)
    offsets = np.zeros(n + 1, dtype=np.uint64)
    np.cumsum(lens, out=offsets[1:])
    bases = np.empty(int(offsets[-1]), dtype=np.uint8)
    lmax = int(lens.max()) if n else 0
    # raw words per read of a chunk: its start, lmax per-base words, the
    # strand, lmax N-call uniforms
    per_read = 1 + lmax + (1 if model.both_strands else 0) + (lmax if model.n_rate > 0 else 0)
    starts = list(range(0, n, chunk))

    def one(r0: int) -> None:
        r1 = min(n, r0 + chunk)
        _sample_chunk(g, model, lens[r0:r1].astype(np.int64), lmax,
                      stream.fork(r0 * per_read), bases[int(offsets[r0]):int(offsets[r1])])

    nt = threads if threads is not None else min(16, os.cpu_count() or 1)
    if nt > 1 and len(starts) > 1:
        with cf.ThreadPoolExecutor(min(nt, len(starts))) as ex:
            list(ex.map(one, starts))
    else:
        for r0 in starts:
            one(r0)
    stream.skip(n * per_read)
    return bases, offsets


def _sample_chunk(g: np.ndarray, model: ReadModel, L: np.ndarray, lmax: int, stream: Stream,
                  out: np.ndarray) -> None:
    """Reads of lengths L (one chunk) into ``out``, drawing from ``stream``."""
    G = len(g)
    nr = len(L)
    # per-base draws come from one raw 64-bit word: bits 32..63 choose the
    # error type against integer thresholds, bits 0..15 the substitution
    # (1, 2 or 3 steps round A,C,G,T), bits 16..17 an inserted base
    t_sub = np.uint64(int(model.sub * 2 ** 32))
    t_ins = np.uint64(int((model.sub + model.ins) * 2 ** 32))
    t_del = np.uint64(int((model.sub + model.ins + model.dele) * 2 ** 32))
    indels = model.ins > 0 or model.dele > 0
    jj = np.arange(lmax, dtype=np.int64)[None, :]
    start = stream.integers(nr, G)
    raw = stream.raw(nr * lmax).reshape(nr, lmax)
    top = raw >> np.uint64(32)
    is_sub = top < t_sub
    if indels:
        is_ins = (top >= t_sub) & (top < t_ins)
        is_del = (top >= t_ins) & (top < t_del)
        adv = np.where(is_ins, 0, np.where(is_del, 2, 1)).astype(np.int64)
        before = np.cumsum(adv, axis=1) - adv
        tidx = (start[:, None] + before + is_del.astype(np.int64)) % G
    else:
        tidx = (start[:, None] + jj) % G
    codes = g[tidx]
    if indels:
        rnd = ((raw >> np.uint64(16)) & np.uint64(3)).astype(np.uint8)
        codes = np.where(is_ins, rnd, codes)
    shift = (((raw & np.uint64(0xFFFF)) * np.uint64(3)) >> np.uint64(16)).astype(np.uint8) + 1
    codes = np.where(is_sub, (codes + shift) & 3, codes).astype(np.uint8)
    if model.both_strands:
        rev = stream.uniform(nr) < 0.5
    else:
        rev = np.zeros(nr, dtype=bool)
    asc = ASCII[codes]
    if model.n_rate > 0:
        asc[stream.uniform(nr * lmax).reshape(nr, lmax) < model.n_rate] = ord("N")
    # opposite strand: complement (A<->T, C<->G, N stays) and reverse each
    # read within its own length
    if rev.any():
        src = np.where(rev[:, None], L[:, None] - 1 - jj, jj)
        np.clip(src, 0, lmax - 1, out=src)
        asc = np.take_along_axis(asc, src, axis=1)
        asc = np.where(rev[:, None], _COMPLEMENT[asc], asc)
    keep = jj < L[:, None]
    out[:] = asc[keep]


_COMPLEMENT = np.arange(256, dtype=np.uint8)
for _a, _b in (("A", "T"), ("C", "G"), ("G", "C"), ("T", "A")):
    _COMPLEMENT[ord(_a)] = ord(_b)


@dataclass
class Workload:
    name: str
    K: int
    m: int                 # counters
    alpha: int             # counter bits
    nhash: int
    tau: int
    genome_len: int
    gc: float
    reads: ReadModel
    seed: int
    repeats: dict | None = None
    note: str = ""
    extra: dict = field(default_factory=dict)

    def generate(self) -> tuple[np.ndarray, np.ndarray]:
        s = Stream(self.seed)
        g = genome(self.genome_len, self.gc, s)
        if self.repeats:
            add_repeat_families(g, stream=s, **self.repeats)
        return sample_reads(g, self.reads, s)


WORKLOADS = {
    "tiny": Workload("tiny", K=21, m=1 << 20, alpha=4, nhash=3, tau=2, genome_len=50_000,
                     gc=0.5, reads=ReadModel(2_000, 100, sub=0.01, n_rate=0.001), seed=1001),
    "single": Workload("single", K=31, m=1 << 28, alpha=4, nhash=4, tau=3,
                       genome_len=5_000_000, gc=0.41,
                       reads=ReadModel(1_000_000, 150, sub=0.005, ins=0.00025, dele=0.00025),
                       seed=2001),
    "repeats": Workload("repeats", K=31, m=1 << 33, alpha=4, nhash=4, tau=3,
                        genome_len=100_000_000, gc=0.5,
                        reads=ReadModel(20_000_000, 150, sub=0.01), seed=3001,
                        repeats=dict(fraction=0.10, len_lo=500, len_hi=5000, copies_lo=2,
                                     copies_hi=200, divergence=0.01)),
    "repeats55": Workload("repeats55", K=55, m=1 << 33, alpha=4, nhash=4, tau=3,
                          genome_len=100_000_000, gc=0.5,
                          reads=ReadModel(20_000_000, 150, sub=0.01), seed=3001,
                          repeats=dict(fraction=0.10, len_lo=500, len_hi=5000, copies_lo=2,
                                       copies_hi=200, divergence=0.01)),
}


def scaled(name: str, n_reads: int, seed_offset: int = 0) -> Workload:
    """The named workload with fewer (or more) reads and an optional new seed."""
    w = WORKLOADS[name]
    r = w.reads
    return Workload(w.name + f"[{n_reads}]", w.K, w.m, w.alpha, w.nhash, w.tau, w.genome_len,
                    w.gc, ReadModel(n_reads, r.read_len, r.sub, r.ins, r.dele, r.n_rate,
                                    r.both_strands), w.seed + seed_offset, w.repeats)


def from_strings(reads: list[str] | list[bytes]) -> tuple[np.ndarray, np.ndarray]:
    """CSR arrays from a list of read strings (for small hand-made cases)."""
    bs = [r.encode() if isinstance(r, str) else bytes(r) for r in reads]
    offsets = np.zeros(len(bs) + 1, dtype=np.uint64)
    np.cumsum([len(b) for b in bs], out=offsets[1:])
    bases = np.frombuffer(b"".join(bs), dtype=np.uint8).copy()
    return bases, offsets


def random_reads(n_reads: int, len_lo: int, len_hi: int, seed: int, alphabet: bytes = b"ACGT",
                 weights: list[float] | None = None) -> tuple[np.ndarray, np.ndarray]:
    """Reads of i.i.d. letters from ``alphabet`` (edge-case inputs: N, IUPAC, lowercase)."""
    s = Stream(seed)
    lens = (len_lo + s.integers(n_reads, len_hi - len_lo + 1)).astype(np.uint64)
    offsets = np.zeros(n_reads + 1, dtype=np.uint64)
    np.cumsum(lens, out=offsets[1:])
    total = int(offsets[-1])
    alpha = np.frombuffer(alphabet, dtype=np.uint8)
    if weights is None:
        idx = s.integers(total, len(alpha))
    else:
        cw = np.cumsum(np.asarray(weights, dtype=np.float64))
        idx = np.searchsorted(cw / cw[-1], s.uniform(total), side="right")
        idx = np.minimum(idx, len(alpha) - 1)
    return alpha[idx].astype(np.uint8), offsets
