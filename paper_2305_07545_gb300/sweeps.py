"""Counter-length and countBF-size sweeps, rerun on synthetic reads.

The paper sweeps the counter length (alpha = 5..16 bits at a fixed countBF
size) and the countBF size (1/8x .. 2x of the size Eq. 1 gives, at 8-bit
counters) on one dataset and reports insertion time and the classification
counts (supplement tables).  This module runs the same two sweeps on the
synthetic `single` read set (28-mers and 55-mers, as in the paper), with the
paper's two-dimensional prime geometry sized by Eq. 1 (FPP = 0.001), and
prints one JSON line per setting.

Each line reports the insertion rate (device time of kmerco_insert), the
distinct / trustworthy / erroneous counts (tau = 5, as in the paper's exact
tables), the saturated counters and, as the accuracy measure, how many
distinct K-mers are classified differently than by their exact
multiplicities (trustworthy when a K-mer occurs more than tau times, the
paper's exact-count ground truth of section 4).  The exact multiplicities
come from a sort of every window's canonical K-mer on the host (numpy), not
from any countBF.

    python -m paper_2305_07545_gb300.sweeps [--reads N] [--K 28 55]
"""
from __future__ import annotations

import argparse
import json

import numpy as np

import readsim

from . import CountBF, kmerco_paper_dims

TAU = 5
NHASH = 3


def _count(bases, offsets, K, alpha, dims, m=0):
    bf = CountBF(K, m, alpha, NHASH, TAU, dims=dims)
    try:
        bf.insert(bases, offsets)
        bf.classify()
        st = bf.stats()
        return bf, st
    except Exception:
        bf.close()
        raise


_CODE = np.full(256, 4, np.uint8)   # 2-bit base codes; 4 marks a base that is not ACGT
for _i, _c in enumerate("ACGT"):
    _CODE[ord(_c)] = _CODE[ord(_c.lower())] = _i


def exact_counts(bases: np.ndarray, offsets: np.ndarray, K: int):
    """Every distinct canonical K-mer of the reads with its multiplicity.

    Windows of K bases inside one read with no base outside ACGT (either
    case); the canonical key is the smaller of the forward and the reverse
    complement 2K-bit values (first base most significant).  Returns
    (keys, counts): keys ascending, uint64 for K <= 32, else rows
    (low word, high word) like the library's two-word keys."""
    c = _CODE[bases[int(offsets[0]):int(offsets[-1])]].astype(np.uint64)
    L = len(c)
    nw = L - K + 1
    if nw <= 0:
        return (np.zeros(0, np.uint64) if K <= 32 else np.zeros((0, 2), np.uint64),
                np.zeros(0, np.int64))
    bad = np.concatenate([[0], np.cumsum(c == 4)])
    ok = bad[K:K + nw] == bad[:nw]
    # a window must not run past the end of its read
    last = np.zeros(L + 1, np.int64)
    ends = offsets[1:-1].astype(np.int64) - int(offsets[0])
    last[ends] = 1
    brk = np.cumsum(last)[:L]                     # read index of each base
    ok &= brk[K - 1:K - 1 + nw] == brk[:nw]
    c = np.where(c == 4, 0, c)
    comp = np.uint64(3) - c
    lo_n = min(K, 32)                            # bases in the low word
    hi_n = K - lo_n

    def pack(arr, first, count, reverse):
        v = np.zeros(nw, np.uint64)
        for j in range(count):
            i = first + (count - 1 - j if reverse else j)
            v = (v << np.uint64(2)) | arr[i:i + nw]
        return v

    # forward: high word = bases 0 .. hi_n-1, low word = the last lo_n bases
    f_hi = pack(c, 0, hi_n, False)
    f_lo = pack(c, hi_n, lo_n, False)
    # reverse complement: base K-1-i complemented at position i
    r_hi = pack(comp, lo_n, hi_n, True)
    r_lo = pack(comp, 0, lo_n, True)
    take_r = (r_hi < f_hi) | ((r_hi == f_hi) & (r_lo < f_lo))
    hi = np.where(take_r, r_hi, f_hi)[ok]
    lo = np.where(take_r, r_lo, f_lo)[ok]
    if K <= 32:
        keys, counts = np.unique(lo, return_counts=True)
        return keys, counts
    order = np.lexsort((lo, hi))
    hi, lo = hi[order], lo[order]
    first = np.ones(len(lo), bool)
    first[1:] = (hi[1:] != hi[:-1]) | (lo[1:] != lo[:-1])
    at = np.flatnonzero(first)
    counts = np.diff(np.append(at, len(lo)))
    return np.stack([lo[at], hi[at]], axis=1), counts


def _rows(keys: np.ndarray) -> np.ndarray:
    """Keys as one comparable value per key (bytes of both words)."""
    k = np.ascontiguousarray(keys)
    return k.view(np.dtype((np.void, 8 * (k.shape[1] if k.ndim == 2 else 1)))).reshape(-1)


def run(n_reads: int, Ks: list[int]) -> None:
    import torch
    w = readsim.scaled("single", n_reads)
    bases, offsets = w.generate()
    d_bases = torch.from_numpy(bases).cuda()
    d_offsets = torch.from_numpy(offsets.view(np.int64)).cuda()
    torch.cuda.synchronize()
    for K in Ks:
        windows = int(np.maximum(np.diff(offsets.astype(np.int64)) - K + 1, 0).sum())
        # Eq. 1 with n = half the K-mer total reproduces the paper's sizes
        n_half = max(1, windows // 2)
        base_dims = kmerco_paper_dims(n_half, 0.001)
        keys, counts = exact_counts(bases, offsets, K)
        exact = _rows(keys[counts > TAU])

        def line(kind, alpha, dims, scale=None):
            bf, st = _count(d_bases, d_offsets, K, alpha, dims)
            got = _rows(bf.trusted())
            bf.close()
            out = {"sweep": kind, "K": K, "alpha": alpha, "dims": list(dims),
                   "countbf_mib": dims[0] * dims[1] * 8 / 2 ** 20,
                   "kmers": st["inserted"], "insert_ms": st["insert_ms"],
                   "kmers_per_s": st["inserted"] / (st["insert_ms"] / 1000.0),
                   "distinct": st["distinct"], "trustworthy": st["trustworthy"],
                   "erroneous": st["erroneous"], "saturated_counters": st["saturated_counters"],
                   "exact_trustworthy": len(exact),
                   "misclassified": len(np.setxor1d(got, exact, assume_unique=True))}
            if scale is not None:
                out["size_factor"] = scale
            print(json.dumps(out), flush=True)

        for alpha in (5, 6, 7, 8, 9, 10, 12, 14, 16):
            line("counter_length", alpha, base_dims)
        for scale in (0.125, 0.25, 0.5, 1.0, 2.0):
            line("countbf_size", 8, kmerco_paper_dims(max(1, int(n_half * scale)), 0.001), scale)


def main(argv=None) -> None:
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--reads", type=int, default=1_000_000)
    ap.add_argument("--K", type=int, nargs="+", default=[28, 55])
    a = ap.parse_args(argv)
    run(a.reads, a.K)


if __name__ == "__main__":
    main()
