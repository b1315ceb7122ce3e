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
distinct K-mers are classified differently than by a countBF 64x larger
(taken as exact: at that size collisions are negligible).

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


def _trusted_set(bf):
    t = bf.trusted()
    return set(map(bytes, t.reshape(len(t), -1))) if len(t) else set()


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
        # reference: 64x the cells, 16-bit counters
        ref, _ = _count(d_bases, d_offsets, K, 16, None, m=base_dims[0] * base_dims[1] * 4 * 64)
        exact = _trusted_set(ref)
        ref.close()

        def line(kind, alpha, dims, scale=None):
            bf, st = _count(d_bases, d_offsets, K, alpha, dims)
            got = _trusted_set(bf)
            bf.close()
            out = {"sweep": kind, "K": K, "alpha": alpha, "dims": list(dims),
                   "countbf_mib": dims[0] * dims[1] * 8 / 2 ** 20,
                   "kmers": st["inserted"], "insert_ms": st["insert_ms"],
                   "kmers_per_s": st["inserted"] / (st["insert_ms"] / 1000.0),
                   "distinct": st["distinct"], "trustworthy": st["trustworthy"],
                   "erroneous": st["erroneous"], "saturated_counters": st["saturated_counters"],
                   "misclassified_vs_large_filter": len(got ^ exact)}
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
