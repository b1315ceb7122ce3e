"""Sharded count of one sample over P ranks (one GPU each, or P handles on
one GPU).

Reads are independent, so a sample's reads are split into P shards of about
equal bases and every rank inserts its shard into a full-size countBF of its
own.  Two exchange steps then give exactly the single-GPU result:

1. countBF: the cells are cut into P equal chunks; rank r owns chunk r.
   Every rank sends chunk j to rank j (all-to-all), the owner merges the P
   copies counter by counter with min(a + b, 2^alpha - 1) (kmerco_merge_cells),
   and the merged chunks are gathered back to every rank (all-gather).  The
   merge is exact because saturating increments commute (Algorithm 3, read per
   counter): min(min(a, M) + min(b, M), M) = min(a + b, M).  A plain sum
   collective cannot do this: it would carry one counter into the next.
2. distinct keys: each rank sorts its own distinct keys (kmerco_classify),
   draws evenly spaced samples, and all ranks agree on P - 1 splitters from
   the gathered samples.  Key range j goes to rank j (all-to-all; the cut
   points come from kmerco_rank_of).  The owner puts the merged countBF and
   the keys it received into a handle (kmerco_set_counters,
   kmerco_add_distinct, which drops duplicates) and classifies them
   (Algorithm 2 with Algorithm 5).  Owner j's ascending lists cover key range
   j, so the lists of ranks 0 .. P-1 in order are the sample's ascending
   trustworthy and erroneous lists.

The collectives go through a ``comm`` object (``TorchComm`` over
torch.distributed, or ``LocalComm`` for P threads of one process), and the
per-rank counting through an ``engine`` (``LibraryEngine``: the CUDA
library), so that the exchange logic is the same for every transport.
"""
from __future__ import annotations

import threading
from dataclasses import dataclass

import numpy as np

from . import (CountBF, kmerco_add_distinct, kmerco_get_counters, kmerco_get_distinct,
               kmerco_get_erroneous, kmerco_get_trusted, kmerco_merge_cells, kmerco_rank_of,
               kmerco_set_counters)


# ---------------------------------------------------------------- host logic
def shard_bounds(offsets, world: int) -> list[int]:
    """Read indices r_0 = 0 <= r_1 <= ... <= r_P = nreads cutting the reads
    into P shards of about equal bases (shard j = reads [r_j, r_{j+1}))."""
    o = np.asarray(offsets, dtype=np.uint64)
    nreads = len(o) - 1
    first, last = int(o[0]), int(o[-1])
    targets = [first + (last - first) * j // world for j in range(1, world)]
    cuts = np.searchsorted(o[:nreads + 1], np.asarray(targets, np.uint64), side="left")
    return [0] + [int(min(c, nreads)) for c in cuts] + [nreads]


def chunk_bounds(words: int, world: int) -> list[int]:
    """Cells w_0 = 0 <= ... <= w_P = words: rank j owns cells [w_j, w_{j+1})."""
    return [words * j // world for j in range(world + 1)]


def sample_keys(keys: np.ndarray, count: int) -> np.ndarray:
    """`count` evenly spaced keys of an ascending key array (rows of kw words)."""
    n = len(keys)
    if n == 0 or count <= 0:
        return keys[:0]
    idx = (np.arange(count, dtype=np.int64) * n) // count
    return keys[idx]


def _as_int(row: np.ndarray, kw: int) -> int:
    return int(row) if kw == 1 else (int(row[1]) << 64) | int(row[0])


def splitters(samples: list[np.ndarray], world: int, kw: int) -> np.ndarray:
    """P - 1 splitter keys from every rank's samples: the samples of all
    ranks sorted, taken at P - 1 evenly spaced places (rows of kw words)."""
    allk = [s for s in samples if len(s)]
    if world <= 1:
        return np.zeros((0,) if kw == 1 else (0, 2), np.uint64)
    if not allk:
        pool = np.zeros((0,) if kw == 1 else (0, 2), np.uint64)
    else:
        pool = np.concatenate(allk)
    vals = sorted(set(_as_int(r, kw) for r in pool))
    out = []
    for j in range(1, world):
        out.append(vals[len(vals) * j // world] if vals else (1 << (64 * kw)) - 1)
    arr = np.zeros((world - 1,) if kw == 1 else (world - 1, 2), np.uint64)
    for i, v in enumerate(out):
        if kw == 1:
            arr[i] = v
        else:
            arr[i, 0], arr[i, 1] = v & ((1 << 64) - 1), v >> 64
    return arr


def split_sizes(cut_ranks: np.ndarray, n: int) -> list[int]:
    """Keys per destination from the ranks of the P - 1 splitters in the
    sender's ascending keys: range j is [cut_{j-1}, cut_j)."""
    c = [0] + [int(x) for x in cut_ranks] + [n]
    return [c[j + 1] - c[j] for j in range(len(c) - 1)]


# ------------------------------------------------------------------ comms
class TorchComm:
    """Collectives over torch.distributed (NCCL for CUDA tensors, gloo for
    CPU tensors)."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)

    def gather_obj(self, obj):
        out = [None] * self.world
        self.dist.all_gather_object(out, obj, group=self.group)
        return out

    def all_to_all(self, parts: list):
        """parts[j] goes to rank j; returns what every rank sent here.  NCCL
        takes one all-to-all; gloo has none, so there the parts travel as
        point-to-point pairs."""
        import torch
        dist = self.dist
        sizes = self.gather_obj([int(p.numel()) for p in parts])
        outs = [torch.empty(sizes[j][self.rank], dtype=parts[0].dtype, device=parts[0].device)
                for j in range(self.world)]
        ins = [p.contiguous() for p in parts]
        if dist.get_backend(self.group) == "nccl":
            dist.all_to_all(outs, ins, group=self.group)
            return outs
        ops = []
        for j in range(self.world):
            if j == self.rank:
                outs[j].copy_(ins[j])
                continue
            if ins[j].numel():
                ops.append(dist.P2POp(dist.isend, ins[j], j, self.group))
            if outs[j].numel():
                ops.append(dist.P2POp(dist.irecv, outs[j], j, self.group))
        if ops:
            for w in dist.batch_isend_irecv(ops):
                w.wait()
        return outs

    def all_gather(self, t):
        import torch
        sizes = self.gather_obj(int(t.numel()))
        m = max(sizes)
        buf = torch.zeros(m, dtype=t.dtype, device=t.device)
        buf[: t.numel()] = t.reshape(-1)
        outs = [torch.empty(m, dtype=t.dtype, device=t.device) for _ in range(self.world)]
        self.dist.all_gather(outs, buf, group=self.group)
        return [o[: sizes[j]] for j, o in enumerate(outs)]


class LocalComm:
    """Collectives among `world` threads of one process (ranks that share a
    GPU or run on the host): each collective is a barrier-separated exchange
    through shared slots."""

    def __init__(self, world: int):
        self.world = world
        self._barrier = threading.Barrier(world)
        self._slots = [None] * world

    def view(self, rank: int) -> "_LocalRank":
        return _LocalRank(self, rank)


class _LocalRank:
    def __init__(self, hub: LocalComm, rank: int):
        self.hub, self.rank, self.world = hub, rank, hub.world

    def _swap(self, obj):
        h = self.hub
        h._barrier.wait()
        h._slots[self.rank] = obj
        h._barrier.wait()
        out = list(h._slots)
        h._barrier.wait()
        return out

    def gather_obj(self, obj):
        return self._swap(obj)

    def all_to_all(self, parts: list):
        got = self._swap(list(parts))
        return [got[j][self.rank] for j in range(self.world)]

    def all_gather(self, t):
        return self._swap(t)


# ----------------------------------------------------------------- engines
class LibraryEngine:
    """A rank's counting on the CUDA library: device tensors in and out."""

    def __init__(self, K: int, m: int, counter_bits: int, nhash: int, tau: int, device: int = 0,
                 **handle_options):
        import torch
        self.torch = torch
        self.params = dict(k=K, m=m, counter_bits=counter_bits, nhash=nhash, threshold=tau)
        self.device = device
        self.kw = 1 if K <= 32 else 2
        self.opts = handle_options
        self.stream = torch.cuda.Stream(device=device)
        self.local = CountBF(K, m, counter_bits, nhash, tau, device=device,
                             stream=self.stream.cuda_stream, **handle_options)
        self.words = self.local.stats()["words"]

    def _sync(self):
        self.torch.cuda.synchronize(self.device)

    def insert(self, bases, offsets):
        self._sync()   # inputs written on torch's streams
        self.local.insert(bases, offsets)

    def sorted_keys(self):
        """The rank's distinct keys, ascending, as a device int64 tensor of
        n * kw words."""
        self.local.classify()
        n = kmerco_get_distinct(self.local.h)
        t = self.torch.empty(max(n, 1) * self.kw, dtype=self.torch.int64, device=self.device)
        self._sync()
        kmerco_get_distinct(self.local.h, t, None, n)
        return t[: n * self.kw]

    def cells(self):
        t = self.torch.empty(self.words, dtype=self.torch.int64, device=self.device)
        self._sync()
        kmerco_get_counters(self.local.h, t, self.words)
        return t

    def merge_cells(self, first: int, words_tensor):
        self._sync()
        kmerco_merge_cells(self.local.h, words_tensor, first, int(words_tensor.numel()))

    def rank_of(self, probes: np.ndarray) -> np.ndarray:
        n = len(probes)
        out = np.zeros(max(n, 1), np.uint64)
        if n:
            kmerco_rank_of(self.local.h, np.ascontiguousarray(probes, np.uint64), n, out)
        return out[:n]

    def own(self, merged_cells, keys_words):
        """Owner step: the merged countBF and the keys of the owned range in a
        new handle, classified.  Returns that handle."""
        p = self.params
        bf = CountBF(p["k"], p["m"], p["counter_bits"], p["nhash"], p["threshold"],
                     device=self.device, stream=self.stream.cuda_stream, **self.opts)
        self._sync()
        kmerco_set_counters(bf.h, merged_cells, self.words)
        n = int(keys_words.numel()) // self.kw
        if n:
            kmerco_add_distinct(bf.h, keys_words, n)
        bf.classify()
        return bf

    def to_host(self, t) -> np.ndarray:
        a = t.cpu().numpy().view(np.uint64)
        return a if self.kw == 1 else a.reshape(-1, 2)

    def from_host(self, a: np.ndarray):
        """Host words (uint64 rows) or bytes (uint8) as a device tensor."""
        a = np.ascontiguousarray(a)
        if a.dtype != np.uint8:
            a = a.view(np.int64).reshape(-1)
        return self.torch.from_numpy(a).to(self.device)

    def stats(self) -> dict:
        return self.local.stats()

    def close(self):
        self.local.close()


@dataclass
class ShardResult:
    rank: int
    owner: object                 # the rank's classified owner handle (CountBF)
    key_range: tuple              # (first splitter or None, last splitter or None)
    windows: int                  # totals over all ranks
    inserted: int
    distinct: int
    trustworthy: int


def shard_of(bases, offsets, rank: int, world: int):
    """This rank's reads (host arrays): the bases and offsets of shard `rank`."""
    rb = shard_bounds(offsets, world)
    r0, r1 = rb[rank], rb[rank + 1]
    o = np.asarray(offsets, np.uint64)
    lo_b, hi_b = int(o[r0]), int(o[r1])
    return (np.ascontiguousarray(np.asarray(bases)[lo_b:hi_b]),
            (o[r0:r1 + 1] - o[r0]).astype(np.uint64))


def count_sharded(engine, comm, bases=None, offsets=None, samples_per_rank: int = 4096,
                  shard=None) -> ShardResult:
    """One rank's part of a sharded count of the whole sample (host bases,
    offsets), or of the rank's shard already on the device (shard = (bases,
    offsets) tensors, as shard_of cuts it): it inserts its shard, takes part
    in both exchanges and returns its owner handle, classified over its key
    range."""
    rank, world = comm.rank, comm.world
    kw = engine.kw
    # 1. insert this rank's shard of the reads
    if shard is None:
        sb, so = shard_of(bases, offsets, rank, world)
        if len(so) > 1 and len(sb):
            engine.insert(engine.from_host(sb), engine.from_host(so))
    elif shard[1].numel() > 1 and shard[0].numel():
        engine.insert(shard[0], shard[1])
    # 2. countBF exchange: chunk j to rank j, saturating merge, gather back
    cb = chunk_bounds(engine.words, world)
    cells = engine.cells()
    parts = [cells[cb[j]:cb[j + 1]] for j in range(world)]
    got = comm.all_to_all(parts)
    for j in range(world):
        if j != rank and got[j].numel():
            engine.merge_cells(cb[rank], got[j])
    mine = engine.cells()[cb[rank]:cb[rank + 1]]
    merged = comm.all_gather(mine)
    import torch
    merged_cells = torch.cat([m.to(cells.device) for m in merged])
    # 3. distinct keys: local sort, splitters from samples, route key ranges
    keys = engine.sorted_keys()
    host_keys_sample = sample_keys(engine.to_host(keys), samples_per_rank)
    spl = splitters(comm.gather_obj(host_keys_sample), world, kw)
    n_local = int(keys.numel()) // kw
    cuts = engine.rank_of(spl)
    sizes = split_sizes(cuts, n_local)
    starts = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    send = [keys[starts[j] * kw:starts[j + 1] * kw] for j in range(world)]
    recv = comm.all_to_all(send)
    owned = torch.cat([r.to(keys.device) for r in recv]) if recv else keys[:0]
    # 4. the owner classifies its range against the merged countBF
    owner = engine.own(merged_cells, owned)
    st_local = engine.stats()
    st_own = owner.stats()
    totals = comm.gather_obj((st_local["windows"], st_local["inserted"], st_own["distinct"],
                              st_own["trustworthy"]))
    rng = (None if rank == 0 else spl[rank - 1], None if rank == world - 1 else spl[rank])
    return ShardResult(rank, owner, rng, sum(t[0] for t in totals), sum(t[1] for t in totals),
                       sum(t[2] for t in totals), sum(t[3] for t in totals))


def trusted_of(res: ShardResult) -> np.ndarray:
    return res.owner.trusted()


def erroneous_of(res: ShardResult) -> np.ndarray:
    return res.owner.erroneous()
