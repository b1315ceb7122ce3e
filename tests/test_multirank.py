"""Multi-rank host logic on CPU with gloo (world size 2).

1. The benchmark's rank logic: every rank times its own sample; the job's
   time is the slowest rank's and the rate counts all ranks' K-mers.
2. Sharding one sample across ranks and merging the countBFs with the
   counter-wise saturating add gives exactly the countBF of the whole sample
   (the exchange step a sharded single-sample count needs).
3. The sharded count itself (paper_2305_07545_gb300.shard.count_sharded):
   read shards, the chunked countBF exchange and the key-range routing of the
   distinct keys, over gloo with 2 and 3 ranks.
The per-rank counting here is the oracle, since no GPU is present; the
exchange, the routing and the merge rule are what is under test.
"""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _init(rank, world, port):
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)


def _bench_logic(rank, world, port, q):
    _init(rank, world, port)
    import bench
    slowest = bench.max_over_ranks([0.25, 0.40][rank], "cpu")
    rate = bench.whole_job_rate(1000, 10, world, slowest)
    q.put((rank, slowest, rate))
    dist.destroy_process_group()


def _sharded_merge(rank, world, port, q):
    _init(rank, world, port)
    import oracle
    import readsim
    w = readsim.WORKLOADS["tiny"]
    bases, offsets = readsim.scaled("tiny", 600, seed_offset=21).generate()
    nreads = len(offsets) - 1
    cut = [0, nreads // 3, nreads]          # uneven shards
    r0, r1 = cut[rank], cut[rank + 1]
    b = bases[int(offsets[r0]):int(offsets[r1])]
    o = offsets[r0:r1 + 1] - offsets[r0]
    ex = oracle.extract(b, o, w.K)
    local = oracle.insert_sequential(ex.hi, ex.lo, w.K, w.m, w.alpha, w.nhash)
    parts = [torch.zeros(len(local), dtype=torch.int64) for _ in range(world)]
    dist.all_gather(parts, torch.from_numpy(local.view(np.int64)))
    if rank == 0:
        merged = parts[0].numpy().view(np.uint64).copy()
        for p in parts[1:]:
            oracle.merge(merged, p.numpy().view(np.uint64), w.m, w.alpha)
        exw = oracle.extract(bases, offsets, w.K)
        whole = oracle.insert_sequential(exw.hi, exw.lo, w.K, w.m, w.alpha, w.nhash)
        q.put(bool(np.array_equal(merged, whole)) and bool(whole.any()))
    dist.destroy_process_group()


class OracleEngine:
    """The engine interface of paper_2305_07545_gb300.shard with the oracle
    doing each rank's counting on the host (CPU torch tensors), so that the
    sharding, the chunked countBF exchange and the key-range routing run
    under gloo without a GPU."""

    def __init__(self, K, m, alpha, nhash, tau):
        import oracle
        self.o = oracle
        self.K, self.m, self.alpha, self.nhash, self.tau = K, m, alpha, nhash, tau
        self.kw = 1 if K <= 32 else 2
        self.words = oracle.words(m, alpha)
        self.filt = np.zeros(self.words, np.uint64)
        self.hi = np.zeros(0, np.uint64)
        self.lo = np.zeros(0, np.uint64)
        self.n_windows = self.n_inserted = 0

    def insert(self, bases, offsets):
        b = bases.numpy().view(np.uint8)
        o = offsets.numpy().view(np.uint64)
        ex = self.o.extract(b, o, self.K)
        self.o.insert_sequential(ex.hi, ex.lo, self.K, self.m, self.alpha, self.nhash, self.filt)
        self.hi = np.concatenate([self.hi, ex.hi])
        self.lo = np.concatenate([self.lo, ex.lo])
        self.n_windows += ex.n_windows
        self.n_inserted += ex.n

    def _rows(self, hi, lo):
        return lo.copy() if self.kw == 1 else np.stack([lo, hi], axis=1)

    def sorted_keys(self):
        dhi, dlo, _ = self.o.distinct(self.hi, self.lo)
        self._sorted = [(int(h) << 64) | int(l) for h, l in zip(dhi, dlo)]
        return self.from_host(self._rows(dhi, dlo))

    def cells(self):
        return torch.from_numpy(self.filt.view(np.int64).copy())

    def merge_cells(self, first, words_tensor):
        src = np.zeros(self.words, np.uint64)
        w = words_tensor.numpy().view(np.uint64)
        src[first:first + len(w)] = w
        self.o.merge(self.filt, src, self.m, self.alpha)

    def rank_of(self, probes):
        import bisect
        rows = probes.reshape(-1) if self.kw == 1 else probes
        vals = [int(r) if self.kw == 1 else (int(r[1]) << 64) | int(r[0]) for r in rows]
        return np.array([bisect.bisect_left(self._sorted, v) for v in vals], np.uint64)

    def own(self, merged_cells, keys_words):
        k = keys_words.numpy().view(np.uint64)
        if self.kw == 1:
            hi, lo = np.zeros(len(k), np.uint64), k.copy()
        else:
            lo, hi = k[0::2].copy(), k[1::2].copy()
        dhi, dlo, _ = self.o.distinct(hi, lo)   # the owner's distinct set drops duplicates
        filt = merged_cells.numpy().view(np.uint64)
        est, tr = self.o.classify(filt, dhi, dlo, self.K, self.m, self.alpha, self.nhash, self.tau)
        return _OwnerResult(self._rows(dhi, dlo), tr, filt.copy())

    def to_host(self, t):
        a = t.numpy().view(np.uint64)
        return a if self.kw == 1 else a.reshape(-1, 2)

    def from_host(self, a):
        a = np.ascontiguousarray(a)
        if a.dtype != np.uint8:
            a = a.view(np.int64).reshape(-1)
        return torch.from_numpy(a.copy())

    def stats(self):
        return dict(windows=self.n_windows, inserted=self.n_inserted)


class _OwnerResult:
    def __init__(self, keys, trusted_mask, cells):
        self.keys, self.mask, self.cells = keys, trusted_mask, cells

    def stats(self):
        return dict(distinct=len(self.keys), trustworthy=int(self.mask.sum()))

    def trusted(self):
        return self.keys[self.mask]

    def erroneous(self):
        return self.keys[~self.mask]


def _sharded_exchange(rank, world, port, q):
    _init(rank, world, port)
    import oracle
    import readsim
    from paper_2305_07545_gb300 import shard
    out = []
    for K, m in ((21, 1 << 14), (40, 1 << 16)):
        bases, offsets = readsim.scaled("tiny", 700, seed_offset=31 + K).generate()
        eng = OracleEngine(K, m, 4, 3, 2)
        res = shard.count_sharded(eng, shard.TorchComm(), bases, offsets, samples_per_rank=64)
        lists = [None] * world
        dist.all_gather_object(lists, (res.owner.trusted(), res.owner.erroneous(),
                                       res.owner.cells))
        if rank == 0:
            tr = np.concatenate([x[0] for x in lists])
            er = np.concatenate([x[1] for x in lists])
            ref = oracle.run(bases, offsets, K, m, 4, 3, 2)
            rows = (lambda h, l: l) if K <= 32 else (lambda h, l: np.stack([l, h], axis=1))
            want_tr = rows(ref.distinct_hi[ref.trusted_mask], ref.distinct_lo[ref.trusted_mask])
            want_er = rows(ref.distinct_hi[~ref.trusted_mask], ref.distinct_lo[~ref.trusted_mask])
            out.append(bool(np.array_equal(tr, want_tr)) and bool(np.array_equal(er, want_er))
                       and all(np.array_equal(x[2], ref.filter) for x in lists)
                       and res.distinct == len(ref.distinct_lo)
                       and res.inserted == ref.n_inserted and res.windows == ref.n_windows
                       and len(want_tr) > 0 and len(want_er) > 0)
    if rank == 0:
        q.put(out)
    dist.destroy_process_group()


def _run(fn, world=2):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=fn, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    out = []
    while not q.empty():
        out.append(q.get())
    return out


def test_bench_rank_logic_gloo():
    out = sorted(_run(_bench_logic))
    assert [r for r, _, _ in out] == [0, 1]
    for _, slowest, rate in out:
        assert slowest == 0.40                       # max over ranks
        assert rate == pytest.approx(1000 * 10 * 2 / 0.40)


def test_sharded_count_merges_to_whole_gloo():
    assert _run(_sharded_merge) == [True]


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_count_exchange_gloo(world):
    # the whole sharded count of paper_2305_07545_gb300.shard (read shards,
    # chunked saturating countBF exchange, key ranges routed to their owners)
    # over gloo, each rank counting with the oracle: the owners' lists in rank
    # order are the whole sample's, and every rank holds the whole countBF
    assert _run(_sharded_exchange, world) == [[True, True]]
