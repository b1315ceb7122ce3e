"""Multi-rank host logic on CPU with gloo (world size 2).

1. The benchmark's rank logic: every rank times its own sample; the job's
   time is the slowest rank's and the rate counts all ranks' K-mers.
2. Sharding one sample across ranks and merging the countBFs with the
   counter-wise saturating add gives exactly the countBF of the whole sample
   (the exchange step a sharded single-sample count needs).  The per-rank
   counting here is the oracle, since no GPU is present; the exchange and the
   merge rule are what is under test.
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
