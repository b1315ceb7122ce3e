"""Continuous-batching counting service over the countBF library.

Counting jobs (one read set each, with its own countBF parameters) arrive
over time.  A job waiting in the queue is admitted as soon as a slot is free
and its device-memory bound fits the HBM budget; jobs that do not fit wait
while smaller ones behind them may go first.  The bound is the library's own
(kmerco_estimate_bytes: the most a handle holds after inserting and
classifying that job's reads), and every handle is created with it as its
hbm_budget, so the library itself refuses to allocate past it.  Every
admitted job runs on its own handle and CUDA stream, so jobs admitted while
others are on the GPU overlap there.  When a job finishes its memory is
released and waiting jobs are admitted.  Handles are pooled by geometry and
reset between jobs; a pooled handle takes only jobs no larger than the one it
was sized for (reads, bases and windows), so it never grows past its budget.

All device work runs in the C library; this module only schedules.  Each
job's result depends on its own reads and parameters alone, so it is the
same whether the job runs alone or mixed with others.
"""
from __future__ import annotations

import collections
import concurrent.futures as cf
import threading
import time
from dataclasses import dataclass, field

import numpy as np

from . import CountBF, kmerco_estimate_bytes


@dataclass(eq=False)
class Job:
    bases: object            # host uint8 array / pinned tensor of all reads
    offsets: object          # host uint64 offsets (nreads + 1)
    K: int
    m: int
    counter_bits: int = 4
    nhash: int = 4
    tau: int = 3
    name: str = ""
    keep_lists: bool = False  # return the trustworthy / erroneous key lists
    windows: int = 0          # filled in by the server

    def sizes(self) -> tuple[int, int, int]:
        """(reads, bases, windows) of the job: what its buffers are sized by."""
        o = np.asarray(self.offsets)
        nreads = max(len(o) - 1, 0)
        nbytes = int(o[-1]) - int(o[0]) if nreads else 0
        return nreads, nbytes, self.windows


@dataclass
class JobResult:
    name: str
    inserted: int
    distinct: int
    trustworthy: int
    erroneous: int
    counters_digest: str      # kmerco_digest of the job's countBF (computed on the device)
    trusted: np.ndarray | None
    erroneous_keys: np.ndarray | None
    submitted: float
    admitted: float
    finished: float
    device_bytes: int = 0     # device memory the job's handle held at the end
    reserved: int = 0         # device memory the server reserved for the job

    @property
    def latency(self) -> float:
        return self.finished - self.submitted


def window_count(offsets, K: int) -> int:
    o = np.asarray(offsets, dtype=np.int64)
    return int(np.maximum(np.diff(o) - K + 1, 0).sum()) if len(o) > 1 else 0


def _is_host(x) -> bool:
    return not (hasattr(x, "is_cuda") and x.is_cuda)


def estimate_bytes(job: Job) -> int:
    """Device bytes a handle for this job holds at most: the library's own
    count (kmerco_estimate_bytes) of the countBF, the distinct set and list
    for every window being distinct, the increment-code and classification
    buffers, and the staged reads."""
    nreads, nbytes, windows = job.sizes()
    return kmerco_estimate_bytes(job.K, job.m, job.counter_bits, job.nhash, job.tau, nreads,
                                 nbytes, windows, _is_host(job.bases))


@dataclass
class _Pooled:
    handle: object
    sized: tuple          # (reads, bases, windows) of the job it was sized for
    budget: int           # its hbm_budget: the most it can ever hold
    held: int = 0         # device bytes it holds now

    def takes(self, sizes: tuple) -> bool:
        return all(a <= b for a, b in zip(sizes, self.sized))


class Server:
    """Continuous-batching service: `slots` jobs at most on the GPU at once,
    the device memory they can hold at most `hbm_budget` bytes."""

    def __init__(self, hbm_budget: int = 120 << 30, slots: int = 8, make_handle=None):
        """``make_handle(job, budget)`` creates a countBF handle for a job that
        may hold at most ``budget`` device bytes; by default a
        :class:`CountBF` with the job's parameters and that hbm_budget."""
        self.budget = int(hbm_budget)
        self.slots = int(slots)
        self._make = make_handle or (lambda job, budget: CountBF(
            job.K, job.m, job.counter_bits, job.nhash, job.tau, hbm_budget=budget))
        self._cv = threading.Condition()
        self._pending: collections.deque = collections.deque()
        self._in_use = 0          # reserved by running jobs
        self._running = 0
        self._pool: dict = collections.defaultdict(list)   # geometry -> idle _Pooled
        self._idle_bytes = 0      # held by idle pooled handles
        self._closed = False
        self.max_running = 0
        self.max_in_use = 0
        self._t0 = time.perf_counter()
        self._threads = [threading.Thread(target=self._worker, daemon=True)
                         for _ in range(self.slots)]
        for t in self._threads:
            t.start()

    def now(self) -> float:
        return time.perf_counter() - self._t0

    # ------------------------------------------------------------ interface
    def submit(self, job: Job) -> cf.Future:
        job.windows = window_count(job.offsets, job.K)
        need = estimate_bytes(job)
        if need > self.budget:
            raise ValueError(f"job {job.name!r} needs {need} bytes, over the budget")
        fut: cf.Future = cf.Future()
        with self._cv:
            if self._closed:
                raise RuntimeError("server is closed")
            self._pending.append((job, need, fut, self.now()))
            self._cv.notify_all()
        return fut

    def close(self) -> None:
        with self._cv:
            self._closed = True
            self._cv.notify_all()
        for t in self._threads:
            t.join()
        for handles in self._pool.values():
            for p in handles:
                p.handle.close()
        self._pool.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ------------------------------------------------------------- internal
    @staticmethod
    def _key(job: Job) -> tuple:
        return (job.K, job.m, job.counter_bits, job.nhash, job.tau)

    def _take_admissible(self):
        """First pending job that fits next to the running ones (caller holds
        the lock), with the pooled handle it will run on (or None).  A job on
        a pooled handle reserves that handle's budget, else its own bound.
        Idle pooled handles are released to make room; jobs cancelled while
        waiting are dropped."""
        if any(it[2].cancelled() for it in self._pending):
            self._pending = collections.deque(it for it in self._pending if not it[2].cancelled())
        for idx, (job, need, fut, t_sub) in enumerate(self._pending):
            sizes = job.sizes()
            cands = [p for p in self._pool[self._key(job)] if p.takes(sizes)]
            pooled = min(cands, key=lambda p: p.budget) if cands else None
            reserve = pooled.budget if pooled else need
            if self._in_use + reserve > self.budget:
                continue
            if pooled:
                self._pool[self._key(job)].remove(pooled)
                self._idle_bytes -= pooled.held
            while self._in_use + self._idle_bytes + reserve > self.budget and self._idle_bytes:
                self._evict_one()
            del self._pending[idx]
            return job, reserve, fut, t_sub, pooled
        return None

    def _evict_one(self) -> None:
        for key, handles in self._pool.items():
            if handles:
                p = handles.pop()
                self._idle_bytes -= p.held
                p.handle.close()
                return

    def _worker(self) -> None:
        while True:
            with self._cv:
                item = None
                while True:
                    if self._pending:
                        item = self._take_admissible()
                    if item is not None or (self._closed and not self._pending):
                        break
                    self._cv.wait()
                if item is None:
                    return
                job, reserve, fut, t_sub, pooled = item
                self._in_use += reserve
                self._running += 1
                self.max_running = max(self.max_running, self._running)
                self.max_in_use = max(self.max_in_use, self._in_use)
            key = self._key(job)
            t_adm = self.now()
            if not fut.set_running_or_notify_cancel():   # cancelled meanwhile
                with self._cv:
                    self._in_use -= reserve
                    self._running -= 1
                    if pooled is not None:
                        self._pool[key].append(pooled)
                        self._idle_bytes += pooled.held
                    self._cv.notify_all()
                continue
            try:
                if pooled is None:
                    pooled = _Pooled(self._make(job, reserve), job.sizes(), reserve)
                res = self._run(job, pooled.handle, t_sub, t_adm)
                res.reserved = reserve
                fut.set_result(res)
            except BaseException as e:   # the job fails, the server goes on
                fut.set_exception(e)
                if pooled is not None:
                    pooled.handle.close()
                    pooled = None
            with self._cv:
                self._in_use -= reserve
                self._running -= 1
                if pooled is not None:
                    pooled.held = pooled.handle.stats()["device_bytes"]
                    self._pool[key].append(pooled)
                    self._idle_bytes += pooled.held
                self._cv.notify_all()

    def _run(self, job: Job, h: CountBF, t_sub: float, t_adm: float) -> JobResult:
        h.reset()
        h.insert(job.bases, job.offsets)
        h.classify()
        st = h.stats()
        digest = h.digest()
        tr = h.trusted() if job.keep_lists else None
        er = h.erroneous() if job.keep_lists else None
        return JobResult(job.name, st["inserted"], st["distinct"], st["trustworthy"],
                         st["erroneous"], digest, tr, er, t_sub, t_adm, self.now(),
                         device_bytes=st["device_bytes"])


def replay(server: Server, jobs: list[Job], arrivals: list[float]) -> list[JobResult]:
    """Submit each job at its arrival time (seconds from now) and wait for all."""
    t0 = time.perf_counter()
    futs = []
    for job, t in sorted(zip(jobs, arrivals), key=lambda x: x[1]):
        delay = t - (time.perf_counter() - t0)
        if delay > 0:
            time.sleep(delay)
        futs.append(server.submit(job))
    return [f.result() for f in futs]
