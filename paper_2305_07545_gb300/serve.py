"""Continuous-batching counting service over the countBF library.

Counting jobs (one read set each, with its own countBF parameters) arrive
over time.  A job waiting in the queue is admitted as soon as a slot is free
and its worst-case device-memory estimate fits the HBM budget; jobs that do
not fit wait while smaller ones behind them may go first.  Every admitted
job runs on its own handle and CUDA stream, so jobs admitted while others
are on the GPU overlap there.  When a job finishes its memory is released
and waiting jobs are admitted.  Handles are pooled by geometry and reset
between jobs, so a busy server does not allocate per job.

All device work runs in the C library; this module only schedules.  Each
job's result depends on its own reads and parameters alone, so it is the
same whether the job runs alone or mixed with others.
"""
from __future__ import annotations

import collections
import concurrent.futures as cf
import hashlib
import threading
import time
from dataclasses import dataclass, field

import numpy as np

from . import CountBF


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


@dataclass
class JobResult:
    name: str
    inserted: int
    distinct: int
    trustworthy: int
    erroneous: int
    counters_sha256: str
    trusted: np.ndarray | None
    erroneous_keys: np.ndarray | None
    submitted: float
    admitted: float
    finished: float

    @property
    def latency(self) -> float:
        return self.finished - self.submitted


def window_count(offsets, K: int) -> int:
    o = np.asarray(offsets, dtype=np.int64)
    return int(np.maximum(np.diff(o) - K + 1, 0).sum()) if len(o) > 1 else 0


def estimate_bytes(job: Job) -> int:
    """Worst-case device bytes of one job: countBF, a distinct set and list
    sized for every window being distinct, classification buffers, and the
    staged reads."""
    kw = 1 if job.K <= 32 else 2
    eta = 64 // job.counter_bits
    cells = (job.m + eta - 1) // eta * 8
    w = job.windows
    return int(cells + w * kw * (16 + 8 + 24) + w * 4 + np.asarray(job.bases).nbytes
               + np.asarray(job.offsets).nbytes + (1 << 20))


class Server:
    """Continuous-batching service: `slots` jobs at most on the GPU at once,
    their estimated device memory at most `hbm_budget` bytes."""

    def __init__(self, hbm_budget: int = 120 << 30, slots: int = 8, make_handle=None):
        """``make_handle(job)`` creates a countBF handle for a job; by default
        a :class:`CountBF` with the job's parameters."""
        self.budget = int(hbm_budget)
        self.slots = int(slots)
        self._make = make_handle or (lambda job: CountBF(job.K, job.m, job.counter_bits,
                                                         job.nhash, job.tau))
        self._cv = threading.Condition()
        self._pending: collections.deque = collections.deque()
        self._in_use = 0
        self._running = 0
        self._pool: dict = collections.defaultdict(list)   # geometry -> idle handles
        self._idle_bytes = 0
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
            for h in handles:
                h.close()
        self._pool.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ------------------------------------------------------------- internal
    def _take_admissible(self):
        """First pending job that fits next to the running ones (caller holds
        the lock).  Idle pooled handles are released to make room; jobs
        cancelled while waiting are dropped."""
        if any(it[2].cancelled() for it in self._pending):
            self._pending = collections.deque(it for it in self._pending if not it[2].cancelled())
        for idx, (job, need, fut, t_sub) in enumerate(self._pending):
            if self._in_use + need > self.budget:
                continue
            while self._in_use + self._idle_bytes + need > self.budget and self._idle_bytes:
                self._evict_one()
            del self._pending[idx]
            return job, need, fut, t_sub
        return None

    def _evict_one(self) -> None:
        for key, handles in self._pool.items():
            if handles:
                h = handles.pop()
                self._idle_bytes -= h._pool_bytes
                h.close()
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
                job, need, fut, t_sub = item
                self._in_use += need
                self._running += 1
                self.max_running = max(self.max_running, self._running)
                self.max_in_use = max(self.max_in_use, self._in_use)
                key = (job.K, job.m, job.counter_bits, job.nhash, job.tau)
                h = self._pool[key].pop() if self._pool[key] else None
                if h is not None:
                    self._idle_bytes -= h._pool_bytes
            t_adm = self.now()
            if not fut.set_running_or_notify_cancel():   # cancelled meanwhile
                with self._cv:
                    self._in_use -= need
                    self._running -= 1
                    if h is not None:
                        self._pool[key].append(h)
                        self._idle_bytes += h._pool_bytes
                    self._cv.notify_all()
                continue
            try:
                if h is None:
                    h = self._make(job)
                res = self._run(job, h, t_sub, t_adm)
                fut.set_result(res)
            except BaseException as e:   # the job fails, the server goes on
                fut.set_exception(e)
                if h is not None:
                    h.close()
                    h = None
            with self._cv:
                self._in_use -= need
                self._running -= 1
                if h is not None:
                    h._pool_bytes = h.stats()["device_bytes"]
                    self._pool[key].append(h)
                    self._idle_bytes += h._pool_bytes
                self._cv.notify_all()

    def _run(self, job: Job, h: CountBF, t_sub: float, t_adm: float) -> JobResult:
        h.reset()
        h.insert(job.bases, job.offsets)
        h.classify()
        st = h.stats()
        digest = hashlib.sha256(h.counters().tobytes()).hexdigest()
        tr = h.trusted() if job.keep_lists else None
        er = h.erroneous() if job.keep_lists else None
        return JobResult(job.name, st["inserted"], st["distinct"], st["trustworthy"],
                         st["erroneous"], digest, tr, er, t_sub, t_adm, self.now())


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
