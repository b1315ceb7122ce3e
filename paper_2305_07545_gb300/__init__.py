"""GB300 countBF K-mer counter (KmerCo, arXiv 2305.07545): Python binding.

A thin ctypes layer over ``libkmerco.so`` (the C ABI in ``include/kmerco.h``).
It only marshals arguments -- numpy arrays, torch tensors (CPU or CUDA) or
raw pointers -- into the C calls, which run every step of the method in
CUDA kernels.  There is no CPU fallback: if the library is missing and
cannot be built, :func:`load` raises.

The functions keep the C names (``kmerco_create`` ... ``kmerco_strerror``)
and raise :class:`KmercoError` on a non-zero status; :class:`CountBF` wraps a
handle with numpy results.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, byref, c_char_p, c_float, c_int, c_uint32, c_uint64, c_void_p

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libkmerco.so")

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, ESTATE, ESIZE = range(7)


# kmerco_alloc_fn / kmerco_free_fn: a handle's device allocator
ALLOC_FN = ctypes.CFUNCTYPE(c_void_p, c_void_p, ctypes.c_size_t, c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, c_void_p, c_void_p, ctypes.c_size_t, c_void_p)


class kmerco_config_t(ctypes.Structure):
    _fields_ = [("k", c_int), ("m", c_uint64), ("counter_bits", c_int), ("nhash", c_int),
                ("threshold", c_uint32), ("forward_only", c_int), ("stream", c_void_p),
                ("hbm_budget", c_uint64), ("device", c_int), ("update_mode", c_int),
                ("dim_x", c_uint64), ("dim_y", c_uint64), ("canonical_hash", c_int),
                ("whole_file", c_int), ("pass_codes", c_uint64), ("retry_limit", c_uint32),
                ("max_distinct", c_uint64), ("dev_alloc", ALLOC_FN), ("dev_free", FREE_FN),
                ("alloc_ctx", c_void_p)]


class TorchAllocator:
    """Device memory of a handle from torch's caching allocator (the
    handle's dev_alloc / dev_free callbacks), so that the library's buffers
    count in torch.cuda.memory_allocated() and come from torch's pool."""

    def __init__(self, device: int | None = None):
        import torch
        self.device = torch.cuda.current_device() if device is None else device

        def _alloc(ctx, nbytes, stream):
            try:
                return torch.cuda.caching_allocator_alloc(int(nbytes), self.device,
                                                          int(stream or 0))
            except Exception:   # out of memory: the library reports ENOMEM
                return None

        def _free(ctx, ptr, nbytes, stream):
            torch.cuda.caching_allocator_delete(ptr)

        self.alloc = ALLOC_FN(_alloc)   # kept alive with the handle
        self.free = FREE_FN(_free)


class kmerco_stats_t(ctypes.Structure):
    _fields_ = [("windows", c_uint64), ("n_skipped", c_uint64), ("inserted", c_uint64),
                ("distinct", c_uint64), ("trustworthy", c_uint64), ("erroneous", c_uint64),
                ("saturated_counters", c_uint64), ("m_actual", c_uint64), ("words", c_uint64),
                ("device_bytes", c_uint64), ("launches", c_uint64), ("dim_x", c_uint64),
                ("dim_y", c_uint64), ("k", c_int), ("counter_bits", c_int),
                ("eta", c_int), ("nhash", c_int), ("threshold", c_uint32),
                ("classified", c_int), ("insert_ms", c_float), ("classify_ms", c_float)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class kmerco_batch_info_t(ctypes.Structure):
    _fields_ = [("samples", c_int), ("chunk", c_int), ("blocks_per_sm", c_int), ("tuned", c_int),
                ("tuned_ms", c_float), ("graph", c_int), ("launches", c_uint64),
                ("total_chunks", c_uint64), ("schedule", c_int), ("streams", c_int)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class KmercoError(RuntimeError):
    def __init__(self, status: int, call: str):
        self.status = status
        super().__init__(f"{call}: {kmerco_strerror(status)} (status {status})")


_lib = None
_u64p = POINTER(c_uint64)
_u32p = POINTER(c_uint32)

# Exported symbols and their signatures (restype, argtypes).
SIGNATURES = {
    "kmerco_create": (c_int, [c_int, c_uint64, c_int, c_int, c_uint32, POINTER(c_void_p)]),
    "kmerco_create_ex": (c_int, [POINTER(kmerco_config_t), POINTER(c_void_p)]),
    "kmerco_paper_dims": (c_int, [c_uint64, ctypes.c_double, _u64p, _u64p]),
    "kmerco_destroy": (None, [c_void_p]),
    "kmerco_insert": (c_int, [c_void_p, c_void_p, c_void_p, c_uint64]),
    "kmerco_classify": (c_int, [c_void_p]),
    "kmerco_stats": (c_int, [c_void_p, POINTER(kmerco_stats_t)]),
    "kmerco_get_counters": (c_int, [c_void_p, c_void_p, c_uint64]),
    "kmerco_get_distinct": (c_int, [c_void_p, c_void_p, c_void_p, c_uint64, _u64p]),
    "kmerco_get_trusted": (c_int, [c_void_p, c_void_p, c_uint64, _u64p]),
    "kmerco_get_erroneous": (c_int, [c_void_p, c_void_p, c_uint64, _u64p]),
    "kmerco_get_lists_async": (c_int, [c_void_p, c_void_p, c_uint64, c_void_p, c_uint64, _u64p,
                                       _u64p]),
    "kmerco_sync": (c_int, [c_void_p]),
    "kmerco_digest": (c_int, [c_void_p, c_void_p]),
    "kmerco_query": (c_int, [c_void_p, c_void_p, c_uint64, c_void_p]),
    "kmerco_merge": (c_int, [c_void_p, c_void_p]),
    "kmerco_reset": (c_int, [c_void_p]),
    "kmerco_strerror": (c_char_p, [c_int]),
    "kmerco_classify_noalloc": (c_int, [c_void_p, c_uint64, c_int, c_int, c_int, c_uint32,
                                        c_void_p, c_uint64, c_void_p, c_void_p, _u64p, c_void_p]),
    "kmerco_batch_create": (c_int, [POINTER(c_void_p), c_int, POINTER(c_void_p)]),
    "kmerco_batch_destroy": (None, [c_void_p]),
    "kmerco_batch_insert": (c_int, [c_void_p, POINTER(c_void_p), POINTER(c_void_p), _u64p, c_int]),
    "kmerco_set_counters": (c_int, [c_void_p, c_void_p, c_uint64]),
    "kmerco_add_distinct": (c_int, [c_void_p, c_void_p, c_uint64]),
    "kmerco_batch_classify": (c_int, [c_void_p]),
    "kmerco_batch_schedule": (c_int, [c_void_p, c_int, c_int]),
    "kmerco_batch_info": (c_int, [c_void_p, c_void_p]),
    "kmerco_merge_cells": (c_int, [c_void_p, c_void_p, c_uint64, c_uint64]),
    "kmerco_rank_of": (c_int, [c_void_p, c_void_p, c_uint64, c_void_p]),
    "kmerco_estimate_bytes": (c_int, [POINTER(kmerco_config_t), c_uint64, c_uint64, c_uint64, c_int,
                                      _u64p]),
    "kmerco_peak_random_cas": (c_int, [c_uint64, c_uint64, c_int, POINTER(ctypes.c_double)]),
    "kmerco_peak_random_read": (c_int, [c_uint64, c_uint64, c_int, POINTER(ctypes.c_double)]),
}

NOALLOC_MAX_KEYS = 1 << 28


def load(build: bool = True) -> ctypes.CDLL:
    """Load libkmerco.so, compiling it first when it is missing or stale."""
    global _lib
    if _lib is None:
        if build:
            from . import build as _build
            try:
                _build.build()
            except Exception:
                if not os.path.exists(LIB_PATH):
                    raise
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"countBF CUDA library not found at {LIB_PATH}")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(status: int, call: str) -> None:
    if status != OK:
        raise KmercoError(status, call)


def _ptr(x) -> int | None:
    """Address of a numpy array, a torch tensor (host or device) or an int."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        if not x.flags.c_contiguous:
            raise ValueError("arrays must be C-contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return x.data_ptr()
    raise TypeError(f"cannot pass {type(x).__name__} as a pointer")


# --------------------------------------------------------------- C-named calls
def kmerco_strerror(status: int) -> str:
    return load().kmerco_strerror(status).decode()


def kmerco_create(k: int, m: int, counter_bits: int, nhash: int, threshold: int) -> int:
    h = c_void_p()
    _check(load().kmerco_create(k, m, counter_bits, nhash, threshold, byref(h)), "kmerco_create")
    return h.value


UPDATE_AUTO, UPDATE_ATOMIC, UPDATE_PARTITIONED = 0, 1, 2


def kmerco_create_ex(k: int, m: int, counter_bits: int, nhash: int, threshold: int,
                     forward_only: bool = False, stream: int | None = None,
                     hbm_budget: int = 0, device: int = -1, update_mode: int = 0,
                     dims: tuple[int, int] | None = None, pass_codes: int = 0,
                     canonical_hash: bool = False, whole_file: bool = False,
                     retry_limit: int = 0, max_distinct: int = 0,
                     allocator: "TorchAllocator | None" = None) -> int:
    dx, dy = dims if dims is not None else (0, 0)
    cfg = kmerco_config_t(k, m, counter_bits, nhash, threshold, int(forward_only),
                          stream or None, hbm_budget, device, update_mode, dx, dy,
                          int(canonical_hash), int(whole_file), pass_codes, retry_limit,
                          max_distinct)
    if allocator is not None:
        cfg.dev_alloc = allocator.alloc
        cfg.dev_free = allocator.free
    h = c_void_p()
    _check(load().kmerco_create_ex(byref(cfg), byref(h)), "kmerco_create_ex")
    return h.value


def kmerco_estimate_bytes(k: int, m: int, counter_bits: int, nhash: int, threshold: int,
                          nreads: int, nbytes: int, windows: int, host_inputs: bool = True,
                          **options) -> int:
    """Most device bytes a handle holds after one insert of these reads and
    one classify (kmerco.h); options as kmerco_create_ex (no allocator)."""
    dims = options.pop("dims", None)
    dx, dy = dims if dims is not None else (0, 0)
    cfg = kmerco_config_t(k, m, counter_bits, nhash, threshold, int(options.pop("forward_only", 0)),
                          None, options.pop("hbm_budget", 0), -1, options.pop("update_mode", 0),
                          dx, dy, int(options.pop("canonical_hash", 0)),
                          int(options.pop("whole_file", 0)), options.pop("pass_codes", 0), 0,
                          options.pop("max_distinct", 0))
    if options:
        raise TypeError(f"unknown options {sorted(options)}")
    out = c_uint64(0)
    _check(load().kmerco_estimate_bytes(byref(cfg), nreads, nbytes, windows, int(host_inputs),
                                        byref(out)), "kmerco_estimate_bytes")
    return out.value


def kmerco_paper_dims(n: int, fpp: float = 0.001) -> tuple[int, int]:
    """Eq. 1 countBF dimensions (X, Y) for n items at false positive probability fpp."""
    x, y = c_uint64(0), c_uint64(0)
    _check(load().kmerco_paper_dims(n, fpp, byref(x), byref(y)), "kmerco_paper_dims")
    return x.value, y.value


def kmerco_destroy(h: int) -> None:
    load().kmerco_destroy(h)


def kmerco_insert(h: int, bases, offsets, nreads: int | None = None) -> None:
    if nreads is None:
        nreads = len(offsets) - 1
    _check(load().kmerco_insert(h, _ptr(bases), _ptr(offsets), nreads), "kmerco_insert")


def kmerco_classify(h: int) -> None:
    _check(load().kmerco_classify(h), "kmerco_classify")


def kmerco_stats(h: int) -> dict:
    s = kmerco_stats_t()
    _check(load().kmerco_stats(h, byref(s)), "kmerco_stats")
    return s.as_dict()


def kmerco_get_counters(h: int, dst, nwords: int) -> None:
    _check(load().kmerco_get_counters(h, _ptr(dst), nwords), "kmerco_get_counters")


def kmerco_get_distinct(h: int, keys=None, est=None, cap: int = 0) -> int:
    n = c_uint64(0)
    _check(load().kmerco_get_distinct(h, _ptr(keys), _ptr(est), cap, byref(n)),
           "kmerco_get_distinct")
    return n.value


def kmerco_get_trusted(h: int, keys=None, cap: int = 0) -> int:
    n = c_uint64(0)
    _check(load().kmerco_get_trusted(h, _ptr(keys), cap, byref(n)), "kmerco_get_trusted")
    return n.value


def kmerco_get_erroneous(h: int, keys=None, cap: int = 0) -> int:
    n = c_uint64(0)
    _check(load().kmerco_get_erroneous(h, _ptr(keys), cap, byref(n)), "kmerco_get_erroneous")
    return n.value


def kmerco_get_lists_async(h: int, trusted=None, tcap: int = 0, erroneous=None,
                           ecap: int = 0) -> tuple[int, int]:
    """Queues the copies of both classified lists and returns (n_trusted,
    n_erroneous) at once; the buffers hold the lists after kmerco_sync(h)."""
    nt, ne = c_uint64(0), c_uint64(0)
    _check(load().kmerco_get_lists_async(h, _ptr(trusted), tcap, _ptr(erroneous), ecap,
                                         byref(nt), byref(ne)), "kmerco_get_lists_async")
    return nt.value, ne.value


def kmerco_sync(h: int) -> None:
    _check(load().kmerco_sync(h), "kmerco_sync")


def kmerco_digest(h: int) -> tuple[int, int]:
    """The countBF's 128-bit device-side digest (two 64-bit sums)."""
    out = np.zeros(2, np.uint64)
    _check(load().kmerco_digest(h, _ptr(out)), "kmerco_digest")
    return int(out[0]), int(out[1])


def kmerco_query(h: int, keys, n: int, est) -> None:
    _check(load().kmerco_query(h, _ptr(keys), n, _ptr(est)), "kmerco_query")


def kmerco_merge(dst: int, src: int) -> None:
    _check(load().kmerco_merge(dst, src), "kmerco_merge")


def kmerco_merge_cells(h: int, src, first_word: int, nwords: int) -> None:
    _check(load().kmerco_merge_cells(h, _ptr(src), first_word, nwords), "kmerco_merge_cells")


def kmerco_rank_of(h: int, probes, n: int, ranks) -> None:
    _check(load().kmerco_rank_of(h, _ptr(probes), n, _ptr(ranks)), "kmerco_rank_of")


def kmerco_set_counters(h: int, src, nwords: int) -> None:
    _check(load().kmerco_set_counters(h, _ptr(src), nwords), "kmerco_set_counters")


def kmerco_add_distinct(h: int, keys, n: int) -> None:
    _check(load().kmerco_add_distinct(h, _ptr(keys), n), "kmerco_add_distinct")


def kmerco_reset(h: int) -> None:
    _check(load().kmerco_reset(h), "kmerco_reset")


def kmerco_classify_noalloc(cells, m: int, k: int, counter_bits: int, nhash: int,
                            threshold: int, keys, n: int, est, out, stream: int | None = None) -> int:
    """Classification over caller-owned device buffers without any allocation
    (for callers that cannot allocate device memory); returns the number of
    trustworthy keys.  See kmerco.h for the contract and its limits."""
    nt = c_uint64(0)
    _check(load().kmerco_classify_noalloc(_ptr(cells), m, k, counter_bits, nhash, threshold,
                                          _ptr(keys), n, _ptr(est), _ptr(out), byref(nt),
                                          stream or None), "kmerco_classify_noalloc")
    return nt.value


def kmerco_batch_create(handles: list[int]) -> int:
    arr = (c_void_p * len(handles))(*handles)
    b = c_void_p()
    _check(load().kmerco_batch_create(arr, len(handles), byref(b)), "kmerco_batch_create")
    return b.value


def kmerco_batch_destroy(b: int) -> None:
    load().kmerco_batch_destroy(b)


def kmerco_batch_insert(b: int, bases: list, offsets: list, nreads: list[int],
                        reset: bool = True) -> None:
    n = len(nreads)
    pb = (c_void_p * n)(*[_ptr(x) for x in bases])
    po = (c_void_p * n)(*[_ptr(x) for x in offsets])
    pn = (c_uint64 * n)(*nreads)
    _check(load().kmerco_batch_insert(b, pb, po, pn, int(reset)), "kmerco_batch_insert")


def kmerco_batch_classify(b: int) -> None:
    _check(load().kmerco_batch_classify(b), "kmerco_batch_classify")


def kmerco_batch_schedule(b: int, schedule: int, streams: int = 0) -> None:
    _check(load().kmerco_batch_schedule(b, schedule, streams), "kmerco_batch_schedule")


def kmerco_batch_info(b: int) -> dict:
    info = kmerco_batch_info_t()
    _check(load().kmerco_batch_info(b, byref(info)), "kmerco_batch_info")
    return info.as_dict()


def kmerco_peak_random_cas(nbytes: int, ops: int, device: int = -1) -> float:
    """Random 64-bit load + compare-and-swap operations per second over a
    buffer of nbytes (kmerco_peaks.h)."""
    r = ctypes.c_double(0.0)
    _check(load().kmerco_peak_random_cas(nbytes, ops, device, byref(r)), "kmerco_peak_random_cas")
    return r.value


def kmerco_peak_random_read(nbytes: int, ops: int, device: int = -1) -> float:
    """Random 8-byte reads per second over a buffer of nbytes (kmerco_peaks.h)."""
    r = ctypes.c_double(0.0)
    _check(load().kmerco_peak_random_read(nbytes, ops, device, byref(r)), "kmerco_peak_random_read")
    return r.value


# ------------------------------------------------------------------ wrapper
class CountBF:
    """One countBF handle with numpy results.

    Keys come back as ``uint64`` arrays: shape ``(n,)`` for K <= 32, shape
    ``(n, 2)`` holding ``[lo, hi]`` words for 33 <= K <= 64.
    """

    def __init__(self, k: int, m: int, counter_bits: int = 4, nhash: int = 4,
                 threshold: int = 3, forward_only: bool = False, stream: int | None = None,
                 hbm_budget: int = 0, device: int = -1, update_mode: int = UPDATE_AUTO,
                 dims: tuple[int, int] | None = None, pass_codes: int = 0,
                 canonical_hash: bool = False, whole_file: bool = False,
                 retry_limit: int = 0, max_distinct: int = 0, allocator=None):
        """``dims = (X, Y)`` makes a two-dimensional countBF of X x Y cells
        (Algorithm 3's addressing; ``m`` is then ignored).  ``allocator="torch"``
        (or a :class:`TorchAllocator`) takes the handle's device memory from
        torch's caching allocator."""
        if allocator == "torch":
            allocator = TorchAllocator(None if device < 0 else device)
        self.allocator = allocator   # its callbacks must outlive the handle
        self.k = k
        self.kw = 1 if k <= 32 else 2
        self.params = dict(k=k, m=m, counter_bits=counter_bits, nhash=nhash,
                           threshold=threshold, forward_only=bool(forward_only),
                           dims=tuple(dims) if dims is not None else None,
                           canonical_hash=bool(canonical_hash), whole_file=bool(whole_file))
        self.h = None
        self.h = kmerco_create_ex(k, m, counter_bits, nhash, threshold, forward_only, stream,
                                  hbm_budget, device, update_mode, dims, pass_codes,
                                  canonical_hash, whole_file, retry_limit, max_distinct,
                                  allocator)

    def save(self, path: str) -> None:
        """Write the countBF, its distinct keys and its parameters to an
        ``.npz`` file (readable back with :meth:`load`)."""
        self.classify()   # the distinct keys are read back after classification
        keys, _ = self.distinct()
        p = dict(self.params)
        dims = p.pop("dims")
        np.savez(path, cells=self.counters(), keys=keys,
                 dims=np.array(dims if dims is not None else (0, 0), np.uint64),
                 params=np.array([p["k"], p["m"], p["counter_bits"], p["nhash"], p["threshold"],
                                  p["forward_only"], p["canonical_hash"], p["whole_file"]],
                                 np.uint64))

    @classmethod
    def load(cls, path: str, **kw) -> "CountBF":
        """A new handle holding the countBF and distinct keys of a saved file
        (``kw``: options of the constructor that do not change the results,
        such as ``stream`` or ``update_mode``)."""
        z = np.load(path)
        k, m, alpha, nhash, tau, fwd, ch, wf = (int(v) for v in z["params"])
        dims = tuple(int(v) for v in z["dims"])
        bf = cls(k, m, alpha, nhash, tau, forward_only=bool(fwd),
                 dims=dims if dims[0] else None, canonical_hash=bool(ch), whole_file=bool(wf),
                 **kw)
        cells = np.ascontiguousarray(z["cells"], np.uint64)
        kmerco_set_counters(bf.h, cells, len(cells))
        keys = np.ascontiguousarray(z["keys"], np.uint64)
        n = len(keys)
        if n:
            kmerco_add_distinct(bf.h, keys, n)
        return bf

    def close(self) -> None:
        if self.h:
            kmerco_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def insert(self, bases, offsets) -> None:
        kmerco_insert(self.h, bases, offsets, len(offsets) - 1)

    def classify(self) -> None:
        kmerco_classify(self.h)

    def reset(self) -> None:
        kmerco_reset(self.h)

    def stats(self) -> dict:
        return kmerco_stats(self.h)

    def counters(self) -> np.ndarray:
        w = self.stats()["words"]
        out = np.zeros(w, np.uint64)
        kmerco_get_counters(self.h, out, w)
        return out

    def _shape(self, n: int) -> tuple:
        return (n,) if self.kw == 1 else (n, 2)

    def distinct(self) -> tuple[np.ndarray, np.ndarray]:
        n = kmerco_get_distinct(self.h)
        keys = np.zeros(self._shape(max(n, 1)), np.uint64)
        est = np.zeros(max(n, 1), np.uint32)
        kmerco_get_distinct(self.h, keys, est, n)
        return keys[:n], est[:n]

    def trusted(self) -> np.ndarray:
        n = kmerco_get_trusted(self.h)
        keys = np.zeros(self._shape(max(n, 1)), np.uint64)
        kmerco_get_trusted(self.h, keys, n)
        return keys[:n]

    def erroneous(self) -> np.ndarray:
        n = kmerco_get_erroneous(self.h)
        keys = np.zeros(self._shape(max(n, 1)), np.uint64)
        kmerco_get_erroneous(self.h, keys, n)
        return keys[:n]

    def digest(self) -> str:
        """Hex digest of the countBF cells, computed on the device."""
        d0, d1 = kmerco_digest(self.h)
        return f"{d0:016x}{d1:016x}"

    def query(self, keys: np.ndarray) -> np.ndarray:
        keys = np.ascontiguousarray(keys, np.uint64)
        n = keys.shape[0]
        est = np.zeros(max(n, 1), np.uint32)
        kmerco_query(self.h, keys, n, est)
        return est[:n]

    def merge(self, other: "CountBF") -> None:
        kmerco_merge(self.h, other.h)


class Batch:
    """Several CountBF handles inserted together (persistent launch or
    per-sample kernels on concurrent streams, as tuned or pinned)."""

    def __init__(self, filters: list[CountBF]):
        self.filters = list(filters)
        self.b = kmerco_batch_create([f.h for f in self.filters])

    def close(self) -> None:
        if self.b:
            kmerco_batch_destroy(self.b)
            self.b = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def insert(self, bases: list, offsets: list, reset: bool = True) -> None:
        kmerco_batch_insert(self.b, bases, offsets, [len(o) - 1 for o in offsets], reset)

    def classify(self) -> None:
        kmerco_batch_classify(self.b)

    def schedule(self, schedule: int, streams: int = 0) -> None:
        kmerco_batch_schedule(self.b, schedule, streams)

    def info(self) -> dict:
        return kmerco_batch_info(self.b)
