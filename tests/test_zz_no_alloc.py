"""The allocation-free classification entry point (kmerco_classify_noalloc).

It serves callers that must not allocate device memory themselves (a
process whose GPU memory is reserved by its own pool, a plug-in inside such a
host, a path that cannot afford cudaMalloc's device-wide synchronisation).
Its results must equal those of the handle-based kmerco_classify on the same
countBF and keys -- exactly, since the work is integer -- on consecutive calls
that reuse its fixed scratch array.  This file is collected last so that a
failure here does not stop the other GPU tests from running first.
"""
import ctypes

import numpy as np
import pytest

import oracle
import readsim

torch = pytest.importorskip("torch")
import paper_2305_07545_gb300 as kc  # noqa: E402

pytestmark = pytest.mark.gpu


def _expected_split(keys: np.ndarray, est: np.ndarray, tau: int):
    t = est > tau
    return np.concatenate([keys[t], keys[~t]]), int(t.sum())


@pytest.mark.parametrize("K", [21, 55])
def test_noalloc_matches_handle_classify(K):
    w = readsim.WORKLOADS["tiny"]
    bases, offsets = readsim.scaled("tiny", 1500, seed_offset=9).generate()
    alpha, nhash, tau = w.alpha, w.nhash, w.tau
    with kc.CountBF(K, w.m, alpha, nhash, tau) as bf:
        bf.insert(bases, offsets)
        bf.classify()
        st = bf.stats()
        keys, est_ref = bf.distinct()
        trusted_ref, erroneous_ref = bf.trusted(), bf.erroneous()
        m = st["m_actual"]
        cells = torch.zeros(st["words"], dtype=torch.int64, device="cuda")
        torch.cuda.synchronize()
        kc.kmerco_get_counters(bf.h, cells, st["words"])
    kw = 1 if K <= 32 else 2
    n = len(keys)
    assert n > 4096   # several split tiles
    d_keys = torch.from_numpy(keys.view(np.int64).reshape(-1).copy()).cuda()
    est = torch.zeros(n, dtype=torch.int32, device="cuda")
    out = torch.zeros(n * kw, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    torch.cuda.synchronize()

    # what the oracle's Algorithm 5 / Algorithm 2 give on the same countBF
    host_cells = cells.cpu().numpy().view(np.uint64)
    hi = keys[:, 1].copy() if kw == 2 else np.zeros(n, np.uint64)
    lo = keys[:, 0].copy() if kw == 2 else keys
    o_est, o_tr = oracle.classify(host_cells, hi, lo, K, m, alpha, nhash, tau)

    # two calls in a row on the same inputs
    for _ in range(2):
        est.zero_()
        out.zero_()
        nt = kc.kmerco_classify_noalloc(cells, m, K, alpha, nhash, tau, d_keys, n, est, out,
                                        stream)
        assert nt == len(trusted_ref) == st["trustworthy"]
        assert np.array_equal(est.cpu().numpy().view(np.uint32), est_ref)
        got = out.cpu().numpy().view(np.uint64).reshape(keys.shape)
        assert np.array_equal(got[:nt], trusted_ref)
        assert np.array_equal(got[nt:], erroneous_ref)
        assert np.array_equal(est.cpu().numpy().view(np.uint32).astype(np.uint64), o_est)
        assert nt == int(o_tr.sum())
        assert np.array_equal(got[:nt], keys[o_tr]) and np.array_equal(got[nt:], keys[~o_tr])

    # a smaller call right after: the scratch left by the larger one is stale
    half = n // 2 + 77
    est.zero_()
    out.zero_()
    nt = kc.kmerco_classify_noalloc(cells, m, K, alpha, nhash, tau, d_keys, half, est, out, stream)
    want, want_t = _expected_split(keys[:half], est_ref[:half], tau)
    assert nt == want_t
    assert np.array_equal(est.cpu().numpy().view(np.uint32)[:half], est_ref[:half])
    got = out.cpu().numpy().view(np.uint64).reshape(keys.shape)[:half]
    assert np.array_equal(got, want)


def test_noalloc_rejects_oversize_and_bad_arguments():
    lib = kc.load()
    nt = ctypes.c_uint64(123)
    big = kc.NOALLOC_MAX_KEYS + 1
    # the size check comes before any pointer is touched or any kernel runs
    assert lib.kmerco_classify_noalloc(8, 1 << 10, 21, 4, 3, 2, 8, big, 8, 8, ctypes.byref(nt),
                                       None) == kc.EINVAL
    assert lib.kmerco_classify_noalloc(8, 1000, 21, 4, 3, 2, 8, 10, 8, 8, ctypes.byref(nt),
                                       None) == kc.EINVAL   # m not a multiple of eta
    assert lib.kmerco_classify_noalloc(8, 1 << 10, 21, 4, 3, 15, 8, 10, 8, 8, ctypes.byref(nt),
                                       None) == kc.EINVAL   # tau >= 2^alpha - 1
    assert lib.kmerco_classify_noalloc(None, 1 << 10, 21, 4, 3, 2, None, 10, None, None,
                                       ctypes.byref(nt), None) == kc.EINVAL
    assert lib.kmerco_classify_noalloc(8, 1 << 10, 21, 4, 3, 2, 8, 0, 8, 8, ctypes.byref(nt),
                                       None) == kc.OK and nt.value == 0
