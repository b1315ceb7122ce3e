"""Saving a countBF with its distinct keys and loading it back gives the same
classification, and the loaded handle keeps counting."""
import numpy as np
import pytest

import readsim

torch = pytest.importorskip("torch")
import paper_2305_07545_gb300 as kc  # noqa: E402
from test_gpu_parity import _dev, check  # noqa: E402

pytestmark = pytest.mark.gpu


def _snapshot(bf):
    bf.classify()
    keys, est = bf.distinct()
    return dict(stats=bf.stats(), counters=bf.counters(), keys=keys, est=est,
                trusted=bf.trusted(), erroneous=bf.erroneous())


@pytest.mark.parametrize("K,opts", [(21, {}), (45, {}), (25, dict(dims=(211, 223))),
                                    (31, dict(canonical_hash=True, whole_file=True))])
def test_save_load_round_trip(tmp_path, K, opts):
    b, o = readsim.scaled("tiny", 1500, seed_offset=31).generate()
    with kc.CountBF(K, 1 << 18, 4, 3, 2, **opts) as bf:
        bf.insert(_dev(b), _dev(o))
        a = _snapshot(bf)
        da = bf.digest()
        bf.save(str(tmp_path / "bf.npz"))
    with kc.CountBF.load(str(tmp_path / "bf.npz")) as bf2:
        c = _snapshot(bf2)
        assert bf2.digest() == da          # the same countBF, 2-D geometries included
    for key in ("counters", "keys", "est", "trusted", "erroneous"):
        assert np.array_equal(a[key], c[key]), key
    assert c["stats"]["distinct"] == a["stats"]["distinct"]


def test_loaded_handle_keeps_counting(tmp_path):
    b, o = readsim.scaled("tiny", 1200, seed_offset=32).generate()
    half = 500
    b1, o1 = b[:int(o[half])].copy(), o[:half + 1].copy()
    b2, o2 = b[int(o[half]):].copy(), (o[half:] - o[half]).copy()
    with kc.CountBF(21, 1 << 16, 4, 3, 2) as bf:
        bf.insert(_dev(b1), _dev(o1))
        bf.save(str(tmp_path / "part.npz"))
    with kc.CountBF.load(str(tmp_path / "part.npz")) as bf2:
        bf2.insert(_dev(b2), _dev(o2))
        g = _snapshot(bf2)
    # countBF, distinct keys and classification of the whole input; the
    # window totals only count what was inserted after loading
    check(g, b, o, 21, 4, 3, 2, totals=False)


def test_set_counters_checks_the_size():
    with kc.CountBF(21, 1 << 12, 4, 3, 2) as bf:
        w = bf.stats()["words"]
        with pytest.raises(kc.KmercoError) as e:
            kc.kmerco_set_counters(bf.h, np.zeros(w + 1, np.uint64), w + 1)
        assert e.value.status == kc.ESIZE


def _fmix64(k):
    k = np.asarray(k, np.uint64)
    k ^= k >> np.uint64(33)
    k *= np.uint64(0xFF51AFD7ED558CCD)
    k ^= k >> np.uint64(33)
    k *= np.uint64(0xC4CEB9FE1A85EC53)
    k ^= k >> np.uint64(33)
    return k


def _digest(cells):
    # the definition in kmerco.h, on the host: two wrapping sums of mixed
    # (index, cell) values
    i = np.arange(len(cells), dtype=np.uint64)
    with np.errstate(over="ignore"):
        s0 = _fmix64(cells ^ (i * np.uint64(0x9E3779B97F4A7C15))).sum(dtype=np.uint64)
        s1 = _fmix64(cells + _fmix64(i + np.uint64(1))).sum(dtype=np.uint64)
    return int(s0), int(s1)


def test_digest_is_its_definition_and_tells_countbfs_apart():
    b, o = readsim.scaled("tiny", 900, seed_offset=17).generate()
    with kc.CountBF(21, (1 << 20) + 48, 5, 3, 2) as bf:   # 12 counters per cell, ragged
        bf.insert(b, o)
        cells = bf.counters()
        d = kc.kmerco_digest(bf.h)
        assert d == _digest(cells)
        assert kc.kmerco_digest(bf.h) == d                  # deterministic
        changed = cells.copy()
        changed[len(changed) // 2] ^= np.uint64(1)           # one counter one step apart
        kc.kmerco_set_counters(bf.h, changed, len(changed))
        d2 = kc.kmerco_digest(bf.h)
        assert d2 == _digest(changed) and d2[0] != d[0] and d2[1] != d[1]
        swapped = cells.copy()                               # the same cells in another order
        swapped[[0, 1]] = swapped[[1, 0]]
        if swapped[0] != swapped[1]:
            kc.kmerco_set_counters(bf.h, swapped, len(swapped))
            assert kc.kmerco_digest(bf.h) != d
