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
        bf.save(str(tmp_path / "bf.npz"))
    with kc.CountBF.load(str(tmp_path / "bf.npz")) as bf2:
        c = _snapshot(bf2)
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
