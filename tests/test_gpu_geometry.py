"""Two-dimensional countBF (Section 2.1, Algorithm 3; sized by Eq. 1): CUDA
path vs the oracle, bit-exact, through the C ABI."""
import numpy as np
import pytest

import oracle
import readsim

torch = pytest.importorskip("torch")
import paper_2305_07545_gb300 as kc  # noqa: E402
from test_gpu_parity import _dev, check, gpu_run  # noqa: E402

pytestmark = pytest.mark.gpu

CASES = [
    # K, (X, Y), alpha, nhash, tau
    (21, (61, 71), 4, 3, 2),
    (31, (1523, 1549), 4, 4, 3),       # Eq. 1 dimensions of a paper-sized filter
    (25, (13, 17), 5, 4, 2),           # eta = 12, 4 wasted bits per cell
    (19, (5, 11), 3, 2, 1),            # eta = 21, a tiny filter: saturation
    (40, (509, 521), 8, 4, 3),         # two-word keys
    (63, (101, 103), 2, 6, 1),
    (17, (97, 97), 4, 2, 2),           # X == Y is legal: only the diagonal cells are used
]


@pytest.mark.parametrize("K,dims,alpha,nhash,tau", CASES)
def test_two_dimensional_parity(K, dims, alpha, nhash, tau):
    b, o = readsim.random_reads(700, 0, 180, seed=sum(dims) + K, alphabet=b"ACGTacgtN",
                                weights=[24, 24, 24, 24, 1, 1, 1, 1, 0.3])
    g = gpu_run(b, o, K, 0, alpha, nhash, tau, dims=dims)
    st = g["stats"]
    assert (st["dim_x"], st["dim_y"]) == dims
    assert st["words"] == dims[0] * dims[1]
    assert st["m_actual"] == dims[0] * dims[1] * (64 // alpha)
    check(g, b, o, K, alpha, nhash, tau)


@pytest.mark.parametrize("mode", [kc.UPDATE_ATOMIC, kc.UPDATE_PARTITIONED])
def test_two_dimensional_both_update_designs(mode):
    # 2711 x 2729 cells: above the partitioned design's automatic threshold
    w = readsim.WORKLOADS["tiny"]
    b, o = readsim.scaled("tiny", 6000, seed_offset=11).generate()
    dims = (2711, 2729)
    g = gpu_run(b, o, w.K, 0, 4, 4, 2, dims=dims, update_mode=mode)
    check(g, b, o, w.K, 4, 4, 2)


def test_paper_sized_filter_from_eq1():
    b, o = readsim.scaled("tiny", 3000, seed_offset=12).generate()
    n = int(oracle.extract(b, o, 21).n)
    dims = kc.kmerco_paper_dims(n, 0.001)
    assert dims == oracle.paper_dims(n, 0.001)
    g = gpu_run(b, o, 21, 0, 8, 4, 2, dims=dims)
    ref = check(g, b, o, 21, 8, 4, 2)
    assert ref.n_inserted == n


def test_two_dimensional_merge():
    b, o = readsim.scaled("tiny", 1000, seed_offset=13).generate()
    half = 400
    b1, o1 = b[:int(o[half])].copy(), o[:half + 1].copy()
    b2, o2 = b[int(o[half]):].copy(), (o[half:] - o[half]).copy()
    dims = (211, 223)
    with kc.CountBF(21, 0, 4, 3, 2, dims=dims) as x, kc.CountBF(21, 0, 4, 3, 2, dims=dims) as y:
        x.insert(_dev(b1), _dev(o1))
        y.insert(_dev(b2), _dev(o2))
        x.merge(y)
        x.classify()
        keys, est = x.distinct()
        g = dict(stats=x.stats(), counters=x.counters(), keys=keys, est=est,
                 trusted=x.trusted(), erroneous=x.erroneous())
    check(g, b, o, 21, 4, 3, 2)
    # same number of cells, other shape: not mergeable
    with kc.CountBF(21, 0, 4, 3, 2, dims=(211, 223)) as x, \
            kc.CountBF(21, 0, 4, 3, 2, dims=(223, 211)) as y:
        with pytest.raises(kc.KmercoError) as e:
            x.merge(y)
        assert e.value.status == kc.EINVAL


def test_two_dimensional_query_entry_point():
    b, o = readsim.scaled("tiny", 500, seed_offset=14).generate()
    dims = (101, 107)
    with kc.CountBF(21, 0, 4, 3, 2, dims=dims) as bf:
        bf.insert(_dev(b), _dev(o))
        filt = bf.counters()
        ex = oracle.extract(b, o, 21)
        probe = np.concatenate([ex.lo[:300], readsim.Stream(3).integers(300, 1 << 42)
                                .astype(np.uint64)])
        est = np.zeros(len(probe), np.uint32)
        kc.kmerco_query(bf.h, probe, len(probe), est)
    want = [oracle.query_2d(filt, 21, 0, int(x), dims, 4, 3) for x in probe]
    assert est.tolist() == want
