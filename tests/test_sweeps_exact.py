"""The sweeps' accuracy ground truth: exact multiplicities of canonical K-mers
computed on the host with numpy (paper_2305_07545_gb300.sweeps.exact_counts)
must equal the oracle's extraction followed by its sort and count, key for
key and count for count, on reads with N and IUPAC codes, lowercase bases,
reads shorter than K and empty reads, for one- and two-word keys."""
import numpy as np
import pytest

import oracle
import readsim
from paper_2305_07545_gb300 import sweeps


def _reads():
    st = readsim.Stream(4242)
    b, o = readsim.random_reads(300, 0, 140, seed=4243)
    b = b.copy()
    pos = st.integers(len(b) // 50, len(b))
    b[pos] = np.frombuffer(b"NRYKMnacgt" * (len(pos) // 10 + 1), np.uint8)[:len(pos)]
    sb, so = readsim.from_strings(["", "ACGT", "acgtacgtacgtNNacgtacgtacgtacgtacgtacgtacgtacgt",
                                   "TTTTTTTTTTTTTTTTTTTTTTTTTTTTTTTTTTTTTTTTTTTTTTTTTTTTTTTTTTTTTTTTTTTT"])
    return np.concatenate([b, sb]), np.concatenate([o, so[1:] + o[-1]])


@pytest.mark.parametrize("K", [1, 7, 21, 31, 32, 33, 47, 55, 64])
def test_exact_counts_equal_the_oracle(K, oracle_lib):
    b, o = _reads()
    keys, cnt = sweeps.exact_counts(b, o, K)
    ex = oracle.extract(b, o, K)
    dhi, dlo, c2 = oracle.distinct(ex.hi, ex.lo)
    assert int(cnt.sum()) == ex.n
    if K <= 32:
        assert np.array_equal(keys, dlo)
    else:
        assert np.array_equal(keys[:, 0], dlo) and np.array_equal(keys[:, 1], dhi)
    assert np.array_equal(cnt, c2)


def test_exact_counts_with_a_non_zero_first_offset(oracle_lib):
    b, o = _reads()
    o2 = o[40:].copy()                      # reads 40.. only; bases before them ignored
    keys, cnt = sweeps.exact_counts(b, o2, 21)
    ex = oracle.extract(b, o2, 21)
    _, dlo, c2 = oracle.distinct(ex.hi, ex.lo)
    assert np.array_equal(keys, dlo) and np.array_equal(cnt, c2)


def test_exact_counts_of_no_window():
    b, o = readsim.from_strings(["ACG", ""])
    keys, cnt = sweeps.exact_counts(b, o, 5)
    assert len(keys) == 0 and len(cnt) == 0
