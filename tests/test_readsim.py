"""The seeded read simulator: determinism and the workload recipes' shape."""
import numpy as np

import readsim


def test_same_seed_same_reads():
    a = readsim.scaled("tiny", 300).generate()
    b = readsim.scaled("tiny", 300).generate()
    c = readsim.scaled("tiny", 300, seed_offset=1).generate()
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert not np.array_equal(a[0], c[0])


def test_tiny_recipe_shape():
    w = readsim.WORKLOADS["tiny"]
    b, o = w.generate()
    assert len(o) == 2001 and int(o[0]) == 0 and int(o[-1]) == len(b) == 200_000
    assert np.all(np.diff(o.astype(np.int64)) == 100)
    n_frac = float(np.mean(b == ord("N")))
    assert 0.0005 < n_frac < 0.002            # 0.1% N calls
    assert set(np.unique(b).tolist()) <= set(b"ACGTN")


def test_error_free_reads_come_from_the_genome_or_its_reverse_complement():
    s = readsim.Stream(3)
    g = readsim.genome(2000, 0.5, s)
    b, o = readsim.sample_reads(g, readsim.ReadModel(200, 50), s)
    gs = bytes(readsim.ASCII[g]).decode()
    circ = gs + gs[:60]
    comp = str.maketrans("ACGT", "TGCA")
    rev = 0
    for i in range(200):
        r = bytes(b[o[i]:o[i + 1]]).decode()
        if r in circ:
            continue
        assert r.translate(comp)[::-1] in circ
        rev += 1
    assert 60 < rev < 140


def test_gc_content_and_variable_lengths():
    s = readsim.Stream(4)
    g = readsim.genome(200_000, 0.41, s)
    assert abs(float(np.mean((g == 1) | (g == 2))) - 0.41) < 0.01
    b, o = readsim.sample_reads(g, readsim.ReadModel(500, (50, 300), sub=0.01), s)
    lens = np.diff(o.astype(np.int64))
    assert lens.min() >= 50 and lens.max() <= 300 and lens.std() > 30
