"""The C-ABI library: it loads, exports every declared entry point, and
rejects bad arguments on the host before touching the GPU.  CPU only."""
import ctypes
import os
import re

import pytest

import paper_2305_07545_gb300 as kc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INCLUDE = os.path.join(ROOT, "include")


def declared_functions():
    """Every kmerco_* function declared in any header of include/."""
    names = set()
    for f in sorted(os.listdir(INCLUDE)):
        if not f.endswith(".h"):
            continue
        text = open(os.path.join(INCLUDE, f)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(kmerco_[a-z_]+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    return kc.load()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 14
    for n in names:
        assert hasattr(lib, n), f"{n} declared in include/ but not exported"
    assert set(names) == set(kc.SIGNATURES)


def test_strerror(lib):
    for code in range(7):
        assert kc.kmerco_strerror(code)
    assert kc.kmerco_strerror(99) == "unknown status"


@pytest.mark.parametrize("args", [
    (0, 1 << 10, 4, 3, 2),      # K < 1
    (65, 1 << 10, 4, 3, 2),     # K > 64
    (21, 0, 4, 3, 2),           # m < 1
    (21, 1 << 10, 0, 3, 2),     # alpha < 1
    (21, 1 << 10, 33, 3, 2),    # alpha > 32
    (21, 1 << 10, 4, 0, 2),     # k_h < 1
    (21, 1 << 10, 4, 33, 2),    # k_h > 32
    (21, 1 << 10, 4, 3, 15),    # tau >= 2^alpha - 1
    (21, 1 << 10, 1, 3, 1),     # tau >= 2^1 - 1
])
def test_create_rejects_bad_parameters(lib, args):
    h = ctypes.c_void_p(123)
    assert lib.kmerco_create(*args, ctypes.byref(h)) == kc.EINVAL
    assert h.value is None


def test_null_handle_calls(lib):
    assert lib.kmerco_insert(None, None, None, 0) == kc.EINVAL
    assert lib.kmerco_classify(None) == kc.EINVAL
    assert lib.kmerco_reset(None) == kc.EINVAL
    assert lib.kmerco_merge(None, None) == kc.EINVAL
    assert lib.kmerco_stats(None, None) == kc.EINVAL
    lib.kmerco_destroy(None)


def test_python_error_type(lib):
    with pytest.raises(kc.KmercoError) as e:
        kc.kmerco_create(21, 1 << 10, 4, 3, 99)
    assert e.value.status == kc.EINVAL


@pytest.mark.parametrize("k,m,nhash", [(33, 1 << 20, 5), (21, 1 << 20, 5), (21, 1 << 35, 4),
                                         (55, (1 << 34) + 16, 4)])
def test_partitioned_mode_limits(lib, k, m, nhash):
    # the partitioned update design needs k_h <= 4 and at most 2^30 cells;
    # asking for it otherwise is rejected before any GPU work
    with pytest.raises(kc.KmercoError) as e:
        kc.kmerco_create_ex(k, m, 4, nhash, 3, update_mode=kc.UPDATE_PARTITIONED)
    assert e.value.status == kc.EINVAL
    with pytest.raises(kc.KmercoError) as e:
        kc.kmerco_create_ex(21, 1 << 20, 4, 3, 2, update_mode=3)
    assert e.value.status == kc.EINVAL


@pytest.mark.parametrize("dims", [(0, 5), (5, 0), ((1 << 24) + 1, 3), (3, (1 << 24) + 1)])
def test_two_dimensional_geometry_limits(lib, dims):
    # both dimensions 1..2^24, or both zero for a flat countBF; checked
    # before any GPU work
    with pytest.raises(kc.KmercoError) as e:
        kc.kmerco_create_ex(21, 1 << 20, 4, 3, 2, dims=dims)
    assert e.value.status == kc.EINVAL
    with pytest.raises(kc.KmercoError) as e:   # over 2^30 cells: too many for the partitioned design
        kc.kmerco_create_ex(21, 0, 4, 3, 2, update_mode=kc.UPDATE_PARTITIONED, dims=(32771, 32783))
    assert e.value.status == kc.EINVAL


def test_paper_dims_entry_point_matches_the_oracle(lib):
    import oracle
    for n in [1, 2, 50, 1000, 123457, 10 ** 6, 20506529, 81936236, 163872472, 10 ** 9]:
        for fpp in (0.001, 0.01, 1e-6):
            assert kc.kmerco_paper_dims(n, fpp) == oracle.paper_dims(n, fpp), (n, fpp)
    for n, fpp in [(0, 0.001), (10, 0.0), (10, 1.0), (10, -1.0), (10 ** 18, 1e-9)]:
        with pytest.raises(kc.KmercoError) as e:
            kc.kmerco_paper_dims(n, fpp)
        assert e.value.status == kc.EINVAL


def test_variant_flags_are_checked(lib):
    for kw in (dict(canonical_hash=True, forward_only=True),):
        with pytest.raises(kc.KmercoError) as e:
            kc.kmerco_create_ex(21, 1 << 12, 4, 3, 2, **kw)
        assert e.value.status == kc.EINVAL
    cfg = kc.kmerco_config_t(21, 1 << 12, 4, 3, 2, 0, None, 0, -1, 0, 0, 0, 0, 2, 0)
    h = ctypes.c_void_p(1)
    assert lib.kmerco_create_ex(ctypes.byref(cfg), ctypes.byref(h)) == kc.EINVAL   # whole_file = 2
    cfg.whole_file, cfg.canonical_hash = 0, 3
    assert lib.kmerco_create_ex(ctypes.byref(cfg), ctypes.byref(h)) == kc.EINVAL
    assert h.value is None
