"""Host-side arithmetic of bench.py (no GPU): the roofline of an insert call."""
import bench


def test_roofline_counts_random_sector_bytes_per_update():
    # 1.2e8 K-mers, k_h = 4: 256 B each in the random-sector model
    r = bench.roofline_of_insert(120_000_000, 23_535_998, 4, 158_000_008, 6.0, 6658.6, None)
    assert r["algorithmic_bytes_per_kmer"] == 256
    assert r["algorithmic_bytes_per_launch"] == 120_000_000 * 256
    assert abs(r["achieved"] - 120_000_000 * 256 / 0.006 / 1e9) < 1e-6
    assert abs(r["frac"] - r["achieved"] / 6658.6) < 1e-12
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["traffic"] is None


def test_word_granular_count():
    r = bench.roofline_of_insert(1000, 200, 3, 5000, 1.0, 1000.0, 123.0)
    wg = r["word_granular"]
    assert wg["bytes_per_launch"] == 5000 + 1000 * (16 * 3 + 8) + 200 * 16
    assert abs(wg["frac"] - wg["bytes_per_launch"] / 1e-3 / 1e9 / 1000.0) < 1e-12
    assert r["traffic"] == 123.0 and r["avg_launch_ms"] == 1.0


def test_traffic_record_is_well_formed():
    # one record line: the code hash it was taken on and the DRAM bytes of one call
    lines = [l for l in open(bench.PROFILE_SUMMARY) if l.startswith("traffic_record")]
    assert len(lines) == 1
    kv = dict(p.split("=", 1) for p in lines[0].split()[1:])
    assert len(kv["source_sha"]) == 16 and int(kv["source_sha"], 16) >= 0
    assert float(kv["dram_bytes_per_launch"]) > 0
    assert len(bench.source_sha()) == 16
