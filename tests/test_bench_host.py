"""Host-side arithmetic of bench.py (no GPU): the roofline of an insert call."""
import bench


def test_word_granular_bytes_are_the_headline():
    # 1.2e8 K-mers, k_h = 4, one-word keys: 4 x 16 B of cell read-modify-write
    # plus the key written and read once (16 B) per K-mer, plus the input
    r = bench.roofline_of_insert(120_000_000, 4, 1, 158_000_008, 6.0, 6658.6, None)
    assert r["algorithmic_bytes_per_kmer"] == 80
    assert r["algorithmic_bytes_per_launch"] == 158_000_008 + 120_000_000 * 80
    assert abs(r["achieved"] - r["algorithmic_bytes_per_launch"] / 0.006 / 1e9) < 1e-6
    assert abs(r["frac"] - r["achieved"] / 6658.6) < 1e-12
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["traffic"] is None


def test_two_word_keys_and_the_sector_model():
    r = bench.roofline_of_insert(1000, 3, 2, 5000, 1.0, 1000.0, 123.0)
    assert r["algorithmic_bytes_per_launch"] == 5000 + 1000 * (16 * 3 + 32)
    sm = r["sector_model"]
    assert sm["bytes_per_launch"] == 1000 * 64 * 3
    assert abs(sm["frac"] - sm["bytes_per_launch"] / 1e-3 / 1e9 / 1000.0) < 1e-12
    assert r["traffic"] == 123.0 and r["avg_launch_ms"] == 1.0
    assert abs(r["traffic_over_algorithmic"] - 123.0 / r["algorithmic_bytes_per_launch"]) < 1e-15


def test_l2_atomic_view():
    r = bench.l2_atomic_roofline(1_000_000, 3, 0.5, 64e9)
    assert r["bound"] == "l2_atomic"
    assert abs(r["achieved"] - 3e6 / 0.0005 / 1e9) < 1e-9
    assert abs(r["frac"] - 3e6 / 0.0005 / 64e9) < 1e-12


def test_host_cpu_reports_model_and_cores():
    c = bench.host_cpu()
    assert c["nproc"] >= 1 and isinstance(c["cpu_model"], str) and c["cpu_model"]


def test_traffic_records_are_well_formed():
    # one record line per workload: the code hash it was taken on and the
    # DRAM bytes of one call (a summary covering several workloads names
    # each record's workload)
    import os
    for wl, path in bench.PROFILE_SUMMARIES.items():
        if not os.path.exists(path):
            continue
        recs = []
        for line in open(path):
            if line.startswith("traffic_record"):
                kv = dict(p.split("=", 1) for p in line.split()[1:])
                if kv.get("workload", wl) == wl:
                    recs.append(kv)
        assert len(recs) == 1, wl
        kv = recs[0]
        assert len(kv["source_sha"]) == 16 and int(kv["source_sha"], 16) >= 0
        assert float(kv["dram_bytes_per_launch"]) > 0
    assert len(bench.source_sha()) == 16


def test_recorded_traffic_matches_by_workload(tmp_path, monkeypatch):
    f = tmp_path / "p.md"
    sha = bench.source_sha()
    f.write_text(f"traffic_record workload=a source_sha={sha} dram_bytes_per_launch=100\n"
                 f"traffic_record workload=b source_sha={sha} dram_bytes_per_launch=200\n"
                 f"traffic_record workload=c source_sha=0000000000000000 dram_bytes_per_launch=1\n")
    monkeypatch.setattr(bench, "PROFILE_SUMMARIES", {"a": str(f), "b": str(f), "c": str(f)})
    assert bench.recorded_traffic("a") == 100.0
    assert bench.recorded_traffic("b") == 200.0
    assert bench.recorded_traffic("c") is None      # taken on other code
    assert bench.recorded_traffic("d") is None      # no summary


def test_batch_groups_respect_the_memory_limit():
    sizes = [5, 5, 5, 20, 1, 1, 9]
    groups = bench.batch_groups(sizes, 10)
    assert [i for g in groups for i in g] == list(range(len(sizes)))   # every sample once, in order
    for g in groups:
        assert len(g) == 1 or sum(sizes[i] for i in g) <= 10
    assert bench.batch_groups(sizes, 1000) == [list(range(len(sizes)))]


def test_l2_note_names_the_regime():
    l2 = 126 << 20
    assert "L2-resident" in bench.l2_note(512 << 10, 200_000, l2)          # tiny: 512 KiB
    assert "about the size of L2" in bench.l2_note(128 << 20, 150e6, l2)   # single: 128 MiB
    assert "larger than L2" in bench.l2_note(4 << 30, 3.16e9, l2)          # repeats: 4 GiB
