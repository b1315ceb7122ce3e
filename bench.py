"""Benchmark: K-mer insertions per second of the whole countBF path on GB300.

One step = one pass of the full hot path over one sample: reset the countBF,
insert every read (pack, canonicalise, hash, saturating counter updates,
distinct-key set), then classify (sort the distinct keys, QcountBF-II per
key, split at tau).  value = K-mer windows inserted / step time.

The default workload is the largest single-GPU one: 20,000,000 reads x 150 bp
of a 100 Mb genome with repeat families, a 2^33-counter (4 GiB) countBF,
counted as 31-mers; the same reads counted as 55-mers (two-word keys) are
timed after it and reported under "secondary".

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload repeats]
    python bench.py --impl reference ...   # the CPU oracle on a bounded sample

Under torchrun (N > 1) the ranks count ONE sample together: rank r inserts
read shard r, the countBFs are merged with a chunked all-to-all and a
saturating merge, and the distinct keys go to the rank owning their key range
(scaling "strong": value = the sample's windows over the slowest rank's
time).  With --replicas every rank counts its own sample instead (scaling
"weak").
"""
from __future__ import annotations

import argparse
import hashlib
import json
import re
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import readsim  # noqa: E402

METRIC = "K-mer insertions/sec on 1 GB300 (bit-exact vs oracle); % of L2-atomic/HBM roofline"
UNIT = "K-mer insertions/s"
FALLBACK_HBM_GBS = 6800.0
L2_FLUSH_BYTES = 256 << 20
PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "insert_phase_single.md")
# per workload: the ncu summary holding the DRAM traffic record of its insert phase
PROFILE_SUMMARIES = {"single": PROFILE_SUMMARY,
                     "repeats": os.path.join(ROOT, "profiles", "insert_phase_repeats.md"),
                     "repeats55": os.path.join(ROOT, "profiles", "insert_phase_repeats.md")}
SECONDARY = {"repeats": "repeats55"}   # workload timed after the headline one, same reads
INSERT_SOURCES = [os.path.join(ROOT, "paper_2305_07545_gb300", "csrc", f)
                  for f in ("kmerco_insert.cu", "kmerco_internal.cuh")]


def describe(w: readsim.Workload) -> str:
    r = w.reads
    rl = r.read_len if isinstance(r.read_len, int) else f"{r.read_len[0]}-{r.read_len[1]}"
    err = f"{r.sub:.2%} substitutions"
    if r.ins or r.dele:
        err += f" + {r.ins + r.dele:.3%} indels"
    if r.n_rate:
        err += f", {r.n_rate:.1%} N"
    rep = ", 10% repeat families" if w.repeats else ""
    return (f"{w.name}: {w.genome_len / 1e6:g} Mb genome ({w.gc:.0%} GC{rep}), "
            f"{r.n_reads:,} reads x {rl} bp, {err}, K={w.K} canonical, "
            f"2^{w.m.bit_length() - 1} {w.alpha}-bit counters, {w.nhash} hashes, tau={w.tau}")


def source_sha() -> str:
    """Hash of the insert kernels' code: the sources without comments and
    blank lines, so that only a change of the code voids a DRAM record."""
    h = hashlib.sha256()
    for f in INSERT_SOURCES:
        with open(f) as fh:
            text = re.sub(r"/\*.*?\*/", "", fh.read(), flags=re.S)
        for line in text.splitlines():
            code = line.split("//", 1)[0].rstrip()
            if code:
                h.update(code.encode() + b"\n")
    return h.hexdigest()[:16]


def measured_peak() -> tuple[float, str]:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            v = float(json.load(f)["hbm_gbs"])
        return v, "measured (MEASURED_PEAKS.json hbm_gbs, STREAM-style copy)"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback (6.8 TB/s earlier GB300 copy measurement)"


def recorded_traffic(workload: str = "single") -> float | None:
    """DRAM bytes per insert call from the committed ncu summary of the
    workload, if it was taken on the current insert-kernel source."""
    path = PROFILE_SUMMARIES.get(workload)
    if not path:
        return None
    try:
        with open(path) as f:
            for line in f:
                if line.startswith("traffic_record"):
                    kv = dict(p.split("=", 1) for p in line.split()[1:])
                    if kv.get("workload", workload) != workload:
                        continue
                    if kv.get("source_sha") == source_sha():
                        return float(kv["dram_bytes_per_launch"])
    except Exception:
        pass
    return None


def roofline_of_insert(inserted: int, nhash: int, key_words: int, input_bytes: int,
                       insert_ms: float, peak_gbs: float, traffic: float | None) -> dict:
    """Roofline of one insert call (every kernel of one kmerco_insert).

    Algorithmic bytes, word-granular: per inserted K-mer k_h read-modify-writes
    of one 8-byte countBF cell (16 B each) and its canonical key written once
    and read once by the exact distinct step (8 B per key word each way), plus
    the input bases and offsets.  The HBM random-sector model (each update
    reads a random 32-byte sector and writes it back: 64 B per update) is
    reported beside it as a secondary bound, not the headline."""
    insert_s = insert_ms / 1000.0
    per_kmer = 16 * nhash + 16 * key_words
    launch_bytes = input_bytes + inserted * per_kmer
    achieved = launch_bytes / insert_s / 1e9
    sector_bytes = inserted * 64 * nhash
    return {"bound": "hbm", "achieved": achieved, "peak": peak_gbs, "unit": "GB/s",
            "frac": achieved / peak_gbs, "traffic": traffic,
            "kernel": "insert phase: every kernel of one kmerco_insert call (insert_kernel: "
                      "pack, canonical, hash, distinct set, increment staging; in the "
                      "partitioned design also repartition_kernel and the apply kernel)",
            "model": "word-granular: k_h x (8-byte cell read + write) + key written and "
                     "read once per inserted K-mer, plus the input",
            "algorithmic_bytes_per_kmer": per_kmer,
            "algorithmic_bytes_per_launch": int(launch_bytes),
            "traffic_over_algorithmic": (traffic / launch_bytes) if traffic else None,
            "sector_model": {"bytes_per_kmer": 64 * nhash,
                             "bytes_per_launch": int(sector_bytes),
                             "achieved": sector_bytes / insert_s / 1e9,
                             "frac": sector_bytes / insert_s / 1e9 / peak_gbs,
                             "note": "HBM random-sector bound of an in-place update design "
                                     "(64 B per counter update); secondary"},
            "avg_launch_ms": insert_ms}


def l2_atomic_roofline(inserted: int, nhash: int, insert_ms: float, cas_peak: float) -> dict:
    """The countBF update against the measured random compare-and-swap rate
    on an L2-resident buffer: k_h updates per inserted K-mer."""
    ups = inserted * nhash / (insert_ms / 1000.0)
    return {"bound": "l2_atomic", "achieved": ups / 1e9, "peak": cas_peak / 1e9,
            "unit": "G updates/s", "frac": ups / cas_peak, "traffic": None,
            "model": "k_h counter updates per inserted K-mer over the insert phase",
            "avg_launch_ms": insert_ms}


def measure_peaks(device: int) -> dict:
    """Random 64-bit load+CAS and random 8-byte read rates on this GPU
    (kmerco_peak_*), over an L2-resident buffer, a 128 MiB one and a 4 GiB
    one: the ceilings of the countBF update and query."""
    import paper_2305_07545_gb300 as kc
    out = {}
    for name, nbytes in (("512KiB", 512 << 10), ("128MiB", 128 << 20), ("4GiB", 4 << 30)):
        out[name] = {"random_cas_per_s": kc.kmerco_peak_random_cas(nbytes, 1 << 28, device),
                     "random_read_per_s": kc.kmerco_peak_random_read(nbytes, 1 << 28, device)}
    return out


def host_link(device: int) -> dict:
    """Pinned host <-> device copy rates of 1 GiB (CUDA events): the link the
    end-to-end number moves its reads and results over."""
    import torch
    n = 1 << 30
    h = torch.empty(n, dtype=torch.uint8).pin_memory()
    d = torch.empty(n, dtype=torch.uint8, device=device)
    out = {}
    for name, dst, src in (("h2d_gbs", d, h), ("d2h_gbs", h, d)):
        dst.copy_(src, non_blocking=True)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(3):
            dst.copy_(src, non_blocking=True)
        e1.record()
        torch.cuda.synchronize()
        out[name] = 3 * n / (e0.elapsed_time(e1) / 1000.0) / 1e9
    del h, d
    return out


def host_cpu() -> dict:
    """CPU model and logical core count of the host."""
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                k = line.split(":", 1)[0].strip().lower()
                if k in ("model name", "cpu model", "hardware"):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    if model is None:   # Arm hosts name the core in lscpu, not in /proc/cpuinfo
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            for line in out.splitlines():
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    if model is None:
        import platform
        model = platform.processor() or platform.machine() or "unknown"
    return {"cpu_model": model, "nproc": os.cpu_count()}


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-i", str(self.gpu)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc is not None:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self) -> dict | None:
        rows = []
        for line in (self.out or "").splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append(dict(sm=float(parts[1]), smax=float(parts[2]),
                                 power=float(parts[3]) if parts[3] not in ("[N/A]", "N/A") else 0.0,
                                 hw=parts[5], hwt=parts[6], swt=parts[7], cap=parts[8]))
            except ValueError:
                continue
        if not rows:
            return None
        busy = [r for r in rows if r["power"] > 0.5 * max(x["power"] for x in rows)] or rows
        reasons = set()
        for r in busy:
            for key, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"),
                              ("swt", "sw_thermal_slowdown"), ("cap", "sw_power_cap")):
                if r[key].lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(r["sm"] for r in busy),
                "sm_max_mhz": max(r["smax"] for r in rows), "reasons": sorted(reasons),
                "samples": len(rows), "samples_under_load": len(busy),
                "power_w_max": max(r["power"] for r in rows)}


def cpu_oracle_rate(bases, offsets, w, n_reads: int) -> dict:
    """The oracle as it stands, single-threaded, on the first n_reads reads:
    extraction, sequential Algorithm 3, sort + unique, Algorithm 2."""
    import oracle
    oracle.build()
    n_reads = min(n_reads, len(offsets) - 1)
    b = bases[:int(offsets[n_reads])]
    o = offsets[:n_reads + 1]
    t0 = time.perf_counter()
    ex = oracle.extract(b, o, w.K)
    filt = oracle.insert_sequential(ex.hi, ex.lo, w.K, w.m, w.alpha, w.nhash)
    dhi, dlo, _ = oracle.distinct(ex.hi, ex.lo)
    oracle.classify(filt, dhi, dlo, w.K, w.m, w.alpha, w.nhash, w.tau)
    dt = time.perf_counter() - t0
    del filt
    # untimed: Algorithm 1's sequential first-seen count (query 0 before the
    # insert) against the exact distinct count, on the first 2e6 K-mers
    n2 = min(ex.n, 2_000_000)
    first_seen = oracle.seq_distinct(ex.hi[:n2], ex.lo[:n2], w.K, w.m, w.alpha, w.nhash)
    exact = len(oracle.distinct(ex.hi[:n2], ex.lo[:n2])[1])
    return {"value": ex.n / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "seconds": round(dt, 3), **host_cpu(),
            "sample": f"first {n_reads:,} reads of the workload ({ex.n:,} K-mers): oracle "
                      f"extraction + sequential Algorithm 3 + sort/unique + Algorithm 2, "
                      f"single-threaded C on the host",
            "distinct_first_K_mers": {"kmers": n2, "exact": exact,
                                      "sequential_first_seen": first_seen}}


# reads per bounded oracle sample, per workload: about 10-20 s of one host core
CPU_READS = {"tiny": 2_000, "single": 150_000, "repeats": 40_000, "repeats55": 40_000}
REF_READS = {"tiny": 2_000, "single": 25_000, "repeats": 10_000, "repeats55": 10_000}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(x: float, device) -> float:
    """Largest value of x over all ranks (identity without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def l2_note(countbf_bytes: int, input_bytes: int, l2_bytes: int) -> str:
    """How the timed steps stand to an L2 of l2_bytes: what the flush between
    them does and which of the step's data can stay resident."""
    flush = (f"{L2_FLUSH_BYTES >> 20} MiB buffer written between timed steps, outside the "
             f"per-step CUDA events; L2 {l2_bytes / 2**20:.0f} MiB (device properties)")
    if countbf_bytes * 2 <= l2_bytes:
        return (f"{flush}; the {countbf_bytes / 2**20:.1f} MiB countBF is L2-resident within a "
                "step by design (the L2-atomic regime); the flush evicts it between steps")
    if countbf_bytes <= 2 * l2_bytes:
        return (f"{flush}; the {countbf_bytes / 2**20:.0f} MiB countBF is about the size of "
                f"L2, the {input_bytes / 1e9:.2f} GB of inputs larger")
    return f"{flush}; inputs ({input_bytes / 1e9:.2f} GB) and countBF larger than L2"


def whole_job_rate(units_per_rank_step: int, steps: int, world: int, slowest_s: float) -> float:
    """Units all ranks processed divided by the slowest rank's time (weak scaling:
    every rank processes its own sample of the same size)."""
    return units_per_rank_step * steps * world / slowest_s


def run_reference(args) -> None:
    world, rank, _ = dist_setup()
    if rank != 0:
        return
    w = readsim.WORKLOADS[args.workload]
    sample = args.ref_reads or REF_READS.get(args.workload, 25_000)
    wl = readsim.scaled(args.workload, sample)
    bases, offsets = wl.generate()
    import oracle
    oracle.build()
    rates = []
    for i in range(args.warmup + args.steps):
        r = cpu_oracle_rate(bases, offsets, w, sample)
        if i >= args.warmup:
            rates.append(r)
    secs = sum(r["seconds"] for r in rates)
    kmers = sum(r["value"] * r["seconds"] for r in rates)
    value = kmers / secs
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000 * secs / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": describe(w), "sample_reads_per_step": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             **host_cpu(), "sample": rates[0]["sample"] + ", per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def time_workload(name: str, args, bases, offsets, d_bases, d_offsets, flush, clock_dev,
                  world: int, e2e: bool) -> dict:
    """Warm-up and timed steps of one workload on the already resident reads;
    optionally the end-to-end steps from pinned host buffers."""
    import torch
    import torch.distributed as dist

    import paper_2305_07545_gb300 as kc

    w = readsim.WORKLOADS[name]
    if args.counters:
        import dataclasses
        w = dataclasses.replace(w, m=args.counters)
    dev = torch.cuda.current_device()
    nreads = len(offsets) - 1
    lens = np.diff(offsets.astype(np.int64))
    windows_expected = int(np.maximum(lens - w.K + 1, 0).sum())
    stream = torch.cuda.current_stream()
    bf = kc.CountBF(w.K, w.m, w.alpha, w.nhash, w.tau, stream=stream.cuda_stream)

    def step():
        bf.reset()
        bf.insert(d_bases, d_offsets)
        bf.classify()

    for _ in range(args.warmup):
        step()
    st = bf.stats()
    inserted, distinct, trusted = st["inserted"], st["distinct"], st["trustworthy"]
    assert st["windows"] == windows_expected, "window count differs from the read lengths"
    stats_cost = bf.stats()["launches"] - st["launches"]   # kernels one stats call launches

    ev_s = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev_e = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    insert_ms, classify_ms = [], []
    launches = 0
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    with ClockSampler(clock_dev) as clk:
        for i in range(args.steps):
            flush.zero_()
            l0 = bf.stats()["launches"]
            ev_s[i].record(stream)
            step()
            ev_e[i].record(stream)
            s = bf.stats()
            launches += s["launches"] - l0 - stats_cost   # less the stats call's own
            insert_ms.append(s["insert_ms"])
            classify_ms.append(s["classify_ms"])
            assert (s["inserted"], s["distinct"], s["trustworthy"]) == (inserted, distinct, trusted)
        torch.cuda.synchronize()
    step_ms = [a.elapsed_time(b) for a, b in zip(ev_s, ev_e)]
    total_ms = max_over_ranks(sum(step_ms), dev)
    if world > 1:
        dist.barrier()
    out = {"workload": w, "inserted": inserted, "distinct": distinct, "trusted": trusted,
           "total_ms": total_ms, "insert_ms": statistics.mean(insert_ms),
           "step_ms": {"min": min(step_ms), "median": statistics.median(step_ms),
                       "max": max(step_ms)},
           "classify_ms": statistics.mean(classify_ms), "launches": launches,
           "clocks": clk.summary(), "e2e": None,
           "device_bytes": bf.stats()["device_bytes"]}

    # end to end through the public API with host (pinned) buffers
    if e2e:
        h_bases = torch.from_numpy(bases).pin_memory()
        h_offsets = torch.from_numpy(offsets.view(np.int64)).pin_memory()
        cap = max(distinct, 1)
        kw = 1 if w.K <= 32 else 2   # 64-bit words per key
        h_tr = torch.empty(cap * kw, dtype=torch.int64).pin_memory()
        h_er = torch.empty(cap * kw, dtype=torch.int64).pin_memory()

        split = {"reset_insert": 0.0, "classify": 0.0, "queue_lists": 0.0, "final_sync": 0.0}

        def e2e_step():
            t = time.perf_counter()
            bf.reset()
            kc.kmerco_insert(bf.h, h_bases, h_offsets, nreads)
            t1 = time.perf_counter()
            bf.classify()   # waits for the insert (it reads the distinct count)
            t2 = time.perf_counter()
            # both lists go to pinned host memory on the result stream, beside
            # the next step's insert; the next classify waits for them
            nt, ne = kc.kmerco_get_lists_async(bf.h, h_tr, cap, h_er, cap)
            t3 = time.perf_counter()
            split["reset_insert"] += t1 - t
            split["classify"] += t2 - t1
            split["queue_lists"] += t3 - t2
            return nt, ne

        for _ in range(max(1, args.warmup // 2)):
            e2e_step()
        kc.kmerco_sync(bf.h)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        for k in split:
            split[k] = 0.0
        t0 = time.perf_counter()
        for _ in range(args.steps):
            nt, ne = e2e_step()
        ts = time.perf_counter()
        kc.kmerco_sync(bf.h)   # the last step's lists are in host memory
        torch.cuda.synchronize()
        split["final_sync"] = time.perf_counter() - ts
        e2e_s = max_over_ranks(time.perf_counter() - t0, dev)
        assert nt == trusted and nt + ne == distinct
        out["e2e"] = {"value": whole_job_rate(inserted, args.steps, world, e2e_s), "unit": UNIT,
                      "h2d_bytes_per_step": int(bases.nbytes + offsets.nbytes),
                      "d2h_bytes_per_step": int(8 * kw * distinct),
                      "note": "reset + insert from pinned host reads + classify + copy of the "
                              "trustworthy and erroneous key lists to pinned host memory "
                              "(queued on the handle's result stream, overlapping the next "
                              "step's insert; the last step's copies end inside the timed "
                              "region); wall clock",
                      "host_ms_per_step": {k: 1000.0 * v / args.steps for k, v in split.items()}}
        del h_bases, h_offsets, h_tr, h_er
    bf.close()
    return out


def workload_roofline(r: dict, name: str, input_bytes: int, peak: float, peak_src: str,
                      peaks: dict | None, full_size: bool) -> dict:
    w = r["workload"]
    kw = 1 if w.K <= 32 else 2
    traffic = recorded_traffic(name) if full_size else None
    roof = roofline_of_insert(r["inserted"], w.nhash, kw, input_bytes, r["insert_ms"], peak,
                              traffic)
    roof["insert_share_of_step"] = r["insert_ms"] / (r["total_ms"] / r["steps"])
    roof["peak_source"] = peak_src + "; frac of measured"
    if peaks:
        cas = peaks["512KiB"]["random_cas_per_s"]
        roof["l2_atomic"] = l2_atomic_roofline(r["inserted"], w.nhash, r["insert_ms"], cas)
        if w.m * w.alpha // 8 <= (1 << 20):   # L2-resident countBF: the update is L2-atomic bound
            l2 = roof.pop("l2_atomic")
            l2["hbm_view"] = roof
            roof = l2
    return roof


def run_sharded(args) -> None:
    """N > 1 ranks count ONE sample: rank r inserts read shard r into a
    full-size countBF, the countBFs are merged by a chunked all-to-all with a
    saturating merge and gathered back, and the distinct keys go to the rank
    owning their key range (paper_2305_07545_gb300.shard).  The total work is
    fixed, so the scaling is strong."""
    import torch
    import torch.distributed as dist
    from paper_2305_07545_gb300 import shard

    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    dist.init_process_group("nccl")
    name = args.workload
    w = readsim.WORKLOADS[name]
    wl = readsim.scaled(name, args.reads or w.reads.n_reads)   # the same sample on every rank
    bases, offsets = wl.generate()
    dev = torch.cuda.current_device()
    sb, so = shard.shard_of(bases, offsets, rank, world)
    d_shard = (torch.from_numpy(sb).to(dev), torch.from_numpy(so.view(np.int64)).to(dev))
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    comm = shard.TorchComm()
    eng = shard.LibraryEngine(w.K, args.counters or w.m, w.alpha, w.nhash, w.tau, device=dev)

    def step():
        eng.local.reset()
        res = shard.count_sharded(eng, comm, shard=d_shard)
        res.owner.close()
        return res

    for _ in range(args.warmup):
        res = step()
    times = []
    torch.cuda.synchronize()
    dist.barrier()
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            res = step()
            torch.cuda.synchronize()
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
    total_ms = max_over_ranks(sum(times), dev)
    dist.barrier()
    if rank == 0:
        line = {"metric": METRIC, "value": res.inserted * args.steps / (total_ms / 1000.0),
                "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "strong", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
                "config": {"workload": describe(wl), "K": w.K, "m": args.counters or w.m,
                           "kmers_per_step": res.inserted, "distinct": res.distinct,
                           "trustworthy": res.trustworthy,
                           "parallelism": f"one sample sharded over {world} GPUs: read shards, "
                                          "countBF chunks all-to-all + saturating merge + "
                                          "all-gather, distinct keys all-to-all by key range",
                           "l2": "256 MiB buffer written between timed steps"},
                "gpu_launches": None, "clocks": clk.summary(),
                "note": "wall time of the whole sharded step between device synchronisations, "
                        "timed with CUDA events; slowest rank"}
        print(json.dumps(line), flush=True)
    eng.close()
    dist.destroy_process_group()


def run_ours(args) -> None:
    import torch
    import torch.distributed as dist

    world, rank, local = dist_setup()
    name = args.workload
    w = readsim.WORKLOADS[name]
    # reads are generated (threads on the host) before CUDA starts
    wl = readsim.scaled(name, args.reads or w.reads.n_reads, seed_offset=rank)
    t_gen = time.perf_counter()
    bases, offsets = wl.generate()
    t_gen = time.perf_counter() - t_gen
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    clock_dev = dev if world == 1 else local

    peaks = None if args.no_peaks else measure_peaks(dev)
    link = None if args.no_e2e else host_link(dev)
    d_bases = torch.from_numpy(bases).to(dev)
    d_offsets = torch.from_numpy(offsets.view(np.int64)).to(dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    torch.cuda.synchronize()

    full_size = not args.reads and not args.counters
    input_bytes = bases.nbytes + offsets.nbytes
    peak, peak_src = measured_peak()
    r = time_workload(name, args, bases, offsets, d_bases, d_offsets, flush, clock_dev, world,
                      e2e=not args.no_e2e)
    r["steps"] = args.steps
    value = whole_job_rate(r["inserted"], args.steps, world, r["total_ms"] / 1000.0)

    secondary = None
    sec_name = SECONDARY.get(name) if not args.no_secondary else None
    if sec_name:
        r2 = time_workload(sec_name, args, bases, offsets, d_bases, d_offsets, flush, clock_dev,
                           world, e2e=False)
        r2["steps"] = args.steps
        w2 = r2["workload"]
        secondary = {
            "workload": describe(readsim.scaled(sec_name, len(offsets) - 1, seed_offset=rank)),
            "K": w2.K, "value": whole_job_rate(r2["inserted"], args.steps, world,
                                                r2["total_ms"] / 1000.0),
            "unit": UNIT, "ms_per_step": r2["total_ms"] / args.steps,
            "kmers_per_step_per_gpu": r2["inserted"], "distinct_per_gpu": r2["distinct"],
            "trustworthy_per_gpu": r2["trusted"],
            "phases": {"insert_ms": r2["insert_ms"], "classify_ms": r2["classify_ms"],
                       "step_ms": r2["step_ms"]},
            "roofline": workload_roofline(r2, sec_name, input_bytes, peak, peak_src, peaks,
                                          full_size),
            "gpu_launches": r2["launches"], "clocks": r2["clocks"],
            "device_bytes": r2["device_bytes"]}
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    roofline = workload_roofline(r, name, input_bytes, peak, peak_src, peaks, full_size)
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        cpu = cpu_oracle_rate(bases, offsets, w, args.cpu_reads or CPU_READS.get(name, 50_000))

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["total_ms"] / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic",
            "config": {"workload": describe(wl), "K": w.K, "m": r["workload"].m,
                       "counter_bits": w.alpha,
                       "nhash": w.nhash, "tau": w.tau, "reads_per_gpu": len(offsets) - 1,
                       "kmers_per_step_per_gpu": r["inserted"], "distinct_per_gpu": r["distinct"],
                       "trustworthy_per_gpu": r["trusted"],
                       "parallelism": f"{world} independent samples, one per GPU",
                       "l2": l2_note(w.m * w.alpha // 8, input_bytes,
                                     getattr(torch.cuda.get_device_properties(dev),
                                             "L2_cache_size", 126 << 20)),
                       "device_bytes": r["device_bytes"],
                       "read_generation_s": round(t_gen, 1)},
            "roofline": roofline, "cpu_baseline": cpu,
            "e2e": dict(r["e2e"], host_link=link) if r["e2e"] else None,
            "phases": {"insert_ms": r["insert_ms"], "classify_ms": r["classify_ms"],
                       "insert_kmers_per_s": r["inserted"] / (r["insert_ms"] / 1000.0),
                       "classify_distinct_per_s": r["distinct"] / (r["classify_ms"] / 1000.0),
                       "step_ms": r["step_ms"]},
            "secondary": secondary,
            "l2_atomic_peak": None if not peaks else {
                "random_cas_per_s": {k: v["random_cas_per_s"] for k, v in peaks.items()},
                "source": "kmerco_peak_random_cas: random 64-bit load + atomicCAS, measured "
                          "in this run"},
            "random_read_peak": None if not peaks else {
                "random_read_per_s": {k: v["random_read_per_s"] for k, v in peaks.items()},
                "source": "kmerco_peak_random_read: random 8-byte loads, measured in this run"},
            "gpu_launches": r["launches"], "clocks": r["clocks"]}
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


# ---------------------------------------------------------------- batched
def _batch_sample(args):
    """One sample of the batched workload (runs in a worker process)."""
    i, n_reads, seed = args
    st = readsim.Stream(seed)
    g = readsim.genome(1_000_000, 0.5, st)
    err = 0.005 + 0.015 * float(st.uniform(1)[0])
    b, o = readsim.sample_reads(g, readsim.ReadModel(n_reads, (50, 300), sub=err), st)
    return i, b, o, err


def batched_workload(n_samples: int, scale: float, seed: int = 4001):
    """Read counts log-normal (median 1.4e5, sigma 1.2) clipped to [1e4, 2e6],
    times `scale`; lengths U[50, 300]; 0.5-2% substitutions; a 1 Mb genome
    per sample."""
    import multiprocessing as mp
    st = readsim.Stream(seed)
    z = np.sqrt(-2 * np.log(st.uniform(n_samples) + 1e-300)) * np.cos(2 * np.pi * st.uniform(n_samples))
    reads = np.clip(np.exp(np.log(1.4e5) + 1.2 * z), 1e4, 2e6)
    reads = np.maximum((reads * scale).astype(np.int64), 1)
    jobs = [(i, int(reads[i]), seed * 1000 + i) for i in range(n_samples)]
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        out = sorted(pool.map(_batch_sample, jobs), key=lambda x: x[0])
    return out


def batch_groups(sizes: list[int], limit: int) -> list[list[int]]:
    """Consecutive groups of sample indices whose summed device bytes stay
    within `limit` (a sample larger than the limit forms its own group)."""
    groups, cur, acc = [], [], 0
    for i, n in enumerate(sizes):
        if cur and acc + n > limit:
            groups.append(cur)
            cur, acc = [], 0
        cur.append(i)
        acc += n
    if cur:
        groups.append(cur)
    return groups


def run_batched(args) -> None:
    samples = batched_workload(args.samples, args.batch_scale)
    import torch
    import paper_2305_07545_gb300 as kc
    torch.cuda.set_device(0)
    K, nhash, alpha, tau = 31, 4, 4, 3
    stream = torch.cuda.Stream()
    # per sample: countBF size, windows and the library's device-memory bound
    specs, need = [], []
    for _, b, o, err in samples:
        lens = np.diff(o.astype(np.int64))
        w = int(np.maximum(lens - K + 1, 0).sum())
        m = int(2 * (1_000_000 + w * min(1.0, err * K)))
        specs.append((m, w))
        need.append(kc.kmerco_estimate_bytes(K, m, alpha, nhash, tau, len(o) - 1, int(o[-1]), w,
                                             False, update_mode=kc.UPDATE_ATOMIC) + b.nbytes + o.nbytes)
    # all samples at once when they fit the device, else consecutive groups
    groups = batch_groups(need, args.batch_mem)

    def timed(fn, steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    t_batched = t_single = ins_batched = ins_single = 0.0
    inserted = windows = reads = 0
    infos = []
    for g in groups:
        filters, dev, nreads = [], [], []
        for i in g:
            _, b, o, _ = samples[i]
            filters.append(kc.CountBF(K, specs[i][0], alpha, nhash, tau,
                                      stream=stream.cuda_stream, update_mode=kc.UPDATE_ATOMIC))
            dev.append((torch.from_numpy(b).cuda(), torch.from_numpy(o.view(np.int64)).cuda()))
            nreads.append(len(o) - 1)
            windows += specs[i][1]
        torch.cuda.synchronize()
        batch = kc.Batch(filters)
        bases = [d[0] for d in dev]
        offs = [d[1] for d in dev]

        def batched_step():
            kc.kmerco_batch_insert(batch.b, bases, offs, nreads, reset=True)
            batch.classify()

        def per_sample_step():
            for f, (bb, oo) in zip(filters, dev):
                f.reset()
                f.insert(bb, oo)
                f.classify()

        def per_sample_insert():
            for f, (bb, oo) in zip(filters, dev):
                f.reset()
                f.insert(bb, oo)

        for _ in range(args.warmup):
            batched_step()
        infos.append(batch.info())
        t_batched += timed(batched_step, args.steps)
        ins_batched += timed(lambda: kc.kmerco_batch_insert(batch.b, bases, offs, nreads, True),
                             args.steps)
        for _ in range(max(1, args.warmup // 2)):
            per_sample_step()
        t_single += timed(per_sample_step, args.steps)
        ins_single += timed(per_sample_insert, args.steps)
        inserted += sum(f.stats()["inserted"] for f in filters)
        reads += sum(nreads)
        batch.close()
        for f in filters:
            f.close()
        del dev, bases, offs
        torch.cuda.synchronize()
    line = {"metric": METRIC, "value": inserted / (t_batched / 1000.0), "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_batched,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic",
            "config": {"workload": f"batched: {len(samples)} samples, reads log-normal "
                                   f"(median 1.4e5, sigma 1.2, clipped 1e4..2e6) x {args.batch_scale}, "
                                   f"50-300 bp, 0.5-2% substitutions, 1 Mb genome each, K=31, "
                                   f"4-bit counters at 8 bits per expected distinct K-mer, 4 hashes, "
                                   f"tau=3",
                       "reads": int(reads), "kmers_per_step": int(inserted),
                       "windows": int(windows),
                       "groups": [len(g) for g in groups],
                       "group_note": "samples whose summed device-memory bound exceeds "
                                     f"{args.batch_mem >> 30} GiB run as consecutive batches; a "
                                     "step is one pass over all groups",
                       "schedule": infos},
            "per_sample_path": {"value": inserted / (t_single / 1000.0), "ms_per_step": t_single},
            "insert_only_ms": {"batched": ins_batched, "per_sample": ins_single}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- serving
def run_serving(args) -> None:
    samples = batched_workload(args.jobs, args.batch_scale, seed=5001)
    import torch
    from paper_2305_07545_gb300 import serve
    torch.cuda.set_device(0)
    K, nhash, alpha, tau = 31, 4, 4, 3
    jobs = []
    for i, b, o, err in samples:
        w = serve.window_count(o, K)
        exp = 1_000_000 + w * min(1.0, err * K)
        m = 1 << int(np.ceil(np.log2(2 * exp)))      # power-of-two classes share pooled handles
        jobs.append(serve.Job(torch.from_numpy(b).pin_memory(),
                              torch.from_numpy(o.view(np.int64)).pin_memory(),
                              K=K, m=m, counter_bits=alpha, nhash=nhash, tau=tau, name=f"job{i}"))
    kmers = None

    def run(arrivals):
        with serve.Server(hbm_budget=args.hbm_budget, slots=args.slots) as srv:
            for j in jobs[:min(4, len(jobs))]:          # warm the handle pool
                srv.submit(j).result()
            t0 = time.perf_counter()
            res = serve.replay(srv, jobs, arrivals)
            wall = time.perf_counter() - t0
            return res, wall, srv.max_running

    res, wall, peak = run([0.0] * len(jobs))
    kmers = sum(r.inserted for r in res)
    capacity = len(jobs) / wall
    rates = []
    st = readsim.Stream(6001)
    for factor in (0.25, 0.5, 1.0, 2.0, 4.0):
        lam = factor * capacity
        gaps = -np.log(st.uniform(len(jobs)) + 1e-300) / lam
        arrivals = np.cumsum(gaps) - gaps[0]
        r, w, pk = run(list(arrivals))
        lat = np.array([x.latency for x in r]) * 1000.0
        rates.append({"load": factor, "arrivals_per_s": lam, "kmers_per_s": kmers / w,
                      "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                      "max_concurrent": pk})
    line = {"metric": METRIC, "value": kmers / wall, "unit": UNIT, "n_gpus": 1, "steps": 1,
            "warmup": 1, "ms_per_step": wall * 1000.0, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": f"serving: {len(jobs)} counting jobs drawn from the batched "
                                   f"workload's sizes (x {args.batch_scale}), K=31, 4 hashes, "
                                   f"tau=3, Poisson arrivals, HBM budget {args.hbm_budget >> 30} GB, "
                                   f"{args.slots} slots",
                       "kmers": int(kmers), "saturated_jobs_per_s": capacity,
                       "saturated_max_concurrent": peak},
            "serving": rates}
    print(json.dumps(line), flush=True)


def main(argv=None) -> None:
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="repeats",
                    choices=sorted(readsim.WORKLOADS) + ["batched", "serving"])
    ap.add_argument("--jobs", type=int, default=64, help="serving workload: jobs")
    ap.add_argument("--slots", type=int, default=16, help="serving workload: concurrent jobs")
    ap.add_argument("--hbm-budget", type=int, default=120 << 30,
                    help="serving workload: device bytes the jobs may hold")
    ap.add_argument("--samples", type=int, default=256, help="batched workload: samples")
    ap.add_argument("--batch-scale", type=float, default=1.0,
                    help="batched workload: factor on every sample's read count")
    ap.add_argument("--batch-mem", type=int, default=160 << 30,
                    help="batched workload: device bytes one group of samples may need")
    ap.add_argument("--cpu-reads", type=int, default=0,
                    help="reads in the bounded CPU-oracle sample (default: per workload)")
    ap.add_argument("--ref-reads", type=int, default=0,
                    help="reads per step of the reference (oracle) arm (default: per workload)")
    ap.add_argument("--reads", type=int, default=0,
                    help="reads per GPU (default: the workload's own count; smaller for profiling)")
    ap.add_argument("--counters", type=int, default=0,
                    help="countBF counters (default: the workload's own; smaller for profiling)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-secondary", action="store_true",
                    help="skip the 55-mer count of the same reads after the headline workload")
    ap.add_argument("--no-peaks", action="store_true",
                    help="skip the random-access peak measurements")
    ap.add_argument("--replicas", action="store_true",
                    help="with N > 1: every rank counts its own sample instead of one "
                         "sample sharded over all ranks")
    args = ap.parse_args(argv)
    if args.warmup < 3 and args.impl == "ours":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "serving":
        run_serving(args)
    elif dist_setup()[0] > 1 and not args.replicas:
        run_sharded(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
