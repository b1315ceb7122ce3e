"""Benchmark: K-mer insertions per second of the whole countBF path on GB300.

One step = one pass of the full hot path over one sample: reset the countBF,
insert every read (pack, canonicalise, hash, saturating counter updates,
distinct-key set), then classify (sort the distinct keys, QcountBF-II per
key, split at tau).  value = K-mer windows inserted / step time.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload single]
    python bench.py --impl reference ...   # the CPU oracle on a bounded sample

Under torchrun (N > 1) every rank counts its own sample (a different seed)
on its own GPU; nothing is exchanged, so scaling is weak and value is the sum
of all ranks' windows over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
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
PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "insert_kernel_single.md")
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
    h = hashlib.sha256()
    for f in INSERT_SOURCES:
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_peak() -> tuple[float, str]:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            v = float(json.load(f)["hbm_gbs"])
        return v, "measured (MEASURED_PEAKS.json hbm_gbs, STREAM-style copy)"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback (6.8 TB/s earlier GB300 copy measurement)"


def recorded_traffic() -> float | None:
    """DRAM bytes per insert launch from the committed ncu summary, if it was
    taken on the current insert-kernel source."""
    try:
        with open(PROFILE_SUMMARY) as f:
            for line in f:
                if line.startswith("traffic_record"):
                    kv = dict(p.split("=", 1) for p in line.split()[1:])
                    if kv.get("source_sha") == source_sha():
                        return float(kv["dram_bytes_per_launch"])
    except Exception:
        pass
    return None


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
    return {"value": ex.n / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "seconds": round(dt, 3),
            "sample": f"first {n_reads:,} reads of the workload ({ex.n:,} K-mers): oracle "
                      f"extraction + sequential Algorithm 3 + sort/unique + Algorithm 2, "
                      f"single-threaded C on the host"}


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


def whole_job_rate(units_per_rank_step: int, steps: int, world: int, slowest_s: float) -> float:
    """Units all ranks processed divided by the slowest rank's time (weak scaling:
    every rank processes its own sample of the same size)."""
    return units_per_rank_step * steps * world / slowest_s


def run_reference(args) -> None:
    world, rank, _ = dist_setup()
    if rank != 0:
        return
    w = readsim.WORKLOADS[args.workload]
    sample = args.ref_reads
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
                             "sample": rates[0]["sample"] + ", per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args) -> None:
    import torch
    import torch.distributed as dist

    import paper_2305_07545_gb300 as kc

    world, rank, local = dist_setup()
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    w = readsim.WORKLOADS[args.workload]
    wl = readsim.scaled(args.workload, args.reads or w.reads.n_reads, seed_offset=rank)
    bases, offsets = wl.generate()
    nreads = len(offsets) - 1
    lens = np.diff(offsets.astype(np.int64))
    windows_expected = int(np.maximum(lens - w.K + 1, 0).sum())

    stream = torch.cuda.current_stream()
    d_bases = torch.from_numpy(bases).to(dev)
    d_offsets = torch.from_numpy(offsets.view(np.int64)).to(dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    torch.cuda.synchronize()

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

    ev_s = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev_e = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    insert_ms = []
    launches = 0
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    with ClockSampler(dev if world == 1 else local) as clk:
        for i in range(args.steps):
            flush.zero_()
            l0 = bf.stats()["launches"]
            ev_s[i].record(stream)
            step()
            ev_e[i].record(stream)
            s = bf.stats()
            launches += s["launches"] - l0 - 1   # the stats call itself launches one kernel
            insert_ms.append(s["insert_ms"])
            assert (s["inserted"], s["distinct"], s["trustworthy"]) == (inserted, distinct, trusted)
        torch.cuda.synchronize()
    step_ms = [a.elapsed_time(b) for a, b in zip(ev_s, ev_e)]
    total_ms = max_over_ranks(sum(step_ms), dev)
    if world > 1:
        dist.barrier()
    value = whole_job_rate(inserted, args.steps, world, total_ms / 1000.0)

    # end to end through the public API with host (pinned) buffers
    e2e = None
    if not args.no_e2e:
        h_bases = torch.from_numpy(bases).pin_memory()
        h_offsets = torch.from_numpy(offsets.view(np.int64)).pin_memory()
        cap = max(distinct, 1)
        h_tr = torch.empty(cap, dtype=torch.int64).pin_memory()
        h_er = torch.empty(cap, dtype=torch.int64).pin_memory()

        def e2e_step():
            bf.reset()
            kc.kmerco_insert(bf.h, h_bases, h_offsets, nreads)
            bf.classify()
            nt = kc.kmerco_get_trusted(bf.h, h_tr, cap)
            ne = kc.kmerco_get_erroneous(bf.h, h_er, cap)
            return nt, ne

        for _ in range(max(1, args.warmup // 2)):
            e2e_step()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            nt, ne = e2e_step()
        torch.cuda.synchronize()
        e2e_s = max_over_ranks(time.perf_counter() - t0, dev)
        assert nt == trusted and nt + ne == distinct
        e2e = {"value": whole_job_rate(inserted, args.steps, world, e2e_s), "unit": UNIT,
               "h2d_bytes_per_step": int(bases.nbytes + offsets.nbytes),
               "d2h_bytes_per_step": int(8 * distinct),
               "note": "reset + insert from pinned host reads + classify + copy of the "
                       "trustworthy and erroneous key lists to pinned host memory; wall clock"}

    bf.close()
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    peak, peak_src = measured_peak()
    kmer_bytes = 16 * w.nhash + 8                 # k_h cell RMWs + one distinct-set probe
    launch_bytes = bases.nbytes + offsets.nbytes + inserted * kmer_bytes + distinct * 16
    avg_insert_ms = statistics.mean(insert_ms)
    achieved = launch_bytes / (avg_insert_ms / 1000.0) / 1e9
    traffic = recorded_traffic()
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic,
                "kernel": "insert_kernel (fused pack/canonical/hash/countBF update/distinct set)",
                "algorithmic_bytes_per_launch": int(launch_bytes),
                "avg_launch_ms": avg_insert_ms, "insert_share_of_step": avg_insert_ms / (total_ms / args.steps),
                "peak_source": peak_src}

    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        cpu = cpu_oracle_rate(bases, offsets, w, args.cpu_reads)

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic",
            "config": {"workload": describe(wl), "K": w.K, "m": w.m, "counter_bits": w.alpha,
                       "nhash": w.nhash, "tau": w.tau, "reads_per_gpu": nreads,
                       "kmers_per_step_per_gpu": inserted, "distinct_per_gpu": distinct,
                       "trustworthy_per_gpu": trusted,
                       "parallelism": f"{world} independent samples, one per GPU",
                       "l2": "256 MiB buffer written between timed steps, outside the "
                             "per-step CUDA events; countBF 128 MiB + distinct set > L2"},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": launches, "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main(argv=None) -> None:
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="single", choices=sorted(readsim.WORKLOADS))
    ap.add_argument("--cpu-reads", type=int, default=150_000,
                    help="reads in the bounded CPU-oracle sample")
    ap.add_argument("--ref-reads", type=int, default=25_000,
                    help="reads per step of the reference (oracle) arm")
    ap.add_argument("--reads", type=int, default=0,
                    help="reads per GPU (default: the workload's own count; smaller for profiling)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args(argv)
    if args.warmup < 3 and args.impl == "ours":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
