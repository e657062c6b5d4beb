"""Benchmark: keys/s sorted + indexed on one GB300, compressed key sort vs a
full-key sort on the same kernels, with the HBM roofline fraction of the
dominant kernel (the onesweep radix pass of the plain path; the partition
passes or the bucket sorts of the learned path).

A step is one index rebuild from stored DS-metadata (Sec. 5 of the paper):
extract the compressed keys with the stored D-bitmap, sort the (compressed
key, row id) pairs, bulk-load the tree and recompute the D-bitmap.  Inputs
are resident in HBM when the timed region starts; they are larger than L2,
except the 1M-key configuration, between whose timed steps a 256 MiB buffer
is written (outside the timed events).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload all|urls64m|int1m|zipf256m|dna200m|table16m|zipfsweep|...]

The default (all) measures the five benchmark configurations in one line:
the headline is the largest single-GPU one, 200M DNA keys through the
learned partition with the fanout-256 bulk load (config C5); 1M uint64 keys
(C1), 64M URL keys (C2), the 16M-row table of six indexes (C3) and 256M Zipf
keys (C4) are sub-records, each with the plain, learned and full-key times.

Under torchrun (N > 1) every rank rebuilds its own replica of the workload
(the path has no exchange step); value is the keys of all ranks over the
slowest rank's time.  ``--impl reference`` times the CPU oracle on a bounded
sample of the same workload (rank 0 only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import platform
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "keys/sec sorted+indexed (1 GB300) and % of HBM roofline, compressed vs full-key sort"
FALLBACK_HBM_GBS = 6800.0
SPEC_HBM_GBS = 7900.0  # nominal HBM3e bandwidth of a GB300, for context beside the measured peak
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "kernel_traffic.json")

WORKLOADS = {
    # name: (description, n, generator, fanout, cpu sample rows, path the headline value uses)
    "urls64m": ("64M 32-byte URL keys ('http://www.' + Zipf(1.1) name over 100k + '.com/' + 0-16 path chars), "
                "fanout 64, compressed keys packed to 128 bits, plain path", 64 * 2**20, "urls", 64, 8_000_000,
                "plain"),
    "urls8m": ("8M 32-byte URL keys (the 64M workload's generator, first 8M rows), fanout 64; profiling size",
               8 * 2**20, "urls", 64, 2_000_000, "plain"),
    "urls32m": ("32M 32-byte URL keys (the 64M workload's generator, first 32M rows), fanout 64; profiling size "
                "for one-launch DRAM counters of a radix pass", 32 * 2**20, "urls", 64, 2_000_000, "plain"),
    "zipf256m": ("256M uint64 keys, Zipf(0.9) over 2^40 values under a constant 12-bit tag, learned partition "
                 "(1% sample, 16-unit CDF model, about 32K key-range buckets) vs plain radix, fanout 64",
                 256 * 2**20, "zipf", 64, 8_000_000, "learned"),
    "dna200m": ("200M 32-byte {A,C,G,T} keys, 20% sharing one of 65536 random 24-char prefixes, learned partition "
                "+ bulk load with fanout 256", 200_000_000, "dna", 256, 4_000_000, "learned"),
    "dna20m": ("20M 32-byte {A,C,G,T} keys (the 200M workload's generator, first 20M rows), learned partition, "
               "fanout 256; profiling size", 20_000_000, "dna", 256, 2_000_000, "learned"),
    "zipfsweep": ("the Zipf(s, n, m) datasets of Table 4 (10M keys each: 8-byte words of m fixed characters and "
                  "Zipf(s, 26) lowercase letters), compressed-key vs full-key rebuild, fanout 64", 10_000_000,
                  "zipfletters", 64, 200_000, "plain"),
    "int1m": ("1M uint64 keys with 24 seeded varying bit positions, fanout 64", 1_000_000, "int", 64, 1_000_000,
              "plain"),
    "table16m": ("one table of 16M rows with 6 indexes of key widths 4, 8, 12, 16, 32, 64 bytes (uint32 uniform, "
                 "uint64 sequential+noise, Zipf-prefixed strings), all rebuilt in one graph-captured batched launch, "
                 "digit width autotuned per index", 16 * 2**20, "table", 64, 1_000_000, "batched"),
}
TABLE_FANOUTS = [64, 64, 64, 64, 256, 256]
DATA_NOTE = {
    "urls": "synthetic (seeded generator standing in for the paper's URL tables)",
    "dna": "synthetic (seeded generator standing in for the paper's genome-string table)",
    "zipf": "synthetic (seeded Zipf generator, the learned-partition workload)",
    "int": "synthetic (seeded generator standing in for a low-entropy integer key column)",
}


def gen_keys(kind: str, n: int):
    import synth
    if kind == "urls":
        return synth.urls(n, synth.BASE_SEED + 2)
    if kind == "int":
        return synth.varying_bits_u64(n, synth.BASE_SEED + 1)[0]
    if kind == "dna":
        return synth.dna(n, synth.BASE_SEED + 5)
    if kind == "zipf":
        return synth.zipf_tagged_u64(n, synth.BASE_SEED + 4, 0.9)
    if kind == "zipfletters":   # Zipf(1.5, 64, 0) of Table 4, the sweep's representative
        return synth.zipf_letters(n, synth.BASE_SEED + 30, 64, 0, 1.5)
    raise ValueError(kind)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def file_sha(path: str) -> str:
    with open(path, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def max_over_ranks(times, world: int) -> np.ndarray:
    """Element-wise maximum of the ranks' timings (every rank gets it); the
    job is as slow as its slowest replica."""
    times = np.asarray(times, np.float64)
    if world <= 1:
        return times
    import torch
    import torch.distributed as dist
    t = torch.from_numpy(times.copy())
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.numpy()


def ncu_traffic(kernel: str, n: int, ck_words: int):
    """DRAM bytes per launch of `kernel` from the committed ncu summary
    (dram__bytes_read.sum + dram__bytes_write.sum of one launch), scaled to n
    keys, if the kernel's source file is unchanged since the capture and the
    key width matches; else None."""
    try:
        with open(TRAFFIC_FILE) as f:
            t = json.load(f)[kernel]
        if t.get("kernel_src_sha") != file_sha(os.path.join(ROOT, t["kernel_src"])) or t.get("ck_words") != ck_words:
            return None
        return t["dram_bytes_per_launch"] * n / t["n"]
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clock / throttle samples while the GPU is busy."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        rows = [l.strip().split(", ") for l in self.file.read().splitlines() if l.strip()]
        os.unlink(self.file.name)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                smax = float(r[2])
            except ValueError:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(nm)
        busy = [s for s in sm if smax and s > 0.3 * smax] or sm
        return {"sm_mhz": statistics.median(busy) if busy else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------- ours
def run_table(args, rank, world, local_rank, own_clocks=True):
    """The batched workload: every index of one table per step, one graph launch."""
    import torch
    import synth
    from paper_2009_11543_gb300 import build as b
    b.build()
    from paper_2009_11543_gb300 import ck, metrics, pipeline

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    desc, n, kind, fanout, cpu_rows, main_path = WORKLOADS[args.workload]
    cols_np = synth.table_columns(n, synth.BASE_SEED + 3)

    def as_tensor(c):
        return torch.from_numpy(c.view(np.int64) if c.dtype == np.uint64 else
                                (c.view(np.int32) if c.dtype == np.uint32 else c))
    hosts = [as_tensor(c).pin_memory() for c in cols_np]
    cols = [h.to(dev) for h in hosts]
    dmasks = [pipeline.first_build_dmask(c) for c in cols]
    cache = os.path.join(tempfile.gettempdir(), "ck_autotune_%d.txt" % os.getpid())
    B = pipeline.BatchedRebuild(cols, dmasks, TABLE_FANOUTS, cache_path=cache, tune_reps=3)
    seq = [pipeline.Rebuild(c, m, fanout=f, digit_bits=8) for c, m, f in zip(cols, dmasks, TABLE_FANOUTS)]
    full = [pipeline.Rebuild(c, pipeline.full_key_mask(8 * (c.shape[1] if c.dim() == 2 else c.element_size())),
                             fanout=f, digit_bits=8) for c, f in zip(cols, TABLE_FANOUTS)]
    stream = torch.cuda.current_stream()

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    def timed(fn, steps, warmup):
        for _ in range(warmup):
            fn()
        barrier()
        l0 = ck.ck_launch_count()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        barrier()
        return e0.elapsed_time(e1) / steps, ck.ck_launch_count() - l0

    clocks = ClockSampler(local_rank)
    if own_clocks:
        clocks.start()
        time.sleep(0.2)
    B.capture()
    graph_ms, graph_launches = timed(B.launch, args.steps, args.warmup)
    streams_ms, stream_launches = timed(B.run, args.steps, args.warmup)

    def seq_run():
        for r in seq:
            r.run()
    seq_ms, _ = timed(seq_run, args.steps, args.warmup)

    def full_run():
        for r in full:
            r.run()
    full_ms, _ = timed(full_run, max(1, args.steps // 2), args.warmup)
    rid_hosts = [torch.empty(n, dtype=torch.int32, pin_memory=True) for _ in cols]

    def e2e_step():
        for c, h in zip(cols, hosts):
            c.copy_(h, non_blocking=True)
        B.launch()
        for r, h in zip(B.parts, rid_hosts):
            h.copy_(r.rid_sorted[:n], non_blocking=True)
    e2e_ms, _ = timed(e2e_step, args.steps, args.warmup)
    clk = clocks.stop() if own_clocks else None
    status, detail = ck.ck_device_status()
    if status != ck.CK_OK:
        raise RuntimeError("device status %s (detail %d)" % (ck.ck_status_string(status), detail))
    B.close()
    times = max_over_ranks([graph_ms, e2e_ms, seq_ms, full_ms], world)
    graph_ms, e2e_ms, seq_ms, full_ms = (float(x) for x in times)
    if rank != 0:
        return None
    keys = 6 * n
    peak, peak_src = peaks()
    alg = 0
    for r in B.parts:
        kb = r.key_bits // 8
        alg += metrics.extract_bytes(n, kb, r.K) + metrics.radix_passes(r.nbits, r.digit_bits) * \
            metrics.pass_bytes(n, r.K) + metrics.build_bytes(n, r.K)
    achieved = alg / (graph_ms / 1e3) / 1e9
    return {
        "metric": METRIC, "value": world * keys / (graph_ms / 1e3), "unit": "keys/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": graph_ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic (seeded generators standing in for a table with integer and title columns)",
        "config": {"workload": desc, "rows": n, "indexes": 6,
                   "key_bytes": [r.key_bits // 8 for r in B.parts], "distinction_bits": [r.nbits for r in B.parts],
                   "ck_words": [r.K for r in B.parts], "digit_bits_autotuned": [r.digit_bits for r in B.parts],
                   "tile_autotuned": [r.tile for r in B.parts],
                   "tuned_digit_tile": [[r.digit_bits, r.tile] for r in B.parts],
                   "fanouts": TABLE_FANOUTS, "l2": "inputs larger than L2 (no flush)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": {"bound": "hbm", "kernel": "whole batched rebuild (all kernels of 6 indexes)",
                     "achieved": achieved, "peak": peak, "peak_source": peak_src, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": None, "alg_bytes_per_launch": alg, "avg_launch_ms": graph_ms},
        "path": "batched graph",
        "batched_streams": {"value": world * keys / (streams_ms / 1e3), "unit": "keys/s", "ms_per_step": streams_ms},
        "plain_sequential": {"value": world * keys / (seq_ms / 1e3), "unit": "keys/s", "ms_per_step": seq_ms,
                             "digit_bits": 8},
        "batched_vs_plain_speedup": seq_ms / graph_ms,
        "full_key": {"value": world * keys / (full_ms / 1e3), "unit": "keys/s", "ms_per_step": full_ms},
        "compressed_vs_full_speedup": full_ms / graph_ms,
        "e2e": {"value": world * keys / (e2e_ms / 1e3), "unit": "keys/s",
                "h2d_bytes_per_step": int(sum(c.nbytes for c in cols_np)), "d2h_bytes_per_step": 4 * n * 6},
        "gpu_launches": int(graph_launches), "clocks": clk,
        "cpu_baseline": None if (world > 1 or args.no_cpu_baseline) else table_cpu_baseline(dmasks, cpu_rows),
    }


def table_cpu_baseline(dmasks, rows):
    import synth
    cols = synth.table_columns(rows, synth.BASE_SEED + 3)
    t = time.perf_counter()
    for c, m, f in zip(cols, dmasks, TABLE_FANOUTS):
        kb = 8 * (c.shape[1] if c.ndim == 2 else c.dtype.itemsize)
        oracle_step(c, m, f, kb)
    dt = time.perf_counter() - t
    return {"value": 6 * rows / dt, "unit": "keys/s", "cores": 1, "kind": "oracle",
            "sample": "first %d rows of the same seeded table, all 6 indexes rebuilt, single thread" % rows}


# Table 4 of the paper (Sec. 6.3): (s, n, m) and its compressed sort key bytes
# (distinction bits + record id variant bits, in 8-byte words) at 10M keys.
# Table 4 leaves the record id's variant bits out; 29 (the top of Table 2's
# 25 to 29) is the value that yields all of its compressed sizes.
ZIPF_RID_VARIANT_BITS = 29
ZIPF_SWEEP = [(2.5, n, 0, 40) for n in range(48, 113, 8)] + [(1.5, 40, m, 24) for m in range(5)] + \
             [(1.5, 64, m, 24) for m in range(6)]


def run_zipf_sweep(args, rank, world, local_rank):
    """Every Zipf(s, n, m) dataset of Table 4: one compressed-key and one
    full-key rebuild per step, timed with CUDA events (device-resident keys)."""
    import torch
    import synth
    from paper_2009_11543_gb300 import build as b
    b.build()
    from paper_2009_11543_gb300 import ck, metrics, pipeline

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    desc, n_keys, _, fanout, _, _ = WORKLOADS[args.workload]
    stream = torch.cuda.current_stream()

    def timed(fn, steps, warmup):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    clocks = ClockSampler(local_rank)
    clocks.start()
    rows, tot_ms, tot_keys, l0 = [], 0.0, 0, ck.ck_launch_count()
    steps = max(1, args.steps // 4)
    for i, (zs, zn, zm, paper_ck_bytes) in enumerate(ZIPF_SWEEP):
        keys = torch.from_numpy(synth.zipf_letters(n_keys, synth.BASE_SEED + 30 + i, zn, zm, zs)).to(dev)
        dmask = pipeline.first_build_dmask(keys, digit_bits=args.digit_bits)
        nbits = ck.popcount(dmask)
        R = pipeline.Rebuild(keys, dmask, fanout=fanout, digit_bits=args.digit_bits)
        F = pipeline.Rebuild(keys, pipeline.full_key_mask(8 * zn), fanout=fanout, digit_bits=args.digit_bits)
        r_ms = timed(R.run, steps, args.warmup)
        f_ms = timed(F.run, max(1, steps // 2), 2)
        ours_ck = metrics.compressed_sort_key_bytes(nbits, ZIPF_RID_VARIANT_BITS)
        full_ck = metrics.full_sort_key_bytes(zn)
        rows.append({"function": "Zipf(%g,%d,%d)" % (zs, zn, zm), "distinction_bits": nbits, "ck_words": R.K,
                     "radix_passes": metrics.radix_passes(nbits, args.digit_bits),
                     "compressed_sort_key_bytes": ours_ck, "paper_compressed_sort_key_bytes": paper_ck_bytes,
                     "pair_bytes": 4 * R.K + 4,
                     "full_sort_key_bytes": full_ck, "sort_key_ratio": full_ck / ours_ck,
                     "compressed_ms": r_ms, "full_key_ms": f_ms, "speedup": f_ms / r_ms})
        tot_ms += r_ms
        tot_keys += n_keys
        del R, F, keys
        torch.cuda.empty_cache()
    clk = clocks.stop()
    status, detail = ck.ck_device_status()
    if status != ck.CK_OK:
        raise RuntimeError("device status %s (detail %d)" % (ck.ck_status_string(status), detail))
    tot_ms = float(max_over_ranks([tot_ms], world)[0])
    if rank != 0:
        return None
    speedups = np.array([r["speedup"] for r in rows])
    return {
        "metric": METRIC, "value": world * tot_keys / (tot_ms / 1e3), "unit": "keys/s", "n_gpus": world, "steps": steps,
        "warmup": args.warmup, "ms_per_step": tot_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32",
        "data": "synthetic (the paper's Zipf(s, n, m) generator definition, Sec. 6.3)",
        "config": {"workload": desc, "n_per_dataset": n_keys, "datasets": len(rows), "fanout": fanout,
                   "rid_variant_bits": ZIPF_RID_VARIANT_BITS,
                   "l2": "inputs larger than L2 (no flush)", "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": None,
        "sweep": rows,
        "speedup_geomean": float(np.exp(np.mean(np.log(speedups)))),
        "paper_sort_key_sizes_matched": int(sum(r["compressed_sort_key_bytes"] == r["paper_compressed_sort_key_bytes"]
                                                for r in rows)),
        "gpu_launches": int(ck.ck_launch_count() - l0),
        "clocks": clk,
    }


LEARNED_PHASE_NAMES = ("sample_model_boundaries", "bucket_ids", "partition", "bucket_sorts_checks", "verdict_fallback")


def learned_phase_bytes(n: int, ck_words: int) -> dict:
    """Algorithmic bytes of the learned sort's two main phases: the partition
    (two radix passes: the first reads the bucket id and the key words and
    writes them with the row id, the second reads all three and writes the key
    words and the row id) and the bucket sorts (every pair read and written
    once)."""
    K = ck_words
    return {"partition": n * ((4 + 4 * K) + (4 + 4 * K + 4)) + n * ((4 + 4 * K + 4) + (4 * K + 4)),
            "bucket_sorts_checks": n * 2 * (4 * K + 4)}


def measure_config(args, workload, world, local_rank, headline=False, extras=False):
    """Times one rebuild configuration: the plain compressed-key path, the
    learned path and the full-key baseline (device-resident keys, CUDA events
    per step on the launching stream), plus end-to-end host transfers for the
    headline workload.  Returns (record, dmask) on every rank after the
    max over ranks."""
    import torch
    from paper_2009_11543_gb300 import ck, metrics, pipeline

    dev = torch.device("cuda", local_rank)
    desc, n, kind, fanout, cpu_rows, main_path = WORKLOADS[workload]
    m_ins = min(1 << 20, n // 16) if extras else 0
    all_np = gen_keys(kind, n + m_ins)
    keys_np, ins_np = all_np[:n], all_np[n:]
    del all_np
    key_bytes = keys_np.shape[1] if keys_np.ndim == 2 else keys_np.dtype.itemsize
    keys_host = torch.from_numpy(keys_np.view(np.int64) if keys_np.dtype == np.uint64 else keys_np)
    if headline:
        keys_host = keys_host.pin_memory()
    keys = keys_host.to(dev)
    fits_l2 = n * key_bytes < 64 * 2**20
    flush_buf = torch.empty(256 * 2**20, dtype=torch.uint8, device=dev) if fits_l2 else None

    # stored DS-metadata: the D-bitmap of a first build (untimed set-up)
    dmask = pipeline.first_build_dmask(keys, digit_bits=args.digit_bits)
    nbits = ck.popcount(dmask)
    R = pipeline.Rebuild(keys, dmask, fanout=fanout, digit_bits=args.digit_bits)
    F = pipeline.Rebuild(keys, pipeline.full_key_mask(8 * key_bytes), fanout=fanout, digit_bits=args.digit_bits)
    L = pipeline.Rebuild(keys, dmask, fanout=fanout, digit_bits=args.digit_bits, learned=True) if R.K <= 8 else None
    passes = metrics.radix_passes(nbits, args.digit_bits)
    fpasses = metrics.radix_passes(8 * key_bytes, args.digit_bits)
    stream = torch.cuda.current_stream()

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    def flush():
        if flush_buf is not None:
            flush_buf.zero_()

    def timed(r, steps, warmup, n_ev):
        """Per-step events around extract / sort / build (an L2 flush between
        steps, outside the events, when the keys fit in L2); n_ev events
        around the sort's passes or phases."""
        for _ in range(warmup):
            r.run()
        barrier()
        ev = [[torch.cuda.Event(enable_timing=True) for _ in range(n_ev)] for _ in range(steps)]
        ph = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(steps)]
        for row in ev + ph:                    # torch creates an event on its first record
            for e in row:
                e.record(stream)
        barrier()
        l0 = ck.ck_launch_count()
        for s in range(steps):
            flush()
            ph[s][0].record(stream)
            r.extract()
            ph[s][1].record(stream)
            r.sort(pass_events=ck.event_handles(ev[s]) if n_ev else None)
            ph[s][2].record(stream)
            r.build()
            ph[s][3].record(stream)
        barrier()
        launches = ck.ck_launch_count() - l0
        phase = np.array([[ph[s][i].elapsed_time(ph[s][i + 1]) for i in range(3)] for s in range(steps)])
        evt = np.array([[ev[s][q].elapsed_time(ev[s][q + 1]) for q in range(n_ev - 1)] for s in range(steps)]) \
            if n_ev > 1 else np.zeros((steps, 1))
        return float(phase.sum(axis=1).mean()), phase.mean(axis=0), evt.mean(axis=0), launches / steps

    p_ms, p_ph, p_pass, p_launch = timed(R, args.steps, args.warmup, passes + 1 if passes else 0)
    f_ms, f_ph, f_pass, _ = timed(F, max(1, args.steps // 2), args.warmup, fpasses + 1)
    l_ms = l_ph = l_phase = None
    l_launch = 0
    variants = {}
    if L is not None:
        l_ms, l_ph, l_phase, l_launch = timed(L, args.steps, args.warmup, ck.CK_LEARNED_PHASES + 1)
        # what the model buys (the same sort with sample-quantile boundaries
        # and no guesses) and, for the learned workloads, the 4096 model
        # buckets the configuration names (quantile cuts then split the
        # over-capacity ones)
        vopts = {"no_model": ck.learned_opts(flags=ck.CK_LEARNED_NO_MODEL)}
        if main_path == "learned":
            vopts["model_buckets_4096"] = ck.learned_opts(bucket_bits=12)
        for name, o in vopts.items():
            Lv = pipeline.Rebuild(keys, dmask, fanout=fanout, digit_bits=args.digit_bits, learned=True,
                                  learned_opts=o)
            v_ms_, _, v_phase, _ = timed(Lv, max(2, args.steps // 2), args.warmup, ck.CK_LEARNED_PHASES + 1)
            vst = Lv.learned_stats
            # a variant may fall back to the plain sort (exact, CK_EVERIFY in
            # the status word): that is its result, recorded here and cleared
            v_status = ck.ck_status_string(ck.ck_device_status()[0])
            ck.ck_clear_device_status()
            variants[name] = {"ms_per_step": v_ms_, "sort_phases_ms": dict(zip(LEARNED_PHASE_NAMES, map(float, v_phase))),
                              "buckets": vst["buckets"], "model_buckets": vst["model_buckets"],
                              "model_boundary_frac": vst["model_boundary_frac"],
                              "mean_search_steps": vst["mean_search_steps"], "max_bucket": vst["max_bucket"],
                              "fell_back": vst["fell_back"], "oversize_buckets": vst["oversize_buckets"],
                              "device_status": v_status}
            del Lv
            torch.cuda.empty_cache()
    headline_learned = main_path == "learned" and L is not None
    v_ms = l_ms if headline_learned else p_ms

    rec = {"workload": desc, "n": n, "key_bytes": key_bytes, "distinction_bits": nbits, "ck_words": R.K,
           "digit_bits": args.digit_bits, "radix_passes": passes, "fanout": fanout,
           "tree_levels": int(R.shape.levels),
           "l2": ("keys fit in L2: a 256 MiB buffer is written between timed steps (outside the timed events)"
                  if fits_l2 else "inputs larger than L2 (no flush)"),
           "path": "learned" if headline_learned else "plain",
           "ms_per_step": v_ms, "value": world * n / (v_ms / 1e3), "unit": "keys/s",
           "plain": {"ms_per_step": p_ms, "value": world * n / (p_ms / 1e3),
                     "phases_ms": dict(zip(("extract", "sort", "build"), map(float, p_ph))),
                     "launches_per_step": p_launch},
           "full_key": {"ms_per_step": f_ms, "value": world * n / (f_ms / 1e3), "radix_passes": fpasses,
                        "ck_words": F.K, "phases_ms": dict(zip(("extract", "sort", "build"), map(float, f_ph)))},
           "compressed_vs_full_speedup": f_ms / v_ms,
           "plain_vs_full_speedup": f_ms / p_ms,
           "compression_ratio": metrics.compression_ratio(8 * key_bytes, nbits) if nbits else None}
    peak, peak_src = peaks()
    # roofline of the plain path's dominant kernel: the radix pass
    sort_bytes = passes * metrics.pass_bytes(n, R.K)
    pass_ms = float(np.sum(p_pass)) if passes else 0.0
    alg = n * key_bytes + sort_bytes   # W read once per key, 2 (c + 4) per pass (extraction's write not counted)
    plain_roof = None
    if passes:
        avg_pass = pass_ms / passes
        plain_roof = {"bound": "hbm", "kernel": "onesweep_pass_kernel<%d, %d>" % (
                          args.digit_bits, 256 if R.K + 1 >= 3 or n > (1 << 22) else 512),
                      "achieved": sort_bytes / (pass_ms / 1e3) / 1e9, "peak": peak, "peak_source": peak_src,
                      "unit": "GB/s", "frac": sort_bytes / (pass_ms / 1e3) / 1e9 / peak,
                      "traffic": ncu_traffic("onesweep_pass_kernel", n, R.K),
                      "alg_bytes_per_launch": sort_bytes / passes,
                      "avg_launch_ms": avg_pass, "launches_per_step": passes}
        rec["plain"]["extract_sort_roofline_frac"] = alg / ((p_ph[0] + p_ph[1]) / 1e3) / 1e9 / peak
        rec["plain"]["extract_sort_alg_bytes"] = alg
    rec["plain"]["roofline"] = plain_roof
    if L is not None:
        st = L.learned_stats
        phases = dict(zip(LEARNED_PHASE_NAMES, map(float, l_phase)))
        pb = learned_phase_bytes(n, R.K)
        dom = max(("partition", "bucket_sorts_checks"), key=lambda k: phases[k])
        kern = {"partition": "onesweep_pass_kernel<8, 256> (2 launches, bucket-id digits)",
                "bucket_sorts_checks": "local_sort_kernel<%d> + const_check_kernel" % R.K}[dom]
        ach = pb[dom] / (phases[dom] / 1e3) / 1e9
        rec["learned"] = {"ms_per_step": l_ms, "value": world * n / (l_ms / 1e3),
                          "phases_ms": dict(zip(("extract", "sort", "build"), map(float, l_ph))),
                          "sort_phases_ms": phases, "stats": st, "speedup_vs_plain": p_ms / l_ms,
                          "launches_per_step": l_launch, "variants": variants,
                          "model_vs_no_model_speedup": variants["no_model"]["ms_per_step"] / l_ms,
                          "roofline": {"bound": "hbm", "kernel": kern, "achieved": ach, "peak": peak,
                                       "peak_source": peak_src, "unit": "GB/s", "frac": ach / peak,
                                       "traffic": ncu_traffic("local_sort_kernel" if dom == "bucket_sorts_checks"
                                                              else "onesweep_pass_kernel_partition", n, R.K),
                                       "alg_bytes_per_launch": pb[dom],
                                       "avg_launch_ms": phases[dom],
                                       "phase_alg_bytes": pb,
                                       "note": ("the bucket sorts move each pair once each way; their time is bound "
                                                "by the chain of block-wide phases per bucket (barrier stalls, "
                                                "shared-memory latency), not by DRAM, which is about 8% busy: "
                                                "profiles/local_sort_dna20m.md") if dom == "bucket_sorts_checks"
                                       else "two radix passes over the bucket id"}}
    rec["roofline"] = rec["learned"]["roofline"] if headline_learned else plain_roof
    rec["gpu_launches_per_step"] = l_launch if headline_learned else p_launch
    V = L if headline_learned else R

    if headline:
        # end to end: every step copies its keys host -> device, rebuilds, and
        # copies the sorted row ids device -> host; the copies of steps i + 1
        # and i - 1 overlap the rebuild of step i (two buffer slots, two copy streams)
        del R, F
        torch.cuda.empty_cache()
        rid_hosts = [torch.empty(n, dtype=torch.int32, pin_memory=True) for _ in range(2)]
        O = pipeline.OverlappedRebuild(keys.shape, keys.dtype, dmask, dev, fanout=fanout, digit_bits=args.digit_bits,
                                       learned=headline_learned)
        for i in range(args.warmup):
            O.submit(keys_host, rid_hosts[i % 2], stream)
        O.finish(stream)
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        O.begin(stream)
        for i in range(args.steps):
            O.submit(keys_host, rid_hosts[i % 2], stream)
        O.finish(stream)
        e1.record(stream)
        barrier()
        e2e_ms = e0.elapsed_time(e1) / args.steps
        e2e_ok = bool(np.array_equal(rid_hosts[(args.steps - 1) % 2].numpy(), ck.u32(V.rid_sorted)[:n].view(np.int32)))
        del O
        torch.cuda.empty_cache()
        h2d_ms = []
        for _ in range(3):
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            keys.copy_(keys_host, non_blocking=True)
            a1.record(stream)
            a1.synchronize()
            h2d_ms.append(a0.elapsed_time(a1))
        rec["e2e"] = {"value": world * n / (e2e_ms / 1e3), "unit": "keys/s", "ms_per_step": e2e_ms,
                      "h2d_bytes_per_step": int(keys_np.nbytes), "d2h_bytes_per_step": 4 * n,
                      "overlap": "pipeline.OverlappedRebuild: the copies of steps i + 1 and i - 1 run beside the "
                                 "rebuild of step i; the timed region spans the first copy in to the last copy out",
                      "last_result_matches_device_run": e2e_ok,
                      "h2d_copy_gbs_alone": keys_np.nbytes / (min(h2d_ms) / 1e3) / 1e9}
        if headline_learned:
            # model-proposed inner separators (verified, the tree keeps the
            # canonical ones), and the whole learned rebuild as one CUDA graph
            seps_ms = []
            for it in range(args.warmup + args.steps):
                a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a0.record(stream)
                prop, hits = L.separators()
                a1.record(stream)
                a1.synchronize()
                if it >= args.warmup:
                    seps_ms.append(a0.elapsed_time(a1))
            ni = int(L.shape.inner_entries)
            rec["learned"]["separators"] = {"inner_entries": ni, "model_hits": int(hits.cpu()[0]),
                                            "hit_rate": int(hits.cpu()[0]) / max(1, ni),
                                            "ms": float(np.median(seps_ms)),
                                            "note": "model proposal of each inner separator's top 24 bits, "
                                                    "checked against the canonical separator (the tree always "
                                                    "keeps the canonical key); timed on the side, not in the step"}
            g = torch.cuda.CUDAGraph()
            side = torch.cuda.Stream(dev)
            side.wait_stream(stream)
            with torch.cuda.stream(side):
                L.run()
            stream.wait_stream(side)
            barrier()
            with torch.cuda.graph(g):
                L.run()
            for _ in range(args.warmup):
                g.replay()
            barrier()
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            for _ in range(args.steps):
                g.replay()
            a1.record(stream)
            barrier()
            rec["learned"]["graph_ms_per_step"] = a0.elapsed_time(a1) / args.steps
            rec["learned"]["graph_note"] = ("extract -> learned sort -> bulk load captured as one CUDA graph "
                                            "(the learned sort decides on the device) and replayed")
            del g
    if extras:
        rec.update(measure_extras(args, keys, ins_np, dmask, V if not headline_learned else pipeline.Rebuild(
            keys, dmask, fanout=fanout, digit_bits=args.digit_bits), n, key_bytes, m_ins, world, stream))
    status, detail = ck.ck_device_status()
    if status != ck.CK_OK:
        raise RuntimeError("device status %s (detail %d)" % (ck.ck_status_string(status), detail))
    # max over ranks of every timing that feeds a value
    t = max_over_ranks([rec["ms_per_step"], rec["plain"]["ms_per_step"], rec["full_key"]["ms_per_step"],
                        rec["learned"]["ms_per_step"] if "learned" in rec else 0.0,
                        rec["e2e"]["ms_per_step"] if "e2e" in rec else 0.0], world)
    rec["ms_per_step"], rec["plain"]["ms_per_step"], rec["full_key"]["ms_per_step"] = (float(x) for x in t[:3])
    rec["value"] = world * n / (rec["ms_per_step"] / 1e3)
    rec["plain"]["value"] = world * n / (rec["plain"]["ms_per_step"] / 1e3)
    rec["full_key"]["value"] = world * n / (rec["full_key"]["ms_per_step"] / 1e3)
    if "learned" in rec:
        rec["learned"]["ms_per_step"] = float(t[3])
        rec["learned"]["value"] = world * n / (float(t[3]) / 1e3)
    if "e2e" in rec:
        rec["e2e"]["ms_per_step"] = float(t[4])
        rec["e2e"]["value"] = world * n / (float(t[4]) / 1e3)
    rec["data"] = DATA_NOTE.get(kind, "synthetic")
    return rec, dmask


def measure_extras(args, keys, ins_np, dmask, R, n, key_bytes, m_ins, world, stream):
    """DS-metadata maintenance (Sec. 4.3), the first build's bitmaps, partial
    keys (Sec. 4.2) and lower-bound search (Sec. 4.3) on the rebuilt index."""
    import torch
    from paper_2009_11543_gb300 import ck
    dev = keys.device
    R.run()
    ins = torch.from_numpy(ins_np.view(np.int64) if ins_np.dtype == np.uint64 else ins_np).to(dev)
    ins_d = torch.from_numpy(np.ascontiguousarray(R.dmask).view(np.int64)).to(dev)
    ins_v = ck.ck_variant_bits(keys, 0)
    ins_ws = torch.empty(max(256, ck._lib().ck_insert_workspace_bytes(m_ins, key_bytes)), dtype=torch.uint8,
                         device=dev)
    ins_ms = []
    for it in range(args.warmup + args.steps):
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        ck.ck_insert_batch(keys, R.rid_sorted[:n], ins, 0, ins_d, ins_v, ws=ins_ws)
        a1.record(stream)
        a1.synchronize()
        if it >= args.warmup:
            ins_ms.append(a0.elapsed_time(a1))
    ins_ms = float(np.median(ins_ms))
    dm_out = torch.empty(ck.mask_words(8 * key_bytes), dtype=torch.int64, device=dev)
    vm_out = torch.empty_like(dm_out)
    db_ms, vb_ms = [], []
    for it in range(args.warmup + args.steps):
        a0, a1, a2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        a0.record(stream)
        ck.ck_distinction_bits(keys, R.rid_sorted[:n], out=dm_out)
        a1.record(stream)
        ck.ck_variant_bits(keys, 0, out=vm_out)
        a2.record(stream)
        a2.synchronize()
        if it >= args.warmup:
            db_ms.append(a0.elapsed_time(a1))
            vb_ms.append(a1.elapsed_time(a2))
    db_ms, vb_ms = float(np.median(db_ms)), float(np.median(vb_ms))
    dmask_ok = bool(np.array_equal(ck.mask_to_host(dm_out), R.dmask))
    pk_bits = 16
    R.run()
    sv = ck.mask_to_host(ck.ck_variant_bits(keys, 0))
    sref = ck.reference_key(keys, 0)
    qidx = torch.from_numpy(np.random.default_rng(9).integers(0, n, 3 * m_ins)).to(dev)
    queries = torch.cat([keys[qidx], ins])
    m_q = int(queries.shape[0])
    spos = torch.empty(m_q, dtype=torch.int32, device=dev)
    srid = torch.empty(m_q, dtype=torch.int32, device=dev)
    R.partial_keys(sv, sref, pk_bits)
    _, _, sder = R.search(queries, pos=spos, rid=srid, want_derefs=True)
    torch.cuda.synchronize()
    derefs_mean = float(sder[:m_q].double().mean())
    hits_frac = float((srid[:m_q] != -1).double().mean())
    _, _, sder_p = R.search(queries, want_derefs=True, inner_partial=True)
    derefs_mean_p = float(sder_p[:m_q].double().mean())
    pk_ms, se_ms, sf_ms = [], [], []
    for it in range(args.warmup + args.steps):
        a0, a1, a2, a3 = (torch.cuda.Event(enable_timing=True) for _ in range(4))
        a0.record(stream)
        R.partial_keys(sv, sref, pk_bits)
        a1.record(stream)
        R.search(queries, pos=spos, rid=srid)
        a2.record(stream)
        R.search(queries, pos=spos, rid=srid, inner_partial=True)
        a3.record(stream)
        a3.synchronize()
        if it >= args.warmup:
            pk_ms.append(a0.elapsed_time(a1))
            se_ms.append(a1.elapsed_time(a2))
            sf_ms.append(a2.elapsed_time(a3))
    pk_ms, se_ms, sf_ms = float(np.median(pk_ms)), float(np.median(se_ms)), float(np.median(sf_ms))
    return {
        "dmask": {"distinction_bits_ms": db_ms, "distinction_bits_keys_per_s": world * n / (db_ms / 1e3),
                  "variant_bits_ms": vb_ms, "variant_bits_gbs": n * key_bytes / (vb_ms / 1e3) / 1e9,
                  "matches_stored_dmask": dmask_ok,
                  "note": "D-bitmap from adjacent keys in sorted order (rows gathered through the permutation), "
                          "variant bitmap (one read of the keys), medians"},
        "insert_batch": {"value": world * m_ins / (ins_ms / 1e3), "unit": "keys/s", "ms": ins_ms, "batch": m_ins,
                         "index_rows": n, "note": "D-bitmap and variant bitmap maintenance (Sec. 4.3), median"},
        "search": {"value": world * m_q / (se_ms / 1e3), "unit": "lookups/s", "ms": se_ms, "queries": m_q,
                   "hits_frac": hits_frac, "full_keys_read_in_leaf_per_query": derefs_mean, "pk_bits": pk_bits,
                   "inner_nodes": "full keys, binary search (Sec. 4.3)",
                   "partial_key_inner_nodes": {"value": world * m_q / (sf_ms / 1e3), "unit": "lookups/s",
                                               "ms": sf_ms, "full_keys_read_per_query": derefs_mean_p},
                   "partial_keys_ms": pk_ms,
                   "partial_keys_per_s": world * (n + int(R.shape.inner_entries)) / (pk_ms / 1e3),
                   "note": "lower-bound search, full-key compares in inner nodes, partial keys in leaves "
                           "(Sec. 4.3), median; every node scanned by partial keys in partial_key_inner_nodes; "
                           "partial keys of every entry (Sec. 4.2) timed separately"},
    }


def headline_line(args, world, rec, workload, clk, launches):
    return {
        "metric": METRIC, "value": rec["value"], "unit": "keys/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": rec["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": rec["data"],
        "config": {k: rec[k] for k in ("workload", "n", "key_bytes", "distinction_bits", "ck_words", "digit_bits",
                                       "radix_passes", "fanout", "tree_levels", "l2", "path")} |
                  {"parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": rec["roofline"],
        "e2e": rec.get("e2e"),
        "gpu_launches": int(launches),
        "clocks": clk,
        "spec_hbm_gbs": SPEC_HBM_GBS,
    }


def run_ours(args, rank, world, local_rank):
    """One workload (--workload): its record is the line."""
    import torch
    from paper_2009_11543_gb300 import build as b
    b.build()
    torch.cuda.set_device(local_rank)
    clocks = ClockSampler(local_rank)
    clocks.start()
    time.sleep(0.2)
    rec, dmask = measure_config(args, args.workload, world, local_rank, headline=True,
                                extras=args.workload == "urls64m")
    clk = clocks.stop()
    if rank != 0:
        return None
    line = headline_line(args, world, rec, args.workload, clk, rec["gpu_launches_per_step"] * args.steps)
    line["detail"] = rec
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.workload, dmask, WORKLOADS[args.workload][4])
    return line


# The five configurations of the benchmark: the headline is the largest
# single-GPU one, 200M DNA keys through the learned path.
ALL_CONFIGS = [("C1", "int1m"), ("C2", "urls64m"), ("C3", "table16m"), ("C4", "zipf256m"), ("C5", "dna200m")]


def run_all(args, rank, world, local_rank):
    """Every configuration in one process and one JSON line: the 200M DNA
    workload (learned partition + bulk load with fanout 256, model
    separators) is the headline; the others are sub-records."""
    import torch
    from paper_2009_11543_gb300 import build as b
    b.build()
    torch.cuda.set_device(local_rank)
    clocks = ClockSampler(local_rank)
    clocks.start()
    time.sleep(0.2)
    subs = {}
    t_run = time.perf_counter()
    for cname, wl in ALL_CONFIGS[:-1]:
        t0 = time.perf_counter()
        if wl == "table16m":
            a2 = argparse.Namespace(**vars(args))
            a2.workload = wl
            a2.no_cpu_baseline = True
            rec = run_table(a2, rank, world, local_rank, own_clocks=False)
        else:
            rec, _ = measure_config(args, wl, world, local_rank, extras=wl == "urls64m")
        if rec is not None:
            rec["wall_s"] = time.perf_counter() - t0
        subs[cname] = rec
        torch.cuda.empty_cache()
    rec, dmask = measure_config(args, "dna200m", world, local_rank, headline=True)
    clk = clocks.stop()
    if rank != 0:
        return None
    line = headline_line(args, world, rec, "dna200m", clk, rec["gpu_launches_per_step"] * args.steps)
    line["config"]["configs"] = "C5 headline (200M DNA, learned); C1-C4 in `configs`"
    line["C5"] = rec
    line["configs"] = subs
    line["learned_vs_plain"] = {c: (subs[c] or {}).get("learned", {}).get("speedup_vs_plain")
                                for c in ("C1", "C2", "C4")} | {"C5": rec["learned"]["speedup_vs_plain"]}
    line["batched_vs_sequential_C3"] = (subs["C3"] or {}).get("batched_vs_plain_speedup")
    line["bench_wall_s"] = time.perf_counter() - t_run
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline("dna200m", dmask, WORKLOADS["dna200m"][4], par_rows=16_000_000)
    return line


# -------------------------------------------------------- oracle (CPU) leg
def oracle_step(keys, dmask, fanout, key_bits):
    """One rebuild of the sample by the CPU oracle: Compress, compressed key
    sort, D refinement, bottom-up bulk load."""
    import oracle
    K = max(1, (oracle.popcount(dmask) + 31) // 32)
    c = oracle.compress(keys, dmask, K)
    perm = oracle.sort_compressed(c)
    oracle.refine(c, perm, dmask, key_bits)
    oracle.btree(keys, perm, fanout)


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.processor() or platform.machine()


def all_cores_sort(keys, dmask, rows):
    """The paper's multi-core CPU comparison (Sec. 6): GCC parallel-mode
    stable sort of the sample's (compressed key, row id) pairs on every host
    core.  The compression before it is set-up, untimed."""
    import oracle
    K = max(1, (oracle.popcount(dmask) + 31) // 32)
    c = oracle.compress(keys, dmask, K)
    oracle.sort_compressed_parallel(c[: min(rows, 100_000)])          # warm-up (thread pool, pages)
    t = time.perf_counter()
    _, used = oracle.sort_compressed_parallel(c)
    dt = time.perf_counter() - t
    return {"value": rows / dt, "unit": "keys/s", "cores": used, "nproc": os.cpu_count(), "cpu_model": cpu_model(),
            "kind": "gcc_parallel_stable_sort",
            "sample": "the compressed-key sort step alone (Sec. 3.2) on the first %d rows of the same seeded "
                      "workload, %d threads" % (rows, used)}


def cpu_baseline(workload, dmask, rows, par_rows=None):
    desc, n, kind, fanout, _, _ = WORKLOADS[workload]
    keys = gen_keys(kind, max(rows, par_rows or 0))   # the first rows of the same seeded column
    kb = 8 * (keys.shape[1] if keys.ndim == 2 else keys.dtype.itemsize)
    t = time.perf_counter()
    oracle_step(keys[:rows], dmask, fanout, kb)
    dt = time.perf_counter() - t
    rec = {"value": rows / dt, "unit": "keys/s", "cores": 1, "kind": "oracle", "cpu_model": cpu_model(),
           "sample": "first %d rows of the same seeded workload, one rebuild (compress, sort, refine, bulk load), "
                     "single thread" % rows}
    if par_rows:
        rec["all_cores_sort"] = all_cores_sort(keys[:par_rows], dmask, par_rows)
    return rec


def run_reference(args, rank, world):
    if rank != 0:
        return None
    import oracle
    workload = "dna200m" if args.workload == "all" else args.workload   # the headline configuration
    desc, n, kind, fanout, rows, _ = WORKLOADS[workload]
    if kind == "table":
        import synth
        rows = min(rows, 500_000)
        cols = synth.table_columns(rows, synth.BASE_SEED + 3)
        dms = [oracle.dmask(c) for c in cols]
        t = time.perf_counter()
        for _ in range(args.steps):
            for c, m, f in zip(cols, dms, TABLE_FANOUTS):
                oracle_step(c, m, f, 8 * (c.shape[1] if c.ndim == 2 else c.dtype.itemsize))
        dt = (time.perf_counter() - t) / args.steps
        v = 6 * rows / dt
        sample = "first %d rows of the same seeded table (6 indexes) per step, single thread" % rows
        return {"metric": METRIC, "value": v, "unit": "keys/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "u32", "data": "synthetic",
                "config": {"workload": desc, "rows": n, "sample_rows": rows}, "impl": "reference",
                "cpu_baseline": {"value": v, "unit": "keys/s", "cores": 1, "kind": "oracle", "sample": sample},
                "e2e": {"value": v, "unit": "keys/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    rows = min(rows, n, 2_000_000)
    keys = gen_keys(kind, rows)
    kb = 8 * (keys.shape[1] if keys.ndim == 2 else keys.dtype.itemsize)
    dmask = oracle.dmask(keys)           # the sample's stored D-bitmap (set-up, untimed)
    for _ in range(args.warmup):
        oracle_step(keys, dmask, fanout, kb)
    t = time.perf_counter()
    for _ in range(args.steps):
        oracle_step(keys, dmask, fanout, kb)
    dt = (time.perf_counter() - t) / args.steps
    v = rows / dt
    sample = "first %d rows of the same seeded workload per step, single thread" % rows
    return {"metric": METRIC, "value": v, "unit": "keys/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": desc, "n": n, "sample_rows": rows}, "impl": "reference",
            "cpu_baseline": {"value": v, "unit": "keys/s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": "keys/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="all", choices=["all"] + sorted(WORKLOADS))
    ap.add_argument("--digit-bits", type=int, default=8)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3) if args.impl == "ours" else args.warmup
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1 and args.impl == "ours":
        import torch.distributed as dist
        dist.init_process_group("gloo")
    if args.impl == "reference":
        line = run_reference(args, rank, world)
    elif args.workload == "all":
        line = run_all(args, rank, world, local_rank)
    elif args.workload == "table16m":
        line = run_table(args, rank, world, local_rank)
    elif args.workload == "zipfsweep":
        line = run_zipf_sweep(args, rank, world, local_rank)
    else:
        line = run_ours(args, rank, world, local_rank)
    if line is not None and rank == 0:
        print(json.dumps(line))
    if world > 1 and args.impl == "ours":
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
