"""Benchmark: sequence pairs filtered per second by the Shouji hot path on GB300.

Workload (synthetic, shaped like the paper's m=100 datasets): 30,000,000 pairs
of length m = 100 at threshold E = 5, half near (k ~ U{0..5} edits) and half
far (k ~ U{6..25}), ASCII reads and references resident in HBM (6 GB, larger
than L2, so no flush is needed between steps).  One step is the whole hot path
over the batch: shouji_pack_filter_results (both packs and the filter in one
warp-specialized kernel, the packed tiles passed through per-CTA rings that
stay in L2), then shouji_compact.  ``e2e`` runs the same batch
through the host pipeline (shouji_pipeline_run: pinned host buffers in, accept
bits, counts and survivor indices out), with every copy inside the timed
region.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) each rank filters its own 30M pairs (weak scaling, no
data exchange); rank 0 prints one JSON line.  ``--impl reference`` times the
CPU oracle on the host cores over a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "sequence pairs filtered/sec on 1 GB300 at m=100,E=5 (bit-exact); % of roofline"
UNIT = "pairs/s"
N_PAIRS = 30_000_000
M = 100
E = 5
# DRAM bytes per filter launch (dram__bytes_read.sum + dram__bytes_write.sum)
# from one ncu capture, keyed by the hash of the filter kernel source it was
# taken on; scaled to a 30M-pair launch.  Reported as null once the kernel
# source changes.
FILTER_TRAFFIC = {"1e05717a759a6a6a": 1.537e9}  # filter_kernel<5>, m=100, 4M-pair capture
# The same for the fused pack + filter kernel, keyed by the hash of its sources.
FUSED_TRAFFIC = {"a9e5bfbf3c497c56": 7.27e9}  # rings, m=100, E=5, 4M-pair capture
FUSED_SOURCES = ("shouji_pack_filter.cu", "shouji_pack.cuh", "shouji_filter.cuh")


def step_bytes_per_pair(m: int) -> float:
    """Algorithmic DRAM bytes per pair of the step from ASCII: both rows in
    (2m), an accept bit and a count byte out."""
    return 2 * m + 1 / 8 + 1


def packed_out_bytes_per_pair(m: int) -> float:
    """Bytes per pair of the packed rows that shouji_pack_filter also writes
    (2 x m/4): an output of the API, kept for reuse, not work of the filter."""
    return 2 * (m / 4)


def filter_bytes_per_pair(m: int, nmask: bool = False) -> float:
    """Algorithmic DRAM bytes per pair of the filter alone: both packed rows
    in (2 bits per base each, plus 1 bit per base of N mask each), an accept
    bit and a count byte out."""
    return 2 * m / 4 + (2 * m / 8 if nmask else 0) + 1 / 8 + 1


def alu_ops_per_pair(m: int, E: int, nmask: bool = False) -> float:
    """Algorithmic integer lane-ops per pair of the bit-sliced formulation.

    Per window and 32 pairs: map 2(2E+1), segment full adders 2(2E+1),
    2E-1 candidate offers of 12 ops, the strict main-diagonal offer 18, the
    Shouji-vector update 8 and the counter 4 -> 32E + 22 (E >= 1; 16 at E=0).
    N masks add one OR per map cell: + (2E+1).
    """
    per_window = (32 * E + 22) if E >= 1 else 16
    if nmask:
        per_window += 2 * E + 1
    return m * per_window / 32.0


def alu_peak(dev):
    """Measured integer issue rates (lane-ops per SM clock, shouji_alu_probe)
    and the ALU peak they give: SMs x LOP3 rate x maximum SM clock."""
    import torch

    import paper_1809_07858_gb300 as sj
    torch.cuda.synchronize(dev)
    rates = {op: round(sj.shouji_alu_probe(op), 2) for op in sj.PROBE_OPS}
    peaks = measured_peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_max = float(peaks.get("sm_max_mhz") or 2070.0)
    return {"lane_ops_per_sm_clk": rates, "sms": sms, "sm_max_mhz": sm_max,
            "peak": sms * rates["lop3"] * sm_max * 1e6, "unit": "lane-ops/s",
            "basis": "SMs x measured LOP3 lane-ops per SM clock (shouji_alu_probe) x max SM clock"}


def source_hash(names=("shouji_filter.cuh",)) -> str:
    h = hashlib.sha256()
    for name in names:
        with open(os.path.join(ROOT, "paper_1809_07858_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def filter_source_hash() -> str:
    return source_hash()


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, period_ms: int = 100):
        self.gpu_index = gpu_index
        self.period_ms = period_ms
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu_index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", str(self.period_ms), "-f", self.path],
                stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            with open(self.path) as f:
                for line in f:
                    parts = [p.strip() for p in line.split(",")]
                    if len(parts) >= 9:
                        rows.append(parts)
            os.unlink(self.path)
        except OSError:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def warm_until_steady(run, tries: int = 10, tol: float = 0.1):
    """Untimed warm-up of an end-to-end leg: at least 3 runs, then more until
    two runs in a row take times within ``tol`` of each other (at most
    ``tries``).  Right after a process that churned tens of GB of pinned host
    memory, single runs of the host pipeline can stall for 100-200 ms."""
    last = None
    for i in range(tries):
        t0 = time.perf_counter()
        run()
        t = time.perf_counter() - t0
        if i >= 2 and last is not None and abs(t - last) <= tol * min(t, last):
            return i + 1
        last = t
    return tries


def h2d_copy_times(h_reads, h_refs, d_reads, d_refs, chunk, steps):
    """Wall times (ms) of copying both pinned host row sets to the device in
    chunks alternating between two streams, as the host pipeline does."""
    import torch
    streams = (torch.cuda.Stream(), torch.cuda.Stream())
    n = h_reads.shape[0]
    out = []
    for _ in range(steps):
        t0 = time.perf_counter()
        for k, base in enumerate(range(0, n, chunk)):
            with torch.cuda.stream(streams[k % 2]):
                d_reads[base:base + chunk].copy_(h_reads[base:base + chunk], non_blocking=True)
                d_refs[base:base + chunk].copy_(h_refs[base:base + chunk], non_blocking=True)
        torch.cuda.synchronize()
        out.append(round(1000 * (time.perf_counter() - t0), 2))
    return out


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def gpu_index_for(local_rank: int) -> int:
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        ids = [v for v in vis.split(",") if v.strip()]
        if local_rank < len(ids) and ids[local_rank].strip().isdigit():
            return int(ids[local_rank])
    return local_rank


def workload_config(n):
    return {"workload": "sweep m=100 E=5: %d pairs, half near (k~U{0..5}) half far (k~U{6..25}), "
                        "ASCII resident in HBM; step = pack reads and refs + filter (one fused "
                        "kernel on the GPU) + compact" % n,
            "n_pairs": n, "m": M, "E": E,
            "l2": "inputs larger than L2 (%.1f GB ASCII per step); no flush" % (2 * n * M / 1e9),
            "step": "results-only fused pack + filter (packed tiles in per-CTA rings) + compact"}


def cpu_oracle_rate(reads, refs, threads, magnet=False):
    import oracle
    t0 = time.perf_counter()
    oracle.shouji_batch(reads, refs, E, threads=threads, magnet=magnet)
    return len(reads) / (time.perf_counter() - t0)


def run_reference(args, world, rank):
    """CPU oracle arm: each step filters a bounded sample on the host cores."""
    if rank != 0:
        return 0
    import oracle  # noqa: F401
    from paper_1809_07858_gb300 import synth
    sample = args.ref_sample
    reads, refs = synth.workload("sweep", sample, E=E)
    threads = os.cpu_count() or 1
    for _ in range(args.warmup):
        cpu_oracle_rate(reads, refs, threads)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        cpu_oracle_rate(reads, refs, threads)
    dt = time.perf_counter() - t0
    value = sample * args.steps / dt
    sample_desc = "pairs 0..%d of the sweep m=100 E=5 workload per step, %d threads" % (sample - 1, threads)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
        "data": "synthetic",
        # the same workload as the GPU arm (args.n pairs); each step times a sample of it
        "config": dict(workload_config(args.n),
                       parallelism="independent shards" if world > 1 else "1 GPU",
                       sample=sample_desc),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": sample_desc},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_batched(args, dev, peak_ops):
    """The batched form: config-4-shaped batch of mixed lengths (40% 100, 40%
    150, 20% 250) and per-pair E uniform in 2..12, unsorted, one CUDA-graph
    launch per batch (bucketing, packing, per-threshold filters, gather)."""
    import numpy as np
    import torch

    import paper_1809_07858_gb300 as sj
    from paper_1809_07858_gb300 import synth
    n = args.batched_n
    lens, Es = synth.mixed_shape(n, seed=4242)
    reads, refs = synth.pairs(n, 250, seed=4242, near=(0, 6), far=(7, 40), far_fraction=0.5,
                              lengths=lens, stride=256)
    ops = float(np.sum(lens.astype(np.float64) * (32.0 * Es.astype(np.float64) + 22.0) / 32.0))
    d_reads = torch.from_numpy(reads).to(dev)
    d_refs = torch.from_numpy(refs).to(dev)
    del reads, refs
    d_lens = torch.from_numpy(lens.astype(np.int16)).to(dev)
    d_E = torch.from_numpy(Es).to(dev)
    acc = torch.empty((n + 31) // 32, dtype=torch.int32, device=dev)
    cnt = torch.empty(n, dtype=torch.uint8, device=dev)
    b = sj.Batch(n, 250, 2, 12)
    b.tune(d_reads, d_refs, d_lens, d_E)
    stream = torch.cuda.current_stream(dev)
    for _ in range(3):
        b.run(d_reads, d_refs, d_lens, d_E, out_accept=acc, out_count=cnt)
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.batched_steps):
        b.run(d_reads, d_refs, d_lens, d_E, out_accept=acc, out_count=cnt)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / args.batched_steps
    stages = b.timing()
    shapes = {E: b.shape(E) for E in range(2, 13)}
    invalid = b.invalid()
    b.close()
    del d_reads, d_refs
    torch.cuda.empty_cache()
    achieved = ops / (ms * 1e-3)
    filt_ms = stages["filters"]
    return {"value": n / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "steps": args.batched_steps,
            "workload": "%d pairs, lengths 40%% 100 / 40%% 150 / 20%% 250, E uniform 2..12, "
                        "unsorted, stride 256, one CUDA-graph launch per batch (tuned)" % n,
            "invalid": invalid,
            "stages_ms": stages,
            "tuned_shapes": shapes,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_ops,
                         "unit": "lane-ops/s", "frac": achieved / peak_ops,
                         "scope": "whole batch step (bucketing, packing, filters, gather)",
                         "filters_frac": ops / (filt_ms * 1e-3) / peak_ops if filt_ms > 0 else None}}


def run_batched_uniform(args, dev, peak_ops, h_reads, h_refs):
    """The batched persistent kernel on a uniform batch: the headline's pairs
    (m=100, E=5), rows at stride 112 (16-byte boundaries), one CUDA-graph
    launch per batch.  The graph records CUDA events around each stage and
    around the E=5 filter kernel; the kernel's roofline fraction uses its own
    recorded time."""
    import numpy as np
    import torch

    import paper_1809_07858_gb300 as sj
    n = h_reads.shape[0]
    stride = 112
    d_reads = torch.zeros((n, stride), dtype=torch.uint8, device=dev)
    d_refs = torch.zeros((n, stride), dtype=torch.uint8, device=dev)
    d_reads[:, :M].copy_(h_reads, non_blocking=True)
    d_refs[:, :M].copy_(h_refs, non_blocking=True)
    d_lens = torch.full((n,), M, dtype=torch.int16, device=dev)
    d_E = torch.full((n,), E, dtype=torch.uint8, device=dev)
    acc = torch.empty((n + 31) // 32, dtype=torch.int32, device=dev)
    cnt = torch.empty(n, dtype=torch.uint8, device=dev)
    b = sj.Batch(n, M, E, E)
    b.tune(d_reads, d_refs, d_lens, d_E)
    stream = torch.cuda.current_stream(dev)
    for _ in range(3):
        b.run(d_reads, d_refs, d_lens, d_E, out_accept=acc, out_count=cnt)
    torch.cuda.synchronize(dev)
    kernel_ms, stage_list = [], []
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.batched_steps):
        b.run(d_reads, d_refs, d_lens, d_E, out_accept=acc, out_count=cnt)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / args.batched_steps
    # the kernel's own time: the graph's event nodes around it, run by run
    for _ in range(args.batched_steps):
        b.run(d_reads, d_refs, d_lens, d_E, out_accept=acc, out_count=cnt)
        st = b.timing()
        stage_list.append(st)
        kernel_ms.append(st["filter_E"][E])
    shape = b.shape(E)
    b.close()
    accepted = int(np.unpackbits(acc.cpu().numpy().view(np.uint8)).sum())
    del d_reads, d_refs
    torch.cuda.empty_cache()
    k_ms = statistics.median(kernel_ms)
    ops = alu_ops_per_pair(M, E) * n
    stages = {k: statistics.median(x[k] for x in stage_list)
              for k in ("graph", "bucketing", "pack", "filters", "finalize")}
    return {"value": n / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "steps": args.batched_steps,
            "workload": "%d pairs m=%d E=%d (the headline's pairs), rows at stride %d, one "
                        "CUDA-graph launch per batch (tuned)" % (n, M, E, stride),
            "accepted": accepted, "stages_ms": stages,
            "kernel": "batch_filter_kernel<%d>" % E, "kernel_ms": k_ms, "tuned_shape": shape,
            "kernel_ms_runs": [round(x, 4) for x in kernel_ms],
            "roofline": {"bound": "alu", "achieved": ops / (k_ms * 1e-3), "peak": peak_ops,
                         "unit": "lane-ops/s", "frac": ops / (k_ms * 1e-3) / peak_ops,
                         "scope": "the E=%d filter kernel alone, timed by CUDA events the graph "
                                  "records around it" % E,
                         "ops_per_pair": alu_ops_per_pair(M, E)},
            "graph_frac": ops / (ms * 1e-3) / peak_ops}


def run_sweep(args, dev, peak_ops, hbm_peak):
    """The E sweep (m=100): for each E, 30M pairs of the sweep recipe at that
    E, packed once, then the filter alone on the packed pairs, resident in
    HBM (CUDA events over --sweep-steps launches)."""
    import numpy as np
    import torch

    import paper_1809_07858_gb300 as sj
    from paper_1809_07858_gb300 import synth
    n = args.sweep_n
    out = []
    h_r = np.empty((n, M), np.uint8)
    h_t = np.empty((n, M), np.uint8)
    d_r = torch.empty((n, M), dtype=torch.uint8, device=dev)
    d_t = torch.empty((n, M), dtype=torch.uint8, device=dev)
    pr = torch.empty(sj.shouji_packed_words(n, M), dtype=torch.int32, device=dev)
    pt = torch.empty_like(pr)
    acc = torch.empty((n + 31) // 32, dtype=torch.int32, device=dev)
    cnt = torch.empty(n, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    for e in args.sweep_E:
        synth.workload("sweep", n, E=e, out=(h_r, h_t))
        d_r.copy_(torch.from_numpy(h_r))
        d_t.copy_(torch.from_numpy(h_t))
        sj.shouji_pack(d_r, M, packed=pr, stream=stream)
        sj.shouji_pack(d_t, M, packed=pt, stream=stream)
        for _ in range(2):
            sj.shouji_filter(pr, pt, M, n, e, out_accept=acc, out_count=cnt, stream=stream)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.sweep_steps):
            sj.shouji_filter(pr, pt, M, n, e, out_accept=acc, out_count=cnt, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / args.sweep_steps
        ops = alu_ops_per_pair(M, e) * n
        accepted = int(np.unpackbits(acc.cpu().numpy().view(np.uint8)).sum())
        out.append({"E": e, "m": M, "n_pairs": n, "ms": ms, "pairs_per_s": n / (ms * 1e-3),
                    "accepted": accepted, "alu_frac": ops / (ms * 1e-3) / peak_ops,
                    "hbm_frac": filter_bytes_per_pair(M) * n / (ms * 1e-3) / 1e9 / hbm_peak})
    del d_r, d_t, pr, pt
    torch.cuda.empty_cache()
    return {"kernel": "shouji_filter (packed pairs resident in HBM)",
            "workload": "sweep recipe per E: %d pairs m=%d, half near k~U{0..E}, half far "
                        "k~U{E+1..25}, seed 1000+E" % (n, M),
            "steps": args.sweep_steps, "points": out}


def run_long(args, dev, peak_ops, hbm_peak):
    """Long reads with 'N' (m = 150 and 250, 0.1% 'N' on each side): per
    (m, E), pairs of the long recipe packed with N masks, then the masked
    filter alone on the packed pairs, resident in HBM."""
    import numpy as np
    import torch

    import paper_1809_07858_gb300 as sj
    from paper_1809_07858_gb300 import synth
    n = args.long_n
    stream = torch.cuda.current_stream(dev)
    out = []
    for m, e in ((150, 7), (150, 15), (250, 12), (250, 15)):
        h_r, h_t = synth.workload("long", n, E=e, m=m)
        d_r = torch.from_numpy(h_r).to(dev)
        d_t = torch.from_numpy(h_t).to(dev)
        pr, nr = sj.shouji_pack(d_r, m, with_n=True, stream=stream)
        pt, nt = sj.shouji_pack(d_t, m, with_n=True, stream=stream)
        del d_r, d_t
        acc = torch.empty((n + 31) // 32, dtype=torch.int32, device=dev)
        cnt = torch.empty(n, dtype=torch.uint8, device=dev)
        for _ in range(2):
            sj.shouji_filter(pr, pt, m, n, e, reads_nmask=nr, refs_nmask=nt, out_accept=acc,
                             out_count=cnt, stream=stream)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.sweep_steps):
            sj.shouji_filter(pr, pt, m, n, e, reads_nmask=nr, refs_nmask=nt, out_accept=acc,
                             out_count=cnt, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / args.sweep_steps
        ops = alu_ops_per_pair(m, e, nmask=True) * n
        accepted = int(np.unpackbits(acc.cpu().numpy().view(np.uint8)).sum())
        out.append({"m": m, "E": e, "n_pairs": n, "ms": ms, "pairs_per_s": n / (ms * 1e-3),
                    "accepted": accepted, "alu_frac": ops / (ms * 1e-3) / peak_ops,
                    "hbm_frac": filter_bytes_per_pair(m, True) * n / (ms * 1e-3) / 1e9 / hbm_peak})
        del pr, pt, nr, nt, acc, cnt, h_r, h_t
        torch.cuda.empty_cache()
    return {"kernel": "shouji_filter with N masks (packed pairs resident in HBM)",
            "workload": "long recipe per (m, E): %d pairs, near k~U{0..E}, far "
                        "k~U{E+1..ceil(m/4)}, 0.1%% N per base and side, seed 2000+m+E" % n,
            "steps": args.sweep_steps, "points": out}


def run_magnet(args, dev, packed_r, packed_t, n, shouji_accept):
    """MAGNET (Supplementary Sec. 7) on the same packed batch as the headline
    step: shouji_magnet alone, inputs packed and resident in HBM."""
    import numpy as np
    import torch

    import paper_1809_07858_gb300 as sj
    acc = torch.empty((n + 31) // 32, dtype=torch.int32, device=dev)
    cnt = torch.empty(n, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    for _ in range(2):
        sj.shouji_magnet(packed_r, packed_t, M, n, E, out_accept=acc, out_count=cnt, stream=stream)
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.magnet_steps):
        sj.shouji_magnet(packed_r, packed_t, M, n, E, out_accept=acc, out_count=cnt, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / args.magnet_steps
    m_words = acc.cpu().numpy().view(np.uint32)
    s_words = shouji_accept.cpu().numpy().view(np.uint32)

    def ones(w):
        return int(np.unpackbits(w.view(np.uint8)).sum())
    return {"value": n / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "steps": args.magnet_steps,
            "kernel": "shouji_magnet", "workload": "the headline's %d pairs (m=%d, E=%d), "
            "packed and resident" % (n, M, E),
            "accepted": ones(m_words), "accepted_shouji": ones(s_words),
            "accepted_magnet_not_shouji": ones(m_words & ~s_words),
            "accepted_shouji_not_magnet": ones(s_words & ~m_words)}


def union_length(spans):
    total, end = 0.0, -1.0
    for a, b in sorted(spans):
        if a > end:
            total += b - a
            end = b
        elif b > end:
            total += b - end
            end = b
    return total


def run_served(args, dev):
    """The served form: requests of log-uniform size in [1e3, 1e6] pairs with
    the batched mix, filtered by the server (continuous batching, admission by
    device memory).  Three loads: closed loop (the server's capacity), Poisson
    arrivals at --serve-rate per second (the offered load of the workload),
    and Poisson arrivals at 80% of the capacity; each with p50/p99 latency
    (submit to results in host memory) and the overlap of requests on the GPU
    (summed GPU time of the requests over the time any was on the GPU).  The
    same at capacity with the reference segments resident on the device
    (requests send reads and offsets only)."""
    import queue as queue_mod
    import threading
    from concurrent.futures import ThreadPoolExecutor

    import numpy as np
    import torch

    import paper_1809_07858_gb300 as sj
    from paper_1809_07858_gb300 import synth
    pool = 1_200_000
    lens, Es = synth.mixed_shape(pool, seed=777)
    h_reads = torch.empty((pool, 256), dtype=torch.uint8, pin_memory=True)
    h_refs = torch.empty((pool, 256), dtype=torch.uint8, pin_memory=True)
    synth.pairs(pool, 250, seed=777, near=(0, 6), far=(7, 40), far_fraction=0.5, lengths=lens,
                stride=256, out=(h_reads, h_refs))
    h_lens = torch.from_numpy(lens.astype(np.int16)).pin_memory()
    h_E = torch.from_numpy(Es).pin_memory()
    h_off = torch.from_numpy(np.arange(pool, dtype=np.int64) * 256).pin_memory()
    ring = 64
    outs = [(torch.empty(31_251, dtype=torch.int32, pin_memory=True),
             torch.empty(1_000_000, dtype=torch.uint8, pin_memory=True)) for _ in range(ring)]
    budget = int(args.serve_budget_gb * (1 << 30))
    srv = sj.Server(1_000_000, 250, 2, 12, max_stride=256, memory_budget=budget,
                    max_slots=args.serve_slots)
    ref_id = srv.add_reference(h_refs.view(-1))
    rng = np.random.default_rng(99)

    def submit(b, size, off, resident):
        a, c = outs[b]
        if resident:
            return srv.submit_at(h_reads[off:off + size], ref_id, h_off[off:off + size],
                                 h_lens[off:off + size], h_E[off:off + size], a, c,
                                 n_pairs=size, stride=256)
        return srv.submit(h_reads[off:off + size], h_refs[off:off + size], h_lens[off:off + size],
                          h_E[off:off + size], a, c, n_pairs=size, stride=256)

    def drive(n_req, rate=None, inflight=None, resident=False):
        """rate: Poisson arrivals per second; inflight: closed loop with that
        many requests outstanding.  Requests are waited for in any order (a
        pool of waiter threads), so that one long request does not hold back
        the admission of the next ones; output buffers come from a free list."""
        sizes = np.exp(rng.uniform(np.log(1e3), np.log(1e6), size=n_req)).astype(np.int64)
        offs = rng.integers(0, pool - sizes + 1)
        gaps = rng.exponential(1.0 / rate, size=n_req) if rate else None
        res = [None] * n_req
        limit = inflight if inflight else ring
        free = threading.Semaphore(limit)
        bufs = queue_mod.SimpleQueue()
        for b in range(ring):
            bufs.put(b)

        def waiter(i, rid, b):
            try:
                res[i] = srv.wait_timed(rid, timeout=120)
            finally:
                bufs.put(b)
                free.release()

        waiters = ThreadPoolExecutor(max_workers=limit)

        def submitter():
            t_next = time.perf_counter()
            for i in range(n_req):
                if rate:
                    t_next += gaps[i]
                    delay = t_next - time.perf_counter()
                    if delay > 0:
                        time.sleep(delay)
                free.acquire()
                b = bufs.get()
                rid = submit(b, int(sizes[i]), int(offs[i]), resident)
                waiters.submit(waiter, i, rid, b)

        t0 = time.perf_counter()
        th = threading.Thread(target=submitter)
        th.start()
        th.join()
        waiters.shutdown(wait=True)
        wall = time.perf_counter() - t0
        assert all(r is not None for r in res)
        lat_ms = np.array([r[0] for r in res]) * 1e3
        spans = [(r[1], r[2]) for r in res]
        busy = union_length(spans)
        return {"value": float(sizes.sum()) / wall, "unit": UNIT, "requests": n_req,
                "duration_s": wall, "p50_ms": float(np.percentile(lat_ms, 50)),
                "p99_ms": float(np.percentile(lat_ms, 99)),
                "mean_request_pairs": float(sizes.mean()),
                "overlap": sum(b - a for a, b in spans) / busy if busy > 0 else None,
                "gpu_busy_frac": busy / wall}

    drive(64, inflight=16)                       # warm-up: workers of every class are made
    drive(32, inflight=16, resident=True)
    n_cap = max(16, int(args.serve_seconds * 600))   # about a second of closed-loop work
    cap = drive(n_cap, inflight=args.serve_inflight)
    cap_res = drive(n_cap, inflight=args.serve_inflight, resident=True)
    mean_pairs = cap["mean_request_pairs"]
    n_off = max(8, int(args.serve_rate * args.serve_seconds))
    offered = drive(n_off, rate=args.serve_rate)
    rate80 = 0.8 * cap["value"] / mean_pairs
    at80 = drive(max(8, int(rate80 * args.serve_seconds / 2)), rate=rate80)
    st = srv.stats()
    srv.close()
    for d, r in ((offered, args.serve_rate), (at80, rate80)):
        d["arrival"] = "Poisson, %.1f requests/s" % r
        d["offered_pairs_per_s"] = r * mean_pairs
    return {"value": offered["value"], "unit": UNIT, "p50_ms": offered["p50_ms"],
            "p99_ms": offered["p99_ms"],
            "workload": "requests of log-uniform size in [1e3, 1e6] pairs; lengths 40% 100 / 40% "
                        "150 / 20% 250, E uniform 2..12; rows at stride 256 in pinned host memory",
            "offered": offered, "capacity": cap,
            "capacity_pairs_per_s": cap["value"], "at_80pct_capacity": at80,
            "capacity_resident_refs": cap_res,
            "memory_budget_gb": args.serve_budget_gb,
            "peak_used_gb": st["peak_used_bytes"] / (1 << 30),
            "peak_concurrent_requests": st["peak_busy_workers"],
            "workers_made": st["workers_made"], "workers_released": st["workers_released"],
            "closed_loop_inflight": args.serve_inflight}


def run_ours(args, world, rank, local):
    import numpy as np
    import torch

    import paper_1809_07858_gb300 as sj
    from paper_1809_07858_gb300 import synth

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    n = args.n

    # Inputs: this rank's shard of the workload, generated into pinned host
    # memory (the e2e leg reads it from there), then made resident in HBM.
    h_reads = torch.empty((n, M), dtype=torch.uint8, pin_memory=True)
    h_refs = torch.empty((n, M), dtype=torch.uint8, pin_memory=True)
    synth.workload("sweep", n, E=E, first=rank * n, out=(h_reads, h_refs))
    d_reads = h_reads.to(dev)
    d_refs = h_refs.to(dev)
    packed_r = torch.empty(sj.shouji_packed_words(n, M), dtype=torch.int32, device=dev)
    packed_t = torch.empty_like(packed_r)
    accept = torch.empty((n + 31) // 32, dtype=torch.int32, device=dev)
    count = torch.empty(n, dtype=torch.uint8, device=dev)
    idx = torch.empty(n, dtype=torch.int32, device=dev)
    n_acc = torch.empty(1, dtype=torch.int32, device=dev)
    ws = torch.empty(max(16, sj.shouji_compact_workspace_size(n)), dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    alu = alu_peak(dev)
    peak_ops = alu["peak"]
    # whether the step's pack + filter is the one fused kernel (else three launches)
    fused = sj.shouji_pack_filter_fused(d_reads, d_refs, M, E)
    # the step wants the results only: the fused kernel's packed tiles go
    # through per-CTA rings in this workspace (about 93 MB, L2-resident)
    ring_ws = torch.empty(max(16, sj.shouji_pack_filter_workspace_size(d_reads, d_refs, M, E, n)),
                          dtype=torch.uint8, device=dev)

    ev = {k: [] for k in ("fused0", "fused1", "compact0", "compact1")}

    def step(timed):
        def mark(k):
            if timed:
                e = torch.cuda.Event(enable_timing=True)
                e.record(stream)
                ev[k].append(e)
        mark("fused0")
        sj.shouji_pack_filter_results(d_reads, d_refs, M, E, workspace=ring_ws,
                                      out_accept=accept, out_count=count, stream=stream)
        mark("fused1")
        mark("compact0")
        sj.shouji_compact(accept, n, out_idx=idx, out_n=n_acc, workspace=ws, stream=stream)
        mark("compact1")

    for _ in range(args.warmup):
        step(False)
    torch.cuda.synchronize(dev)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    barrier()
    torch.cuda.synchronize(dev)
    with ClockSampler(gpu_index_for(local)) as clk:
        t_start = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        t_start.record(stream)
        for _ in range(args.steps):
            step(True)
        t_end.record(stream)
        torch.cuda.synchronize(dev)
    barrier()
    elapsed_ms = t_start.elapsed_time(t_end)
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([elapsed_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        elapsed_ms = float(t.item())

    def avg(a, b):
        return sum(x.elapsed_time(y) for x, y in zip(ev[a], ev[b])) / max(1, len(ev[a]))

    fused_ms, compact_ms = avg("fused0", "fused1"), avg("compact0", "compact1")
    n_accepted = int(n_acc.item())

    # For comparison, outside the timed region: the same kernel writing the
    # packed rows as outputs (shouji_pack_filter), and the same pack and
    # filter as separate launches (shouji_pack twice, then shouji_filter).
    wp = []
    for r in range(13):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sj.shouji_pack_filter(d_reads, d_refs, M, E, packed_reads=packed_r,
                              packed_refs=packed_t, out_accept=accept, out_count=count,
                              stream=stream)
        e1.record(stream)
        if r >= 3:
            wp.append((e0, e1))
    torch.cuda.synchronize(dev)
    with_packed_ms = sum(a.elapsed_time(b) for a, b in wp) / len(wp)
    sep = {k: [] for k in ("p0", "p1", "f1")}
    for r in range(13):
        for k in ("p0", "p1", "f1"):
            e = torch.cuda.Event(enable_timing=True)
            if k == "p0":
                e.record(stream)
                sj.shouji_pack(d_reads, M, packed=packed_r, stream=stream)
                sj.shouji_pack(d_refs, M, packed=packed_t, stream=stream)
            elif k == "p1":
                e.record(stream)
                sj.shouji_filter(packed_r, packed_t, M, n, E, out_accept=accept, out_count=count,
                                 stream=stream)
            else:
                e.record(stream)
            if r >= 3:
                sep[k].append(e)
    torch.cuda.synchronize(dev)
    pack_ms = sum(a.elapsed_time(b) for a, b in zip(sep["p0"], sep["p1"])) / len(sep["p0"])
    filter_ms = sum(a.elapsed_time(b) for a, b in zip(sep["p1"], sep["f1"])) / len(sep["p1"])

    # End to end through the host pipeline: pinned host ASCII in, accept words,
    # counts and survivor indices out, every copy inside the timed region.
    pipe = sj.Pipeline(M, chunk_pairs=args.chunk, max_pairs=n)
    h_acc = torch.empty((n + 31) // 32, dtype=torch.int32, pin_memory=True)
    h_cnt = torch.empty(n, dtype=torch.uint8, pin_memory=True)
    h_idx = torch.empty(n, dtype=torch.int32, pin_memory=True)
    warm_until_steady(lambda: pipe.run(h_reads, h_refs, n, E, h_acc, count=h_cnt, idx=h_idx))
    # The host link alone: the same input bytes as bare pinned host -> device
    # copies (chunks on two streams, no kernel), timed like the e2e steps.
    # Both show the same sporadic stalls on some boxes.
    copy_ms = h2d_copy_times(h_reads, h_refs, d_reads, d_refs, args.chunk, args.e2e_steps)
    barrier()
    e2e_steps_ms = []
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        t1 = time.perf_counter()
        e2e_acc = pipe.run(h_reads, h_refs, n, E, h_acc, count=h_cnt, idx=h_idx)
        e2e_steps_ms.append(round(1000 * (time.perf_counter() - t1), 2))
    e2e_s = time.perf_counter() - t0
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([e2e_s], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    assert e2e_acc == n_accepted, (e2e_acc, n_accepted)

    # The same through shouji_pipeline_run_packed, for callers that keep their
    # pairs in the packed 2-bit layout (a quarter of the ASCII bytes): the
    # packed words written above by shouji_pack, copied to pinned host memory
    # before the timed region.
    hp_r = torch.empty(packed_r.numel(), dtype=torch.int32, pin_memory=True)
    hp_t = torch.empty_like(hp_r, pin_memory=True)
    hp_r.copy_(packed_r)
    hp_t.copy_(packed_t)
    warm_until_steady(lambda: pipe.run_packed(hp_r, hp_t, n, E, h_acc, count=h_cnt, idx=h_idx))
    barrier()
    e2e_packed_ms = []
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        t1 = time.perf_counter()
        packed_acc = pipe.run_packed(hp_r, hp_t, n, E, h_acc, count=h_cnt, idx=h_idx)
        e2e_packed_ms.append(round(1000 * (time.perf_counter() - t1), 2))
    e2e_packed_s = time.perf_counter() - t0
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([e2e_packed_s], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_packed_s = float(t.item())
    pipe.close()
    assert packed_acc == n_accepted, (packed_acc, n_accepted)
    packed_h2d = 2 * hp_r.numel() * 4
    del hp_r, hp_t

    if rank != 0:
        return 0

    clocks = clk.summary()
    peaks = measured_peaks()
    ops_launch = alu_ops_per_pair(M, E) * n
    achieved = ops_launch / (filter_ms * 1e-3)
    src = filter_source_hash()
    traffic = FILTER_TRAFFIC.get(src)
    hbm_peak = float(peaks.get("hbm_gbs") or 6800.0)
    fused_src = source_hash(FUSED_SOURCES)
    # The step's roofline: the larger of its two algorithmic lower bounds,
    # the bytes it must move (ASCII in, accept bits and counts out) at the
    # measured HBM copy bandwidth and the filter's lane-ops at the measured
    # integer peak.
    step_bytes = step_bytes_per_pair(M) * n
    t_hbm = step_bytes / (hbm_peak * 1e9)
    t_alu = ops_launch / peak_ops
    fused_s = fused_ms * 1e-3
    hbm_frac = step_bytes / fused_s / 1e9 / hbm_peak
    alu_frac = ops_launch / fused_s / peak_ops
    with_packed = (step_bytes_per_pair(M) + packed_out_bytes_per_pair(M)) * n
    with_packed_s = with_packed_ms * 1e-3
    if t_hbm >= t_alu:
        roofline = {"bound": "hbm", "achieved": step_bytes / fused_s / 1e9, "peak": hbm_peak,
                    "unit": "GB/s", "frac": hbm_frac,
                    "peak_basis": "measured HBM copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"}
    else:
        roofline = {"bound": "alu", "achieved": ops_launch / fused_s, "peak": peak_ops,
                    "unit": "lane-ops/s", "frac": alu_frac, "peak_basis": alu["basis"]}
    # traffic: DRAM bytes per launch from one ncu capture of this kernel source
    roofline.update({
        "traffic": FUSED_TRAFFIC.get(fused_src),
        "kernel": "shouji_pack_filter_results (%s)" % (
            "pack_filter_kernel, packed tiles in per-CTA rings" if fused else
            "separate pack x2 + filter launches"),
        "fused_kernel": fused,
        "bytes_per_pair": step_bytes_per_pair(M),
        "bytes_basis": "2m ASCII in + 1/8 accept + 1 count out per pair",
        "hbm_frac": hbm_frac, "alu_frac": alu_frac,
        "alu_ops_per_pair": alu_ops_per_pair(M, E),
        "with_packed_out": {"call": "shouji_pack_filter (the same kernel, packed rows written "
                                    "as outputs for reuse)",
                            "ms": with_packed_ms,
                            "bytes_per_pair": step_bytes_per_pair(M) + packed_out_bytes_per_pair(M),
                            "achieved": with_packed / with_packed_s / 1e9, "unit": "GB/s",
                            "frac": with_packed / with_packed_s / 1e9 / hbm_peak,
                            "frac_on_step_bytes": step_bytes / with_packed_s / 1e9 / hbm_peak},
        "src": fused_src})
    value = world * n * args.steps / (elapsed_ms * 1e-3)
    e2e_value = world * n * args.e2e_steps / e2e_s
    h2d = 2 * n * M
    d2h = h_acc.numel() * 4 + n + 4 * n_accepted
    batched = batched_uniform = served = magnet = sweep = long_reads = None
    if world == 1 and args.magnet_steps > 0:
        magnet = run_magnet(args, dev, packed_r, packed_t, n, accept)
    if world == 1:
        del d_reads, d_refs, packed_r, packed_t, idx
        torch.cuda.empty_cache()
        if args.batched_steps > 0:
            batched_uniform = run_batched_uniform(args, dev, peak_ops, h_reads, h_refs)
            batched = run_batched(args, dev, peak_ops)
        if args.sweep_steps > 0:
            sweep = run_sweep(args, dev, peak_ops, hbm_peak)
            long_reads = run_long(args, dev, peak_ops, hbm_peak)
        if args.serve_seconds > 0:
            served = run_served(args, dev)
    cpu = None
    if world == 1:
        sample = args.cpu_sample
        threads = os.cpu_count() or 1
        rate = cpu_oracle_rate(h_reads[:sample].numpy(), h_refs[:sample].numpy(), threads)
        cpu = {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": "pairs 0..%d of the same workload (%d threads)" % (sample - 1, threads)}
        one = max(1, sample // 10)
        cpu["single_thread"] = {
            "value": cpu_oracle_rate(h_reads[:one].numpy(), h_refs[:one].numpy(), 1),
            "unit": UNIT, "sample": "pairs 0..%d, one thread" % (one - 1)}
        if magnet is not None:
            msample = max(1, sample // 10)
            mrate = cpu_oracle_rate(h_reads[:msample].numpy(), h_refs[:msample].numpy(), threads,
                                    magnet=True)
            magnet["cpu_baseline"] = {"value": mrate, "unit": UNIT, "cores": threads,
                                      "kind": "oracle", "sample": "pairs 0..%d (%d threads)" % (
                                          msample - 1, threads)}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": dict(workload_config(n), parallelism="independent shards" if world > 1 else "1 GPU"),
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "steps": args.e2e_steps, "step_ms": e2e_steps_ms,
                "h2d_copy_only_ms": copy_ms,
                "path": "shouji_pipeline_run, pinned host buffers, chunks of %d pairs" % args.chunk},
        "e2e_packed_input": {
            "value": world * n * args.e2e_steps / e2e_packed_s, "unit": UNIT,
            "h2d_bytes_per_step": packed_h2d, "d2h_bytes_per_step": d2h,
            "steps": args.e2e_steps, "step_ms": e2e_packed_ms,
            "path": "shouji_pipeline_run_packed, pairs held in pinned host memory in the "
                    "packed 2-bit layout, chunks of %d pairs" % args.chunk},
        "gpu_launches": (4 if fused else 6) * args.steps,
        "roofline": roofline,
        "alu_peak": alu,
        "kernels_ms": {"pack_filter": fused_ms, "compact": compact_ms},
        "separate": {"pack_x2_ms": pack_ms, "filter_ms": filter_ms,
                     "filter_roofline": {"bound": "alu", "achieved": achieved, "peak": peak_ops,
                                         "unit": "lane-ops/s", "frac": achieved / peak_ops,
                                         "traffic": traffic, "filter_src": src}},
        "accepted": n_accepted,
        "clocks": clocks,
        "cpu_baseline": cpu,
        "batched_uniform": batched_uniform,
        "batched": batched,
        "sweep": sweep,
        "long_reads": long_reads,
        "served": served,
        "magnet": magnet,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=N_PAIRS)
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--chunk", type=int, default=1 << 22)
    ap.add_argument("--cpu-sample", type=int, default=1_000_000)
    ap.add_argument("--ref-sample", type=int, default=200_000)
    ap.add_argument("--batched-n", type=int, default=50_000_000)
    ap.add_argument("--batched-steps", type=int, default=10, help="0 skips the batched legs")
    ap.add_argument("--sweep-n", type=int, default=30_000_000)
    ap.add_argument("--long-n", type=int, default=10_000_000)
    ap.add_argument("--sweep-E", type=lambda v: [int(x) for x in v.split(",")],
                    default=[0, 2, 5, 8, 10])
    ap.add_argument("--sweep-steps", type=int, default=10,
                    help="0 skips the E-sweep and long-read legs")
    ap.add_argument("--serve-seconds", type=float, default=3.0, help="0 skips the served leg")
    ap.add_argument("--serve-rate", type=float, default=200.0)
    ap.add_argument("--serve-budget-gb", type=float, default=40.0)
    ap.add_argument("--serve-slots", type=int, default=64)
    ap.add_argument("--serve-inflight", type=int, default=32)
    ap.add_argument("--magnet-steps", type=int, default=5, help="0 skips the MAGNET leg")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    world, rank, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, world, rank)
    return run_ours(args, world, rank, local)


if __name__ == "__main__":
    sys.exit(main())
