#!/usr/bin/env python
"""Throughput benchmark of the GB300 windowed GenASM aligner.

One step aligns a whole batch: every pair of the workload goes through the
windowing loop (GenASM-DC with ET, DENT/SENE storage, GenASM-TB, slide).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload long_reads]
                  [--impl ours|reference] [--pairs P] [--scaling weak|strong]
                  [--no-e2e] [--no-cpu-baseline]

Prints one JSON line (rank 0). ``value`` is alignments/s of the device-resident
batch (CUDA events around each launch on the launching stream, max over
ranks); ``e2e`` is the same metric through the C ABI with pinned host buffers
(host-to-device copies of the packed inputs and device-to-host copies of all
outputs inside the timed region). ``--impl reference`` times the CPU oracle on
the host cores instead. With N > 1 (torchrun, or launched by this script when
WORLD_SIZE is unset), each rank aligns its own batch of the same size (weak
scaling), or its cost-balanced shard of one batch (--scaling strong, results
gathered on rank 0 and checked against a single-GPU run of the whole batch);
there is no collective on the data path.
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

from paper_2208_09985_gb300 import synth  # noqa: E402

WORKLOADS = {
    "long_reads": dict(
        make=lambda n, seed: synth.long_reads(n, seed=seed), n=100_000, seed=2, W=64, O=24,
        desc="100,000 pairs: 10 kbp patterns vs 10.5 kbp texts, 10% edits (50/25/25, 20% homopolymer "
             "indels of 1-5 bases), W=64 O=24 k=64"),
    "short_reads": dict(
        make=lambda n, seed: synth.short_reads(n, seed=seed), n=1_000_000, seed=1, W=64, O=24,
        desc="1,000,000 pairs: patterns U{100..250} bp, texts +5% padding, 5% edits, W=64 O=24 k=64"),
    "uneven_reads": dict(
        make=lambda n, seed: synth.uneven_reads(n, seed=seed), n=200_000, seed=3, W=64, O=24,
        desc="200,000 pairs: log-normal lengths (median 8 kbp, 1-100 kbp), per-pair error U[1%,15%], W=64 O=24"),
    "tiny_windows": dict(
        make=lambda n, seed: synth.tiny_windows(n, seed=seed), n=1000, seed=0, W=64, O=24,
        desc="1,000 pairs: 110 bp texts, 100 bp patterns, 2% edits, W=64 O=24"),
}

METRIC = "alignments/s and Gbases/s on 1 GB300 (10 kbp, 10% err), learned+persistent vs plain"
INT_LOGIC_OPS_PER_CLK_PER_SM = 64  # LOP3/SHF pipe per SM per clock (scrooge_logic_peak measures it on the GPU)
PAPER_OPS_PER_CELL = 7  # bit-vector ops of one GenASM-DC cell: 3 shifts, 1 OR, 3 AND


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--scaling", choices=["weak", "strong"], default="weak",
                    help="weak: each rank aligns a batch of the workload's size; strong: the ranks share one batch")
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="long_reads")
    ap.add_argument("--pairs", type=int, default=0, help="override the workload's pair count")
    ap.add_argument("--W", type=int, default=0, help="override the workload's window size (k = W)")
    ap.add_argument("--O", type=int, default=-1, help="override the workload's window overlap")
    ap.add_argument("--flags", type=int, default=0, help="extra SCROOGE_* flags (ablations)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the built-in kernel settings (default: autotune on a separate sample first)")
    ap.add_argument("--lanes", type=int, default=0,
                    help="with --no-autotune: lanes per pair of the 64-base banded kernel (persistent launches and "
                         "the learned launches' rest bucket), with --rows and --wpb")
    ap.add_argument("--rows", type=int, default=8)
    ap.add_argument("--wpb", type=int, default=2)
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="time budget of the CPU baseline")
    ap.add_argument("--model", default="", help="saved ordering model (JSON); default: train one first")
    ap.add_argument("--train-pairs", type=int, default=50_000)
    ap.add_argument("--train-epochs", type=int, default=30)
    return ap.parse_args()


def self_launch(args) -> int:
    """Run this script as args.gpus ranks on this node under torch.distributed.run (127.0.0.1)."""
    import socket
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={args.gpus}",
           "--master-addr=127.0.0.1", f"--master-port={port}", os.path.abspath(__file__), *sys.argv[1:]]
    return subprocess.call(cmd)


def sharded_results(batch, world: int, rank: int, align_fn, cost=None, group=None):
    """Strong scaling: this rank's shard of one batch (longest-processing-time-first on `cost`, else
    contiguous), aligned by align_fn(sub_batch) -> result dict with a dense CIGAR, gathered on rank
    0 in pair order (None on the other ranks). Returns (pair indices of this rank, merged result)."""
    from paper_2208_09985_gb300 import shard
    idx = shard.shard_indices(batch.n_pairs, world, rank, cost)
    res = align_fn(batch.subset(idx))
    return idx, shard.gather_to_rank0(batch.n_pairs, idx, res, group)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while alive."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={gpu_index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        rows = [r.split(",") for r in out.strip().splitlines() if r.count(",") >= 8]
        if not rows:
            return None
        sm = [float(r[1]) for r in rows]
        mx = [float(r[2]) for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].strip().lower() == "active"})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": reasons, "samples": len(rows)}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def kernel_traffic(kernel: str, workload: str, n_pairs: int):
    """DRAM bytes per launch of an alignment kernel on `n_pairs` pairs of a workload, from the
    committed ncu summary (profiles/<kernel>_traffic.txt). The counters come from a capture of
    one launch on a smaller batch of the same workload and are scaled by the pairs processed.
    None when the kernel source changed since the counters were taken."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_traffic.txt")
    try:
        rec = dict(line.split(": ", 1) for line in open(path).read().splitlines()
                   if line and not line.startswith("#"))
    except (OSError, ValueError):
        return None
    h = hashlib.sha256()
    for name in KERNEL_SOURCES[kernel]:
        h.update(open(os.path.join(ROOT, "paper_2208_09985_gb300", "csrc", name), "rb").read())
    if (rec.get("source_sha256") != h.hexdigest() or rec.get("workload") != workload
            or "pairs_captured" not in rec or "dram_bytes_captured" not in rec):
        return None
    captured = int(rec["pairs_captured"])
    return {"bytes": int(rec["dram_bytes_captured"]) * n_pairs / captured, "pairs_captured": captured,
            "bytes_captured": int(rec["dram_bytes_captured"])}


def cpu_model() -> str:
    """Model name of the host CPU (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def cpu_baseline(batch, W, O, budget_s: float):
    """The oracle as it stands on all host cores, over a time-bounded prefix of the batch."""
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    chunk = 1024
    done, t0 = 0, time.perf_counter()
    while done < batch.n_pairs and time.perf_counter() - t0 < budget_s:
        hi = min(batch.n_pairs, done + chunk)
        oracle.align_batch(batch.subset(np.arange(done, hi)), W, O, threads=cores)
        done = hi
    dt = time.perf_counter() - t0
    bases = int(np.diff(batch.pattern_off)[:done].sum())
    return {"value": done / dt, "unit": "alignments/s", "cores": cores, "kind": "oracle",
            "cpu_model": cpu_model(), "gbases_per_s": bases / dt / 1e9,
            "sample": f"first {done} pairs of the workload (time-bounded at {budget_s:g} s), {cores} threads"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    wl = WORKLOADS[args.workload]
    n_total = args.pairs or wl["n"]
    per_step = min(n_total, 2048 if args.workload in ("long_reads", "uneven_reads") else 65536)
    batch = wl["make"](per_step, wl["seed"])
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    for _ in range(args.warmup):
        oracle.align_batch(batch, wl["W"], wl["O"], threads=cores)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.align_batch(batch, wl["W"], wl["O"], threads=cores)
        times.append(time.perf_counter() - t0)
    ms = 1e3 * sum(times) / len(times)
    value = per_step / (ms / 1e3)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "alignments/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32 bit-vectors", "data": "synthetic",
        "config": {"workload": args.workload, "desc": wl["desc"], "pairs_per_step": per_step,
                   "W": wl["W"], "O": wl["O"], "k": wl["W"]},
        "gbases_per_s": float(np.diff(batch.pattern_off).sum()) / (ms / 1e3) / 1e9,
        "cpu_baseline": {"value": value, "unit": "alignments/s", "cores": cores, "kind": "oracle",
                         "cpu_model": cpu_model(),
                         "sample": f"first {per_step} pairs of the workload per step, {cores} threads"},
        "e2e": {"value": value, "unit": "alignments/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


PATHS = ("plain", "persistent", "learned", "learned_graph", "full_width_persistent")


def path_flags(sc, name: str) -> int:
    return {"plain": 0, "persistent": sc.SCROOGE_PERSISTENT, "learned": sc.SCROOGE_LEARNED,
            "learned_graph": sc.SCROOGE_LEARNED | sc.SCROOGE_GRAPH,
            "full_width_persistent": sc.SCROOGE_PERSISTENT | sc.SCROOGE_NO_BAND}[name]


# sources of each alignment kernel, hashed to tell whether committed ncu counters still apply
KERNEL_SOURCES = {"align_band_kernel": ("align_band.cu", "align_kernel.cuh"),
                  "align_lane_kernel": ("align_lane.cu", "align_kernel.cuh"),
                  "align_kernel": ("align_kernel.cuh",)}


def kernel_name(sc, ctx, W: int, flags: int) -> str:
    """The alignment kernel that serves most pairs of a learned call with these flags (on 33..64-base
    windows: the rest bucket's kernel, or the persistent launch's when the model order is off)."""
    slot = sc.settings_slot(W, flags)
    if slot == 0 and sc.scrooge_get_learned_order(ctx):
        kind, lanes, _, _ = sc.scrooge_get_bucket_config(ctx, 1)
        if kind == 1:
            return "align_kernel"
        return "align_lane_kernel" if lanes == 1 else "align_band_kernel"
    if slot == 0:
        return "align_lane_kernel" if sc.scrooge_get_kernel_config(ctx, 0)[0] == 1 else "align_band_kernel"
    return "align_band_kernel" if slot == 3 else "align_kernel"


def prepare_model(sc, ctx, args):
    """Install the ordering model: from --model, else trained on 50,000 uneven pairs (seed 40)."""
    from paper_2208_09985_gb300 import learned
    if args.model:
        return {"source": args.model, **learned.load_model(ctx, args.model)}
    t0 = time.perf_counter()
    train = synth.uneven_reads(args.train_pairs, seed=40)
    tdb = sc.DeviceBatch(sc.PackedBatch(train))
    _, hist = learned.train(ctx, tdb, 64, 24, epochs=args.train_epochs, batch=1024, lr=2e-3, seed=1)
    del tdb
    return {"source": f"trained here on {args.train_pairs} uneven pairs (seed 40), {args.train_epochs} epochs",
            "final_mse": float(hist[-1]), "first_mse": float(hist[0]), "seconds": time.perf_counter() - t0}


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        if args.impl == "ours":
            import torch
            have = torch.cuda.device_count()
            if have < args.gpus:
                raise SystemExit(f"bench: --gpus {args.gpus} needs {args.gpus} GPUs; {have} visible")
        raise SystemExit(self_launch(args))
    if world != args.gpus:
        raise SystemExit(f"bench: --gpus {args.gpus} but WORLD_SIZE={world}")
    if args.impl == "reference":
        return run_reference(args)
    import torch
    import paper_2208_09985_gb300 as sc

    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    wl = WORKLOADS[args.workload]
    n_pairs = args.pairs or wl["n"]
    W = args.W or wl["W"]
    O = args.O if args.O >= 0 else wl["O"]
    k = W
    strong = args.scaling == "strong" and world > 1
    full_batch = None
    if strong:
        # one batch for the whole job; this rank aligns its cost-balanced shard
        full_batch = wl["make"](n_pairs, wl["seed"])
    batch = full_batch if strong else wl["make"](n_pairs, wl["seed"] + 1000 * rank)
    pb = sc.PackedBatch(batch)
    stream = torch.cuda.Stream()  # graph capture needs a stream other than the legacy default one
    torch.cuda.set_stream(stream)
    ctx = sc.scrooge_create(local, stream)
    words = 1 if W <= 32 else (2 if W <= 64 else 4)
    model_info = prepare_model(sc, ctx, args)
    flags = args.flags
    n_job = world * n_pairs  # pairs of the whole job
    if strong:
        # shard by predicted work: (pattern length + 1) x (predicted DP rows per window + 1), computed on
        # rank 0 with the ordering model and broadcast, so every rank sees the same partition
        from paper_2208_09985_gb300 import learned
        cost_t = torch.zeros(n_pairs, dtype=torch.float32, device="cuda")
        if rank == 0:
            fdb = sc.DeviceBatch(pb)
            feat = learned.device_features(ctx, fdb)
            pred = torch.zeros(n_pairs, dtype=torch.float32, device="cuda")
            sc.scrooge_model_predict(ctx, feat, n_pairs, pred)
            torch.cuda.synchronize()
            cost_t = (fdb.pat_len.to(torch.float32) + 1.0) * torch.expm1(pred).clamp_min(0.0).add(1.0)
            del fdb, feat, pred
        torch.distributed.broadcast(cost_t, src=0)
        cost_np = cost_t.cpu().numpy().astype(np.float64)
        from paper_2208_09985_gb300 import shard
        batch = full_batch.subset(shard.shard_indices(n_pairs, world, rank, cost_np))
        pb = sc.PackedBatch(batch)
        n_job = n_pairs
        n_pairs = batch.n_pairs  # this rank's pairs
    tune_info = None
    if not args.no_autotune:
        # kernel settings and the heavy load classes, tuned on a same-size sample drawn with another seed
        t0 = time.perf_counter()
        sample = wl["make"](n_pairs, wl["seed"] + 7 + 1000 * rank)
        sdb = sc.DeviceBatch(sc.PackedBatch(sample))
        table = sc.autotune_device(ctx, sdb, W, O, k, flags=flags | sc.SCROOGE_LEARNED, repeats=3)
        del sdb, sample
        tune_info = {"sample_pairs": n_pairs, "sample_seed": wl["seed"] + 7 + 1000 * rank, "configs_timed": len(table),
                     "class_ms": [[r[1], r[3] / 1e3] for r in table if r[4] == 2],
                     "best_settings_ms": sorted([[r[0], r[1], r[2], r[3] / 1e3] for r in table if r[4] == 1],
                                                key=lambda r: r[3])[:3],
                     "heavy_class": sc.scrooge_get_heavy_class(ctx), "long_class": sc.scrooge_get_long_class(ctx),
                     "buckets": {name: dict(zip(("kind", "lanes", "rows", "warps"),
                                                sc.scrooge_get_bucket_config(ctx, b)))
                                 for b, name in ((0, "heavy"), (1, "rest"))},
                     "bucket_best_ms": {name: sorted([[r[0] % 1000, r[1], r[2], r[3] / 1e3] for r in table
                                                      if r[4] == 3 and r[0] // 1000 == b], key=lambda r: r[3])[:3]
                                        for b, name in ((0, "heavy"), (1, "rest"))},
                     "learned_order": sc.scrooge_get_learned_order(ctx),
                     "order_ms": {"model": [r[3] / 1e3 for r in table if r[4] == 4 and r[0] == 1],
                                  "input": [r[3] / 1e3 for r in table if r[4] == 4 and r[0] == 0]},
                     "long_class_ms": [[r[1], r[3] / 1e3] for r in table if r[4] == 5],
                     "seconds": time.perf_counter() - t0}
    if args.no_autotune and args.lanes:
        sc.scrooge_set_kernel_config(ctx, 0, args.lanes, args.rows, args.wpb)
        sc.scrooge_set_bucket_config(ctx, 1, 0, args.lanes, args.rows, args.wpb)
    db = sc.DeviceBatch(pb)

    # untimed run with per-pair statistics: algorithmic DP cells of the method
    cells = torch.zeros(n_pairs, dtype=torch.int64, device="cuda")
    rows = torch.zeros(n_pairs, dtype=torch.int64, device="cuda")
    sc.scrooge_set_stats(ctx, None, rows, cells, None)
    sc.align_device(ctx, db, W, O, k, flags | sc.SCROOGE_SYNC)
    sc.scrooge_set_stats(ctx)
    total_cells = int(cells.sum().item())
    total_rows = int(rows.sum().item())
    ec = db.edit_counts.cpu().numpy()
    ref_off = db.cigar_off.cpu().numpy()
    total_runs = int(ref_off[-1])
    if (ec < 0).any() or total_runs > db.cigar_capacity:
        raise SystemExit("bench: some pairs failed or the CIGAR buffer is too small")
    ref_tc = db.text_consumed.clone()
    ref_cig = db.cigar[:total_runs].clone()

    def same_as_reference(tag):
        """Every timed path must give the stats run's results: edit counts, text consumed, CIGAR
        offsets and every CIGAR run (compared on the device, outside the timed region)."""
        import torch
        ok = (np.array_equal(db.edit_counts.cpu().numpy(), ec) and np.array_equal(db.cigar_off.cpu().numpy(), ref_off)
              and torch.equal(db.text_consumed, ref_tc) and torch.equal(db.cigar[:total_runs], ref_cig))
        if not ok:
            raise SystemExit(f"bench: {tag} changed the results")

    def timed(fl, sampler=False, kernel_events=False):
        """W warm-up steps, then K steps between CUDA events on the stream; max over ranks."""
        for _ in range(args.warmup):
            sc.align_device(ctx, db, W, O, k, fl)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        clocks = ClockSampler(local) if sampler else None
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        kev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        for a, b in kev:
            a.record(stream)
            b.record(stream)
        torch.cuda.synchronize()
        for i, (a, b) in enumerate(evs):
            if kernel_events:
                sc.scrooge_set_timing_events(ctx, kev[i][0], kev[i][1])
            a.record(stream)
            sc.align_device(ctx, db, W, O, k, fl)
            b.record(stream)
        torch.cuda.synchronize()
        sc.scrooge_set_timing_events(ctx)
        if world > 1:
            torch.distributed.barrier()
        clk = clocks.stop() if clocks else None
        step_ms = [a.elapsed_time(b) for a, b in evs]
        ker_ms = [a.elapsed_time(b) for a, b in kev] if kernel_events else None
        ms = sum(step_ms) / len(step_ms)
        if world > 1:
            t = torch.tensor([ms], device="cuda")
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
            ms = float(t.item())
        same_as_reference(f"flags {fl}")
        return ms, step_ms, ker_ms, clk, sc.scrooge_last_kernel_count(ctx)

    paths = {}
    for name in PATHS:
        fl = flags | path_flags(sc, name)
        ms, step_ms, _, clk, nk = timed(fl, sampler=(name == "learned_graph"))
        paths[name] = {"ms_per_step": ms, "alignments_per_s": n_job / (ms / 1e3),
                       "kernels_per_step": nk, "step_ms": [round(x, 4) for x in step_ms]}
        if name == "learned_graph":
            head_ms, head_steps, head_clk, head_kernels = ms, step_ms, clk, nk
    # the alignment kernel alone, timed inside the learned (non-graph) steps
    _, _, ker_ms, _, _ = timed(flags | sc.SCROOGE_LEARNED, kernel_events=True)
    kernel_ms = sum(ker_ms) / len(ker_ms)
    value = n_job / (head_ms / 1e3)
    bases = int(np.diff(batch.pattern_off).sum())
    bases_job = int(np.diff(full_batch.pattern_off).sum()) if strong else world * bases

    # end to end through the C ABI with pinned host buffers (learned + graph)
    e2e = None
    if not args.no_e2e:
        fl = flags | sc.SCROOGE_LEARNED | sc.SCROOGE_GRAPH
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
        h_in = [pin(x) for x in (pb.texts, pb.text_off, pb.text_len, pb.patterns, pb.pat_off, pb.pat_len)]
        cap = db.cigar_capacity
        h_ec = torch.zeros(n_pairs, dtype=torch.int32).pin_memory().numpy()
        h_tc = torch.zeros(n_pairs, dtype=torch.int32).pin_memory().numpy()
        h_off = torch.zeros(n_pairs + 1, dtype=torch.int64).pin_memory().numpy()
        h_cig = torch.zeros(cap, dtype=torch.int32).pin_memory().numpy().view(np.uint32)

        def call():
            sc.scrooge_align_batch(ctx, h_in[0], h_in[1], h_in[2], h_in[3], h_in[4], h_in[5], n_pairs, W, O,
                                   k, fl, h_ec, h_tc, h_cig, cap, h_off)
        for _ in range(args.warmup):
            call()
        e2e_steps = max(2, min(args.steps, 5))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            call()
        torch.cuda.synchronize()
        e2e_s = (time.perf_counter() - t0) / e2e_steps
        if world > 1:
            t = torch.tensor([e2e_s], device="cuda")
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
            e2e_s = float(t.item())
        h2d = sum(int(x.nbytes) for x in h_in)
        d2h = int(h_ec.nbytes + h_tc.nbytes + h_off.nbytes) + 4 * int(h_off[-1])
        if not (np.array_equal(h_ec, ec) and np.array_equal(h_off, ref_off)
                and np.array_equal(h_tc, ref_tc.cpu().numpy())
                and np.array_equal(h_cig[:total_runs], ref_cig.cpu().numpy().view(np.uint32))):
            raise SystemExit("bench: end-to-end results differ from the device-resident run")
        e2e = {"value": n_job / e2e_s, "unit": "alignments/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "gbases_per_s": bases_job / e2e_s / 1e9,
               "path": "learned + persistent + graph, host buffers"}

    # strong scaling: the shards' results, gathered on rank 0, equal a single-GPU run of the whole batch
    scaling_check = None
    if strong:
        mine = sc.device_results(db)
        tot = int(mine["cigar_off"][-1])
        local_res = {"edit_counts": mine["edit_counts"], "text_consumed": mine["text_consumed"],
                     "cigar": mine["cigar"][:tot], "cigar_off": mine["cigar_off"]}
        _, merged = sharded_results(full_batch, world, rank, lambda sub: local_res, cost_np)
        if rank == 0:
            fdb = sc.DeviceBatch(sc.PackedBatch(full_batch))
            sc.align_device(ctx, fdb, W, O, k, flags | sc.SCROOGE_SYNC)
            ref = sc.device_results(fdb)
            tot = int(ref["cigar_off"][-1])
            if not (np.array_equal(merged["edit_counts"], ref["edit_counts"])
                    and np.array_equal(merged["text_consumed"], ref["text_consumed"])
                    and np.array_equal(merged["cigar_off"], ref["cigar_off"])
                    and np.array_equal(merged["cigar"], ref["cigar"][:tot])):
                raise SystemExit("bench: the gathered shards differ from a single-GPU run of the whole batch")
            scaling_check = {"pairs": n_job, "shard": "LPT on predicted work", "identical_to_single_gpu": True}
            del fdb

    if rank != 0:
        sc.scrooge_destroy(ctx)
        if world > 1:
            torch.distributed.destroy_process_group()
        return

    # roofline of the alignment kernel: the integer logic pipe (LOP3/SHF)
    props = torch.cuda.get_device_properties(local)
    peaks = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz") or (head_clk or {}).get("sm_max_mhz") or 2070.0)
    peak_ops = props.multi_processor_count * INT_LOGIC_OPS_PER_CLK_PER_SM * sm_max * 1e6
    # algorithmic work: the paper's count of 7 bit-vector ops per DP cell (3 shifts, 1 OR, 3 AND,
    # Section 2.3.1 / its operational-intensity estimate), over the cells computed up to each
    # window's edit distance; the kernel basis is the full-width kernel's own 3*words-1 LOP3/SHF
    ops_per_cell = PAPER_OPS_PER_CELL
    kernel_ops_per_cell = 3 * words - 1
    kernel = kernel_name(sc, ctx, W, flags)
    achieved = total_cells * ops_per_cell / (kernel_ms / 1e3)
    probe = sc.scrooge_logic_peak(ctx, 4096)
    traffic = kernel_traffic(kernel, args.workload, n_pairs)
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(batch, W, O, args.cpu_seconds)
    plain = paths["plain"]["alignments_per_s"]
    line = {
        "metric": METRIC, "value": value, "unit": "alignments/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": head_ms, "higher_is_better": True,
        "scaling": "strong" if strong else "weak",
        "vs_baseline": None, "dtype": "u32 bit-vectors", "data": "synthetic",
        "config": {"workload": args.workload, "desc": wl["desc"], "pairs_per_gpu": n_pairs, "pairs_per_job": n_job,
                   "W": W, "O": O, "k": k,
                   "path": "learned ordering + persistent work queue + CUDA graph (value); plain, persistent and "
                           "learned without graph in `paths`", "flags": flags,
                   "kernel": kernel, "kernel_config": list(sc.scrooge_get_kernel_config(ctx, sc.settings_slot(W, flags))),
                   "l2": "inputs larger than L2 (packed inputs %.0f MB)" % (pb.texts.nbytes / 1e6 + pb.patterns.nbytes / 1e6),
                   "parallelism": f"dp{world}" if world > 1 else "single GPU"},
        "gbases_per_s": bases_job / (head_ms / 1e3) / 1e9,
        "paths": paths, "learned_gain_vs_plain": value / plain,
        "learned_gain_vs_persistent": value / paths["persistent"]["alignments_per_s"],
        "model": model_info, "autotune": tune_info,
        "mean_edits_per_pair": float(ec.mean()), "cigar_runs_per_step": total_runs,
        "dp_cells_per_step": total_cells, "dp_rows_per_step": total_rows,
        "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": peak_ops / 1e12, "unit": "Tops/s",
                     "frac": achieved / peak_ops, "frac_survey_basis": achieved / peak_ops,
                     "frac_kernel_basis": total_cells * kernel_ops_per_cell / (kernel_ms / 1e3) / peak_ops,
                     "traffic": None if traffic is None else traffic["bytes"],
                     "traffic_basis": None if traffic is None else
                     f"ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch on the first "
                     f"{traffic['pairs_captured']} pairs ({traffic['bytes_captured']} B), scaled by pairs",
                     "kernel": kernel, "kernel_ms": kernel_ms,
                     "basis": f"{ops_per_cell} bit-vector ops per DP cell (the paper's count) over the cells "
                              f"computed up to each window's edit distance ({total_cells} per step); "
                              f"frac_kernel_basis: {kernel_ops_per_cell} LOP3/SHF per cell; alignment kernel timed "
                              f"alone (events around it, learned order); peak = {props.multi_processor_count} SMs x "
                              f"{INT_LOGIC_OPS_PER_CLK_PER_SM} logic ops/clk x {sm_max:.0f} MHz (unit counts and "
                              f"clocks; peak_probe measures the per-SM rate on this GPU)",
                     "peak_probe": {"ops_per_s": probe["ops_per_s"] / 1e12,
                                    "ops_per_clk_per_sm": probe["ops_per_clk_per_sm"], "unit": "Tops/s",
                                    "what": "scrooge_logic_peak: 8 independent LOP3+SHF chains per thread, "
                                            "one wave of blocks"}},
        "clocks": head_clk,
        "gpu_launches": args.steps * head_kernels,
        "e2e": e2e,
        "cpu_baseline": cpu,
        "step_ms": [round(x, 4) for x in head_steps],
    }
    if scaling_check:
        line["sharding"] = scaling_check
    print(json.dumps(line), flush=True)
    sc.scrooge_destroy(ctx)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
