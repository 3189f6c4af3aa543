"""Every pair of the full-size workloads against the CPU oracle (needs a GB300).

The short-read (1,000,000 pairs), long-read (100,000) and uneven-read
(200,000) workloads, and the fixed-error sweep (20,000 pairs at each of 5, 10
and 15% edits) at the operating points W/O = 64/24, 64/33 and 32/17, are
aligned on the GPU in the launch configurations the benchmark times (plain,
persistent, learned ordering with CUDA-graph replay) and compared with the
oracle pair by pair: edit counts, text consumed, CIGAR run counts and every
CIGAR run, bit for bit. The oracle runs once per workload and operating point
on all host cores.
"""
import os

import numpy as np
import pytest

import oracle
import paper_2208_09985_gb300 as sc
from paper_2208_09985_gb300 import learned, synth
from tests._compare import assert_same_all

pytestmark = pytest.mark.gpu

THREADS = os.cpu_count() or 4


@pytest.fixture(scope="module")
def ctx():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    oracle.build()
    s = torch.cuda.Stream()  # graph capture needs a stream other than the legacy default one
    h = sc.scrooge_create(0, s)
    # an ordering model trained on the method's own statistics (uneven reads, another seed)
    train = sc.DeviceBatch(sc.PackedBatch(synth.uneven_reads(4000, seed=40)))
    with torch.cuda.stream(s):
        learned.train(h, train, 64, 24, epochs=8, batch=512, lr=2e-3, seed=1)
    s.synchronize()
    del train
    yield h, s
    sc.scrooge_destroy(h)


def _gpu(ctx, db, W, O, flags):
    import torch
    h, s = ctx
    with torch.cuda.stream(s):
        sc.align_device(h, db, W, O, W, flags | sc.SCROOGE_SYNC)
    s.synchronize()
    return sc.device_results(db)


def _check_paths(ctx, batch, W, O, paths, label):
    pb = sc.PackedBatch(batch)
    ref = oracle.align_batch(batch, W, O, W, threads=THREADS)
    # capacity for every run of the batch (the oracle's count) so no call is cut short
    db = sc.DeviceBatch(pb, cigar_capacity=int(np.asarray(ref["cigar_lens"]).astype(np.int64).sum()) + 16)
    h, _ = ctx
    for path in paths:
        name, flags = path[:2]
        cfg = path[2] if len(path) > 2 else None  # kernel settings of the 33..64-base windows' slot
        saved = sc.scrooge_get_kernel_config(h, 0)
        try:
            if cfg:
                sc.scrooge_set_kernel_config(h, 0, *cfg)
            got = _gpu(ctx, db, W, O, flags)
        finally:
            sc.scrooge_set_kernel_config(h, 0, *saved)
        assert_same_all(got, ref, label=f"{label} {name} W={W} O={O}")
    return ref


PLAIN = ("plain", 0)
PERSISTENT = ("persistent", sc.SCROOGE_PERSISTENT)
LEARNED_GRAPH = ("learned+graph", sc.SCROOGE_LEARNED | sc.SCROOGE_GRAPH)


# the one-lane-per-pair kernel with one, two and three shared-memory row slots: every row the
# traceback reads then goes through the device area, so the eviction copies are exercised at scale
LANE_SLOTS = tuple((f"persistent lanes 1 rows {r} warps {w}", sc.SCROOGE_PERSISTENT, (1, r, w))
                   for r, w in ((1, 1), (2, 1), (3, 2)))


def test_long_reads_every_pair(ctx):
    """100,000 pairs of 10 kbp at 10% edits: the benchmark's workload."""
    ref = _check_paths(ctx, synth.long_reads(100_000), 64, 24, (PLAIN, PERSISTENT, LEARNED_GRAPH) + LANE_SLOTS,
                       "long_reads")
    assert (ref["edit_counts"] >= 0).all()


def test_short_reads_every_pair(ctx):
    """1,000,000 short-read pairs (100-250 bp, 5% edits)."""
    _check_paths(ctx, synth.short_reads(1_000_000), 64, 24, (PLAIN, PERSISTENT, LEARNED_GRAPH), "short_reads")


def test_uneven_reads_every_pair(ctx):
    """200,000 uneven pairs (log-normal lengths, 1-15% edits): learned ordering + persistent queue +
    CUDA graph against the unsorted plain launch and the oracle."""
    _check_paths(ctx, synth.uneven_reads(200_000), 64, 24, (PLAIN, LEARNED_GRAPH), "uneven_reads")


@pytest.mark.parametrize("rate,seed", [(0.05, 5), (0.10, 6), (0.15, 7)])
def test_fixed_error_sweep_every_pair(ctx, rate, seed):
    """20,000 pairs of 10 kbp at one error rate, at the benchmark's operating point and at the
    paper's two (W=64/O=33 for long reads, W=32/O=17 for short reads)."""
    b = synth.fixed_error(20_000, rate, seed=seed)
    for W, O in ((64, 24), (64, 33), (32, 17)):
        _check_paths(ctx, b, W, O, (PLAIN, LEARNED_GRAPH), f"fixed_error {rate:.0%}")
