"""Parity of the CUDA path with the CPU oracle (needs a GB300).

Every comparison is bit-exact: edit counts, text consumed, CIGAR lengths and
every CIGAR run. Inputs are the seeded synthetic workloads; the oracle sees
codes 0..3, the CUDA library the packed form produced by its own packer.
"""
import os

import numpy as np
import pytest

import oracle
import paper_2208_09985_gb300 as sc
from paper_2208_09985_gb300 import synth
from tests._compare import assert_same

pytestmark = pytest.mark.gpu

THREADS = os.cpu_count() or 4


@pytest.fixture(scope="module")
def ctx():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    oracle.build()
    h = sc.scrooge_create(0)
    yield h
    sc.scrooge_destroy(h)


def _both(ctx, batch, W=64, O=24, k=None, flags=0):
    pb = sc.PackedBatch(batch)
    g = sc.align_host(ctx, pb, W, O, k, flags)
    r = oracle.align_batch(batch, W, O, k, threads=THREADS)
    return g, r


def test_tiny_windows_full(ctx):
    b = synth.tiny_windows(1000, seed=0)
    g, r = _both(ctx, b)
    assert_same(g, r, label="tiny_windows")
    assert (g["edit_counts"] >= 0).all()


def _kernels(W):
    """(settings slot, extra flags, label) of every kernel that serves windows of W bases."""
    words = 1 if W <= 32 else (2 if W <= 64 else 4)
    out = [(words, sc.SCROOGE_NO_BAND if words > 1 else 0, f"full{words}")]
    if words == 2:
        out.append((0, 0, "band64"))
    if words == 4:
        out.append((3, 0, "band128"))
    return out


@pytest.mark.parametrize("W", [32, 64, 128, 16, 40, 100, 1, 2, 33])
def test_random_edge_cases_all_lane_configs(ctx, W):
    rng = np.random.default_rng(W)
    b = synth.random_pairs(300, max_text=4 * W + 5, max_pattern=4 * W + 5, seed=100 + W)
    for slot, flags, name in _kernels(W):
        lanes_opts = {1: [1, 2, 4], 2: [2, 4, 8], 4: [8, 16], 0: [1, 2, 4, 8], 3: [8, 16]}[slot]
        saved = sc.scrooge_get_kernel_config(ctx, slot)
        try:
            for lanes in lanes_opts:
                for rows in (1, 3, 40):
                    sc.scrooge_set_kernel_config(ctx, slot, lanes, rows, 2)
                    O = int(rng.integers(0, W))
                    for k in (W, max(0, W // 8), 16, 15, 32, 31):
                        if k > W:
                            continue
                        g, r = _both(ctx, b, W, O, k, flags)
                        assert_same(g, r, label=f"{name} W={W} O={O} k={k} lanes={lanes} rows={rows}")
        finally:
            sc.scrooge_set_kernel_config(ctx, slot, *saved)


@pytest.mark.parametrize("lanes", [1, 2, 4, 8])
def test_band_fallback_windows(ctx, lanes):
    """Windows whose edit distance exceeds the band (d_opt > 15) are recomputed at full width."""
    b = synth.concat([synth.fixed_error(30, 0.25, length=600, seed=61), synth.fixed_error(30, 0.35, length=400, seed=62),
                      synth.random_pairs(150, 300, 300, seed=63), synth.long_reads(4, seed=64)])
    pb = sc.PackedBatch(b)
    saved = sc.scrooge_get_kernel_config(ctx, 0)
    try:
        for rows in (1, 5, 16):
            sc.scrooge_set_kernel_config(ctx, 0, lanes, rows, 2)
            for O, k in ((24, 64), (24, 16), (24, 17), (33, 40), (24, 15), (0, 64), (63, 64)):
                g = sc.align_host(ctx, pb, 64, O, k)
                r = oracle.align_batch(b, 64, O, k, threads=THREADS)
                assert_same(g, r, label=f"band lanes={lanes} rows={rows} O={O} k={k}")
    finally:
        sc.scrooge_set_kernel_config(ctx, 0, *saved)


@pytest.mark.parametrize("flags", list(range(16)))
def test_ablation_flags_identical(ctx, flags):
    f = (sc.SCROOGE_NO_SENE if flags & 1 else 0) | (sc.SCROOGE_NO_DENT if flags & 2 else 0) | \
        (sc.SCROOGE_NO_ET if flags & 4 else 0) | (sc.SCROOGE_NO_BAND if flags & 8 else 0)
    b = synth.concat([synth.tiny_windows(200, seed=5), synth.long_reads(6, seed=9),
                      synth.random_pairs(100, 200, 200, seed=8)])
    for W, O in ((64, 24), (64, 33), (32, 17), (128, 64)):
        g, r = _both(ctx, b, W, O, flags=f)
        assert_same(g, r, label=f"flags={f} W={W} O={O}")


def test_kernel_shapes_w64(ctx):
    b = synth.concat([synth.long_reads(8, seed=21), synth.short_reads(300, seed=22),
                      synth.fixed_error(4, 0.15, seed=23)])
    r = oracle.align_batch(b, 64, 24, threads=THREADS)
    pb = sc.PackedBatch(b)
    for slot, flags, name in _kernels(64):
        saved = sc.scrooge_get_kernel_config(ctx, slot)
        try:
            for lanes in ((1, 2, 4, 8) if slot == 0 else (2, 4, 8)):
                for rows in (1, 6, 12, 65):
                    for wpb in (1, 2):
                        sc.scrooge_set_kernel_config(ctx, slot, lanes, rows, wpb)
                        g = sc.align_host(ctx, pb, 64, 24, flags=flags)
                        assert_same(g, r, label=f"{name} lanes={lanes} rows={rows} wpb={wpb}")
        finally:
            sc.scrooge_set_kernel_config(ctx, slot, *saved)


def test_device_pointers_match_host(ctx):
    import torch
    b = synth.short_reads(5000, seed=31)
    pb = sc.PackedBatch(b)
    h = sc.align_host(ctx, pb)
    db = sc.DeviceBatch(pb)
    sc.align_device(ctx, db, 64, 24, flags=sc.SCROOGE_SYNC)
    torch.cuda.synchronize()
    d = sc.device_results(db)
    np.testing.assert_array_equal(d["edit_counts"], h["edit_counts"])
    np.testing.assert_array_equal(d["text_consumed"], h["text_consumed"])
    np.testing.assert_array_equal(d["cigar_lens"], h["cigar_lens"])
    np.testing.assert_array_equal(d["cigar_off"], h["cigar_off"])
    tot = int(h["cigar_off"][-1])
    assert np.array_equal(d["cigar"][:tot], h["cigar"][:tot])


def test_workload_subsets(ctx):
    for b in (synth.short_reads(20_000), synth.long_reads(200), synth.uneven_reads(120),
              synth.fixed_error(100, 0.05, seed=5), synth.fixed_error(100, 0.15, seed=7)):
        g, r = _both(ctx, b)
        assert_same(g, r, label=b.name)


def test_k_failures(ctx):
    b = synth.concat([synth.random_pairs(200, 150, 150, seed=41, rate_max=0.6), synth.tiny_windows(100, seed=3)])
    for k in (0, 1, 3, 8):
        g, r = _both(ctx, b, 64, 24, k)
        assert_same(g, r, label=f"k={k}")
        assert (g["edit_counts"] == -1).any() or k == 8


def test_cigar_capacity_too_small(ctx):
    """A short output buffer is reported; alignments and offsets stay valid; fitting pairs are written."""
    b = synth.random_pairs(300, 200, 200, seed=43, rate_max=0.4)
    pb = sc.PackedBatch(b)
    full = sc.align_host(ctx, pb)
    total = int(full["cigar_off"][-1])
    for cap in (0, 1, total // 2, total - 1):
        n = b.n_pairs
        ec, tc, off = np.zeros(n, np.int32), np.zeros(n, np.int32), np.zeros(n + 1, np.int64)
        cig = np.zeros(max(cap, 1), np.uint32)
        with pytest.raises(sc.ScroogeError) as e:
            sc.scrooge_align_batch(ctx, pb.texts, pb.text_off, pb.text_len, pb.patterns, pb.pat_off, pb.pat_len, n,
                                   64, 24, 64, 0, ec, tc, cig, cap, off)
        assert e.value.code == sc.SCROOGE_E_CAPACITY
        np.testing.assert_array_equal(ec, full["edit_counts"])
        np.testing.assert_array_equal(off, full["cigar_off"])
        fits = np.flatnonzero(off[1:] <= cap)
        for p in fits:
            assert np.array_equal(cig[off[p]:off[p + 1]], full["cigar"][off[p]:off[p + 1]])
    # device pointers: the total tells the caller
    import torch
    db = sc.DeviceBatch(pb, cigar_capacity=total - 1)
    sc.align_device(ctx, db, 64, 24)
    torch.cuda.synchronize()
    assert int(db.cigar_off[-1]) == total


def test_bad_arguments(ctx):
    b = synth.tiny_windows(4)
    pb = sc.PackedBatch(b)
    for W, O, k in ((0, 0, 0), (129, 0, 10), (64, 64, 64), (64, -1, 64), (64, 24, 65), (64, 24, -1)):
        with pytest.raises(sc.ScroogeError) as e:
            sc.align_host(ctx, pb, W, O, k)
        assert e.value.code == sc.SCROOGE_E_INVAL
    bad = sc.PackedBatch(b)
    bad.text_off = bad.text_off.copy()
    bad.text_off[1] += 16
    with pytest.raises(sc.ScroogeError) as e:
        sc.align_host(ctx, bad)
    assert e.value.code == sc.SCROOGE_E_INVAL


def test_allocation_failure_is_reported_and_recovers(ctx):
    ctx2 = sc.scrooge_create(0)
    try:
        b = synth.tiny_windows(50)
        pb = sc.PackedBatch(b)
        sc.scrooge_debug_fail_next_allocs(ctx2, 1)
        with pytest.raises(sc.ScroogeError) as e:
            sc.align_host(ctx2, pb)
        assert e.value.code == sc.SCROOGE_E_NOMEM
        g = sc.align_host(ctx2, pb)
        r = oracle.align_batch(b, 64, 24, threads=THREADS)
        assert_same(g, r, label="after injected allocation failure")
    finally:
        sc.scrooge_destroy(ctx2)


def test_stats_count_rows(ctx):
    import torch
    b = synth.long_reads(16, seed=77)
    pb = sc.PackedBatch(b)
    n = b.n_pairs
    win = torch.zeros(n, dtype=torch.int32, device="cuda")
    rows = torch.zeros(n, dtype=torch.int64, device="cuda")
    cells = torch.zeros(n, dtype=torch.int64, device="cuda")
    cyc = torch.zeros(n, dtype=torch.int64, device="cuda")
    sc.scrooge_set_stats(ctx, win, rows, cells, cyc)
    try:
        sc.align_host(ctx, pb)
    finally:
        sc.scrooge_set_stats(ctx)
    for p in range(n):
        r = oracle.align_pair(b.text(p), b.pattern(p), 64, 24)
        assert int(win[p]) == r["d_opt"].shape[0]
        assert int(rows[p]) == int((r["d_opt"] + 1).sum())
    assert (cyc.cpu().numpy() > 0).all()


@pytest.mark.parametrize("rows", [1, 4, 8])
def test_warp_specialized_blocks(ctx, rows):
    """Persistent banded launches as DC + traceback warps give the oracle's results."""
    b = synth.concat([synth.long_reads(6, seed=71), synth.short_reads(600, seed=72),
                      synth.fixed_error(20, 0.2, length=1500, seed=73), synth.random_pairs(300, 300, 300, seed=74),
                      synth.tiny_windows(50, seed=75)])
    pb = sc.PackedBatch(b)
    saved = sc.scrooge_get_kernel_config(ctx, 0)
    try:
        sc.scrooge_set_kernel_config(ctx, 0, 4, rows, 2)
        for O, k in ((24, 64), (33, 64), (24, 12), (40, 20), (0, 64)):
            r = oracle.align_batch(b, 64, O, k, threads=THREADS)
            g = sc.align_host(ctx, pb, 64, O, k, sc.SCROOGE_PERSISTENT | sc.SCROOGE_WARP_SPECIALIZED)
            assert_same(g, r, label=f"warp-specialised rows={rows} O={O} k={k}")
    finally:
        sc.scrooge_set_kernel_config(ctx, 0, *saved)


def test_bounded_wait_times_out_and_recovers(ctx):
    """A barrier wait of the warp-specialised blocks that runs out of polls makes the call return
    SCROOGE_E_TIMEOUT (no fault, no hang: every warp leaves); with the default bound restored the
    same context gives the oracle's results. One poll per wait is far too few: the traceback warp
    waits for a window the DC warps have only begun."""
    b = synth.concat([synth.long_reads(4, seed=91), synth.short_reads(300, seed=92)])
    pb = sc.PackedBatch(b)
    r = oracle.align_batch(b, 64, 24, threads=THREADS)
    fl = sc.SCROOGE_PERSISTENT | sc.SCROOGE_WARP_SPECIALIZED
    codes = []
    try:
        sc.scrooge_set_wait_limit(ctx, 1)
        for _ in range(3):
            try:
                sc.align_host(ctx, pb, 64, 24, None, fl)
                codes.append(0)
            except sc.ScroogeError as e:
                codes.append(e.code)
    finally:
        sc.scrooge_set_wait_limit(ctx, 0)
    assert sc.SCROOGE_E_TIMEOUT in codes and set(codes) <= {0, sc.SCROOGE_E_TIMEOUT}, codes
    g = sc.align_host(ctx, pb, 64, 24, None, fl)
    assert_same(g, r, label="after a timed-out wait")


def test_warp_specialized_few_pairs(ctx):
    """Fewer pairs than slots, a single pair, and empty patterns."""
    for b in (synth.tiny_windows(1, seed=81), synth.tiny_windows(7, seed=82), synth.short_reads(65, seed=83),
              synth.from_lists(["ACGT" * 30, "", "ACG"], ["", "ACGT", "ACGTT"])):
        r = oracle.align_batch(b, 64, 24, threads=THREADS)
        g = sc.align_host(ctx, sc.PackedBatch(b), 64, 24, None, sc.SCROOGE_PERSISTENT | sc.SCROOGE_WARP_SPECIALIZED)
        assert_same(g, r, label=f"warp-specialised {b.n_pairs} pairs")


@pytest.mark.parametrize("lanes", [8, 16])
def test_band128_windows_and_fallback(ctx, lanes):
    """The 64-diagonal band for 65..128-base windows, with windows beyond it (d_opt > 31)."""
    b = synth.concat([synth.fixed_error(20, 0.12, length=2000, seed=101), synth.fixed_error(20, 0.3, length=800, seed=102),
                      synth.random_pairs(120, 500, 500, seed=103), synth.long_reads(3, seed=104)])
    pb = sc.PackedBatch(b)
    saved = sc.scrooge_get_kernel_config(ctx, 3)
    try:
        for rows in (1, 6, 32):
            sc.scrooge_set_kernel_config(ctx, 3, lanes, rows, 2)
            for W, O, k in ((128, 32, 128), (128, 64, 32), (128, 48, 31), (100, 37, 100), (65, 1, 65), (128, 0, 128),
                            (128, 127, 40)):
                g = sc.align_host(ctx, pb, W, O, k)
                r = oracle.align_batch(b, W, O, k, threads=THREADS)
                assert_same(g, r, label=f"band128 lanes={lanes} rows={rows} W={W} O={O} k={k}")
    finally:
        sc.scrooge_set_kernel_config(ctx, 3, *saved)


@pytest.mark.parametrize("lanes", [4, 8])
def test_wide_band_for_64_base_windows(ctx, lanes):
    """SCROOGE_WIDE_BAND: 64 diagonals for 64-base windows, exact for d_opt <= 31, full width beyond."""
    b = synth.concat([synth.fixed_error(20, 0.25, length=600, seed=111), synth.fixed_error(20, 0.4, length=400, seed=112),
                      synth.random_pairs(150, 300, 300, seed=113), synth.long_reads(3, seed=114),
                      synth.short_reads(200, seed=115)])
    pb = sc.PackedBatch(b)
    saved = sc.scrooge_get_kernel_config(ctx, 0)
    try:
        for rows in (1, 8, 32):
            sc.scrooge_set_kernel_config(ctx, 0, lanes, rows, 2)
            for W, O, k in ((64, 24, 64), (64, 24, 32), (64, 24, 31), (64, 33, 16), (48, 10, 48), (64, 0, 64)):
                for extra in (0, sc.SCROOGE_PERSISTENT):
                    g = sc.align_host(ctx, pb, W, O, k, sc.SCROOGE_WIDE_BAND | extra)
                    r = oracle.align_batch(b, W, O, k, threads=THREADS)
                    assert_same(g, r, label=f"wide band lanes={lanes} rows={rows} W={W} O={O} k={k} flags={extra}")
    finally:
        sc.scrooge_set_kernel_config(ctx, 0, *saved)


@pytest.mark.parametrize("W,O", [(16, 12), (32, 24), (32, 31), (64, 56), (64, 63), (100, 90), (128, 120)])
def test_extended_dent_row_cycle(ctx, W, O):
    """DENT extended to rows (Supplementary Section 1): each window of a full-width kernel keeps
    max(W-O+lanes, ceil((k+1)/2)) row slots (row d in slot d mod that), which these high-error
    windows with small W-O wrap around. Results equal the oracle's, and those of the ablation
    keeping all k+1 rows; the banded kernels, which keep all rows, are checked beside them."""
    b = synth.concat([synth.random_pairs(200, 3 * W, 3 * W, seed=900 + W + O),
                      synth.fixed_error(20, 0.35, length=8 * W, seed=901 + O),
                      synth.fixed_error(20, 0.10, length=8 * W, seed=902)])
    pb = sc.PackedBatch(b)
    r = oracle.align_batch(b, W, O, W, threads=THREADS)
    # these small W-O give the floor of ceil((k+1)/2) slots; windows this deep wrap the cycle
    deep = max(int(oracle.align_pair(b.text(p), b.pattern(p), W, O, W)["d_opt"].max(initial=-1)) for p in range(40))
    assert deep >= (W + 2) // 2
    for slot, flags, name in _kernels(W):
        lanes_opts = {1: [1, 2, 4], 2: [2, 4, 8], 4: [8, 16], 0: [1, 2, 4, 8], 3: [8, 16]}[slot]
        saved = sc.scrooge_get_kernel_config(ctx, slot)
        try:
            for lanes in lanes_opts:
                for rows in (1, 4, 64):
                    sc.scrooge_set_kernel_config(ctx, slot, lanes, rows, 2)
                    g = sc.align_host(ctx, pb, W, O, W, flags)
                    assert_same(g, r, label=f"{name} W={W} O={O} lanes={lanes} rows={rows}")
                    shape = sc.scrooge_last_launch_shape(ctx)
                    cycle = min(W + 1, max(W - O + shape["lanes"], (W + 2) // 2))
                    assert shape["row_slots"] == (W + 1 if name.startswith("band") else cycle), shape
                    g = sc.align_host(ctx, pb, W, O, W, flags | sc.SCROOGE_NO_EXT_DENT)
                    assert_same(g, r, label=f"{name} W={W} O={O} lanes={lanes} rows={rows} all rows")
                    assert sc.scrooge_last_launch_shape(ctx)["row_slots"] == W + 1
        finally:
            sc.scrooge_set_kernel_config(ctx, slot, *saved)
    if W == 64:
        for extra in (sc.SCROOGE_PERSISTENT | sc.SCROOGE_WARP_SPECIALIZED, sc.SCROOGE_WIDE_BAND):
            g = sc.align_host(ctx, pb, W, O, W, extra)
            assert_same(g, r, label=f"W={W} O={O} flags={extra}")
