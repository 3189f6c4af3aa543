"""Host-pointer calls in parts (copies under the kernels) against one launch and the oracle
(needs a GB300).

A persistent call with host pointers on at least 8,192 pairs runs as launches over 2 to 4 parts
of its pairs (a part holds at least a wave of the kernel's pair slots where the batch allows),
each part's copies overlapping the other parts' kernels.
The results must be those of the one-launch path and of the oracle, bit for bit: with pairs laid
out in order, with sequences out of pair order (the first part then needs the whole arrays), and
with a CIGAR buffer that ends inside any part.
"""
import copy
import os

import numpy as np
import pytest

import oracle
import paper_2208_09985_gb300 as sc
from paper_2208_09985_gb300 import synth
from tests._compare import assert_same_all

pytestmark = pytest.mark.gpu

THREADS = os.cpu_count() or 4


@pytest.fixture(scope="module")
def ctx():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    oracle.build()
    h = sc.scrooge_create(0)
    yield h
    sc.scrooge_set_host_overlap(h, True)
    sc.scrooge_destroy(h)


def _run(ctx, pb, overlap, cap=None, W=64, O=24):
    sc.scrooge_set_host_overlap(ctx, overlap)
    return sc.align_host(ctx, pb, W, O, W, sc.SCROOGE_PERSISTENT, cigar_capacity=cap)


def _same(a, b, label):
    for key in ("edit_counts", "text_consumed", "cigar_off"):
        assert np.array_equal(a[key], b[key]), f"{label}: {key}"
    tot = int(a["cigar_off"][-1])
    assert np.array_equal(a["cigar"][:tot], b["cigar"][:tot]), f"{label}: cigar"


def test_two_halves_equal_one_launch_and_oracle(ctx):
    b = synth.concat([synth.long_reads(6000, seed=71), synth.short_reads(6000, seed=72),
                      synth.uneven_reads(2000, seed=73)])
    pb = sc.PackedBatch(b)
    assert pb.n_pairs >= 8192
    split = _run(ctx, pb, True)
    one = _run(ctx, pb, False)
    _same(split, one, "two halves vs one launch")
    assert_same_all(split, oracle.align_batch(b, 64, 24, 64, threads=THREADS), label="two halves vs oracle")
    again = _run(ctx, pb, True)  # a second call on the same context and buffers
    _same(again, split, "second call")


@pytest.mark.parametrize("W,O,extra", [(32, 17, 0), (64, 24, sc.SCROOGE_NO_BAND), (64, 33, sc.SCROOGE_NO_SENE),
                                        (128, 64, 0)])
def test_two_halves_other_kernels(ctx, W, O, extra):
    """The two halves on the full-width kernels, the SENE-off ablation and the 128-base band."""
    b = synth.concat([synth.long_reads(2500, seed=81), synth.short_reads(7000, seed=82)])
    pb = sc.PackedBatch(b)
    got = {}
    for overlap in (True, False):
        sc.scrooge_set_host_overlap(ctx, overlap)
        got[overlap] = sc.align_host(ctx, pb, W, O, W, sc.SCROOGE_PERSISTENT | extra)
    _same(got[True], got[False], f"W={W} O={O} flags={extra}")


def test_two_halves_sequences_out_of_order(ctx):
    """Pairs whose sequences lie out of pair order: the first half's prefix of the arrays is all of them."""
    b = synth.concat([synth.long_reads(3000, seed=74), synth.short_reads(7000, seed=75)])
    pb = sc.PackedBatch(b)
    perm = np.random.default_rng(76).permutation(pb.n_pairs)
    q = copy.copy(pb)
    q.text_off, q.text_len = pb.text_off[perm].copy(), pb.text_len[perm].copy()
    q.pat_off, q.pat_len = pb.pat_off[perm].copy(), pb.pat_len[perm].copy()
    ref = _run(ctx, pb, False)
    got = _run(ctx, q, True)
    lens = np.diff(ref["cigar_off"])
    assert np.array_equal(got["edit_counts"], ref["edit_counts"][perm])
    assert np.array_equal(got["text_consumed"], ref["text_consumed"][perm])
    assert np.array_equal(np.diff(got["cigar_off"]), lens[perm])
    for i in range(0, pb.n_pairs, 97):
        p = perm[i]
        a = got["cigar"][got["cigar_off"][i]:got["cigar_off"][i + 1]]
        r = ref["cigar"][ref["cigar_off"][p]:ref["cigar_off"][p + 1]]
        assert np.array_equal(a, r), f"pair {i}"


@pytest.mark.parametrize("where", ["second half", "first half"])
def test_two_halves_capacity_too_small(ctx, where):
    """A CIGAR buffer that ends inside one half: the call reports the capacity needed, every offset is
    the one-launch path's, and the pairs that fit are written as there."""
    b = synth.concat([synth.long_reads(4000, seed=77), synth.short_reads(6000, seed=78)])
    pb = sc.PackedBatch(b)
    full = _run(ctx, pb, False)
    off = full["cigar_off"]
    h = pb.n_pairs // 2
    cap = int(off[h] + (off[-1] - off[h]) // 3) if where == "second half" else int(off[h] // 2)
    out = {}
    for overlap in (True, False):
        sc.scrooge_set_host_overlap(ctx, overlap)
        n = pb.n_pairs
        ec, tc = np.zeros(n, np.int32), np.zeros(n, np.int32)
        o, cig = np.zeros(n + 1, np.int64), np.zeros(cap, np.uint32)
        with pytest.raises(sc.ScroogeError) as err:
            sc.scrooge_align_batch(ctx, pb.texts, pb.text_off, pb.text_len, pb.patterns, pb.pat_off, pb.pat_len, n,
                                   64, 24, 64, sc.SCROOGE_PERSISTENT, ec, tc, cig, cap, o)
        assert err.value.code == sc.SCROOGE_E_CAPACITY
        assert np.array_equal(o, off)
        assert np.array_equal(ec, full["edit_counts"])
        out[overlap] = cig
    fits = np.flatnonzero(off[1:] <= cap)
    for p in fits[::53]:
        s, e = off[p], off[p + 1]
        assert np.array_equal(out[True][s:e], full["cigar"][s:e]), f"pair {p}"
        assert np.array_equal(out[False][s:e], full["cigar"][s:e]), f"pair {p}"


def test_large_batch_layout_checked_by_threads(ctx):
    """Batches of 65,536 pairs or more have their layout checked by several host threads: the results are
    those of the one-launch path, and a broken pair is reported by its index (the first broken one)."""
    b = synth.short_reads(120_000, seed=83)
    pb = sc.PackedBatch(b)
    got = {}
    for overlap in (True, False):
        sc.scrooge_set_host_overlap(ctx, overlap)
        got[overlap] = sc.align_host(ctx, pb, 64, 24, 64, sc.SCROOGE_PERSISTENT)
    _same(got[True], got[False], "120,000 short reads")
    for q in (119_990, 61_000):
        bad = copy.copy(pb)
        bad.pat_off = pb.pat_off.copy()
        bad.pat_off[q] += 16
        bad.pat_off[119_995] += 32  # a later broken pair: the first one is named
        for overlap in (True, False):
            sc.scrooge_set_host_overlap(ctx, overlap)
            with pytest.raises(sc.ScroogeError) as err:
                sc.align_host(ctx, bad, 64, 24, 64, sc.SCROOGE_PERSISTENT)
            assert err.value.code == sc.SCROOGE_E_INVAL
            assert f"pair {q}:" in str(err.value), str(err.value)


@pytest.mark.parametrize("part", [0, 2, 3])
def test_four_parts_capacity_too_small(ctx, part):
    """Four parts (at least four waves of the lane kernel's 38,912 pair slots) with a CIGAR buffer that
    ends inside part `part`."""
    b = synth.concat([synth.long_reads(1500, seed=84), synth.short_reads(160_000, seed=85)])
    pb = sc.PackedBatch(b)
    n = pb.n_pairs
    assert n >= 4 * 38_912
    full = _run(ctx, pb, False)
    off = full["cigar_off"]
    lo, hi = n * part // 4, n * (part + 1) // 4
    cap = int((off[lo] + off[hi]) // 2)
    got = {}
    for overlap in (True, False):
        sc.scrooge_set_host_overlap(ctx, overlap)
        ec, tc = np.zeros(n, np.int32), np.zeros(n, np.int32)
        o, cig = np.zeros(n + 1, np.int64), np.zeros(cap, np.uint32)
        with pytest.raises(sc.ScroogeError) as err:
            sc.scrooge_align_batch(ctx, pb.texts, pb.text_off, pb.text_len, pb.patterns, pb.pat_off, pb.pat_len, n,
                                   64, 24, 64, sc.SCROOGE_PERSISTENT, ec, tc, cig, cap, o)
        assert err.value.code == sc.SCROOGE_E_CAPACITY
        assert np.array_equal(o, off) and np.array_equal(ec, full["edit_counts"])
        assert np.array_equal(tc, full["text_consumed"])
        got[overlap] = cig
    fits = np.flatnonzero(off[1:] <= cap)
    end = int(off[fits[-1] + 1]) if fits.size else 0
    assert np.array_equal(got[True][:end], full["cigar"][:end])
    assert np.array_equal(got[False][:end], full["cigar"][:end])
    split = _run(ctx, pb, True)
    _same(split, full, "four parts, full capacity")
