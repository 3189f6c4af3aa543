"""Comparison of CUDA results with oracle results, pair by pair."""
import numpy as np


def pair_runs(res, p):
    o = int(res["cigar_off"][p])
    n = int(res["cigar_lens"][p])
    return res["cigar"][o:o + max(n, 0)].view(np.uint32)


def assert_same(gpu, ref, pairs=None, label=""):
    """Edit counts, text consumed, CIGAR lengths and CIGAR runs must be identical.

    ``ref`` holds the oracle results of the pairs ``pairs`` of ``gpu`` (all
    pairs, in order, when ``pairs`` is None).
    """
    idx = np.arange(len(ref["edit_counts"])) if pairs is None else np.asarray(pairs)
    for key in ("edit_counts", "text_consumed", "cigar_lens"):
        g = np.asarray(gpu[key])[idx]
        r = np.asarray(ref[key])
        bad = np.flatnonzero(g != r)
        assert bad.size == 0, (f"{label}: {key} differs at pairs {idx[bad[:10]]}: "
                               f"gpu {g[bad[:10]]} oracle {r[bad[:10]]}")
    for q, p in enumerate(idx):
        a = pair_runs(gpu, int(p))
        b = pair_runs(ref, q)
        if not np.array_equal(a, b):
            raise AssertionError(f"{label}: CIGAR of pair {p} differs (gpu {len(a)} runs, oracle {len(b)} runs)")


def dense_runs(res):
    """The runs of every pair back to back in pair order (the oracle lays pairs out at capacity
    offsets; the library writes them densely)."""
    lens = np.asarray(res["cigar_lens"]).astype(np.int64)
    off = np.asarray(res["cigar_off"]).astype(np.int64)[:-1]
    total = int(lens.sum())
    idx = np.repeat(off, lens) + (np.arange(total, dtype=np.int64) - np.repeat(np.cumsum(lens) - lens, lens))
    return np.asarray(res["cigar"]).view(np.uint32)[idx]


def assert_same_all(gpu, ref, label=""):
    """assert_same over every pair at once: edit counts, text consumed and run counts compared
    array-wise, then every run of the dense CIGARs (the first differing pair is named on failure)."""
    for key in ("edit_counts", "text_consumed", "cigar_lens"):
        g = np.asarray(gpu[key])
        r = np.asarray(ref[key])
        assert g.shape == r.shape, f"{label}: {key} shapes {g.shape} vs {r.shape}"
        bad = np.flatnonzero(g != r)
        assert bad.size == 0, (f"{label}: {key} differs at {bad.size} pairs, first {bad[:10]}: "
                               f"gpu {g[bad[:10]]} oracle {r[bad[:10]]}")
    lens = np.asarray(ref["cigar_lens"]).astype(np.int64)
    off = np.zeros(lens.size + 1, np.int64)
    np.cumsum(lens, out=off[1:])
    np.testing.assert_array_equal(np.asarray(gpu["cigar_off"]).astype(np.int64), off, err_msg=f"{label}: offsets")
    a = np.asarray(gpu["cigar"]).view(np.uint32)[:int(off[-1])]
    b = dense_runs(ref)
    diff = np.flatnonzero(a != b)
    if diff.size:
        p = int(np.searchsorted(off, diff[0], side="right") - 1)
        raise AssertionError(f"{label}: CIGAR runs differ at {diff.size} positions, first in pair {p}")
