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


def run_totals(res, n_pairs):
    """Per pair: pattern bases, text bases and edits implied by the CIGAR runs."""
    pat = np.zeros(n_pairs, np.int64)
    txt = np.zeros(n_pairs, np.int64)
    ed = np.zeros(n_pairs, np.int64)
    lens = np.asarray(res["cigar_lens"]).astype(np.int64)
    off = np.asarray(res["cigar_off"]).astype(np.int64)
    cig = np.asarray(res["cigar"]).view(np.uint32)
    ok = lens > 0
    starts = off[:-1][ok]
    cnt = lens[ok]
    idx = np.repeat(starts, cnt) + (np.arange(int(cnt.sum())) - np.repeat(np.cumsum(cnt) - cnt, cnt))
    owner = np.repeat(np.flatnonzero(ok), cnt)
    runs = cig[idx]
    op = (runs & 15).astype(np.int64)
    ln = (runs >> 4).astype(np.int64)
    np.add.at(pat, owner, np.where((op == 7) | (op == 8) | (op == 1), ln, 0))
    np.add.at(txt, owner, np.where((op == 7) | (op == 8) | (op == 2), ln, 0))
    np.add.at(ed, owner, np.where(op != 7, ln, 0))
    return pat, txt, ed
