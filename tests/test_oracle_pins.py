"""Pins of the CPU oracle against what the paper and plain mathematics fix.

* Theorem 1 (Section 2.2.1): every bit of every entry R[i][d] of Algorithm 1
  equals [dist(text[i:n), pattern[j:m)) <= d] for the free-text-end distance,
  checked by brute force on every window of many tiny inputs (and a few
  windows of up to 128 characters, which need two machine words).
* Figure 1's example (text ACGT, pattern ACGA, k = 4) with hand-derived values.
* The traceback (Section 2.2.2) and windowing (Section 2.2.3): every CIGAR is a
  valid alignment of the whole pattern against a text prefix whose edit count
  is the reported score, never below the optimum, and exactly optimal when a
  single window covers the pattern.
* Lemma S3 (Supplementary Section 10): the edit distance of a window is at
  most the Hamming distance of equal-length strings.
"""
import json
import os

import numpy as np
import pytest

from paper_2208_09985_gb300 import synth
from tests import _brute as brute

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _bits(s):
    return np.array([int(c) for c in s], dtype=np.uint8)


def test_free_end_recurrence_matches_definition():
    """The O(nm) free-end table used for bigger windows equals the literal definition."""
    rng = np.random.default_rng(11)
    for _ in range(60):
        n, m = rng.integers(0, 7, 2)
        t = rng.integers(0, 3, n)
        p = rng.integers(0, 3, m)
        assert np.array_equal(brute.free_end_table_literal(t, p), brute.free_end_table(t, p))
        assert brute.free_end_distance(t, p) == brute.free_end_table(t, p)[0, 0]


def test_fig1_example(oracle_mod):
    g = json.load(open(os.path.join(GOLDEN, "fig1_example.json")))
    text, pat, k = synth.encode(g["text"]), synth.encode(g["pattern"]), g["k"]
    pm = oracle_mod.pattern_masks(pat)
    for x, c in enumerate("ACGT"):
        assert np.array_equal(pm[x], _bits(g["pattern_masks_msb_first"][c])), c
    bits, d_opt = oracle_mod.window_table(text, pat, k)
    assert d_opt == g["edit_distance"]
    for key, val in g["entries_msb_first"].items():
        i, d = [int(x) for x in key[2:-1].split("][")]
        assert np.array_equal(bits[i, d], _bits(val)), key
    # the caption's highlighted 0 at d=1, i=2, j=2
    assert bits[2, 1, 2] == 0


def _check_theorem1(oracle_mod, t, p, k):
    bits, d_opt = oracle_mod.window_table(t, p, k)
    dist = brute.free_end_table(t, p)[:, : len(p)]  # (n+1) x m
    expect = (dist[:, None, :] > np.arange(k + 1)[None, :, None]).astype(np.uint8)
    assert np.array_equal(bits, expect), (synth.decode(t), synth.decode(p), k)
    best = int(brute.free_end_table(t, p)[0, 0])
    assert d_opt == (best if best <= k else -1)


def test_theorem1_tiny_exhaustive_random(oracle_mod):
    rng = np.random.default_rng(1)
    for _ in range(1500):
        n, m = int(rng.integers(0, 10)), int(rng.integers(0, 10))
        alpha = int(rng.integers(1, 5))
        t = rng.integers(0, alpha, n).astype(np.uint8)
        p = rng.integers(0, alpha, m).astype(np.uint8)
        k = int(rng.integers(0, max(n, m) + 2))
        _check_theorem1(oracle_mod, t, p, k)


def test_theorem1_all_binary_strings_len3(oracle_mod):
    for a in range(1 << 3):
        for b in range(1 << 3):
            t = np.array([(a >> s) & 1 for s in range(3)], np.uint8)
            p = np.array([(b >> s) & 1 for s in range(3)], np.uint8)
            _check_theorem1(oracle_mod, t, p, 3)


@pytest.mark.parametrize("n,m", [(64, 64), (70, 65), (100, 97), (128, 128), (127, 40), (5, 128)])
def test_theorem1_multiword(oracle_mod, n, m):
    rng = np.random.default_rng(n * 1000 + m)
    t = rng.integers(0, 4, n).astype(np.uint8)
    p, _ = synth.mutate(rng, t[:m].copy(), np.array([0, min(m, n)]), 0.1)
    p = np.concatenate([p, rng.integers(0, 4, 200).astype(np.uint8)])[:m]
    _check_theorem1(oracle_mod, t, p, min(128, max(n, m)))


def test_window_hamming_bound(oracle_mod):
    """Lemma S3: for equal lengths, edit distance <= Hamming distance; d_opt is at most that."""
    rng = np.random.default_rng(5)
    tot = 0
    for _ in range(200):
        t = rng.integers(0, 4, 64).astype(np.uint8)
        p = rng.integers(0, 4, 64).astype(np.uint8)
        _, d_opt = oracle_mod.window_table(t, p, 64)
        assert 0 <= d_opt <= int((t != p).sum())
        tot += d_opt
    # Lemma S1/S2: expected Hamming distance of random pairs is 3W/4
    assert tot / 200 <= 0.75 * 64


def _check_pair(oracle_mod, t, p, W, O, k=None):
    r = oracle_mod.align_pair(t, p, W, O, k)
    if r["status"] == 1:
        return r
    assert r["status"] == 0
    err = brute.check_cigar(t, p, r["cigar"], r["text_consumed"], r["edit_count"])
    assert not err, (err, synth.decode(t), synth.decode(p), W, O)
    assert r["edit_count"] >= brute.free_end_distance(t, p)
    assert r["edit_count"] >= brute.lev(t[: r["text_consumed"]], p)
    return r


def test_windowed_invariants_random(oracle_mod):
    rng = np.random.default_rng(3)
    for it in range(400):
        W = int(rng.choice([4, 8, 12, 16, 32, 64]))
        O = int(rng.integers(0, W))
        b = synth.random_pairs(1, max_text=int(rng.integers(0, 3 * W + 3)),
                               max_pattern=int(rng.integers(0, 3 * W + 3)), seed=1000 + it)
        t, p = b.text(0), b.pattern(0)
        r = _check_pair(oracle_mod, t, p, W, O)
        assert r["status"] == 0  # k = W never fails
        # one window covering the whole pattern gives the optimal distance
        if len(p) <= W - O and len(t) <= W:
            assert r["edit_count"] == brute.free_end_distance(t, p)


def test_single_window_is_optimal(oracle_mod):
    rng = np.random.default_rng(8)
    for _ in range(200):
        W = int(rng.choice([8, 16, 32, 64, 128]))
        O = int(rng.integers(0, W // 2))
        n = int(rng.integers(0, W + 1))
        m = int(rng.integers(0, W - O + 1))
        t = rng.integers(0, 4, n).astype(np.uint8)
        p, _ = synth.mutate(rng, t[:m].copy(), np.array([0, min(m, n)]), float(rng.uniform(0, 0.4)))
        p = p[:m]
        r = _check_pair(oracle_mod, t, p, W, O)
        assert r["edit_count"] == brute.free_end_distance(t, p)
        assert r["d_opt"].shape[0] == (1 if len(p) else 0)
        if len(p):
            assert r["d_opt"][0] == r["edit_count"]


def test_special_cases(oracle_mod):
    rng = np.random.default_rng(4)
    t = rng.integers(0, 4, 500).astype(np.uint8)
    # error-free pair: pattern is a text prefix
    r = oracle_mod.align_pair(t, t[:400], 64, 24)
    assert r["edit_count"] == 0 and oracle_mod.cigar_string(r["cigar"]) == "400="
    assert r["text_consumed"] == 400
    # empty pattern
    r = oracle_mod.align_pair(t, t[:0], 64, 24)
    assert r["edit_count"] == 0 and r["cigar"].shape[0] == 0 and r["text_consumed"] == 0
    # empty text: the pattern is all insertions
    r = oracle_mod.align_pair(t[:0], t[:150], 64, 24)
    assert r["edit_count"] == 150 and oracle_mod.cigar_string(r["cigar"]) == "150I"
    # homopolymer text, unrelated pattern
    r = _check_pair(oracle_mod, np.zeros(300, np.uint8), np.full(200, 2, np.uint8), 64, 24)
    assert r["edit_count"] == 200
    # k smaller than a window's distance fails the pair
    q = t[:100].copy()
    q[10:30] = (q[10:30] + 1) % 4
    r = oracle_mod.align_pair(t, q, 64, 24, k=5)
    assert r["status"] == 1 and r["edit_count"] == -1 and r["cigar"].shape[0] == 0


def test_tie_break_convention(oracle_mod):
    """M before S before I before D (a reading; the paper leaves ties open)."""
    r = oracle_mod.align_pair(synth.encode("AAAC"), synth.encode("AAC"), 8, 0)
    assert oracle_mod.cigar_string(r["cigar"]) == "2=1X" and r["text_consumed"] == 3
    r = oracle_mod.align_pair(synth.encode("ACGT"), synth.encode("AGT"), 8, 0)
    assert oracle_mod.cigar_string(r["cigar"]) == "1=1D2="
    r = oracle_mod.align_pair(synth.encode("AGTT"), synth.encode("ACGT"), 8, 0)
    assert oracle_mod.cigar_string(r["cigar"]) == "1=1I2="


def test_window_stop_rule(oracle_mod):
    """The first window keeps exactly W-O characters of progress on an error-free pair."""
    t = synth.encode("ACGT" * 40)
    r = oracle_mod.align_pair(t, t[:100], 16, 6)
    assert r["d_opt"].shape[0] == 10  # 100 pattern bases / (W-O = 10) per window
    assert oracle_mod.cigar_string(r["cigar"]) == "100="
    # a deletion makes the text run one ahead: the first window stops at i == W-O
    # with 9 pattern bases, then 10 per window: 9 + 9 * 10 = 99, one more for 100
    q = np.concatenate([t[:2], t[3:]])[:100]
    r = oracle_mod.align_pair(t, q, 16, 6)
    assert r["d_opt"].shape[0] == 11
    assert oracle_mod.cigar_string(r["cigar"]) == "2=1D98="


def test_batch_matches_single(oracle_mod):
    b = synth.random_pairs(60, 200, 200, seed=77)
    res = oracle_mod.align_batch(b, 32, 12, threads=3)
    for p in range(b.n_pairs):
        r = oracle_mod.align_pair(b.text(p), b.pattern(p), 32, 12)
        assert res["edit_counts"][p] == r["edit_count"]
        assert res["text_consumed"][p] == r["text_consumed"]
        assert np.array_equal(oracle_mod.pair_cigar(res, p), r["cigar"])


def test_cigar_overflow_reported(oracle_mod):
    b = synth.random_pairs(5, 200, 200, seed=9, rate_max=0.4)
    res = oracle_mod.align_batch(b, 32, 12, threads=1, cigar_capacity=1)
    for p in range(b.n_pairs):
        full = oracle_mod.align_pair(b.text(p), b.pattern(p), 32, 12)
        if len(full["cigar"]) > 1:
            assert res["cigar_lens"][p] == -1
        else:
            assert res["cigar_lens"][p] == len(full["cigar"])
        # the alignment itself is unaffected by the capacity
        assert res["edit_counts"][p] == full["edit_count"]
        assert res["text_consumed"][p] == full["text_consumed"]


def test_free_end_row_recurrence_matches_its_definition():
    """The vectorised free-end DP used by the edit-distance tests equals the row-by-row one."""
    from tests._brute import free_end_distance, free_end_distance_rows
    rng = np.random.default_rng(17)
    for _ in range(200):
        n, m = int(rng.integers(0, 50)), int(rng.integers(0, 50))
        t, p = rng.integers(0, 4, n), rng.integers(0, 4, m)
        assert free_end_distance_rows(t, p) == free_end_distance(t, p)


def _first_window_extent(runs, n, m, W, O):
    """(text chars, pattern chars, edits) of the first window's kept traceback.

    The traceback of a window stops at the first point where j == m_w, i == W-O
    or j == W-O (Section 2.2.3), so walking the stitched CIGAR one operation at
    a time and stopping at the first such point recovers the first window.
    """
    L, mw = W - O, min(W, m)
    i = j = e = 0
    for op, ln in brute.cigar_ops(runs):
        for _ in range(ln):
            if j >= mw or i >= L or j >= L:
                return i, j, e
            i += op in (7, 8, 2)
            j += op in (7, 8, 1)
            e += op != 7
    return i, j, e


def test_traceback_rows_extended_dent(oracle_mod):
    """Supplementary Section 1 (DENT extended to rows): a window's kept traceback descends at most
    W-O rows below d_opt, so only rows d_opt-(W-O) .. d_opt are ever read.

    Why: the traceback path is part of an optimal alignment, so its part up to (i, j) costs
    lev(text[:i], pattern[:j]) <= max(i, j) <= W-O. Checked by brute force on the first window of
    every pair (the edits logged for it equal that Levenshtein distance), on every window (logged
    edits <= W-O, and they sum to the edit count), and shown tight: an all-substitution window
    descends exactly W-O rows.
    """
    rng = np.random.default_rng(17)
    for it in range(300):
        W = int(rng.choice([8, 12, 16, 32]))
        O = int(rng.integers(0, W))
        # from unrelated strings (edit rates near 3/4) down to close copies
        rate = float(rng.choice([0.0, 0.1, 0.3, 1.0]))
        m = int(rng.integers(1, 3 * W))
        t = rng.integers(0, 4, m + int(rng.integers(0, W))).astype(np.uint8)
        p = t[:m].copy()
        hit = rng.random(m) < rate
        p[hit] = rng.integers(0, 4, int(hit.sum())).astype(np.uint8)
        r = oracle_mod.align_pair(t, p, W, O, W)
        assert r["status"] == 0
        we = r["window_edits"]
        assert len(we) == len(r["d_opt"]) and (we >= 0).all()
        assert (we <= W - O).all(), (W, O, we)
        assert (we <= r["d_opt"]).all()
        assert int(we.sum()) == r["edit_count"]
        i1, j1, e1 = _first_window_extent(r["cigar"], len(t), len(p), W, O)
        assert e1 == we[0] == brute.lev(t[:i1], p[:j1]), (W, O, i1, j1)
    # tight: text all A, pattern all C -> every traceback step is a substitution
    for W, O in ((8, 3), (16, 0), (32, 17), (64, 33), (64, 24)):
        r = oracle_mod.align_pair(np.zeros(3 * W, np.uint8), np.ones(2 * W, np.uint8), W, O, W)
        assert r["status"] == 0 and int(r["window_edits"].max()) == W - O
