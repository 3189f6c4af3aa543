"""The row cycle of DENT extended to rows (Supplementary Section 1) against the oracle.

The full-width kernels store row d of a window in slot d mod R. Their DC runs the rows in a
pipeline over the G lanes of a pair, so when early termination stops a window at d_opt, rows up
to min(k, d_opt + G - 1) have been stored. The traceback (SENE) reads row d - 1 at each edit
step taken from row d, so the lowest row it reads is d_opt - e, with e the window's edits. Row y
is still in its slot when no later stored row shares it:

    y + R > min(k, d_opt + G - 1).

This checks that condition for every window of random pairs, with the oracle's per-window d_opt
and edit counts. It uses R = max(W-O+G, ceil((k+1)/2)), the slot count the library uses. It
also shows that one slot fewer than W-O+G fails on windows whose traceback spends all W-O edits.
"""
import numpy as np

import oracle
from paper_2208_09985_gb300 import synth


def _slots(W, O, k, G):
    return min(k + 1, max(W - O + G, (k + 2) // 2))


def _survives(d_opt, edits, k, G, R):
    lowest_read = d_opt - edits
    if edits == 0:
        return True  # no edge read
    return lowest_read + R > min(k, d_opt + G - 1)


def test_row_cycle_holds_every_row_the_traceback_reads(oracle_mod):
    rng = np.random.default_rng(23)
    windows = 0
    for it in range(250):
        W = int(rng.choice([8, 16, 32, 64]))
        O = int(rng.integers(0, W))
        k = W
        rate = float(rng.choice([0.05, 0.2, 0.5, 1.0]))
        m = int(rng.integers(1, 4 * W))
        t = rng.integers(0, 4, m + int(rng.integers(0, W))).astype(np.uint8)
        p = t[:m].copy()
        hit = rng.random(m) < rate
        p[hit] = rng.integers(0, 4, int(hit.sum())).astype(np.uint8)
        r = oracle_mod.align_pair(t, p, W, O, k)
        assert r["status"] == 0
        for G in (1, 2, 4, 8, 16):
            R = _slots(W, O, k, G)
            for d, e in zip(r["d_opt"], r["window_edits"]):
                assert _survives(int(d), int(e), k, G, R), (W, O, G, R, d, e)
        windows += len(r["d_opt"])
    assert windows > 1000


def test_one_slot_fewer_loses_a_row():
    """A window of W-O mismatched bases and then a shared tail has d_opt = W-O, and its traceback
    takes W-O substitutions. With W-O+G-1 slots the run-ahead row d_opt+G-1 overwrites the lowest
    row the traceback reads; W-O+G slots keep it."""
    rng = np.random.default_rng(5)
    for W, O, G in ((16, 4, 4), (32, 17, 2), (64, 33, 4), (64, 24, 8), (64, 40, 16)):
        k, L = W, W - O
        tail = rng.integers(0, 4, 3 * W).astype(np.uint8)
        t = np.concatenate([np.zeros(L, np.uint8), tail])
        p = np.concatenate([np.ones(L, np.uint8), tail])
        r = oracle.align_pair(t, p, W, O, k)
        d, e = int(r["d_opt"][0]), int(r["window_edits"][0])
        assert (d, e) == (L, L), (W, O, d, e)
        assert d + G - 1 <= k
        assert not _survives(d, e, k, G, W - O + G - 1)
        assert _survives(d, e, k, G, W - O + G)
