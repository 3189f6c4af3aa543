"""Exact edit distances (scrooge_edit_distance) against brute force (needs a GB300).

The free-end distance is pinned by the O(nm) numpy recurrence and the plain
Levenshtein DP of tests/_brute.py; the windowed alignment can never beat it.
"""
import numpy as np
import pytest

import oracle
import paper_2208_09985_gb300 as sc
from paper_2208_09985_gb300 import synth
from tests._brute import free_end_distance, free_end_distance_rows, lev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    assert torch.cuda.is_available()
    h = sc.scrooge_create(0)
    yield h
    sc.scrooge_destroy(h)


def _edit(ctx, b):
    import torch
    db = sc.DeviceBatch(sc.PackedBatch(b))
    fe, gl = sc.edit_distance_device(ctx, db)
    torch.cuda.synchronize()
    return fe.cpu().numpy(), gl.cpu().numpy()


def test_small_pairs_match_brute_force(ctx):
    rng = np.random.default_rng(5)
    texts, pats = [], []
    for t in range(300):
        n, m = int(rng.integers(0, 160)), int(rng.integers(0, 160))
        if t % 2:
            src = rng.integers(0, 4, max(n, m) + 3)
            tx, pt = src[:n].copy(), src[:m].copy()
            for _ in range(int(rng.integers(0, 12))):
                if len(pt):
                    pt[int(rng.integers(0, len(pt)))] = int(rng.integers(0, 4))
        else:
            tx, pt = rng.integers(0, 4, n), rng.integers(0, 4, m)
        texts.append(tx.astype(np.uint8))
        pats.append(pt.astype(np.uint8))
    texts += [np.zeros(0, np.uint8), np.zeros(70, np.uint8), np.arange(130, dtype=np.uint8) % 4]
    pats += [np.zeros(5, np.uint8), np.zeros(0, np.uint8), (np.arange(129, dtype=np.uint8) + 1) % 4]
    b = synth.from_lists(texts, pats)
    fe, gl = _edit(ctx, b)
    for p in range(b.n_pairs):
        t, q = b.text(p), b.pattern(p)
        assert fe[p] == (free_end_distance(t, q) if len(q) else 0), p
        assert gl[p] == lev(t, q), p


@pytest.mark.parametrize("length", [700, 2500, 9000])
def test_long_pairs_every_word_split_and_bound_on_the_windowed_method(ctx, length):
    import torch
    b = synth.fixed_error(3, 0.12, length=length, seed=length)
    db = sc.DeviceBatch(sc.PackedBatch(b))
    m_max = int(db.pat_len.max().item())
    ref = [free_end_distance_rows(b.text(p), b.pattern(p)) for p in range(b.n_pairs)]
    # max_pattern_length picks 1, 2, 4 or 8 words per lane; every split gives the same distances
    for bound in sorted({m_max, 2 * 2048 + 1, 4 * 2048 + 1, sc.SCROOGE_EDIT_DISTANCE_MAX_M}):
        if bound < m_max:
            continue
        fe = torch.zeros(b.n_pairs, dtype=torch.int32, device="cuda")
        gl = torch.zeros_like(fe)
        sc.scrooge_edit_distance(ctx, db.texts, db.text_off, db.text_len, db.patterns, db.pat_off, db.pat_len,
                                 b.n_pairs, bound, sc.SCROOGE_DEVICE_PTRS | sc.SCROOGE_SYNC, fe, gl)
        got = fe.cpu().numpy()
        assert list(got) == ref, bound
        assert (got <= gl.cpu().numpy()).all()
    r = oracle.align_batch(b, 64, 24)
    assert (np.asarray(ref) <= r["edit_counts"]).all()


def test_rejects_host_pointers_and_long_patterns(ctx):
    import torch
    b = synth.tiny_windows(4, seed=1)
    pb = sc.PackedBatch(b)
    out = np.zeros(4, np.int32)
    with pytest.raises(sc.ScroogeError):  # host pointers are refused before any launch
        sc.scrooge_edit_distance(ctx, pb.texts, pb.text_off, pb.text_len, pb.patterns, pb.pat_off, pb.pat_len, 4,
                                 200, 0, out, out)
    db = sc.DeviceBatch(pb)
    dout = torch.zeros(4, dtype=torch.int32, device="cuda")
    with pytest.raises(sc.ScroogeError):
        sc.scrooge_edit_distance(ctx, db.texts, db.text_off, db.text_len, db.patterns, db.pat_off, db.pat_len, 4,
                                 sc.SCROOGE_EDIT_DISTANCE_MAX_M + 1, sc.SCROOGE_DEVICE_PTRS, dout, dout)
    # a pattern above max_pattern_length gets -1
    sc.scrooge_edit_distance(ctx, db.texts, db.text_off, db.text_len, db.patterns, db.pat_off, db.pat_len, 4,
                             1, sc.SCROOGE_DEVICE_PTRS | sc.SCROOGE_SYNC, dout, dout)
    got = dout.cpu().numpy()
    assert ((got == -1) | (pb.pat_len <= 1)).all()
