"""Seeded synthetic read/reference pairs for the windowed GenASM aligner.

This module only draws inputs: random bases and a streaming edit model. It
holds none of the alignment arithmetic, so the CPU oracle (under ``oracle/``)
and the CUDA path can both be fed from it without sharing any code.

Bases are codes 0..3 (A, C, G, T), one per byte. A batch is stored as two
concatenated code arrays (texts = references, patterns = reads) plus int64
start offsets with one trailing entry, so pair ``p`` is
``texts[text_off[p]:text_off[p+1]]`` and likewise for patterns.

The paper's datasets (simulated PacBio reads, minimap2 candidate chains,
Illumina short-read chains; Section 3.1.1) are not available, so the recipes
below stand in for them with the same length and error structure:

* ``short_reads``  -- pattern lengths U{100..250}, 5 % edits (short-read chains);
* ``long_reads``   -- 10 kbp patterns, 10 % edits, 20 % of edit events are
  homopolymer indels of 1-5 bases (PacBio-like long reads);
* ``uneven_reads`` -- log-normal lengths (median 8 kbp, clipped to 1-100 kbp)
  with a per-pair error rate drawn from U[1 %, 15 %];
* ``fixed_error``  -- 10 kbp pairs at one error rate (for sweeps);
* ``tiny_windows`` -- a 110 bp text with a 100 bp pattern at 2 % edits.

Generation is chunked: pairs are produced in chunks of ``CHUNK`` pairs, each
chunk from its own ``numpy.random.default_rng([seed, chunk_index])`` stream and
always drawn in full before it is cut, so the first N pairs of any batch are
identical whatever the total size asked for.
That lets a test regenerate a prefix of a million-pair workload cheaply.
"""
from __future__ import annotations

import os
from dataclasses import dataclass

import numpy as np

CHUNK = 4096


@dataclass
class PairBatch:
    """Concatenated text/pattern codes of a batch of pairs."""

    texts: np.ndarray  # uint8 codes 0..3
    text_off: np.ndarray  # int64 [n_pairs + 1]
    patterns: np.ndarray  # uint8 codes 0..3
    pattern_off: np.ndarray  # int64 [n_pairs + 1]
    name: str = ""

    @property
    def n_pairs(self) -> int:
        return int(self.text_off.shape[0] - 1)

    def text(self, p: int) -> np.ndarray:
        return self.texts[self.text_off[p]:self.text_off[p + 1]]

    def pattern(self, p: int) -> np.ndarray:
        return self.patterns[self.pattern_off[p]:self.pattern_off[p + 1]]

    @property
    def text_lengths(self) -> np.ndarray:
        return np.diff(self.text_off).astype(np.int32)

    @property
    def pattern_lengths(self) -> np.ndarray:
        return np.diff(self.pattern_off).astype(np.int32)

    def subset(self, idx) -> "PairBatch":
        """Pairs ``idx`` (any integer index array) as a new batch."""
        idx = np.asarray(idx, dtype=np.int64)
        t = [self.text(int(p)) for p in idx]
        q = [self.pattern(int(p)) for p in idx]
        return from_lists(t, q, name=f"{self.name}[subset]")


def _offsets(lengths: np.ndarray) -> np.ndarray:
    off = np.zeros(lengths.shape[0] + 1, dtype=np.int64)
    np.cumsum(lengths, out=off[1:])
    return off


def from_lists(texts, patterns, name: str = "") -> PairBatch:
    """Build a batch from per-pair code arrays (or ACGT strings)."""
    conv = lambda s: encode(s) if isinstance(s, str) else np.asarray(s, dtype=np.uint8)
    t = [conv(s) for s in texts]
    q = [conv(s) for s in patterns]
    tl = np.array([len(s) for s in t], dtype=np.int64)
    ql = np.array([len(s) for s in q], dtype=np.int64)
    tc = np.concatenate(t) if t and tl.sum() else np.zeros(0, np.uint8)
    qc = np.concatenate(q) if q and ql.sum() else np.zeros(0, np.uint8)
    return PairBatch(tc.astype(np.uint8), _offsets(tl), qc.astype(np.uint8), _offsets(ql), name)


_ENC = np.full(256, 255, dtype=np.uint8)
for _i, _c in enumerate("ACGT"):
    _ENC[ord(_c)] = _i
    _ENC[ord(_c.lower())] = _i


def encode(s: str) -> np.ndarray:
    """ACGT string -> codes 0..3. Other letters raise ValueError."""
    a = _ENC[np.frombuffer(s.encode("ascii"), dtype=np.uint8)]
    if (a == 255).any():
        raise ValueError("only A, C, G, T are accepted")
    return a


def decode(codes) -> str:
    return "".join("ACGT"[int(c)] for c in codes)


def concat(batches, name: str = "") -> PairBatch:
    tl = np.concatenate([np.diff(b.text_off) for b in batches])
    ql = np.concatenate([np.diff(b.pattern_off) for b in batches])
    return PairBatch(np.concatenate([b.texts for b in batches]), _offsets(tl),
                     np.concatenate([b.patterns for b in batches]), _offsets(ql), name)


def mutate(rng: np.random.Generator, src: np.ndarray, src_off: np.ndarray, rate,
           homopolymer_frac: float = 0.0, max_hp: int = 5):
    """Streaming edit model applied to every source sequence of a batch.

    Walk each source; at each base an edit event happens with probability q.
    A plain event is a substitution (50 %; one of the three other bases,
    uniformly), an insertion (25 %; a uniform base placed before the current
    one) or a deletion (25 %; the current base is dropped). With
    ``homopolymer_frac`` > 0 that fraction of events is instead a homopolymer
    indel of r ~ U{1..max_hp} copies of the current base: an insertion adds r
    copies, a deletion removes the current base and up to r-1 following bases
    of the same run. Each inserted or deleted base counts as one edit, so q is
    chosen to make the expected edit count ``rate`` per source base.

    ``rate`` is a scalar or one rate per sequence. Returns (codes, offsets).
    """
    n = src_off.shape[0] - 1
    lens = np.diff(src_off)
    total = int(src_off[-1])
    if total == 0:
        return np.zeros(0, np.uint8), np.zeros(n + 1, np.int64)
    src = np.asarray(src, dtype=np.uint8)
    mean_bases = (1.0 - homopolymer_frac) + homopolymer_frac * (1 + max_hp) / 2.0
    rate = np.asarray(rate, dtype=np.float64)
    u = rng.random(total, dtype=np.float32)
    if rate.ndim == 0:
        ev = np.flatnonzero(u < np.float32(rate / mean_bases))
    else:
        q = (np.broadcast_to(rate, (n,)) / mean_bases).astype(np.float32)
        ev = np.flatnonzero(u < np.repeat(q, lens))
    del u
    nev = ev.shape[0]
    hp = rng.random(nev) < homopolymer_frac
    kind = rng.random(nev)
    rlen = rng.integers(1, max_hp + 1, nev)
    hp_ins = rng.random(nev) < 0.5
    new_base = rng.integers(0, 4, nev).astype(np.uint8)
    sub_shift = rng.integers(1, 4, nev).astype(np.uint8)

    # per source position: bases emitted before it (insertions) and whether it is kept
    pre_count = np.zeros(nev, dtype=np.int64)  # only event positions can have insertions
    pre_base = np.zeros(nev, dtype=np.uint8)
    keep = np.ones(total, dtype=bool)
    main_base = src.copy()

    plain = ~hp
    sub = plain & (kind < 0.5)
    ins = plain & (kind >= 0.5) & (kind < 0.75)
    dele = plain & (kind >= 0.75)
    s = ev[sub]
    main_base[s] = (src[s] + sub_shift[sub]) % 4
    pre_count[ins] = 1
    pre_base[ins] = new_base[ins]
    keep[ev[dele]] = False
    # homopolymer insertions: r extra copies of the current base before it
    hi = hp & hp_ins
    pre_count[hi] = rlen[hi]
    pre_base[hi] = src[ev[hi]]
    # homopolymer deletions: the current base and up to r-1 more of its run
    hd = hp & ~hp_ins
    if hd.any():
        is_start = np.ones(total, dtype=bool)
        is_start[1:] = src[1:] != src[:-1]
        is_start[src_off[:-1][lens > 0]] = True
        starts = np.flatnonzero(is_start)
        s = ev[hd]
        nxt = np.searchsorted(starts, s, side="right")
        run_end = np.where(nxt < starts.size, starts[np.minimum(nxt, starts.size - 1)], total)
        dl = np.minimum(rlen[hd], run_end - s)
        diff = np.zeros(total + 1, dtype=np.int32)
        np.add.at(diff, s, 1)
        np.add.at(diff, s + dl, -1)
        keep &= np.cumsum(diff[:-1]) == 0
    # an insertion before a deleted base is dropped with it
    pre_count[~keep[ev]] = 0
    cnt = keep.astype(np.int64)
    np.add.at(cnt, ev, pre_count)
    ends = np.cumsum(cnt)
    out = np.empty(int(ends[-1]) if total else 0, dtype=np.uint8)
    out[ends[keep] - 1] = main_base[keep]
    has_pre = pre_count > 0
    if has_pre.any():
        first = ends[ev[has_pre]] - cnt[ev[has_pre]]
        k = pre_count[has_pre]
        pos = np.repeat(first, k) + (np.arange(int(k.sum())) - np.repeat(np.cumsum(k) - k, k))
        out[pos] = np.repeat(pre_base[has_pre], k)
    per = np.add.reduceat(cnt, src_off[:-1]) if n else np.zeros(0, np.int64)
    per = np.where(lens > 0, per, 0)
    return out, _offsets(per.astype(np.int64))


def _random_codes(rng, lengths):
    lengths = np.asarray(lengths, dtype=np.int64)
    return rng.integers(0, 4, int(lengths.sum()), dtype=np.uint8), _offsets(lengths)


def _run_chunk(args):
    """One full chunk from its own stream, cut to the first ``cnt`` pairs."""
    fn, seed, c, cnt, kw = args
    b = globals()[fn](np.random.default_rng([seed, c]), CHUNK, **kw)
    if cnt < CHUNK:
        b = PairBatch(b.texts[: b.text_off[cnt]], b.text_off[: cnt + 1].copy(),
                      b.patterns[: b.pattern_off[cnt]], b.pattern_off[: cnt + 1].copy())
    return b


def _chunked(seed: int, n_pairs: int, fn: str, name: str, **kw) -> PairBatch:
    """Generate ``n_pairs`` pairs chunk by chunk with the module function ``fn``.

    Large batches are generated by a pool of spawned worker processes; the
    result does not depend on how many workers run.
    """
    jobs = [(fn, seed, c, min(CHUNK, n_pairs - c * CHUNK), kw) for c in range((n_pairs + CHUNK - 1) // CHUNK)]
    if not jobs:
        z = np.zeros(1, np.int64)
        return PairBatch(np.zeros(0, np.uint8), z, np.zeros(0, np.uint8), z.copy(), name)
    workers = min(len(jobs), os.cpu_count() or 1, 16)
    if workers >= 4 and len(jobs) >= 8:
        import multiprocessing as mp
        from concurrent.futures import ProcessPoolExecutor
        with ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn")) as ex:
            parts = list(ex.map(_run_chunk, jobs))
    else:
        parts = [_run_chunk(j) for j in jobs]
    return concat(parts, name)


def _with_padding(rng, src, src_off, pad_frac):
    """text = source followed by ceil(pad_frac * len) uniform bases."""
    lens = np.diff(src_off)
    pad = np.ceil(pad_frac * lens).astype(np.int64)
    padc, pad_off = _random_codes(rng, pad)
    tl = lens + pad
    out = np.empty(int(tl.sum()), np.uint8)
    toff = _offsets(tl)
    # interleave source and padding per pair
    idx_src = np.repeat(toff[:-1], lens) + (np.arange(int(lens.sum())) - np.repeat(src_off[:-1], lens))
    out[idx_src] = src
    idx_pad = np.repeat(toff[:-1] + lens, pad) + (np.arange(int(pad.sum())) - np.repeat(pad_off[:-1], pad))
    out[idx_pad] = padc
    return out, toff


def _chunk_tiny(rng, cnt):
    t, toff = _random_codes(rng, np.full(cnt, 110))
    src = t.reshape(cnt, 110)[:, :100].ravel()
    q, qoff = mutate(rng, src, _offsets(np.full(cnt, 100)), 0.02)
    return PairBatch(t, toff, q, qoff)


def tiny_windows(n_pairs: int = 1000, seed: int = 0) -> PairBatch:
    """110 bp uniform text; pattern = its first 100 bp with 2 % edits."""
    return _chunked(seed, n_pairs, "_chunk_tiny", "tiny_windows")


def _chunk_short(rng, cnt):
    L = rng.integers(100, 251, cnt)
    src, soff = _random_codes(rng, L)
    t, toff = _with_padding(rng, src, soff, 0.05)
    q, qoff = mutate(rng, src, soff, 0.05)
    return PairBatch(t, toff, q, qoff)


def short_reads(n_pairs: int = 1_000_000, seed: int = 1) -> PairBatch:
    """L ~ U{100..250}; text = L-bp source + 5 % padding; pattern = source at 5 % edits."""
    return _chunked(seed, n_pairs, "_chunk_short", "short_reads")


def _chunk_long(rng, cnt, text_len, pattern_len, rate):
    t, toff = _random_codes(rng, np.full(cnt, text_len))
    q, qoff = mutate(rng, t, toff, rate, homopolymer_frac=0.2)
    ql = np.diff(qoff)
    if (ql < pattern_len).any():
        raise RuntimeError("mutated read shorter than the requested pattern length")
    keep = np.repeat(qoff[:-1], pattern_len) + np.tile(np.arange(pattern_len), cnt)
    return PairBatch(t, toff, q[keep], _offsets(np.full(cnt, pattern_len)))


def long_reads(n_pairs: int = 100_000, seed: int = 2, text_len: int = 10_500,
               pattern_len: int = 10_000, rate: float = 0.10) -> PairBatch:
    """10.5 kbp text; pattern = text at 10 % edits (20 % homopolymer indels), cut to 10 kbp."""
    return _chunked(seed, n_pairs, "_chunk_long", "long_reads", text_len=text_len,
                    pattern_len=pattern_len, rate=rate)


def _chunk_uneven(rng, cnt, sigma):
    L = np.clip(np.exp(rng.normal(np.log(8000.0), sigma, cnt)), 1000, 100_000).astype(np.int64)
    rate = rng.uniform(0.01, 0.15, cnt)
    src, soff = _random_codes(rng, L)
    t, toff = _with_padding(rng, src, soff, 0.05)
    q, qoff = mutate(rng, src, soff, rate)
    return PairBatch(t, toff, q, qoff)


def uneven_reads(n_pairs: int = 200_000, seed: int = 3, sigma: float = 0.75) -> PairBatch:
    """Log-normal lengths (median 8 kbp, clipped to [1, 100] kbp), per-pair rate U[1 %, 15 %]."""
    return _chunked(seed, n_pairs, "_chunk_uneven", "uneven_reads", sigma=sigma)


def _chunk_fixed(rng, cnt, rate, length):
    src, soff = _random_codes(rng, np.full(cnt, length))
    t, toff = _with_padding(rng, src, soff, 0.05)
    q, qoff = mutate(rng, src, soff, rate)
    return PairBatch(t, toff, q, qoff)


def fixed_error(n_pairs: int = 20_000, rate: float = 0.10, seed: int = 6,
                length: int = 10_000) -> PairBatch:
    """length-bp source + 5 % padding as text; pattern = source at ``rate`` edits."""
    return _chunked(seed, n_pairs, "_chunk_fixed", f"fixed_error_{rate:g}", rate=rate, length=length)


def random_pairs(n_pairs: int, max_text: int, max_pattern: int, seed: int,
                 rate_max: float = 0.5) -> PairBatch:
    """Small pairs of mixed length and error for edge-case sweeps.

    Text length U{0..max_text}; the pattern is a mutated prefix of the text
    (or an unrelated random string for a quarter of the pairs), cut to at most
    ``max_pattern`` bases. Includes empty sequences.
    """
    rng = np.random.default_rng(seed)
    texts, pats = [], []
    for _ in range(n_pairs):
        n = int(rng.integers(0, max_text + 1))
        t = rng.integers(0, 4, n).astype(np.uint8)
        if rng.random() < 0.25:
            q = rng.integers(0, 4, int(rng.integers(0, max_pattern + 1))).astype(np.uint8)
        else:
            q, _ = mutate(rng, t, np.array([0, n]), float(rng.uniform(0, rate_max)))
            q = q[: int(rng.integers(0, max_pattern + 1))]
        texts.append(t)
        pats.append(q)
    return from_lists(texts, pats, name=f"random_pairs_{seed}")
