"""The seeded input generators: deterministic, prefix-stable, and with the stated structure.

Full-size GPU parity tests regenerate samples of a workload at a smaller size, which is only
valid if any prefix of a workload is identical whatever pair count is asked for (generation is
chunked with one seeded stream per chunk). The generators hold none of the alignment arithmetic.
"""
import numpy as np
import pytest

from paper_2208_09985_gb300 import synth


def _same(a, b, n):
    for p in range(n):
        assert np.array_equal(a.text(p), b.text(p)), p
        assert np.array_equal(a.pattern(p), b.pattern(p)), p


@pytest.mark.parametrize("make", [lambda n: synth.tiny_windows(n, seed=0), lambda n: synth.short_reads(n, seed=1),
                                  lambda n: synth.long_reads(n, seed=2), lambda n: synth.uneven_reads(n, seed=3)])
def test_prefix_stable_and_deterministic(make):
    small, large = make(50), make(5000)
    assert small.n_pairs == 50 and large.n_pairs == 5000
    _same(small, large, 50)
    _same(make(5000), large, 5000)


def test_structure_of_the_workloads():
    t = synth.tiny_windows(200, seed=0)
    # 110 bp texts; patterns are their first 100 bp at 2% edits, so indels move the length a little
    assert all(len(t.text(p)) == 110 and 94 <= len(t.pattern(p)) <= 106 for p in range(200))
    lr = synth.long_reads(40, seed=2)
    assert all(len(lr.text(p)) == 10_500 and len(lr.pattern(p)) == 10_000 for p in range(40))
    sr = synth.short_reads(2000, seed=1)
    lens = np.array([len(sr.pattern(p)) for p in range(2000)])
    assert lens.min() >= 90 and lens.max() <= 270  # U{100..250} at 5% edits
    for b in (t, lr, sr):
        for p in range(min(b.n_pairs, 50)):
            assert b.text(p).max(initial=0) <= 3 and b.pattern(p).max(initial=0) <= 3


@pytest.mark.parametrize("rate", [0.05, 0.10, 0.15])
def test_fixed_error_rate(rate):
    """Each source base draws an edit with probability q: the patterns' Hamming distance to the text
    prefix stays far above zero and the length changes average out (25% insertions vs 25% deletions)."""
    b = synth.fixed_error(60, rate, seed=7, length=4000)
    dl = np.array([len(b.pattern(p)) - 4000 for p in range(60)], dtype=float)
    assert abs(dl.mean()) < 0.02 * 4000 * rate + 20
    b0 = synth.fixed_error(60, 0.0, seed=7, length=4000)
    for p in range(10):
        assert np.array_equal(b0.pattern(p), b0.text(p)[:4000])
