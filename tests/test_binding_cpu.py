"""Host-side checks of the CUDA library that need no GPU.

The library must build for sm_103a, load, and export every function that
include/scrooge.h declares; the host packer must produce the documented
bit-plane layout.
"""
import ctypes

import numpy as np
import pytest

import paper_2208_09985_gb300 as sc
from paper_2208_09985_gb300 import build as sc_build
from paper_2208_09985_gb300 import synth


@pytest.fixture(scope="module")
def lib():
    sc_build.build()
    return sc.load()


def test_exports_every_header_function(lib):
    names = sc.header_functions()
    assert "scrooge_align_batch" in names and "scrooge_create" in names
    raw = ctypes.CDLL(sc.LIB_PATH)
    missing = [n for n in names if not hasattr(raw, n)]
    assert not missing, f"declared but not exported: {missing}"


def _unpack(packed, off, length):
    """Decode the documented layout: 32-base blocks, plane 0 then plane 1, base t at bit 31-t."""
    out = np.zeros(length, np.uint8)
    w0 = off // 16
    for pos in range(length):
        blk, t = divmod(pos, 32)
        lo = (int(packed[w0 + 2 * blk]) >> (31 - t)) & 1
        hi = (int(packed[w0 + 2 * blk + 1]) >> (31 - t)) & 1
        out[pos] = lo | (hi << 1)
    return out


def test_pack_roundtrip(lib):
    b = synth.random_pairs(40, 300, 300, seed=3)
    packed, off, ln = sc.scrooge_pack_2bit(b.texts, b.text_off)
    assert np.all(off % 64 == 0)
    assert np.array_equal(ln, np.diff(b.text_off))
    for s in range(b.n_pairs):
        assert np.array_equal(_unpack(packed, int(off[s]), int(ln[s])), b.text(s))
        # bits past the end of a sequence are zero
        words = sc.scrooge_packed_words(int(ln[s]))
        tail = np.zeros(words * 16, np.uint8)
        tail[: ln[s]] = 1
        seg = packed[off[s] // 16: off[s] // 16 + words]
        if ln[s] % 32:
            last_blk = (int(ln[s]) // 32)
            keep = int(ln[s]) % 32
            mask = (0xFFFFFFFF >> keep) if keep else 0
            assert int(seg[2 * last_blk]) & mask == 0 and int(seg[2 * last_blk + 1]) & mask == 0


def test_pack_ascii_and_reject(lib):
    s = np.frombuffer(b"ACGTacgtTTGA", dtype=np.uint8)
    packed, off, ln = sc.scrooge_pack_2bit(s, np.array([0, 12]), ascii=True)
    assert np.array_equal(_unpack(packed, 0, 12), synth.encode("ACGTACGTTTGA"))
    with pytest.raises(sc.ScroogeError):
        sc.scrooge_pack_2bit(np.frombuffer(b"ACGN", dtype=np.uint8), np.array([0, 4]), ascii=True)
    with pytest.raises(sc.ScroogeError):
        sc.scrooge_pack_2bit(np.array([0, 1, 4], np.uint8), np.array([0, 3]))


def test_packed_words(lib):
    assert sc.scrooge_packed_words(0) == 0
    assert sc.scrooge_packed_words(1) == 4
    assert sc.scrooge_packed_words(64) == 4
    assert sc.scrooge_packed_words(65) == 8
    assert sc.scrooge_packed_words(-1) == -1
