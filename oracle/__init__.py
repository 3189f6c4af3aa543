"""CPU oracle of Scrooge's windowed GenASM (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package. It never serves the product path, and it shares
no code with the CUDA library: ``genasm_oracle.c`` is built on its own with
gcc into ``oracle/_build/liboracle.so``.

Functions take sequences as numpy code arrays (0..3 for A, C, G, T, one per
byte), never the 2-bit packed form the CUDA path reads.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "genasm_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None
_lock = threading.Lock()

OP_I, OP_D, OP_EQ, OP_X = 1, 2, 7, 8
OP_CHAR = {OP_I: "I", OP_D: "D", OP_EQ: "=", OP_X: "X"}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (portable flags only). Returns the .so path."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if (force or not os.path.exists(_LIB_PATH)
            or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-Wall", "-Wextra", "-fPIC", "-shared",
                               "-pthread", _SRC, "-o", tmp])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def bind(path: str):
    """Load an oracle shared library from ``path`` and declare its signatures."""
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    i32, i64 = ctypes.c_int, ctypes.c_int64
    lib.orc_window_table.argtypes = [P, i32, P, i32, i32, P, P]
    lib.orc_pattern_masks.argtypes = [P, i32, P]
    lib.orc_align_pair.argtypes = [P, i64, P, i64, i32, i32, i32, P, P, P, i64, P, P, P, i64, P]
    lib.orc_align_batch.argtypes = [P, P, P, P, i64, i32, i32, i32, i32, P, P, P, P, P]
    for f in (lib.orc_window_table, lib.orc_pattern_masks, lib.orc_align_pair, lib.orc_align_batch):
        f.restype = ctypes.c_int
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = bind(build())
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _codes(s) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(s, dtype=np.uint8))
    if a.size and a.max() > 3:
        raise ValueError("codes must be 0..3")
    return a


def window_table(text, pattern, k: int):
    """Algorithm 1's full table for one window.

    Returns (bits, d_opt): bits[i, d, j] is bit j of R[i][d] for
    0 <= i <= n, 0 <= d <= k, 0 <= j < m; d_opt is -1 if no d <= k qualifies.
    """
    t, p = _codes(text), _codes(pattern)
    n, m = t.shape[0], p.shape[0]
    bits = np.zeros((n + 1, k + 1, max(m, 1)), dtype=np.uint8)
    d = ctypes.c_int(0)
    if _load().orc_window_table(_ptr(t), n, _ptr(p), m, k, _ptr(bits), ctypes.byref(d)) != 0:
        raise ValueError("bad window arguments")
    return bits[:, :, :m], d.value


def pattern_masks(pattern) -> np.ndarray:
    """PM[x, j] for x in 0..3 (A, C, G, T), j < m."""
    p = _codes(pattern)
    m = p.shape[0]
    pm = np.zeros((4, max(m, 1)), dtype=np.uint8)
    if _load().orc_pattern_masks(_ptr(p), m, _ptr(pm)) != 0:
        raise ValueError("bad pattern")
    return pm[:, :m]


def align_pair(text, pattern, W: int = 64, O: int = 24, k: int | None = None):
    """Windowed alignment of one pair.

    Returns dict(edit_count, text_consumed, cigar (uint32 runs, len << 4 | op),
    d_opt (per window), window_edits (per window: edits of its kept
    traceback, i.e. how many rows it descended below d_opt), status).
    status 0 = aligned, 1 = some window had no d <= k (edit_count -1),
    -2 = CIGAR overflow.
    """
    k = W if k is None else k
    t, p = _codes(text), _codes(pattern)
    n, m = t.shape[0], p.shape[0]
    cap = n + m + 1
    cig = np.zeros(cap, dtype=np.uint32)
    nwin_cap = m + 1
    dopt = np.full(nwin_cap, -1, dtype=np.int32)
    wed = np.full(nwin_cap, -1, dtype=np.int32)
    ec = ctypes.c_int32(0)
    tc, cl, nw = ctypes.c_int64(0), ctypes.c_int64(0), ctypes.c_int64(0)
    st = _load().orc_align_pair(_ptr(t), n, _ptr(p), m, W, O, k, ctypes.byref(ec), ctypes.byref(tc),
                                _ptr(cig), cap, ctypes.byref(cl), _ptr(dopt), _ptr(wed), nwin_cap,
                                ctypes.byref(nw))
    if st == -1:
        raise ValueError("bad arguments or internal oracle error")
    return {"edit_count": ec.value, "text_consumed": tc.value,
            "cigar": cig[: max(cl.value, 0)].copy(), "d_opt": dopt[: min(nw.value, nwin_cap)].copy(),
            "window_edits": wed[: min(nw.value, nwin_cap)].copy(),
            "status": st}


def align_batch(batch, W: int = 64, O: int = 24, k: int | None = None, threads: int | None = None,
                cigar_capacity=None):
    """Windowed alignment of a ``synth.PairBatch`` on ``threads`` host threads.

    ``cigar_capacity`` is the run capacity of each pair (default n + m + 1).
    Returns dict(edit_counts, text_consumed, cigar, cigar_off, cigar_lens).
    """
    k = W if k is None else k
    threads = threads or os.cpu_count() or 1
    n_pairs = batch.n_pairs
    if cigar_capacity is None:
        cap = (np.diff(batch.text_off) + np.diff(batch.pattern_off) + 1).astype(np.int64)
    else:
        cap = np.broadcast_to(np.asarray(cigar_capacity, dtype=np.int64), (n_pairs,))
    cig_off = np.zeros(n_pairs + 1, dtype=np.int64)
    np.cumsum(cap, out=cig_off[1:])
    cig = np.zeros(int(cig_off[-1]), dtype=np.uint32)
    ec = np.zeros(n_pairs, dtype=np.int32)
    tc = np.zeros(n_pairs, dtype=np.int32)
    cl = np.zeros(n_pairs, dtype=np.int32)
    texts, patterns = _codes(batch.texts), _codes(batch.patterns)
    toff = np.ascontiguousarray(batch.text_off, dtype=np.int64)
    poff = np.ascontiguousarray(batch.pattern_off, dtype=np.int64)
    st = _load().orc_align_batch(_ptr(texts), _ptr(toff), _ptr(patterns), _ptr(poff), n_pairs, W, O, k,
                                 int(threads), _ptr(ec), _ptr(tc), _ptr(cig), _ptr(cig_off), _ptr(cl))
    if st != 0:
        raise ValueError("bad arguments or internal oracle error")
    return {"edit_counts": ec, "text_consumed": tc, "cigar": cig, "cigar_off": cig_off, "cigar_lens": cl}


def cigar_string(runs) -> str:
    """uint32 runs -> text CIGAR such as '12=1X3=1I'."""
    return "".join(f"{int(r) >> 4}{OP_CHAR[int(r) & 15]}" for r in runs)


def pair_cigar(result: dict, p: int) -> np.ndarray:
    """Runs of pair p from an ``align_batch`` result."""
    o = int(result["cigar_off"][p])
    return result["cigar"][o:o + max(int(result["cigar_lens"][p]), 0)]
