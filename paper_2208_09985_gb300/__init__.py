"""Python binding of ``libscrooge.so``, the GB300 windowed GenASM aligner.

The functions below carry the names of the C ABI in ``include/scrooge.h`` and
only marshal arguments: every step of the alignment runs in the CUDA library.
There is no fallback: if the library is not built, calls raise.

Arrays may be numpy arrays (host memory) or torch tensors. With
``SCROOGE_DEVICE_PTRS`` in ``flags`` every array of ``scrooge_align_batch``
must be a CUDA tensor; otherwise every array must be in host memory.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(_HERE)
LIB_PATH = os.path.join(_HERE, "_build", "libscrooge.so")
HEADER = os.path.join(ROOT, "include", "scrooge.h")

SCROOGE_OK = 0
SCROOGE_E_INVAL = -1
SCROOGE_E_NOMEM = -2
SCROOGE_E_CUDA = -3
SCROOGE_E_TIMEOUT = -4
SCROOGE_E_NOMODEL = -5
SCROOGE_E_INTERNAL = -6
SCROOGE_E_CAPACITY = -7

SCROOGE_DEVICE_PTRS = 1 << 0
SCROOGE_SYNC = 1 << 1
SCROOGE_NO_SENE = 1 << 2
SCROOGE_NO_DENT = 1 << 3
SCROOGE_NO_ET = 1 << 4
SCROOGE_PERSISTENT = 1 << 5
SCROOGE_LEARNED = 1 << 6
SCROOGE_GRAPH = 1 << 7
SCROOGE_NO_BAND = 1 << 8
SCROOGE_WARP_SPECIALIZED = 1 << 9
SCROOGE_WIDE_BAND = 1 << 10
SCROOGE_NO_EXT_DENT = 1 << 11

SCROOGE_OP_I, SCROOGE_OP_D, SCROOGE_OP_EQ, SCROOGE_OP_X = 1, 2, 7, 8

_lib = None
_lock = threading.Lock()


class ScroogeError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"scrooge error {code}: {msg}")
        self.code = code


def load():
    """The loaded CUDA library. Raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"CUDA library missing at {LIB_PATH}: build it with "
                                   "`python -c 'import __graft_entry__ as g; g.build()'`")
            lib = ctypes.CDLL(LIB_PATH)
            P, i32, i64, u32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32
            sig = {
                "scrooge_create": ([ctypes.POINTER(P), ctypes.c_int, P], ctypes.c_int),
                "scrooge_destroy": ([P], ctypes.c_int),
                "scrooge_last_error": ([P], ctypes.c_char_p),
                "scrooge_set_stream": ([P, P], ctypes.c_int),
                "scrooge_packed_words": ([i64], i64),
                "scrooge_pack_2bit": ([P, P, i32, ctypes.c_int, P, i64, P, P], ctypes.c_int),
                "scrooge_align_batch": ([P, P, P, P, P, P, P, i32, i32, i32, i32, u32, P, P, P, i64, P],
                                        ctypes.c_int),
                "scrooge_set_kernel_config": ([P, i32, i32, i32, i32], ctypes.c_int),
                "scrooge_get_kernel_config": ([P, i32, P, P, P], ctypes.c_int),
                "scrooge_set_stats": ([P, P, P, P, P], ctypes.c_int),
                "scrooge_set_order": ([P, P, i32], ctypes.c_int),
                "scrooge_model_floats": ([], i32),
                "scrooge_set_timing_events": ([P, P, P], ctypes.c_int),
                "scrooge_last_kernel_count": ([P], i32),
                "scrooge_model_set": ([P, P, i32], ctypes.c_int),
                "scrooge_model_get": ([P, P, i32], ctypes.c_int),
                "scrooge_features": ([P, P, P, P, P, P, P, i32, P], ctypes.c_int),
                "scrooge_model_predict": ([P, P, i32, P], ctypes.c_int),
                "scrooge_model_grad": ([P, P, P, i32, P, P], ctypes.c_int),
                "scrooge_model_train": ([P, P, P, i32, i32, i32, ctypes.c_float, ctypes.c_uint64, P], ctypes.c_int),
                "scrooge_learned_order": ([P, P, P, P, P, P, P, i32, P], ctypes.c_int),
                "scrooge_debug_fail_next_allocs": ([P, i32], ctypes.c_int),
                "scrooge_autotune": ([P, P, P, P, P, P, P, i32, i32, i32, i32, u32, P, P, P, i64, P, i32, P, i32,
                                      P], ctypes.c_int),
                "scrooge_align_batch_noalloc": ([P, P, P, P, P, P, i32, i32, i32, i32, u32, P, P, P, P, P, P, P],
                                                ctypes.c_int),
                "scrooge_edit_distance": ([P, P, P, P, P, P, P, i32, i32, u32, P, P], ctypes.c_int),
                "scrooge_last_launch_shape": ([P, P, i32], ctypes.c_int),
                "scrooge_set_heavy_class": ([P, i32], ctypes.c_int),
                "scrooge_get_heavy_class": ([P], i32),
                "scrooge_set_long_class": ([P, i32], ctypes.c_int),
                "scrooge_get_long_class": ([P], i32),
                "scrooge_logic_peak": ([P, i32, P, P], ctypes.c_int),
                "scrooge_set_wait_limit": ([P, i32], ctypes.c_int),
                "scrooge_set_bucket_config": ([P, i32, i32, i32, i32, i32], ctypes.c_int),
                "scrooge_get_bucket_config": ([P, i32, P, P, P, P], ctypes.c_int),
                "scrooge_set_learned_order": ([P, i32], ctypes.c_int),
                "scrooge_get_learned_order": ([P], i32),
                "scrooge_set_host_overlap": ([P, i32], ctypes.c_int),
                "scrooge_get_host_overlap": ([P], i32),
            }
            for name, (args, res) in sig.items():
                f = getattr(lib, name)
                f.argtypes = args
                f.restype = res
            _lib = lib
    return _lib


def header_functions() -> list[str]:
    """Names of every function declared in include/scrooge.h."""
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(scrooge_\w+)\s*\(", src)))


def _ptr(a):
    """Raw address of a numpy array or torch tensor (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return a.data_ptr()
    if isinstance(a, int):
        return a
    raise TypeError(f"unsupported array type {type(a)}")


def _check(ctx, rc: int):
    if rc != SCROOGE_OK:
        msg = load().scrooge_last_error(ctx).decode() if ctx else ""
        raise ScroogeError(rc, msg)
    return rc


def scrooge_create(device: int = 0, stream=None):
    """New context on ``device``; ``stream`` is a torch.cuda.Stream, a raw handle or None."""
    h = ctypes.c_void_p()
    s = getattr(stream, "cuda_stream", stream)
    rc = load().scrooge_create(ctypes.byref(h), int(device), s)
    if rc != SCROOGE_OK:
        raise ScroogeError(rc, "scrooge_create failed (no usable CUDA device?)")
    return h


def scrooge_destroy(ctx):
    return load().scrooge_destroy(ctx)


def scrooge_last_error(ctx) -> str:
    return load().scrooge_last_error(ctx).decode()


def scrooge_set_stream(ctx, stream):
    return _check(ctx, load().scrooge_set_stream(ctx, getattr(stream, "cuda_stream", stream)))


def scrooge_packed_words(n_bases: int) -> int:
    return int(load().scrooge_packed_words(int(n_bases)))


def scrooge_pack_2bit(seqs: np.ndarray, offsets: np.ndarray, ascii: bool = False):
    """Pack concatenated sequences; returns (packed uint32, base offsets int64, lengths int32)."""
    seqs = np.ascontiguousarray(seqs, dtype=np.uint8)
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    n = offsets.shape[0] - 1
    lens = np.diff(offsets)
    total = int(sum((int(x) + 63) // 64 * 4 for x in lens)) if n < 4096 else \
        int((((lens + 63) // 64) * 4).sum())
    packed = np.zeros(max(total, 1), dtype=np.uint32)
    poff = np.zeros(max(n, 1), dtype=np.int64)
    plen = np.zeros(max(n, 1), dtype=np.int32)
    rc = load().scrooge_pack_2bit(_ptr(seqs), _ptr(offsets), n, 1 if ascii else 0, _ptr(packed),
                                  packed.shape[0], _ptr(poff), _ptr(plen))
    if rc != SCROOGE_OK:
        raise ScroogeError(rc, "scrooge_pack_2bit: bad sequence or offsets")
    return packed, poff[:n], plen[:n]


def scrooge_align_batch(ctx, texts, text_offsets, text_lengths, patterns, pattern_offsets, pattern_lengths,
                        n_pairs: int, W: int, O: int, k: int, flags: int, edit_counts, text_consumed, cigar,
                        cigar_capacity: int, cigar_offsets):
    """Direct call of the C entry point; raises ScroogeError on a non-zero return."""
    rc = load().scrooge_align_batch(ctx, _ptr(texts), _ptr(text_offsets), _ptr(text_lengths), _ptr(patterns),
                                    _ptr(pattern_offsets), _ptr(pattern_lengths), int(n_pairs), int(W), int(O),
                                    int(k), int(flags), _ptr(edit_counts), _ptr(text_consumed), _ptr(cigar),
                                    int(cigar_capacity), _ptr(cigar_offsets))
    return _check(ctx, rc)


def scrooge_set_kernel_config(ctx, words: int, lanes_per_pair: int, smem_rows: int, warps_per_block: int):
    return _check(ctx, load().scrooge_set_kernel_config(ctx, words, lanes_per_pair, smem_rows, warps_per_block))


def scrooge_get_kernel_config(ctx, words: int):
    a, b, c = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _check(ctx, load().scrooge_get_kernel_config(ctx, words, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return a.value, b.value, c.value


def scrooge_autotune(ctx, texts, text_offsets, text_lengths, patterns, pattern_offsets, pattern_lengths,
                     n_pairs: int, W: int, O: int, k: int, flags: int, edit_counts, text_consumed, cigar,
                     cigar_capacity: int, cigar_offsets, repeats: int = 2, max_results: int = 512):
    """Time every kernel configuration on a device batch; returns rows (a, b, c, microseconds, kind): kind 1
    kernel settings (lanes, rows, warps), 2 heavy load classes (0, class, 0), 3 bucket settings (bucket*1000 +
    kernel kind*100 + lanes, rows, warps), 4 learned order on/off (1 or 0, 0, 0), 5 long-pair classes
    (0, class, 1); see include/scrooge.h."""
    res = np.zeros((max_results, 5), dtype=np.int32)
    nres = ctypes.c_int32(0)
    rc = load().scrooge_autotune(ctx, _ptr(texts), _ptr(text_offsets), _ptr(text_lengths), _ptr(patterns),
                                 _ptr(pattern_offsets), _ptr(pattern_lengths), int(n_pairs), int(W), int(O), int(k),
                                 int(flags), _ptr(edit_counts), _ptr(text_consumed), _ptr(cigar),
                                 int(cigar_capacity), _ptr(cigar_offsets), int(repeats), _ptr(res), max_results,
                                 ctypes.byref(nres))
    _check(ctx, rc)
    return [tuple(int(x) for x in r) for r in res[: nres.value]]


def settings_slot(W: int, flags: int = 0) -> int:
    """The kernel-settings slot (``words`` of scrooge_set_kernel_config) a call with W and flags uses."""
    if 32 < W <= 128 and not flags & (SCROOGE_NO_SENE | SCROOGE_NO_ET | SCROOGE_NO_BAND):
        return 0 if W <= 64 else 3
    return 1 if W <= 32 else (2 if W <= 64 else 4)


def autotune_device(ctx, db: "DeviceBatch", W: int = 64, O: int = 24, k: int | None = None, flags: int = 0,
                    repeats: int = 2):
    """scrooge_autotune on a DeviceBatch; the fastest configuration stays installed in ``ctx``."""
    k = W if k is None else k
    return scrooge_autotune(ctx, db.texts, db.text_off, db.text_len, db.patterns, db.pat_off, db.pat_len,
                            db.n_pairs, W, O, k, flags, db.edit_counts, db.text_consumed, db.cigar,
                            db.cigar_capacity, db.cigar_off, repeats)


def scrooge_set_order(ctx, order=None, n_pairs: int = 0):
    """Pair order (device int32 tensor) of later SCROOGE_PERSISTENT calls; None = input order."""
    return _check(ctx, load().scrooge_set_order(ctx, _ptr(order), int(n_pairs) if order is not None else 0))


def scrooge_set_timing_events(ctx, start=None, stop=None):
    """torch.cuda.Event pair recorded around the alignment kernel of later calls (None, None = off)."""
    h = lambda ev: None if ev is None else ev.cuda_event
    return _check(ctx, load().scrooge_set_timing_events(ctx, h(start), h(stop)))


LAUNCH_SHAPE_KEYS = ("kernel", "lanes", "smem_rows", "warps_per_block", "smem_bytes_per_block", "blocks",
                     "stored_columns", "stored_words", "table_bytes_per_warp", "scratch_bytes_per_warp",
                     "fallback_bytes_per_warp", "pairs_per_warp", "row_slots")


def scrooge_last_launch_shape(ctx) -> dict:
    """Launch shape of the context's last alignment call (see include/scrooge.h)."""
    a = np.zeros(len(LAUNCH_SHAPE_KEYS), dtype=np.int64)
    _check(ctx, load().scrooge_last_launch_shape(ctx, _ptr(a), len(a)))
    return dict(zip(LAUNCH_SHAPE_KEYS, (int(x) for x in a)))


def scrooge_set_heavy_class(ctx, load_class: int):
    """Learned launches: load classes >= load_class run on the full-width kernel (16: none)."""
    return _check(ctx, load().scrooge_set_heavy_class(ctx, int(load_class)))


def scrooge_get_heavy_class(ctx) -> int:
    return int(load().scrooge_get_heavy_class(ctx))


def scrooge_set_long_class(ctx, work_class: int):
    """Learned launches: pairs in work classes >= work_class get a warp each (16: off)."""
    return _check(ctx, load().scrooge_set_long_class(ctx, int(work_class)))


def scrooge_get_long_class(ctx) -> int:
    return int(load().scrooge_get_long_class(ctx))


def scrooge_last_kernel_count(ctx) -> int:
    return int(load().scrooge_last_kernel_count(ctx))


def scrooge_model_floats() -> int:
    return int(load().scrooge_model_floats())


def scrooge_model_set(ctx, params: np.ndarray):
    params = np.ascontiguousarray(params, dtype=np.float32)
    return _check(ctx, load().scrooge_model_set(ctx, _ptr(params), params.shape[0]))


def scrooge_model_get(ctx) -> np.ndarray:
    out = np.zeros(scrooge_model_floats(), dtype=np.float32)
    _check(ctx, load().scrooge_model_get(ctx, _ptr(out), out.shape[0]))
    return out


def scrooge_features(ctx, texts, text_offsets, text_lengths, patterns, pattern_offsets, pattern_lengths, n_pairs,
                     features):
    return _check(ctx, load().scrooge_features(ctx, _ptr(texts), _ptr(text_offsets), _ptr(text_lengths),
                                               _ptr(patterns), _ptr(pattern_offsets), _ptr(pattern_lengths),
                                               int(n_pairs), _ptr(features)))


def scrooge_model_predict(ctx, features, n: int, pred):
    return _check(ctx, load().scrooge_model_predict(ctx, _ptr(features), int(n), _ptr(pred)))


def scrooge_model_grad(ctx, features, targets, n: int, grad) -> float:
    loss = ctypes.c_float(0.0)
    _check(ctx, load().scrooge_model_grad(ctx, _ptr(features), _ptr(targets), int(n), _ptr(grad),
                                          ctypes.byref(loss)))
    return loss.value


def scrooge_model_train(ctx, features, targets, n: int, epochs: int = 30, batch: int = 1024, lr: float = 2e-3,
                        seed: int = 1) -> np.ndarray:
    hist = np.zeros(epochs, dtype=np.float32)
    _check(ctx, load().scrooge_model_train(ctx, _ptr(features), _ptr(targets), int(n), int(epochs), int(batch),
                                           float(lr), int(seed), _ptr(hist)))
    return hist


def scrooge_learned_order(ctx, texts, text_offsets, text_lengths, patterns, pattern_offsets, pattern_lengths,
                          n_pairs, order):
    return _check(ctx, load().scrooge_learned_order(ctx, _ptr(texts), _ptr(text_offsets), _ptr(text_lengths),
                                                    _ptr(patterns), _ptr(pattern_offsets), _ptr(pattern_lengths),
                                                    int(n_pairs), _ptr(order)))


def scrooge_set_stats(ctx, windows=None, rows=None, cells=None, cycles=None):
    return _check(ctx, load().scrooge_set_stats(ctx, _ptr(windows), _ptr(rows), _ptr(cells), _ptr(cycles)))


SCROOGE_EDIT_DISTANCE_MAX_M = 16384


def scrooge_edit_distance(ctx, texts, text_offsets, text_lengths, patterns, pattern_offsets, pattern_lengths,
                          n_pairs: int, max_pattern_length: int, flags: int, free_end, global_distance):
    """Exact free-end and global edit distances (device tensors; flags must include SCROOGE_DEVICE_PTRS)."""
    return _check(ctx, load().scrooge_edit_distance(ctx, _ptr(texts), _ptr(text_offsets), _ptr(text_lengths),
                                                    _ptr(patterns), _ptr(pattern_offsets), _ptr(pattern_lengths),
                                                    int(n_pairs), int(max_pattern_length), int(flags),
                                                    _ptr(free_end), _ptr(global_distance)))


def edit_distance_device(ctx, db: "DeviceBatch", sync: bool = True):
    """(free_end, global) int32 device tensors of a DeviceBatch: the optimal scores of its pairs."""
    import torch
    fe = torch.empty(db.n_pairs, dtype=torch.int32, device=db.texts.device)
    gl = torch.empty(db.n_pairs, dtype=torch.int32, device=db.texts.device)
    max_m = int(db.pat_len.max().item()) if db.n_pairs else 0
    scrooge_edit_distance(ctx, db.texts, db.text_off, db.text_len, db.patterns, db.pat_off, db.pat_len, db.n_pairs,
                          min(max_m, SCROOGE_EDIT_DISTANCE_MAX_M), SCROOGE_DEVICE_PTRS | (SCROOGE_SYNC if sync else 0),
                          fe, gl)
    return fe, gl


def scrooge_set_bucket_config(ctx, bucket: int, kind: int, lanes_per_pair: int, smem_rows: int,
                              warps_per_block: int):
    """Kernel settings of one load bucket of learned launches (0 heavy, 1 rest; kind 0 banded, 1 full width)."""
    return _check(ctx, load().scrooge_set_bucket_config(ctx, bucket, kind, lanes_per_pair, smem_rows,
                                                        warps_per_block))


def scrooge_get_bucket_config(ctx, bucket: int):
    a = [ctypes.c_int32() for _ in range(4)]
    _check(ctx, load().scrooge_get_bucket_config(ctx, bucket, *[ctypes.byref(x) for x in a]))
    return tuple(x.value for x in a)


def scrooge_set_learned_order(ctx, on: bool):
    """SCROOGE_LEARNED launches in the model's order (True) or in input order (False)."""
    return _check(ctx, load().scrooge_set_learned_order(ctx, 1 if on else 0))


def scrooge_get_learned_order(ctx) -> bool:
    return load().scrooge_get_learned_order(ctx) == 1


def scrooge_set_host_overlap(ctx, on: bool):
    """Host-pointer persistent calls of 8,192 pairs or more in 2 to 4 parts, copies under the kernels (True, the
    default), or as one launch (False)."""
    return _check(ctx, load().scrooge_set_host_overlap(ctx, 1 if on else 0))


def scrooge_get_host_overlap(ctx) -> bool:
    return load().scrooge_get_host_overlap(ctx) == 1


def scrooge_set_wait_limit(ctx, polls: int = 0):
    """Polls per bounded device wait of later calls (0: the default bound)."""
    return _check(ctx, load().scrooge_set_wait_limit(ctx, polls))


def scrooge_logic_peak(ctx, iterations: int = 4096) -> dict:
    """Measured rate of the integer logic pipe: ops/s and ops per clock per SM."""
    ops = ctypes.c_double(0.0)
    per_clk = ctypes.c_double(0.0)
    _check(ctx, load().scrooge_logic_peak(ctx, iterations, ctypes.byref(ops), ctypes.byref(per_clk)))
    return {"ops_per_s": ops.value, "ops_per_clk_per_sm": per_clk.value}


def scrooge_debug_fail_next_allocs(ctx, count: int):
    return _check(ctx, load().scrooge_debug_fail_next_allocs(ctx, int(count)))


def scrooge_align_batch_noalloc(texts, text_offsets, text_lengths, patterns, pattern_offsets, pattern_lengths,
                                n_pairs: int, W: int, O: int, k: int, flags: int, edit_counts, text_consumed, cigar,
                                cigar_offsets, cigar_lens, status=None, stream=None):
    """Allocation-free alignment (device tensors only); raises ScroogeError on a non-zero return."""
    rc = load().scrooge_align_batch_noalloc(_ptr(texts), _ptr(text_offsets), _ptr(text_lengths), _ptr(patterns),
                                            _ptr(pattern_offsets), _ptr(pattern_lengths), int(n_pairs), int(W),
                                            int(O), int(k), int(flags), _ptr(edit_counts), _ptr(text_consumed),
                                            _ptr(cigar), _ptr(cigar_offsets), _ptr(cigar_lens), _ptr(status),
                                            getattr(stream, "cuda_stream", stream))
    if rc != SCROOGE_OK:
        raise ScroogeError(rc, "scrooge_align_batch_noalloc failed")
    return rc


# --------------------------------------------------------------- helpers


class PackedBatch:
    """A synth.PairBatch packed for the library (host numpy arrays)."""

    def __init__(self, batch):
        self.n_pairs = batch.n_pairs
        self.texts, self.text_off, self.text_len = scrooge_pack_2bit(batch.texts, batch.text_off)
        self.patterns, self.pat_off, self.pat_len = scrooge_pack_2bit(batch.patterns, batch.pattern_off)

    def cigar_guess(self) -> int:
        """A CIGAR capacity (runs) that holds typical outputs: a quarter run per pattern base."""
        return int(self.pat_len.astype(np.int64).sum()) // 4 + 16 * self.n_pairs + 1024


def align_host(ctx, pb: PackedBatch, W: int = 64, O: int = 24, k: int | None = None, flags: int = 0,
               cigar_capacity: int | None = None) -> dict:
    """Align a PackedBatch from host memory; returns host numpy results.

    Without ``cigar_capacity`` the CIGAR buffer starts at ``pb.cigar_guess()``
    runs and the call is repeated once with the exact size if that was short.
    """
    k = W if k is None else k
    n = pb.n_pairs
    ec = np.zeros(n, np.int32)
    tc = np.zeros(n, np.int32)
    off = np.zeros(n + 1, np.int64)
    cap = pb.cigar_guess() if cigar_capacity is None else int(cigar_capacity)
    cig = np.zeros(max(cap, 1), np.uint32)
    args = (pb.texts, pb.text_off, pb.text_len, pb.patterns, pb.pat_off, pb.pat_len, n, W, O, k,
            flags & ~SCROOGE_DEVICE_PTRS, ec, tc)
    try:
        scrooge_align_batch(ctx, *args, cig, cap, off)
    except ScroogeError as e:
        if e.code != SCROOGE_E_CAPACITY or cigar_capacity is not None:
            raise
        cap = int(off[-1])
        cig = np.zeros(max(cap, 1), np.uint32)
        scrooge_align_batch(ctx, *args, cig, cap, off)
    return {"edit_counts": ec, "text_consumed": tc, "cigar": cig, "cigar_off": off,
            "cigar_lens": np.diff(off).astype(np.int32)}


class DeviceBatch:
    """A PackedBatch resident on a CUDA device (torch tensors), with output buffers."""

    def __init__(self, pb: PackedBatch, device="cuda", cigar_capacity: int | None = None):
        import torch
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(device)
        self.n_pairs = pb.n_pairs
        self.texts, self.text_off, self.text_len = t(pb.texts), t(pb.text_off), t(pb.text_len)
        self.patterns, self.pat_off, self.pat_len = t(pb.patterns), t(pb.pat_off), t(pb.pat_len)
        self.cigar_capacity = pb.cigar_guess() if cigar_capacity is None else int(cigar_capacity)
        self.cigar_off = torch.zeros(self.n_pairs + 1, dtype=torch.int64, device=device)
        self.edit_counts = torch.zeros(self.n_pairs, dtype=torch.int32, device=device)
        self.text_consumed = torch.zeros_like(self.edit_counts)
        self.cigar = torch.zeros(max(self.cigar_capacity, 1), dtype=torch.int32, device=device)


def align_device(ctx, db: DeviceBatch, W: int = 64, O: int = 24, k: int | None = None, flags: int = 0):
    """Align a DeviceBatch in place (asynchronous unless SCROOGE_SYNC is in flags)."""
    k = W if k is None else k
    return scrooge_align_batch(ctx, db.texts, db.text_off, db.text_len, db.patterns, db.pat_off, db.pat_len,
                               db.n_pairs, W, O, k, flags | SCROOGE_DEVICE_PTRS, db.edit_counts, db.text_consumed,
                               db.cigar, db.cigar_capacity, db.cigar_off)


def device_results(db: DeviceBatch) -> dict:
    """Copy a DeviceBatch's outputs to host numpy arrays."""
    off = db.cigar_off.cpu().numpy()
    return {"edit_counts": db.edit_counts.cpu().numpy(), "text_consumed": db.text_consumed.cpu().numpy(),
            "cigar": db.cigar.cpu().numpy().view(np.uint32), "cigar_off": off,
            "cigar_lens": np.diff(off).astype(np.int32)}
