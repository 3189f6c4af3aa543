"""Training and persistence of the learned pair-ordering model.

The model predicts, from cheap per-pair features, the pair's mean number of
DP rows per window (the early-termination work of the method), as
``log1p(rows / windows)``. Labels come from the method itself: an alignment
run with per-pair statistics switched on. Features, training (forward,
backward, Adam) and inference all run in the library's CUDA kernels; this
module only moves tensors between those calls and reads/writes JSON.
"""
from __future__ import annotations

import json
import os

import numpy as np

import paper_2208_09985_gb300 as sc


def device_features(ctx, db) -> "torch.Tensor":
    """(n_pairs, 6) float32 features of a DeviceBatch (on its device)."""
    import torch
    feat = torch.zeros((db.n_pairs, 6), dtype=torch.float32, device=db.texts.device)
    sc.scrooge_features(ctx, db.texts, db.text_off, db.text_len, db.patterns, db.pat_off, db.pat_len, db.n_pairs,
                        feat)
    return feat


def method_labels(ctx, db, W: int = 64, O: int = 24, k: int | None = None):
    """Per-pair statistics of one alignment run: (windows, rows, cells, cycles) device tensors."""
    import torch
    dev = db.texts.device
    n = db.n_pairs
    win = torch.zeros(n, dtype=torch.int32, device=dev)
    rows = torch.zeros(n, dtype=torch.int64, device=dev)
    cells = torch.zeros(n, dtype=torch.int64, device=dev)
    cyc = torch.zeros(n, dtype=torch.int64, device=dev)
    sc.scrooge_set_stats(ctx, win, rows, cells, cyc)
    try:
        sc.align_device(ctx, db, W, O, k, sc.SCROOGE_SYNC)
    finally:
        sc.scrooge_set_stats(ctx)
    return win, rows, cells, cyc


def load_target(win, rows) -> "torch.Tensor":
    """log1p of the mean DP rows per window (0 for pairs without windows)."""
    import torch
    w = win.to(torch.float32).clamp_min(1.0)
    return torch.log1p(rows.to(torch.float32) / w)


def train(ctx, db, W: int = 64, O: int = 24, epochs: int = 40, batch: int = 1024, lr: float = 2e-3,
          seed: int = 1):
    """Label a DeviceBatch with the method's statistics and train a model on it.

    Returns (params float32 array, per-epoch loss array). The model stays
    installed in ``ctx``.
    """
    win, rows, _, _ = method_labels(ctx, db, W, O)
    target = load_target(win, rows).contiguous()
    feat = device_features(ctx, db)
    hist = sc.scrooge_model_train(ctx, feat, target, db.n_pairs, epochs, batch, lr, seed)
    return sc.scrooge_model_get(ctx), hist


def save_model(path: str, params: np.ndarray, meta: dict | None = None) -> None:
    doc = {"format": "scrooge-order-mlp-1", "floats": int(params.shape[0]), "params": [float(x) for x in params],
           "meta": meta or {}}
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(doc, f)
    os.replace(tmp, path)


def load_model(ctx, path: str) -> dict:
    """Install a saved model in ``ctx``; returns its metadata."""
    with open(path) as f:
        doc = json.load(f)
    if doc.get("format") != "scrooge-order-mlp-1" or doc.get("floats") != sc.scrooge_model_floats():
        raise ValueError(f"{path}: not a model of this library")
    sc.scrooge_model_set(ctx, np.asarray(doc["params"], dtype=np.float32))
    return doc.get("meta", {})


def _tune_key(gpu: str, W: int, O: int, flags: int) -> str:
    return f"{gpu}|W={W}|O={O}|flags={flags}"


def autotune_cached(ctx, db, W: int, O: int, flags: int = 0, cache_path: str | None = None, gpu: str = "gpu",
                    repeats: int = 2):
    """Kernel settings for (gpu, W, O, flags): from the JSON cache, else by scrooge_autotune (and stored)."""
    words = sc.settings_slot(W, flags)
    cache = {}
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as f:
            cache = json.load(f)
    key = _tune_key(gpu, W, O, flags)
    if key in cache:
        lanes, rows, wpb = cache[key]["config"]
        sc.scrooge_set_kernel_config(ctx, words, lanes, rows, wpb)
        if "heavy_class" in cache[key]:
            sc.scrooge_set_heavy_class(ctx, cache[key]["heavy_class"])
        return cache[key]
    table = sc.autotune_device(ctx, db, W, O, flags=flags, repeats=repeats)
    cfg = sc.scrooge_get_kernel_config(ctx, words)
    entry = {"config": list(cfg), "table": [list(r) for r in table], "pairs": db.n_pairs,
             "heavy_class": sc.scrooge_get_heavy_class(ctx)}
    if cache_path:
        cache[key] = entry
        tmp = cache_path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1)
        os.replace(tmp, cache_path)
    return entry
