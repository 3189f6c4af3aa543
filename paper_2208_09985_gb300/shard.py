"""Sharding a batch of pairs over ranks and gathering the results (host side).

Pairs are independent and no window crosses a pair, so a batch splits into
per-rank shards with no exchange on the data path; only the final results are
concatenated, with CIGAR offsets rebased. Two partitions are offered:
contiguous slices, and a cost-balanced one (longest-processing-time-first on a
per-pair cost such as the predicted work).
"""
from __future__ import annotations

import heapq

import numpy as np


def shard_indices(n_pairs: int, world: int, rank: int, cost=None) -> np.ndarray:
    """Pair indices of ``rank``: contiguous slices, or LPT on ``cost`` (ascending indices either way)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad world/rank")
    if cost is None:
        bounds = np.linspace(0, n_pairs, world + 1).round().astype(np.int64)
        return np.arange(bounds[rank], bounds[rank + 1], dtype=np.int64)
    cost = np.asarray(cost, dtype=np.float64)
    if cost.shape != (n_pairs,):
        raise ValueError("one cost per pair")
    heap = [(0.0, r) for r in range(world)]
    owner = np.empty(n_pairs, dtype=np.int64)
    for p in np.argsort(-cost, kind="stable"):
        load, r = heapq.heappop(heap)
        owner[p] = r
        heapq.heappush(heap, (load + float(cost[p]), r))
    return np.flatnonzero(owner == rank)


def merge_results(n_pairs: int, parts) -> dict:
    """Concatenate per-shard results [(indices, result dict)] into one result in pair order.

    A result dict has edit_counts, text_consumed, cigar (runs) and cigar_off
    (n_local + 1 offsets into cigar). The merged CIGAR is dense in pair order.
    """
    ec = np.zeros(n_pairs, np.int32)
    tc = np.zeros(n_pairs, np.int32)
    lens = np.zeros(n_pairs, np.int64)
    seen = np.zeros(n_pairs, bool)
    for idx, res in parts:
        idx = np.asarray(idx, dtype=np.int64)
        if seen[idx].any():
            raise ValueError("a pair appears in two shards")
        seen[idx] = True
        ec[idx] = res["edit_counts"]
        tc[idx] = res["text_consumed"]
        lens[idx] = np.diff(np.asarray(res["cigar_off"], dtype=np.int64))
    if not seen.all():
        raise ValueError("some pairs are in no shard")
    off = np.zeros(n_pairs + 1, np.int64)
    np.cumsum(lens, out=off[1:])
    cig = np.zeros(int(off[-1]), np.uint32)
    for idx, res in parts:
        loc_off = np.asarray(res["cigar_off"], dtype=np.int64)
        runs = np.asarray(res["cigar"]).view(np.uint32)
        for q, p in enumerate(np.asarray(idx, dtype=np.int64)):
            cig[off[p]:off[p + 1]] = runs[loc_off[q]:loc_off[q + 1]]
    return {"edit_counts": ec, "text_consumed": tc, "cigar": cig, "cigar_off": off,
            "cigar_lens": np.diff(off).astype(np.int32)}


def gather_to_rank0(n_pairs: int, indices: np.ndarray, result: dict, group=None):
    """Collect every rank's (indices, result) on rank 0 with torch.distributed; merged result there, None elsewhere."""
    import torch.distributed as dist
    payload = (np.asarray(indices), {k: np.asarray(result[k]) for k in ("edit_counts", "text_consumed", "cigar",
                                                                         "cigar_off")})
    world = dist.get_world_size(group)
    out = [None] * world if dist.get_rank(group) == 0 else None
    dist.gather_object(payload, out, dst=0, group=group)
    if dist.get_rank(group) != 0:
        return None
    return merge_results(n_pairs, out)
