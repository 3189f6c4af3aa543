"""Sharding across ranks (world_size 2, gloo on CPU).

Each rank aligns only its shard (here with the CPU oracle, since the host-side
logic is what is under test); rank 0 gathers and must obtain exactly the
single-process result, for contiguous and cost-balanced shards.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2208_09985_gb300 import shard, synth


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _oracle_result(batch, idx):
    import oracle
    res = oracle.align_batch(batch.subset(idx), 32, 12, threads=2)
    lens = res["cigar_lens"].astype(np.int64)
    off = np.zeros(len(idx) + 1, np.int64)
    np.cumsum(lens, out=off[1:])
    runs = np.concatenate([res["cigar"][res["cigar_off"][q]:res["cigar_off"][q] + lens[q]] for q in range(len(idx))]) \
        if len(idx) else np.zeros(0, np.uint32)
    return {"edit_counts": res["edit_counts"], "text_consumed": res["text_consumed"], "cigar": runs, "cigar_off": off}


def _worker(rank, world, port, mode, outdir):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        b = synth.random_pairs(120, 150, 150, seed=21)
        cost = np.diff(b.pattern_off).astype(np.float64) if mode == "lpt" else None
        idx = shard.shard_indices(b.n_pairs, world, rank, cost)
        merged = shard.gather_to_rank0(b.n_pairs, idx, _oracle_result(b, idx))
        if rank == 0:
            np.savez(os.path.join(outdir, f"merged_{mode}.npz"), **merged)
    finally:
        dist.destroy_process_group()


def _bench_worker(rank, world, port, outdir):
    """The benchmark's strong-scaling step with the oracle standing in for the GPU aligner."""
    import sys
    import torch.distributed as dist
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        b = synth.concat([synth.random_pairs(60, 200, 200, seed=31), synth.short_reads(40, seed=32)])
        cost = np.diff(b.pattern_off).astype(np.float64) * (1.0 + (np.arange(b.n_pairs) % 5))
        idx, merged = bench.sharded_results(b, world, rank, lambda sub: _oracle_result(sub, np.arange(sub.n_pairs)),
                                            cost)
        np.save(os.path.join(outdir, f"idx_{rank}.npy"), idx)
        if rank == 0:
            np.savez(os.path.join(outdir, "merged_bench.npz"), **merged)
    finally:
        dist.destroy_process_group()


def test_bench_strong_scaling_two_ranks(tmp_path):
    """bench.py --scaling strong: each rank aligns its LPT shard of one batch; rank 0 gathers the single-process
    result (here with the CPU oracle as the aligner, on gloo)."""
    import oracle
    oracle.build()
    mp.spawn(_bench_worker, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    got = dict(np.load(tmp_path / "merged_bench.npz"))
    b = synth.concat([synth.random_pairs(60, 200, 200, seed=31), synth.short_reads(40, seed=32)])
    ref = _oracle_result(b, np.arange(b.n_pairs))
    for key in ("edit_counts", "text_consumed", "cigar_off", "cigar"):
        np.testing.assert_array_equal(got[key], ref[key], err_msg=key)
    i0, i1 = np.load(tmp_path / "idx_0.npy"), np.load(tmp_path / "idx_1.npy")
    assert len(i0) and len(i1) and np.array_equal(np.sort(np.concatenate([i0, i1])), np.arange(b.n_pairs))


@pytest.mark.parametrize("mode", ["contiguous", "lpt"])
def test_two_rank_shards_gather_to_the_single_process_result(tmp_path, mode):
    import oracle
    oracle.build()
    mp.spawn(_worker, args=(2, _free_port(), mode, str(tmp_path)), nprocs=2, join=True)
    got = dict(np.load(tmp_path / f"merged_{mode}.npz"))
    b = synth.random_pairs(120, 150, 150, seed=21)
    ref = _oracle_result(b, np.arange(b.n_pairs))
    np.testing.assert_array_equal(got["edit_counts"], ref["edit_counts"])
    np.testing.assert_array_equal(got["text_consumed"], ref["text_consumed"])
    np.testing.assert_array_equal(got["cigar_off"], ref["cigar_off"])
    np.testing.assert_array_equal(got["cigar"], ref["cigar"])


def test_shard_partitions():
    for n, w in ((10, 3), (0, 2), (7, 7), (100, 4)):
        parts = [shard.shard_indices(n, w, r) for r in range(w)]
        assert np.array_equal(np.sort(np.concatenate(parts)), np.arange(n))
        cost = np.arange(n, dtype=float)[::-1]
        lpt = [shard.shard_indices(n, w, r, cost) for r in range(w)]
        assert np.array_equal(np.sort(np.concatenate(lpt)), np.arange(n))
        if n >= w:  # LPT keeps the loads within the largest single cost
            loads = [cost[p].sum() for p in lpt]
            assert max(loads) - min(loads) <= cost.max() + 1e-9
    with pytest.raises(ValueError):
        shard.merge_results(3, [(np.array([0, 1]), {"edit_counts": [0, 0], "text_consumed": [0, 0],
                                                     "cigar": np.zeros(0, np.uint32), "cigar_off": [0, 0, 0]})])
