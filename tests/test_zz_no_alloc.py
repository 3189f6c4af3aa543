"""The allocation-free entry point against the allocating one.

Some callers cannot allocate device memory: code that runs while a stream is
being captured into a CUDA graph, or an application that hands out all device
memory through its own allocator. ``scrooge_align_batch_noalloc`` serves them
by keeping its only scratch (deep DP rows, one status word) in a fixed static
array compiled into the library. Called twice in a row through the C ABI, it
must give exactly the results of ``scrooge_align_batch``; the second call also
shows that the shared array's leftover contents do not leak into results.
"""
import numpy as np
import pytest

import paper_2208_09985_gb300 as sc
from paper_2208_09985_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("W,O,k,extra", [(64, 24, 64, 0), (32, 17, 32, 0), (128, 64, 128, 0), (64, 33, 12, 0),
                                         (64, 60, 64, 0), (32, 28, 32, 0), (64, 60, 64, sc.SCROOGE_NO_EXT_DENT),
                                         (32, 17, 32, sc.SCROOGE_NO_EXT_DENT)])
def test_noalloc_matches_allocating_entry_point(W, O, k, extra):
    import torch
    assert torch.cuda.is_available()
    batch = synth.concat([synth.tiny_windows(300, seed=1), synth.long_reads(24, seed=4),
                          synth.random_pairs(200, 300, 300, seed=6), synth.fixed_error(8, 0.15, seed=2)])
    pb = sc.PackedBatch(batch)
    ctx = sc.scrooge_create(0)
    try:
        ref = sc.align_host(ctx, pb, W, O, k, extra)
    finally:
        sc.scrooge_destroy(ctx)
    n = batch.n_pairs
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    texts, toff, tlen = dev(pb.texts), dev(pb.text_off), dev(pb.text_len)
    pats, poff, plen = dev(pb.patterns), dev(pb.pat_off), dev(pb.pat_len)
    cap = pb.text_len.astype(np.int64) + pb.pat_len.astype(np.int64) + 1
    coff_h = np.zeros(n + 1, np.int64)
    np.cumsum(cap, out=coff_h[1:])
    coff = dev(coff_h)
    stream = torch.cuda.current_stream()
    for call in range(2):
        ec = torch.full((n,), -7, dtype=torch.int32, device="cuda")
        tc = torch.full((n,), -7, dtype=torch.int32, device="cuda")
        lens = torch.full((n,), -7, dtype=torch.int32, device="cuda")
        cig = torch.zeros(int(coff_h[-1]), dtype=torch.int32, device="cuda")
        status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
        sc.scrooge_align_batch_noalloc(texts, toff, tlen, pats, poff, plen, n, W, O, k, sc.SCROOGE_SYNC | extra, ec, tc,
                                       cig, coff, lens, status, stream)
        torch.cuda.synchronize()
        assert int(status.item()) == 0, f"call {call}: status {int(status.item())}"
        np.testing.assert_array_equal(ec.cpu().numpy(), ref["edit_counts"])
        np.testing.assert_array_equal(tc.cpu().numpy(), ref["text_consumed"])
        got_lens = lens.cpu().numpy()
        np.testing.assert_array_equal(got_lens, ref["cigar_lens"])
        runs = cig.cpu().numpy().view(np.uint32)
        for p in range(n):
            a = runs[coff_h[p]:coff_h[p] + got_lens[p]]
            b = ref["cigar"][ref["cigar_off"][p]:ref["cigar_off"][p + 1]]
            assert np.array_equal(a, b), f"call {call}: CIGAR of pair {p} differs"


def test_noalloc_rejects_bad_arguments():
    import torch
    z = torch.zeros(4, dtype=torch.int64, device="cuda")
    with pytest.raises(sc.ScroogeError) as e:
        sc.scrooge_align_batch_noalloc(z, z, z, z, z, z, 1, 64, 64, 64, 0, z, z, z, z, z)
    assert e.value.code == sc.SCROOGE_E_INVAL
    with pytest.raises(sc.ScroogeError) as e:
        sc.scrooge_align_batch_noalloc(z, z, z, z, z, z, 1, 64, 24, 64, sc.SCROOGE_NO_SENE, z, z, z, z, z)
    assert e.value.code == sc.SCROOGE_E_INVAL
