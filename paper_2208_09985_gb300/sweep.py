"""Ablation sweep of the windowed alignment on 10 kbp pairs.

The grid:
- edit rates 5%, 10% and 15% (50/25/25 substitutions/insertions/deletions);
- W in {32, 64, 128}, with O in {W/4, 3W/8, W/2, W/2+1} (W/2+1 is the paper's
  operating point: the DENT entry of W-O+1 bits fits one word at W = 64, O = 33);
- each of SENE, DENT and ET on or off (the paper's ablations, Sections 2.4.1-2.4.3);
- the plain launch and the learned-ordering persistent launch side by side.

Each point reports:
- throughput;
- the DP-table footprint per pair;
- the mean edit count against the exact free-end distance of the same pairs
  (scrooge_edit_distance), and the paper's quantile scores (Section 5): the
  0.5, 0.1, 0.01 and 0.001 quantiles counted from the worst pair (for 20,000
  pairs, 0.01 is the 200th worst) of the windowed edit count, of the exact
  distance, and of the excess of one over the other, pair by pair;
- the full-width kernel with every improvement on beside the plain
  launch, so that SENE on and off (GenASM's edge vectors) compare on the same
  kernel.

SENE, DENT, ET and the launch form never change results, and each run checks
that its edit counts and CIGAR offsets match the first run of the same
(rate, W, O).

    python -m paper_2208_09985_gb300.sweep --pairs 20000 --out sweep.jsonl

This prints one JSON line per run and a markdown summary at the end. The
library's CUDA kernels do all the work; this module only drives them.

With --ext-dent it measures DENT extended to rows (Supplementary Section 1)
instead: the full-width kernels at (W, O) = (32, 17), (32, 8), (64, 33) and
(64, 24), each with the cycle of row slots (the default) and with
SCROOGE_NO_EXT_DENT, on one batch per edit rate. It checks that the results are
identical, and reports throughput, row slots and scratch bytes per pair.

    python -m paper_2208_09985_gb300.sweep --ext-dent --pairs 20000 --rates 0.10,0.15
"""
from __future__ import annotations

import argparse
import json
import sys

import numpy as np

import paper_2208_09985_gb300 as sc
from paper_2208_09985_gb300 import learned, synth

TOGGLES = [(sene, dent, et) for sene in (1, 0) for dent in (1, 0) for et in (1, 0)]
QUANTILES = (0.5, 0.1, 0.01, 0.001)


def worst_quantile(values, q: float) -> float:
    """The q quantile counted from the worst (largest) value: the ceil(q * n)-th largest of n values."""
    v = np.sort(np.asarray(values, dtype=np.float64))[::-1]
    if v.size == 0:
        return float("nan")
    return float(v[max(1, int(np.ceil(q * v.size))) - 1])


def toggle_flags(sene: int, dent: int, et: int) -> int:
    return (0 if sene else sc.SCROOGE_NO_SENE) | (0 if dent else sc.SCROOGE_NO_DENT) | (0 if et else sc.SCROOGE_NO_ET)


def method_footprint(W: int, O: int, k: int, sene: int, dent: int, mean_rows: float) -> float:
    """Bytes of the DP table the method keeps per window, by the paper's accounting.

    Three W-bit edge vectors per cell are stored without SENE, and one entry
    with it (Section 2.4.1). DENT keeps columns and bits 0..W-O only
    (Section 2.4.2). Rows run to d_opt with ET (the measured mean) and to k
    without it.
    """
    L = W - O
    cols = min(L + 1, W) if dent else W
    bits = min(L + 1, W) if dent else W
    vectors = 1 if sene else 3
    return mean_rows * cols * vectors * bits / 8.0


def align_grow(ctx, db, W, O, k, flags):
    """Synchronous align_device that grows the batch's CIGAR buffer when it is too small."""
    import torch
    try:
        sc.align_device(ctx, db, W, O, k, flags | sc.SCROOGE_SYNC)
    except sc.ScroogeError as e:
        if e.code != sc.SCROOGE_E_CAPACITY:
            raise
        need = int(db.cigar_off[-1].item())
        db.cigar = torch.zeros(need, dtype=torch.int32, device=db.cigar.device)
        db.cigar_capacity = need
        sc.align_device(ctx, db, W, O, k, flags | sc.SCROOGE_SYNC)


def timed(ctx, db, W, O, k, flags, steps, stream):
    import torch
    align_grow(ctx, db, W, O, k, flags)
    ts = []
    for _ in range(steps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        sc.align_device(ctx, db, W, O, k, flags)
        b.record(stream)
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    return float(np.median(ts))


def main(argv=None):
    import torch
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--pairs", type=int, default=20_000)
    ap.add_argument("--length", type=int, default=10_000)
    ap.add_argument("--rates", default="0.05,0.10,0.15")
    ap.add_argument("--W", default="32,64,128")
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--train-pairs", type=int, default=20_000)
    ap.add_argument("--model", default="", help="saved ordering model (JSON); default: train one first")
    ap.add_argument("--out", default="")
    ap.add_argument("--ext-dent", action="store_true", help="measure DENT extended to rows instead of the grid")
    args = ap.parse_args(argv)
    if args.ext_dent:
        return ext_dent(args)

    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    ctx = sc.scrooge_create(0, stream)
    if args.model:
        learned.load_model(ctx, args.model)
    else:
        tb = sc.DeviceBatch(sc.PackedBatch(synth.uneven_reads(args.train_pairs, seed=40)))
        learned.train(ctx, tb, epochs=20, batch=1024)
        del tb
    out = open(args.out, "w") if args.out else None
    rows = []
    for rate in (float(x) for x in args.rates.split(",")):
        batch = synth.fixed_error(args.pairs, rate, seed=500 + int(rate * 1000), length=args.length)
        db = sc.DeviceBatch(sc.PackedBatch(batch))
        fe, gl = sc.edit_distance_device(ctx, db)
        fe_mean, gl_mean = float(fe.double().mean()), float(gl.double().mean())
        bases = int(np.diff(batch.pattern_off).sum())
        for W in (int(x) for x in args.W.split(",")):
            k = W
            for O in (W // 4, 3 * W // 8, W // 2, W // 2 + 1):
                ref = None
                # statistics of the method (rows per window) from one run with ET
                win = torch.zeros(db.n_pairs, dtype=torch.int32, device="cuda")
                rws = torch.zeros(db.n_pairs, dtype=torch.int64, device="cuda")
                sc.scrooge_set_stats(ctx, win, rws, None, None)
                align_grow(ctx, db, W, O, k, 0)
                sc.scrooge_set_stats(ctx)
                mean_rows = float(rws.sum().item()) / max(1, int(win.sum().item()))
                for sene, dent, et in TOGGLES:
                    forms = ("plain", "learned", "full") if (sene, dent, et) == (1, 1, 1) else ("plain", "learned")
                    for form in forms:
                        fl = toggle_flags(sene, dent, et) | {"plain": 0, "learned": sc.SCROOGE_LEARNED,
                                                             "full": sc.SCROOGE_NO_BAND}[form]
                        ms = timed(ctx, db, W, O, k, fl, args.steps, stream)
                        shape = sc.scrooge_last_launch_shape(ctx)
                        res = sc.device_results(db)
                        if ref is None:
                            ref = res
                            ec = res["edit_counts"].astype(np.float64)
                            fe_np = fe.cpu().numpy()
                            ok = ec >= 0
                            acc = {"mean_edits": float(ec[ok].mean()), "failed_pairs": int((~ok).sum()),
                                   "mean_excess_over_free_end": float((ec[ok] - fe_np[ok]).mean()),
                                   "pairs_at_optimum": float((ec[ok] == fe_np[ok]).mean()),
                                   "quantiles": {str(q): {"windowed": worst_quantile(ec[ok], q),
                                                          "exact": worst_quantile(fe_np[ok], q),
                                                          "excess": worst_quantile(ec[ok] - fe_np[ok], q)}
                                                 for q in QUANTILES}}
                        elif not (np.array_equal(res["edit_counts"], ref["edit_counts"])
                                  and np.array_equal(res["cigar_off"], ref["cigar_off"])):
                            raise SystemExit(f"sweep: rate {rate} W {W} O {O} flags {fl} changed the results")
                        rows_per_window = mean_rows if et else k + 1
                        pps = shape["pairs_per_warp"]
                        rec = {"rate": rate, "W": W, "O": O, "k": k, "sene": sene, "dent": dent, "et": et,
                               "form": form, "ms": ms, "alignments_per_s": db.n_pairs / (ms / 1e3),
                               "gbases_per_s": bases / (ms / 1e3) / 1e9,
                               "method_table_bytes_per_window": method_footprint(W, O, k, sene, dent,
                                                                                 rows_per_window),
                               "smem_bytes_per_pair": shape["table_bytes_per_warp"] / pps,
                               "scratch_bytes_per_pair": shape["scratch_bytes_per_warp"] / pps,
                               "kernel": (("lane" if shape["lanes"] == 1 else "band") if shape["kernel"] == 0
                                          else f"full{shape['kernel']}"),
                               "lanes": shape["lanes"], "smem_rows": shape["smem_rows"],
                               "row_slots": shape["row_slots"],
                               "mean_rows_per_window": mean_rows,
                               "free_end_mean": fe_mean, "global_mean": gl_mean, **acc}
                        rows.append(rec)
                        line = json.dumps(rec)
                        print(line, flush=True)
                        if out:
                            out.write(line + "\n")
                            out.flush()
        del db
    sc.scrooge_destroy(ctx)
    print(summary(rows))


def ext_dent(args):
    """DENT extended to rows on the full-width kernels: the cycle of row slots against all k+1 rows."""
    import torch
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    ctx = sc.scrooge_create(0, stream)
    lines = ["| rate | W | O | kernel | row slots | scratch B/pair | aln/s | all k+1 rows: slots | scratch B/pair | "
             "aln/s |", "|---|---|---|---|---|---|---|---|---|---|"]
    for rate in (float(x) for x in args.rates.split(",")):
        batch = synth.fixed_error(args.pairs, rate, seed=500 + int(rate * 1000), length=args.length)
        db = sc.DeviceBatch(sc.PackedBatch(batch))
        for W, O in ((32, 17), (32, 8), (64, 33), (64, 24)):
            k = W
            cells = []
            ref = None
            for extra in (0, sc.SCROOGE_NO_EXT_DENT):
                fl = sc.SCROOGE_NO_BAND | extra
                ms = timed(ctx, db, W, O, k, fl, args.steps, stream)
                shape = sc.scrooge_last_launch_shape(ctx)
                res = sc.device_results(db)
                if ref is None:
                    ref = res
                elif not (np.array_equal(res["edit_counts"], ref["edit_counts"])
                          and np.array_equal(res["cigar_off"], ref["cigar_off"])):
                    raise SystemExit(f"ext-dent: rate {rate} W {W} O {O} changed the results")
                rec = {"rate": rate, "W": W, "O": O, "k": k, "ext_dent": int(extra == 0), "ms": ms,
                       "alignments_per_s": db.n_pairs / (ms / 1e3), "row_slots": shape["row_slots"],
                       "smem_rows": shape["smem_rows"], "lanes": shape["lanes"],
                       "scratch_bytes_per_pair": shape["scratch_bytes_per_warp"] / shape["pairs_per_warp"],
                       "kernel": f"full{shape['kernel']}"}
                print(json.dumps(rec), flush=True)
                cells.append(rec)
            a, b = cells
            lines.append(f"| {rate:.2f} | {W} | {O} | {a['kernel']} | {a['row_slots']} | "
                         f"{a['scratch_bytes_per_pair']:.0f} | {a['alignments_per_s'] / 1e6:.3f}M | {b['row_slots']} | "
                         f"{b['scratch_bytes_per_pair']:.0f} | {b['alignments_per_s'] / 1e6:.3f}M |")
        del db
    sc.scrooge_destroy(ctx)
    print("\n".join(lines))


def summary(rows) -> str:
    """Markdown tables of a sweep's JSON records."""
    lines = ["| rate | W | O | mean edits | exact free-end | excess | at optimum | rows/window |",
             "|---|---|---|---|---|---|---|---|"]
    qlines = ["| rate | W | O | " + " | ".join(f"q={q}: windowed / exact / excess" for q in QUANTILES) + " |",
              "|---|---|---|" + "---|" * len(QUANTILES)]
    seen = set()
    for r in rows:
        key = (r["rate"], r["W"], r["O"])
        if key in seen:
            continue
        seen.add(key)
        lines.append(f"| {r['rate']:.2f} | {r['W']} | {r['O']} | {r['mean_edits']:.1f} | {r['free_end_mean']:.1f} | "
                     f"{r['mean_excess_over_free_end']:.2f} | {100 * r['pairs_at_optimum']:.1f}% | "
                     f"{r['mean_rows_per_window']:.2f} |")
        qs = r["quantiles"]
        qlines.append(f"| {r['rate']:.2f} | {r['W']} | {r['O']} | " + " | ".join(
            f"{qs[str(q)]['windowed']:.0f} / {qs[str(q)]['exact']:.0f} / {qs[str(q)]['excess']:.0f}"
            for q in QUANTILES) + " |")
    lines += ["", "Quantile scores, counted from the worst pair (edit counts; lower is better):", ""] + qlines
    lines += ["", "| rate | W | O | SENE | DENT | ET | plain aln/s | learned aln/s | table B/window (method) | "
              "smem B/pair (kernel) | kernel |", "|---|---|---|---|---|---|---|---|---|---|---|"]
    by = {}
    for r in rows:
        by.setdefault((r["rate"], r["W"], r["O"], r["sene"], r["dent"], r["et"]), {})[r["form"]] = r
    for key, d in by.items():
        p, q = d.get("plain"), d.get("learned")
        base = p or q
        lines.append(f"| {key[0]:.2f} | {key[1]} | {key[2]} | {key[3]} | {key[4]} | {key[5]} | "
                     f"{p['alignments_per_s'] / 1e6:.3f}M | {q['alignments_per_s'] / 1e6:.3f}M | "
                     f"{base['method_table_bytes_per_window']:.0f} | {base['smem_bytes_per_pair']:.0f} | "
                     f"{base['kernel']} |" if p and q else "")
    # SENE on and off on the same kernel (the full-width kernel serves both)
    lines += ["", "SENE on and off on the full-width kernel (Scrooge's entries against GenASM's edges):", "",
              "| rate | W | O | SENE on, full width | SENE off (full width) | ratio |", "|---|---|---|---|---|---|"]
    for key, d in by.items():
        if key[3:] != (1, 1, 1):
            continue
        on = d.get("full")
        off = by.get(key[:3] + (0, 1, 1), {}).get("plain")
        if on and off:
            lines.append(f"| {key[0]:.2f} | {key[1]} | {key[2]} | {on['alignments_per_s'] / 1e6:.3f}M | "
                         f"{off['alignments_per_s'] / 1e6:.3f}M | {on['alignments_per_s'] / off['alignments_per_s']:.2f} |")
    return "\n".join(x for x in lines if x is not None)


if __name__ == "__main__":
    sys.exit(main())
