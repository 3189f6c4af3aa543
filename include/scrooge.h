/*
 * scrooge.h -- C ABI of a GB300 (sm_103a) library for Scrooge's windowed
 * GenASM pairwise alignment (Lindegger et al., "Scrooge: A Fast and Memory-
 * Frugal Genomic Sequence Aligner for CPUs, GPUs, and ASICs", arXiv 2208.09985).
 *
 * The library aligns many (text = reference, pattern = read) pairs. For each
 * pair it runs the windowing heuristic of Section 2.2.3: a W-character window
 * of both strings is aligned by GenASM-DC (Algorithm 1, Section 2.2.1) with
 * early termination at the first edit count d that reaches the window start
 * (ET, Section 2.4.3), the DP entries that the traceback can reach are kept
 * (SENE, Section 2.4.1; DENT, Section 2.4.2), and GenASM-TB (Section 2.2.2)
 * walks them to emit CIGAR operations for the first W-O characters; the next
 * window starts where the traceback stopped. The problem solved in each
 * window is edit distance with the whole pattern and a free end in the text
 * (Theorem 1 with the initial column R[n][d] = 1..1 << d).
 *
 * Conventions fixed where the paper is silent (identical to the CPU oracle):
 * the traceback prefers M, then S (substitution), then I, then D when several
 * edges hold a 0; it stops as soon as W-O text characters, or W-O pattern
 * characters, or the whole pattern window are consumed; text and pattern
 * cursors advance by the characters consumed.
 *
 * Thread safety: a context may be used by one host thread at a time.
 * All entry points return 0 (SCROOGE_OK) or a negative SCROOGE_E_* code;
 * scrooge_last_error() then describes the failure.
 */
#ifndef SCROOGE_H
#define SCROOGE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct scrooge_ctx scrooge_ctx; /* opaque, owned by the library */

/* ------------------------------------------------------------ status codes */
#define SCROOGE_OK 0
#define SCROOGE_E_INVAL (-1)    /* bad argument (sizes, alignment, W/O/k, null pointer) */
#define SCROOGE_E_NOMEM (-2)    /* device or host allocation failed */
#define SCROOGE_E_CUDA (-3)     /* a CUDA call failed; see scrooge_last_error */
#define SCROOGE_E_TIMEOUT (-4)  /* a bounded device wait gave up */
#define SCROOGE_E_NOMODEL (-5)  /* SCROOGE_LEARNED without a loaded or trained model */
#define SCROOGE_E_INTERNAL (-6) /* a kernel reported an impossible state */
#define SCROOGE_E_CAPACITY (-7) /* the CIGAR output buffer is too small (see scrooge_align_batch) */

/* ------------------------------------------------------------------- flags */
/* All pointers passed to scrooge_align_batch are device pointers and the
 * call is asynchronous on the context stream. Without it, all pointers are
 * host pointers: inputs are copied to the device, outputs back, and the call
 * returns when the results are in host memory. */
#define SCROOGE_DEVICE_PTRS (1u << 0)
/* With SCROOGE_DEVICE_PTRS: synchronise the stream before returning. */
#define SCROOGE_SYNC (1u << 1)
/* Ablation switches (Section 3.3); results are identical with any of them. */
#define SCROOGE_NO_SENE (1u << 2) /* store GenASM's three edge vectors instead of entries */
#define SCROOGE_NO_DENT (1u << 3) /* store every column and every bit of each entry */
#define SCROOGE_NO_ET (1u << 4)   /* compute all k+1 rows of every window */
/* Scheduling (results are identical): */
#define SCROOGE_PERSISTENT (1u << 5) /* pair slots pull pairs from a device work queue (see scrooge_set_order) */
#define SCROOGE_LEARNED (1u << 6)    /* order pairs by the MLP's predicted load (implies PERSISTENT) */
/* Capture the launch sequence (ordering, alignment, CIGAR offsets and gather)
 * in a CUDA graph, kept in the context and replayed while the same call
 * (pointers, sizes, W/O/k, flags, kernel settings) repeats. Needs a stream
 * other than the legacy default stream. */
#define SCROOGE_GRAPH (1u << 7)
/* Implementation choice, never a change of results: windows of 33..128 bases
 * with SENE and ET use the banded kernels unless this flag asks for the
 * full-width ones (see "kernel settings"). */
#define SCROOGE_NO_BAND (1u << 8)
/* Implementation choice, never a change of results: persistent launches of
 * the banded kernel run as blocks of four DC warps and one traceback warp,
 * which hand windows over through shared-memory barriers (4 lanes per pair,
 * the banded kernel settings' shared-memory rows). Every barrier wait is
 * bounded; if one gives up, the synchronous call returns SCROOGE_E_TIMEOUT. */
#define SCROOGE_WARP_SPECIALIZED (1u << 9)
/* Implementation choice, never a change of results: windows of 33..64 bases
 * use the 64-diagonal band (two words per entry, exact for d_opt <= 31)
 * instead of the 32-diagonal one; lanes_per_pair 4 or 8. */
#define SCROOGE_WIDE_BAND (1u << 10)
/* Ablation switch, results identical: keep every full-width row of a window
 * instead of DENT extended to rows (Supplementary Section 1). By default,
 * with SENE, DENT and ET all on, the row store of a full-width kernel's window
 * (and of the allocation-free entry point) is a
 * cycle of R = max(W-O+G, ceil((k+1)/2)) row slots (G = lanes per pair; row d
 * in slot d mod R) instead of k+1 rows: the traceback only reads rows
 * d_opt-(W-O)..d_opt, and the row pipeline over a pair's lanes stores at most
 * G-1 rows past d_opt. The lower bound lets a row wrap at most once. */
#define SCROOGE_NO_EXT_DENT (1u << 11)

/* CIGAR run encoding: (length << 4) | op, op in SAM codes. */
#define SCROOGE_OP_I 1  /* base only in the pattern (read): insertion */
#define SCROOGE_OP_D 2  /* base only in the text (reference): deletion */
#define SCROOGE_OP_EQ 7 /* '=' match */
#define SCROOGE_OP_X 8  /* 'X' substitution */

/* Create a context on CUDA device `cuda_device`, issuing work on
 * `cuda_stream` (a cudaStream_t; NULL = the legacy default stream).
 * *out receives the context; free it with scrooge_destroy. */
int scrooge_create(scrooge_ctx **out, int cuda_device, void *cuda_stream);

/* Free a context and all device memory it owns (NULL is accepted). */
int scrooge_destroy(scrooge_ctx *ctx);

/* Description of the last failure on this context ("" if none). The string
 * is owned by the context and valid until the next call on it. */
const char *scrooge_last_error(const scrooge_ctx *ctx);

/* Replace the stream used by later calls. */
int scrooge_set_stream(scrooge_ctx *ctx, void *cuda_stream);

/* ---------------------------------------------------------- input packing
 * Sequences are read in a 2-bit packed form (Section 2.5: the GPU version
 * transfers two bits per base): every 32 bases form one block of two 32-bit
 * words, the low-bit plane then the high-bit plane of the codes A=0, C=1,
 * G=2, T=3; base t of a block sits at bit 31-t of both words. A packed
 * sequence starts at a base offset that is a multiple of 64 (16 bytes) and
 * its unused tail bits are 0. */

/* 32-bit words that scrooge_pack_2bit uses for a sequence of n bases
 * (rounded up to a 64-base boundary). */
int64_t scrooge_packed_words(int64_t n_bases);

/* Host-side packer. seqs[offsets[s] .. offsets[s+1]) is sequence s, as codes
 * 0..3 (ascii = 0) or letters ACGT/acgt (ascii = 1; anything else is
 * SCROOGE_E_INVAL). Writes the packed words of all n_seqs sequences
 * back to back into `packed` (capacity `packed_words`), their base offsets
 * into packed_offsets[n_seqs] and their lengths into lengths[n_seqs].
 * All pointers are host pointers owned by the caller. */
int scrooge_pack_2bit(const uint8_t *seqs, const int64_t *offsets, int32_t n_seqs, int ascii,
                      uint32_t *packed, int64_t packed_words, int64_t *packed_offsets, int32_t *lengths);

/* ------------------------------------------------------------- alignment
 * Align pair p = (text p, pattern p) for p in [0, n_pairs).
 *
 *   texts, patterns      packed sequences (see above)
 *   *_offsets[n_pairs]   base offset of each sequence (multiple of 64)
 *   *_lengths[n_pairs]   its length in bases (>= 0)
 *   W                    window size, 1..128 (Section 2.2.3)
 *   O                    window overlap, 0..W-1
 *   k                    largest edit count tried per window, 0..W; a window
 *                        with no d <= k fails the pair (k = W never fails)
 *   flags                SCROOGE_* flags above
 * Outputs (caller-owned):
 *   edit_counts[n_pairs]     X + I + D operations of the pair's CIGAR, or -1
 *                            if some window failed (the pair then has no runs)
 *   text_consumed[n_pairs]   text bases covered by the CIGAR (the text end is free)
 *   cigar[cigar_capacity]    run-length CIGAR runs (SCROOGE_OP_*) of all pairs,
 *                            back to back in pair order
 *   cigar_offsets[n_pairs+1] runs of pair p are cigar[cigar_offsets[p] ..
 *                            cigar_offsets[p+1]); cigar_offsets[n_pairs] is the
 *                            total. A pair whose runs do not fit entirely below
 *                            cigar_capacity is not written; a synchronous call
 *                            then returns SCROOGE_E_CAPACITY (all other outputs
 *                            are valid and cigar_offsets[n_pairs] tells the
 *                            capacity needed). An asynchronous call reports it
 *                            only through cigar_offsets[n_pairs].
 * Device scratch: the library keeps per-pair run buffers of m + n + 1 runs.
 * With SCROOGE_DEVICE_PTRS the call reads the pairs' total length back to
 * size that scratch (one small synchronous copy before the alignment kernel);
 * the rest is queued on the stream.
 * Returns SCROOGE_E_INVAL before any work on bad arguments. */
int scrooge_align_batch(scrooge_ctx *ctx, const uint32_t *texts, const int64_t *text_offsets,
                        const int32_t *text_lengths, const uint32_t *patterns, const int64_t *pattern_offsets,
                        const int32_t *pattern_lengths, int32_t n_pairs, int32_t W, int32_t O, int32_t k,
                        uint32_t flags, int32_t *edit_counts, int32_t *text_consumed, uint32_t *cigar,
                        int64_t cigar_capacity, int64_t *cigar_offsets);

/* ------------------------------------------------------- kernel settings
 * Implementation parameters of the alignment kernels. They never change
 * results. words = 1, 2 or 4 selects the full-width kernel for windows of up
 * to 32 * words bases. The banded kernels serve windows of 33..128 bases when
 * SENE and ET are on (and SCROOGE_NO_BAND is not given):
 *   - words = 0 selects the one for 33..64-base windows (lanes_per_pair 1, 2,
 *     4 or 8). It keeps the 32 diagonals j - i = -15..16 of each DP entry in one
 *     word, which is exact for every window whose edit distance is at most 15.
 *     lanes_per_pair = 1 selects a kernel with one lane per pair: each lane
 *     computes its own window's 64 columns, and the warp's 32 pairs trace
 *     back on all 32 lanes; smem_rows is then the number of a pair's latest
 *     rows kept in shared memory, older rows being copied to device scratch.
 *   - words = 3 selects the one for 65..128-base windows (lanes_per_pair 8 or
 *     16). It keeps the 64 diagonals -31..32 in two words, exact up to 31.
 * Both recompute the other windows at full width.
 *   lanes_per_pair   threads that share one pair's window (words=1: 1,2,4;
 *                    words=2: 2,4,8; words=4: 8,16; words=0: 1,2,4,8;
 *                    words=3: 8,16)
 *   smem_rows        DP rows of each pair kept in shared memory (>= 1); rows
 *                    beyond go to a device scratch area
 *   warps_per_block  1 or 2 (the kernel is compiled for blocks of at most 64 threads)
 * Defaults: words 1 = (2, 8, 2), 2 = (4, 4, 2), 4 = (8, 8, 2), 0 = (1, 4, 1),
 * 3 = (8, 6, 2). scrooge_get_kernel_config reports the current values. */
int scrooge_set_kernel_config(scrooge_ctx *ctx, int32_t words, int32_t lanes_per_pair, int32_t smem_rows,
                              int32_t warps_per_block);
int scrooge_get_kernel_config(const scrooge_ctx *ctx, int32_t words, int32_t *lanes_per_pair,
                              int32_t *smem_rows, int32_t *warps_per_block);

/* Kernel per load bucket (no counterpart in the paper; never changes
 * results). With SCROOGE_LEARNED on windows the banded kernel serves, the
 * pairs whose predicted load class (see "learned pair ordering") is at least
 * load_class come first in the order and run on the full-width kernel; the
 * rest run on the banded one, and the two launches overlap on two streams. 16 (the
 * default) sends every pair to the banded kernel, 0 every pair to the
 * full-width one. scrooge_autotune with SCROOGE_LEARNED also picks this
 * class. */
int scrooge_set_heavy_class(scrooge_ctx *ctx, int32_t load_class);
int32_t scrooge_get_heavy_class(const scrooge_ctx *ctx);

/* Kernel settings per load bucket of learned launches (no counterpart in the
 * paper; never changes results). With SCROOGE_LEARNED on windows of 33..64
 * bases, bucket 0 is the heavy pairs (load class >= scrooge_set_heavy_class,
 * when that splits any off) and bucket 1 the rest of the order; each runs on
 * kind 0 = the banded kernel (lanes_per_pair 1, 2, 4 or 8; 1 = one lane per
 * pair) or kind 1 = the full-width kernel (lanes_per_pair 2, 4 or 8), with its
 * own smem_rows and warps_per_block (1 or 2). Defaults: heavy = full width,
 * 4 lanes, 4 rows, 2 warps; rest = banded, 1 lane, 4 rows, 1 warp.
 * scrooge_autotune with SCROOGE_LEARNED sets them. */
int scrooge_set_bucket_config(scrooge_ctx *ctx, int32_t bucket, int32_t kind, int32_t lanes_per_pair,
                              int32_t smem_rows, int32_t warps_per_block);
int scrooge_get_bucket_config(const scrooge_ctx *ctx, int32_t bucket, int32_t *kind, int32_t *lanes_per_pair,
                              int32_t *smem_rows, int32_t *warps_per_block);

/* Whether SCROOGE_LEARNED launches take pairs in the model's order (1, the
 * default) or in input order (0: the call then runs as SCROOGE_PERSISTENT,
 * without the ordering pipeline; the model must still be installed).
 * scrooge_autotune with SCROOGE_LEARNED sets it from measurement. Results
 * never change. */
int scrooge_set_learned_order(scrooge_ctx *ctx, int32_t on);
int32_t scrooge_get_learned_order(const scrooge_ctx *ctx);

/* Host-pointer calls in parts (no counterpart in the paper; never changes
 * results). A scrooge_align_batch call with host pointers, a persistent
 * launch in input order (SCROOGE_PERSISTENT, or SCROOGE_LEARNED with the
 * model's order switched off, no order set by scrooge_set_order for this
 * batch, not SCROOGE_WARP_SPECIALIZED) and at least 8,192 pairs is run as 2
 * to 4 parts of its pair range when this is on (1, the default); a part
 * holds at least as many pairs as the kernel has pair slots on the GPU where
 * the batch allows. Each part's sequences are copied to the device while the
 * parts before it run, and its outputs are gathered and copied back while
 * the parts after it run. Each part has its own launch; consecutive parts
 * alternate between two kernel streams with their own row scratch, and a
 * part's blocks take the SMs that the previous part's blocks free. The
 * sequence words a part needs are the prefix of the texts and patterns
 * arrays that its pairs and the earlier ones reach, so the overlap needs
 * pairs laid out in pair order. Such calls are not captured in a CUDA graph
 * (SCROOGE_GRAPH is ignored for them). 0 runs them as one launch. */
int scrooge_set_host_overlap(scrooge_ctx *ctx, int32_t on);
int32_t scrooge_get_host_overlap(const scrooge_ctx *ctx);

/* Long pairs (no counterpart in the paper; never changes results). The
 * windows of a pair are sequential, so a batch can take no less time than
 * its longest pair. With SCROOGE_LEARNED on windows the banded kernel
 * serves, the pairs whose predicted work class (see "learned pair ordering")
 * is at least work_class come first in the order. A first launch on a
 * high-priority stream gives each of them a warp of its own (one pair per
 * warp, three one-warp blocks per SM), so each of their windows costs only
 * its own rows and traceback steps, not the worst of a warp's pairs.
 * 16 (the default) turns this off; 13 selects pattern length x rows per
 * window of at least 2^19. */
int scrooge_set_long_class(scrooge_ctx *ctx, int32_t work_class);
int32_t scrooge_get_long_class(const scrooge_ctx *ctx);

/* Launch shape of the last scrooge_align_batch call on this context, for
 * reports: up to 13 int64 into shape[0..n): kernel (0 banded, else the words
 * of the full-width kernel), lanes per pair, DP rows kept in shared memory,
 * warps per block, dynamic shared memory per block (bytes), blocks, stored
 * columns per row, stored words per entry, shared-memory table bytes per
 * warp, device-scratch row bytes per warp, full-width fallback bytes per
 * warp, pairs per warp, row slots of a window's full-width rows (see
 * SCROOGE_NO_EXT_DENT; k+1 without it). */
int scrooge_last_launch_shape(const scrooge_ctx *ctx, int64_t *shape, int32_t n);

/* Autotuner (no counterpart in the paper: it picks implementation
 * parameters only, so results never change). Times every supported
 * (lanes_per_pair, smem_rows, warps_per_block) for the window width of W on
 * the given batch -- arguments as for scrooge_align_batch with
 * SCROOGE_DEVICE_PTRS, outputs overwritten -- keeping the fastest of
 * `repeats` timed runs per configuration (CUDA events on the context stream,
 * after one untimed run), and installs the fastest configuration in the
 * context. If `results` is not NULL it receives up to max_results rows of 5
 * int32: lanes, rows, warps, microseconds, 1. With SCROOGE_LEARNED on windows
 * the banded kernel serves, that sweep times persistent launches in input
 * order (learned launches take the per-bucket settings below), and it then:
 *   - times the heavy load classes (scrooge_set_heavy_class) 16, 15, ..., 10,
 *     0 before and again after the settings sweep (at least 3 timed runs
 *     each), as rows 0, class, 0, microseconds, 2, and installs the fastest
 *     class of the second pass if it beats class 16 (no split) by at least
 *     10%, else 16;
 *   - sweeps the kernel settings of each load bucket of learned launches
 *     (scrooge_set_bucket_config; the rest, then the heavy bucket if there is
 *     one), kind x lanes x rows {2, 4, 8} x warps {1, 2}, as rows
 *     bucket*1000 + kind*100 + lanes, rows, warps, microseconds, 3, keeping
 *     the fastest per bucket;
 *   - times the long pairs' own launch (scrooge_set_long_class) 16 (off), 14,
 *     13, 12, as rows 0, class, 1, microseconds, 5, and keeps the fastest if
 *     it beats 16 by at least 5%;
 *   - times the learned launch with the model's order and in input order, as
 *     rows 1, 0, 0, microseconds, 4 and 0, 0, 0, microseconds, 4, and keeps
 *     the model's order (scrooge_set_learned_order) only if it is at least 2%
 *     faster.
 * *n_results gets the row count.
 * Synchronous. */
int scrooge_autotune(scrooge_ctx *ctx, const uint32_t *texts, const int64_t *text_offsets,
                     const int32_t *text_lengths, const uint32_t *patterns, const int64_t *pattern_offsets,
                     const int32_t *pattern_lengths, int32_t n_pairs, int32_t W, int32_t O, int32_t k,
                     uint32_t flags, int32_t *edit_counts, int32_t *text_consumed, uint32_t *cigar,
                     int64_t cigar_capacity, int64_t *cigar_offsets, int32_t repeats, int32_t *results,
                     int32_t max_results, int32_t *n_results);

/* Pair order of later SCROOGE_PERSISTENT calls: order[s] is the pair taken
 * s-th from the device work queue (a DEVICE array holding a permutation of
 * 0..n_pairs-1, owned by the caller and read during each call). It applies to
 * calls with exactly n_pairs pairs; NULL restores the input order. Results do
 * not depend on the order. */
int scrooge_set_order(scrooge_ctx *ctx, const int32_t *order, int32_t n_pairs);

/* ------------------------------------------------- learned pair ordering
 * No counterpart in the paper: a small MLP predicts each pair's per-window
 * load from cheap features, and SCROOGE_LEARNED launches hand pairs to the
 * persistent kernel in the order of an 8-bit bucket key, stable within a
 * bucket. From the most significant bit down the key holds:
 *   - the long pairs first (work class >= scrooge_set_long_class);
 *   - then the heavy pairs (load class >= scrooge_set_heavy_class);
 *   - then the pattern length, longest first, in eighths of an octave below
 *     the batch's longest pattern (6 bits): the windows of a pair are
 *     sequential, so the longest pairs must start first, and pairs of
 *     similar length share warps and finish together. On uneven batches this
 *     measured faster than orders that mix in the predicted load, even the
 *     true load.
 * Here rows is the predicted mean DP rows per window, the load class is
 * floor(4 log2(rows + 1)) and the work class is
 * floor(log2((m + 1)(rows + 1))) - 6, both clipped to 0..15; they choose the
 * launches and kernels of the buckets (scrooge_set_bucket_config). The
 * order never changes results.
 *
 * Features (float32, 6 per pair, row-major): log2(m+1), log2(n+1),
 * (n-m)/max(m,1), the fraction of sampled pattern 12-mers found in the text
 * within +-64 positions of the same offset, the spread of the offsets of
 * those hits (standard deviation / 64), and the fraction of hits within +-16
 * of their mean offset. Model: 6 -> 64 -> 64 -> 1 with ReLU, inputs
 * standardised by stored feature means and deviations; the output estimates
 * log(1 + mean DP rows per window). Parameters (scrooge_model_floats()
 * floats): W1[64][6], b1[64], W2[64][64], b2[64], w3[64], b3, mean[6], sd[6]. */
int32_t scrooge_model_floats(void);
/* Install / read the model (host arrays of scrooge_model_floats() floats). */
int scrooge_model_set(scrooge_ctx *ctx, const float *params, int32_t n);
int scrooge_model_get(scrooge_ctx *ctx, float *params, int32_t n);
/* Features of n_pairs packed pairs (device pointers, as for
 * scrooge_align_batch) into the DEVICE array features[n_pairs * 6];
 * asynchronous on the context stream. */
int scrooge_features(scrooge_ctx *ctx, const uint32_t *texts, const int64_t *text_offsets,
                     const int32_t *text_lengths, const uint32_t *patterns, const int64_t *pattern_offsets,
                     const int32_t *pattern_lengths, int32_t n_pairs, float *features);
/* Model output for n feature rows (device arrays); asynchronous. */
int scrooge_model_predict(scrooge_ctx *ctx, const float *features, int32_t n, float *pred);
/* Gradient of the mean squared error of the installed model over n rows
 * (device features and targets) into the DEVICE array grad (model layout;
 * the mean/sd entries stay 0); *loss (host, may be NULL) gets the mean
 * squared error. Synchronous. */
int scrooge_model_grad(scrooge_ctx *ctx, const float *features, const float *targets, int32_t n, float *grad,
                       float *loss);
/* Train a new model on n rows (device features and targets): feature
 * scaling from the data, seeded initialisation, `epochs` passes of Adam over
 * shuffled mini-batches of `batch` rows with learning rate lr. The model is
 * installed in the context; loss_history (host, may be NULL) receives the
 * mean squared error of each epoch. Synchronous. */
int scrooge_model_train(scrooge_ctx *ctx, const float *features, const float *targets, int32_t n, int32_t epochs,
                        int32_t batch, float lr, uint64_t seed, float *loss_history);
/* The order SCROOGE_LEARNED would use for these pairs, into the DEVICE array
 * order[n_pairs]; asynchronous. */
int scrooge_learned_order(scrooge_ctx *ctx, const uint32_t *texts, const int64_t *text_offsets,
                          const int32_t *text_lengths, const uint32_t *patterns, const int64_t *pattern_offsets,
                          const int32_t *pattern_lengths, int32_t n_pairs, int32_t *order);

/* Events (cudaEvent_t, caller-owned, may both be NULL) that later
 * scrooge_align_batch calls record on the context stream right before and
 * after the alignment kernel, so callers can time that kernel alone. Not
 * recorded in SCROOGE_GRAPH mode. */
int scrooge_set_timing_events(scrooge_ctx *ctx, void *start, void *stop);

/* Kernels launched (or replayed in a graph) by the last scrooge_align_batch
 * call on this context. */
int32_t scrooge_last_kernel_count(const scrooge_ctx *ctx);

/* Per-pair statistics of the next scrooge_align_batch calls, written to
 * caller-owned DEVICE arrays of n_pairs entries (any may be NULL; all NULL
 * switches statistics off): windows aligned, DP rows computed up to each
 * window's edit distance (sum of d_opt + 1), DP cells in those rows (sum of
 * (d_opt + 1) * text window length), and SM clock cycles the pair took. */
int scrooge_set_stats(scrooge_ctx *ctx, int32_t *windows, int64_t *rows, int64_t *cells, int64_t *cycles);

/* ------------------------------------------------ allocation-free variant
 * No counterpart in the paper. For callers that cannot allocate device
 * memory -- code running while a stream is being captured into a CUDA graph,
 * or a host application whose device memory is handed out by its own
 * allocator -- this entry point aligns without calling cudaMalloc, cudaFree
 * or any allocating routine, and needs no context.
 *
 * It runs the same alignment kernel. All pointers are device pointers; the
 * work is queued on `cuda_stream` (a cudaStream_t, NULL = default stream) on
 * the current device and the call returns at once unless flags holds
 * SCROOGE_SYNC. Allowed flags: SCROOGE_SYNC, SCROOGE_NO_DENT, SCROOGE_NO_ET,
 * SCROOGE_NO_EXT_DENT (every row of a window kept instead of the cycle of row
 * slots; results are the same) (SCROOGE_DEVICE_PTRS is implied and ignored).
 *
 * Scratch: DP rows that do not fit in shared memory go to a fixed 16 MiB
 * array (plus one status word) compiled into the library; every GPU that
 * loads the library holds it until the process exits. The static size caps
 * how many pairs are resident at once, never how many pairs a call takes;
 * a W/O/k whose rows would not fit for even one block of pairs returns
 * SCROOGE_E_INVAL (no supported setting reaches that: the largest, W = 128
 * without DENT, needs under 2 MiB per block).
 * Every call shares that array and it keeps the last call's contents, so
 * calls whose work overlaps on the GPU (different streams, or different
 * host threads) race; queue them on one stream. The first call on each
 * device looks up the array's device address and sets kernel attributes;
 * make that first call before any stream capture.
 *
 * Outputs are those of scrooge_align_batch except the CIGAR layout: pair p
 * writes at most cigar_offsets[p+1] - cigar_offsets[p] runs (cigar_offsets
 * is an input capacity layout; m + n + 1 runs per pair always suffice) to
 * cigar[cigar_offsets[p] ..], and cigar_lens[p] receives the runs written.
 * `status` (device int32, may be NULL) receives 0, or bit 0 if a traceback
 * found no open edge (should never happen), or bit 1 if some pair's capacity
 * was too small (its runs are cut at the capacity). */
int scrooge_align_batch_noalloc(const uint32_t *texts, const int64_t *text_offsets, const int32_t *text_lengths,
                                const uint32_t *patterns, const int64_t *pattern_offsets,
                                const int32_t *pattern_lengths, int32_t n_pairs, int32_t W, int32_t O, int32_t k,
                                uint32_t flags, int32_t *edit_counts, int32_t *text_consumed, uint32_t *cigar,
                                const int64_t *cigar_offsets, int32_t *cigar_lens, int32_t *status,
                                void *cuda_stream);

/* ------------------------------------------------- exact edit distances
 * No counterpart in the paper's hot path. It is the optimal score that the
 * windowed heuristic is measured against, as in the paper's accuracy study
 * (Section 5). For every pair it computes
 *   free_end[p]        = min over t of lev(pattern, text[0:t]): the whole
 *                        pattern against a text prefix, the problem that
 *                        scrooge_align_batch solves window by window, so
 *                        free_end[p] <= edit_counts[p] always;
 *   global_distance[p] = lev(pattern, text).
 * Unit costs; Myers' bit-vector algorithm, one warp per pair. Inputs are in
 * the packed layout of scrooge_align_batch and must be DEVICE pointers
 * (flags must contain SCROOGE_DEVICE_PTRS; SCROOGE_SYNC is honoured), as
 * must the two int32 outputs of n_pairs entries.
 * max_pattern_length bounds the pattern lengths (at most
 * SCROOGE_EDIT_DISTANCE_MAX_M); a pair above it gets -1 in both outputs.
 * Asynchronous on the context stream. */
#define SCROOGE_EDIT_DISTANCE_MAX_M 16384
int scrooge_edit_distance(scrooge_ctx *ctx, const uint32_t *texts, const int64_t *text_offsets,
                          const int32_t *text_lengths, const uint32_t *patterns, const int64_t *pattern_offsets,
                          const int32_t *pattern_lengths, int32_t n_pairs, int32_t max_pattern_length,
                          uint32_t flags, int32_t *free_end, int32_t *global_distance);

/* Bounded device waits (no counterpart in the paper). The warp-specialised
 * blocks (SCROOGE_WARP_SPECIALIZED) hand windows between warps through
 * shared-memory barriers, and every wait on one is bounded: when it gives up,
 * the warp leaves and a synchronous call returns SCROOGE_E_TIMEOUT. `polls`
 * = 0 (the default) allows 2^24 polls with mbarrier.try_wait, which may
 * suspend the waiting thread between polls; polls > 0 allows that many
 * polls with the non-suspending mbarrier.test_wait, so a wait that nothing
 * completes ends after a short, bounded time (a small value makes the waits
 * give up, which is how the time-out path is tested). Applies to later calls
 * on this context. */
int scrooge_set_wait_limit(scrooge_ctx *ctx, int32_t polls);

/* ------------------------------------------------ logic-pipe peak probe
 * No counterpart in the paper. It measures the peak the alignment kernels'
 * roofline is taken against: the integer logic pipe of the context's device
 * (3-input logic ops and funnel shifts). One full wave of blocks runs
 * 8 independent chains per thread, one logic op and one funnel shift per
 * chain step, `iterations` x 16 steps per chain (1..2^20); a first launch
 * with one iteration warms up. Outputs (host, either may be NULL):
 *   *ops_per_s           logic ops of the timed launch / its duration
 *                        (CUDA events on the context stream);
 *   *ops_per_clk_per_sm  median over SMs of the ops an SM's blocks executed
 *                        divided by the SM clock cycles between the first
 *                        block's start and the last block's end on that SM
 *                        (independent of the clock frequency).
 * Allocates and frees a few bytes of device memory. Synchronous. */
int scrooge_logic_peak(scrooge_ctx *ctx, int32_t iterations, double *ops_per_s, double *ops_per_clk_per_sm);

/* Testing hook: make the next `count` device allocations of this context
 * fail with SCROOGE_E_NOMEM (0 switches it off). */
int scrooge_debug_fail_next_allocs(scrooge_ctx *ctx, int32_t count);

#ifdef __cplusplus
}
#endif

#endif /* SCROOGE_H */
