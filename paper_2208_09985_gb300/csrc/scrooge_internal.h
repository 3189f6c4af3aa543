// Internal declarations shared by the host side of the library and its kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace scrooge {

// Learned ordering model: kFeatures -> kHidden -> kHidden -> 1, ReLU.
constexpr int kFeatures = 6;
constexpr int kHidden = 64;
// W1, b1, W2, b2, w3, b3, then the feature means and standard deviations
constexpr int kModelFloats = kHidden * kFeatures + kHidden + kHidden * kHidden + kHidden + kHidden + 1 + 2 * kFeatures;

// Everything one alignment launch needs. All pointers are device pointers.
struct AlignParams {
    const uint32_t *texts;     // packed bit-plane blocks
    const int64_t *text_off;   // [n_pairs] base offset, multiple of 64
    const int32_t *text_len;   // [n_pairs]
    const uint32_t *patterns;
    const int64_t *pat_off;
    const int32_t *pat_len;
    int32_t n_pairs;
    int32_t W, O, k;
    int32_t ncol;   // DP columns stored per row (DENT: W-O+1 rounded up to whole lane chunks, else all)
    int32_t rstride;  // cells between two stored rows (ncol x pairs per warp, padded against bank conflicts)
    int32_t sw;     // 32-bit words stored per vector (a power of two, the SWP template parameter)
    int32_t rcap;   // rows per pair held in shared memory
    int32_t ring;   // full-width row slots per window: row d is stored in slot d mod ring (k + 1: every row)
    int32_t et;     // 1: stop at the first row that reaches the window start
    int32_t sene;   // 1: store entries; 0: store GenASM's I, D, M edge vectors
    int32_t *edit_counts;
    int32_t *text_consumed;
    uint32_t *cigar;            // per-pair run scratch
    const int64_t *cigar_off;   // [n_pairs + 1] scratch offsets (capacity m + n + 1 each)
    int32_t *cigar_lens;        // [n_pairs] runs written
    uint32_t *spill;                // rows >= rcap, one region per resident warp
    int64_t spill_words_per_pair;   // words of that region per warp
    uint32_t *fb;                   // banded kernel: full-width rows and state of windows beyond the band
    int64_t fb_words_per_warp;      // words of that region per warp
    int32_t fb_ncol;                // one-lane-per-pair kernel: stored columns of a full-width fallback row
    int32_t smem_words_per_warp;
    int32_t table_words_per_warp;
    const int32_t *order;   // optional pair order (slot -> pair id)
    int32_t *queue;         // persistent mode: next slot to hand out (nullptr: static)
    const int64_t *range_lo;  // persistent mode: only slots [*range_lo, *range_hi) of the order
    const int64_t *range_hi;  // (nullptr: 0 and n_pairs)
    int32_t slots_per_warp;   // pair slots of a warp that take pairs (0: all 32/G)
    int32_t wait_limit;       // warp-specialised kernel: polls per barrier wait (0: the default bound)
    int32_t *status;        // bit 0: traceback found no edge (impossible by Theorem 1)
    int32_t *st_windows;
    int64_t *st_rows;
    int64_t *st_cells;
    int64_t *st_cycles;
};

// Geometry of the stored DP table for one launch.
struct TableShape {
    int ncol;  // stored columns (multiple of the lane chunk)
    int swp;   // stored 32-bit words per vector: 1, 2 or 4
    int nv;    // stored vectors per cell: 1 (entries) or 3 (GenASM edges)
};

inline TableShape table_shape(int W, int O, int words, int lanes, bool dent, bool sene) {
    const int wmax = 32 * words, chunk = wmax / lanes, L = W - O;
    TableShape t;
    const int ncol = dent ? (L + 1 < W ? L + 1 : W) : W;
    t.ncol = ((ncol + chunk - 1) / chunk) * chunk;
    if (t.ncol > wmax) t.ncol = wmax;
    int sw = dent ? (L + 1 + 31) / 32 : words;
    if (sw > words) sw = words;
    t.swp = sw <= 1 ? 1 : (sw <= 2 ? 2 : 4);
    t.nv = sene ? 1 : 3;
    return t;
}

// Cells between two rows of one warp's table: ncol x pairs-per-warp, padded so
// that the lanes of a pair, which store row d - l at column chunk G-1-l in the
// same step, fall on different shared-memory banks.
inline int row_stride_cells(const TableShape &t, int ppw, int chunk) {
    const int cell = t.nv * t.swp;
    const int group = ppw * cell;  // words one lane slot of all pairs writes per column
    int rs = t.ncol * ppw;
    if (group < 32) {
        for (int pad = 0; pad < 32; ++pad) {
            const int off = ((rs + pad + chunk * ppw) * cell) % 32;
            if (off == group % 32) {
                rs += pad;
                break;
            }
        }
    }
    return rs;
}

// Words of one warp's stored rows.
inline int64_t table_words_per_warp(int rows, const TableShape &t, int ppw, int chunk) {
    const int64_t w = (int64_t)rows * row_stride_cells(t, ppw, chunk) * t.nv * t.swp;
    return (w + 3) & ~(int64_t)3;  // keep 16-byte alignment
}

inline int stage_words_per_warp(int nw, int ppw) { return ((ppw * 4 * (nw + 1)) + 3) & ~3; }

// Per-width launchers of the alignment kernel (align_w32.cu, align_w64.cu,
// align_w128.cu). `swp` is TableShape::swp. launch_* returns
// cudaErrorInvalidValue for a combination that is not instantiated.
cudaError_t launch_align_w32(const AlignParams &, int lanes, bool sene, int swp, int wpb, int blocks, size_t smem,
                             cudaStream_t);
cudaError_t launch_align_w64(const AlignParams &, int lanes, bool sene, int swp, int wpb, int blocks, size_t smem,
                             cudaStream_t);
cudaError_t launch_align_w128(const AlignParams &, int lanes, bool sene, int swp, int wpb, int blocks, size_t smem,
                              cudaStream_t);
cudaError_t occupancy_w32(int lanes, bool sene, int swp, int wpb, size_t smem, int *blocks_per_sm);
cudaError_t occupancy_w64(int lanes, bool sene, int swp, int wpb, size_t smem, int *blocks_per_sm);
cudaError_t occupancy_w128(int lanes, bool sene, int swp, int wpb, size_t smem, int *blocks_per_sm);
// Banded kernels (align_band.cu): windows of up to 32 * nww bases, a band of 32 * bw diagonals
// per entry. (nww, bw) = (2, 1) for windows of 33..64 bases (lanes 2, 4 or 8), (2, 2) for the
// same windows with the wide band (lanes 4 or 8), (4, 2) for 65..128 bases (lanes 8 or 16).
// Rows d < 16 * bw are exact inside the band; other windows are recomputed at full width (nww
// words).
inline int band_rows_for(int bw) { return 16 * bw; }
cudaError_t launch_align_band(const AlignParams &, int nww, int bw, int lanes, int wpb, int blocks, size_t smem,
                              cudaStream_t);
cudaError_t occupancy_band(int nww, int bw, int lanes, int wpb, size_t smem, int *blocks_per_sm);
bool supported_band(int nww, int bw, int lanes);
// words of the full-width fallback region of one warp of a banded kernel
inline int64_t band_fallback_words(int k, int ncol, int ppw, int nww, int bw) {
    return k >= band_rows_for(bw) ? (int64_t)(k + 1) * ncol * ppw * nww : 0;
}
// Row slots of a window's full-width row store. DENT extended to rows (Supplementary Section 1):
// the part of a window's traceback that is kept spends at most W-O edits (it is part of an optimal
// alignment, so its cost up to (i, j) is lev(text[:i], pattern[:j]) <= max(i, j) <= W-O), so with
// early termination it reads rows d_opt-(W-O) .. d_opt only. The DC pipeline over the G lanes of a
// pair stores up to G-1 rows past d_opt before the stop reaches its first lane, so W-O+G slots,
// row d in slot d mod (W-O+G), never overwrite a row the traceback reads. The cycle has at least
// ceil((k+1)/2) slots, so a row wraps at most once and its slot is one compare and subtract
// (ring_slot); that keeps the full W-O+G at every operating point with W-O+G >= (k+1)/2, which
// includes the paper's. Without it: k+1 rows.
inline int ext_dent_ring(int W, int O, int k, int lanes, bool on) {
    int ring = W - O + lanes;
    if (ring < (k + 2) / 2) ring = (k + 2) / 2;
    return on && ring < k + 1 ? ring : k + 1;
}
// Banded kernel with one lane per pair (align_lane.cu) for windows of 33..64 bases: ncol (at most
// 64; see SCROOGE_LANE_NCOLS) stored columns per row, rcap rows per lane in shared memory after a
// per-warp table of kLaneTableBytes; windows beyond the band are recomputed at full width by
// groups of 4 lanes (fb: k+1 rows of fb_ncol columns x 8 windows x 2 words per warp).
constexpr int kLaneTableBytes = 3072;
// Stored-column counts the lane kernel is compiled for: the multiples of 8, and W-O+1 at the
// operating points W=64/O=24 (41) and W=64/O=32 (33), which would otherwise round up to 48 and 40.
#define SCROOGE_LANE_NCOLS \
    SCROOGE_LANE_NCOL(8)       \
    SCROOGE_LANE_NCOL(16)      \
    SCROOGE_LANE_NCOL(24)      \
    SCROOGE_LANE_NCOL(32)      \
    SCROOGE_LANE_NCOL(33)      \
    SCROOGE_LANE_NCOL(40)      \
    SCROOGE_LANE_NCOL(41)      \
    SCROOGE_LANE_NCOL(48)      \
    SCROOGE_LANE_NCOL(56)      \
    SCROOGE_LANE_NCOL(64)
cudaError_t launch_align_lane(const AlignParams &, int wpb, int blocks, size_t smem, cudaStream_t);
cudaError_t occupancy_lane(int ncol, int wpb, size_t smem, int *blocks_per_sm);
bool lane_ncol_supported(int ncol);
// Warp-specialised banded kernel (align_band.cu): blocks of 4 DC warps (4 lanes per pair, two
// sets of 8 pairs each) and one traceback warp; persistent launches only. Shared memory per block:
// 8 sets x smem_words_per_warp words, then ws_meta_bytes().
constexpr int kWsSets = 8;
cudaError_t launch_align_ws(const AlignParams &, int blocks, size_t smem, cudaStream_t);
cudaError_t occupancy_ws(size_t smem, int *blocks_per_sm);
size_t ws_meta_bytes();
bool supported_w32(int lanes, bool sene, int swp);
bool supported_w64(int lanes, bool sene, int swp);
bool supported_w128(int lanes, bool sene, int swp);

bool align_supported(int words, int lanes);

// Occupancy of `kernel` at `threads` threads and `smem` bytes of dynamic shared memory, first
// raising the kernel's dynamic shared-memory limit to `smem` if it is lower. The limit is never
// lowered: launches of one kernel with different settings (the buckets of a learned call, the
// allocation-free entry point) may be planned in any order and run concurrently.
template <typename K>
inline cudaError_t occupancy_raising_smem(K *kernel, int threads, size_t smem, int *blocks_per_sm) {
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, kernel);
    if (e != cudaSuccess) return e;
    if ((size_t)a.maxDynamicSharedSizeBytes < smem &&
        (e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
        return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, kernel, threads, smem);
}

// Dense CIGAR output (cigar_compact.cu).
int64_t scan_temp_words(int64_t n);
int scan_kernel_count(int64_t n);
// out[0..n]: exclusive prefix sums of in[0..n) (int32 if wide == 0, else int64) and the total.
cudaError_t exclusive_scan(const void *in, int wide, int64_t n, int64_t *out, int64_t *tmp, cudaStream_t s);
// cap[p] = text_len[p] + pat_len[p] + 1
cudaError_t launch_capacity(const int32_t *text_len, const int32_t *pat_len, int32_t n, int64_t *cap, cudaStream_t s);
// v[i] += *base for i < n (base: a device pointer)
cudaError_t launch_add_base(int64_t *v, int64_t n, const int64_t *base, cudaStream_t s);
// copies each pair's runs to dense[dense_off[p] ..] when they fit below capacity
cudaError_t launch_compact(const uint32_t *scratch, const int64_t *scratch_off, const int32_t *lens,
                           const int64_t *dense_off, int32_t n, uint32_t *dense, int64_t capacity, int sm_count,
                           cudaStream_t s);

// Learned ordering (learn.cu).
cudaError_t launch_features(const uint32_t *texts, const int64_t *text_off, const int32_t *text_len,
                            const uint32_t *patterns, const int64_t *pat_off, const int32_t *pat_len, int32_t n,
                            float *feat, int sm_count, cudaStream_t s);
cudaError_t launch_mlp_forward(const float *model, const float *feat, int32_t n, float *pred, cudaStream_t s);
// gradient of the mean squared error over feat/target rows `rows[0..n)` (rows == nullptr: 0..n)
cudaError_t launch_mlp_grad(const float *model, const float *feat, const float *target, const int32_t *rows,
                            int32_t n, float *grad, float *loss_sum, int sm_count, cudaStream_t s);
cudaError_t launch_adam(float *model, const float *grad, float *m1, float *m2, float lr, int step, cudaStream_t s);
cudaError_t launch_feature_stats(const float *feat, int32_t n, float *model, cudaStream_t s);
int64_t sort_temp_words(int32_t n);
int learned_kernel_count(int32_t n);
// Device address of the first position of bucket `key` in the order that launch_learned_order
// wrote with scratch `tmp` (the number of pairs with a smaller key).
const int64_t *learned_bucket_start(const int64_t *tmp, int32_t n, int key);
cudaError_t launch_learned_order(const float *pred, const int32_t *pat_len, int32_t n, int heavy_class, int long_class,
                                 uint8_t *key, int32_t *order, int64_t *tmp, cudaStream_t s);

}  // namespace scrooge
