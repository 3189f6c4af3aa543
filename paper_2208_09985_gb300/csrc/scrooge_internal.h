// Internal declarations shared by the host side of the library and its kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace scrooge {

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
    int32_t ncol;   // DP columns stored per row (DENT: W-O+1, else W)
    int32_t sw;     // 32-bit words stored per entry (DENT: ceil((W-O+1)/32), else all)
    int32_t rcap;   // rows per pair held in shared memory
    int32_t et;     // 1: stop at the first row that reaches the window start
    int32_t sene;   // 1: store entries; 0: store GenASM's I, D, M edge vectors
    int32_t *edit_counts;
    int32_t *text_consumed;
    uint32_t *cigar;            // per-pair run scratch
    const int64_t *cigar_off;   // [n_pairs + 1] scratch offsets (capacity m + n + 1 each)
    int32_t *cigar_lens;        // [n_pairs] runs written
    uint32_t *spill;                // rows >= rcap, one region per resident pair slot
    int64_t spill_words_per_pair;
    int32_t smem_words_per_warp;
    int32_t table_words_per_warp;
    const int32_t *order;   // optional pair order (slot -> pair id)
    int32_t *queue;         // persistent mode: next slot to hand out (nullptr: static)
    int32_t *status;        // bit 0: traceback found no edge (impossible by Theorem 1)
    int32_t *st_windows;
    int64_t *st_rows;
    int64_t *st_cells;
    int64_t *st_cycles;
};

// Words of a stored table row block: rows x columns x words x pairs-per-warp.
inline int64_t table_words_per_warp(int rcap, int ncol, int sw, int sene, int ppw) {
    return (int64_t)rcap * ncol * sw * (sene ? 1 : 3) * ppw;
}

inline int stage_words_per_warp(int nw, int ppw) { return ppw * 4 * (nw + 1); }

// Launches the alignment kernel for `words` 32-bit words per bitvector and
// `lanes` threads per pair. Returns cudaErrorInvalidValue for an unsupported
// combination.
cudaError_t launch_align(const AlignParams &p, int words, int lanes, int warps_per_block, int blocks,
                         size_t smem_bytes, cudaStream_t stream);

// Resident blocks per SM for that kernel with `smem_bytes` dynamic shared memory.
cudaError_t align_occupancy(int words, int lanes, int warps_per_block, size_t smem_bytes, int *blocks_per_sm);

bool align_supported(int words, int lanes);

// Dense CIGAR output (cigar_compact.cu).
int64_t scan_temp_words(int64_t n);
// out[0..n]: exclusive prefix sums of in[0..n) (int32 if wide == 0, else int64) and the total.
cudaError_t exclusive_scan(const void *in, int wide, int64_t n, int64_t *out, int64_t *tmp, cudaStream_t s);
// cap[p] = text_len[p] + pat_len[p] + 1
cudaError_t launch_capacity(const int32_t *text_len, const int32_t *pat_len, int32_t n, int64_t *cap, cudaStream_t s);
// copies each pair's runs to dense[dense_off[p] ..] when they fit below capacity
cudaError_t launch_compact(const uint32_t *scratch, const int64_t *scratch_off, const int32_t *lens,
                           const int64_t *dense_off, int32_t n, uint32_t *dense, int64_t capacity, int sm_count,
                           cudaStream_t s);

}  // namespace scrooge
