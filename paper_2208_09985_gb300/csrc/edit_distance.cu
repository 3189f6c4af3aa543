// Exact edit distances of whole pairs, for measuring the windowed heuristic's
// accuracy. This has no counterpart in Scrooge's hot path. The paper measures
// accuracy against optimal alignments (Section 5); this is the GPU stand-in for
// those optimal scores.
//
// For pattern P (m bases) and text T (n bases) it computes
//   free_end = min over t of lev(P, T[0:t])  (the whole pattern against a text
//              prefix: the problem the windowed method approximates), and
//   global   = lev(P, T).
// Method: Myers' bit-vector algorithm (J. ACM 1999) in Hyyro's formulation of
// the vertical and horizontal deltas, with +1 entering the top row of every
// column because the text start is fixed (D[0][j] = j). Pattern row r is bit
// r % 64 of 64-bit word r / 64 (least significant first, so the addition
// carries and the shifts run from row r to row r+1).
//
// One warp per pair. Lane l holds words [l*K, (l+1)*K); a column's carries
// (the addition carry and the top bits of the horizontal deltas) move from lane
// to lane, so the lanes form a pipeline over the text columns: in step s lane l
// works on column s - l and takes its carries from lane l-1 by warp shuffles.
#include <algorithm>

#include "scrooge_ctx.h"

namespace scrooge {
namespace {

constexpr uint32_t kAll = 0xffffffffu;

__device__ __forceinline__ uint2 block_at(const uint2 *seq, int64_t b, int64_t nblk) {
    return (b >= 0 && b < nblk) ? __ldg(seq + b) : make_uint2(0u, 0u);
}

template <int K>
__global__ void __launch_bounds__(256) edit_distance_kernel(const uint32_t *texts, const int64_t *text_off,
                                                            const int32_t *text_len, const uint32_t *patterns,
                                                            const int64_t *pat_off, const int32_t *pat_len,
                                                            int32_t n_pairs, int32_t max_m, int32_t *free_end,
                                                            int32_t *global_d) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t pair = warp; pair < n_pairs; pair += nwarps) {
        const int n = text_len[pair], m = pat_len[pair];
        if (m == 0 || m > max_m || m > 64 * 32 * K) {
            if (lane == 0) {
                free_end[pair] = m == 0 ? 0 : -1;
                global_d[pair] = m == 0 ? n : -1;
            }
            continue;
        }
        const uint2 *tseq = reinterpret_cast<const uint2 *>(texts + (text_off[pair] >> 4));
        const uint2 *pseq = reinterpret_cast<const uint2 *>(patterns + (pat_off[pair] >> 4));
        const int64_t tblk = (n + 31) >> 5, pblk = (m + 31) >> 5;
        const int last_word = (m - 1) >> 6;
        const int last_lane = last_word / K, last_w = last_word - last_lane * K, last_bit = (m - 1) & 63;
        // the pattern's two bit planes, row-ordered (bit reversal of the packed blocks)
        uint64_t p0[K], p1[K], Pv[K], Mv[K];
#pragma unroll
        for (int w = 0; w < K; ++w) {
            const int64_t word = (int64_t)lane * K + w;
            const uint2 a = block_at(pseq, 2 * word, pblk), b = block_at(pseq, 2 * word + 1, pblk);
            p0[w] = ((uint64_t)__brev(b.x) << 32) | __brev(a.x);
            p1[w] = ((uint64_t)__brev(b.y) << 32) | __brev(a.y);
            Pv[w] = ~0ull;
            Mv[w] = 0ull;
        }
        int score = m, best = m;
        uint32_t carry_o = 0u, ph_o = 0u, mh_o = 0u;
        uint2 blk = make_uint2(0u, 0u);
        const bool works = lane <= last_lane;
        for (int s = 0; s < n + last_lane; ++s) {
            uint32_t cin = __shfl_up_sync(kAll, carry_o, 1);
            uint32_t pin = __shfl_up_sync(kAll, ph_o, 1);
            uint32_t hin = __shfl_up_sync(kAll, mh_o, 1);
            if (lane == 0) {
                cin = 0u;
                pin = 1u;  // D[0][j] - D[0][j-1] = +1: the text start is fixed
                hin = 0u;
            }
            const int j = s - lane;
            if (works && j >= 0 && j < n) {
                if ((j & 31) == 0) blk = block_at(tseq, j >> 5, tblk);
                const int sh = 31 - (j & 31);
                const uint64_t c0 = 0ull - (uint64_t)((blk.x >> sh) & 1u);
                const uint64_t c1 = 0ull - (uint64_t)((blk.y >> sh) & 1u);
                uint64_t carry = cin, ph_in = pin, mh_in = hin;
#pragma unroll
                for (int w = 0; w < K; ++w) {
                    const uint64_t eq = ~((p0[w] ^ c0) | (p1[w] ^ c1));
                    const uint64_t xv = eq | Mv[w];
                    const uint64_t a = eq & Pv[w];
                    const uint64_t t = a + Pv[w];
                    const uint64_t u = t + carry;
                    carry = (uint64_t)((t < a) | (u < t));
                    const uint64_t xh = (u ^ Pv[w]) | eq;
                    uint64_t ph = Mv[w] | ~(xh | Pv[w]);
                    uint64_t mh = Pv[w] & xh;
                    if (lane == last_lane && w == last_w)
                        score += (int)((ph >> last_bit) & 1ull) - (int)((mh >> last_bit) & 1ull);
                    const uint64_t pt = ph >> 63, mt = mh >> 63;
                    ph = (ph << 1) | ph_in;
                    mh = (mh << 1) | mh_in;
                    ph_in = pt;
                    mh_in = mt;
                    Pv[w] = mh | ~(xv | ph);
                    Mv[w] = ph & xv;
                }
                carry_o = (uint32_t)carry;
                ph_o = (uint32_t)ph_in;
                mh_o = (uint32_t)mh_in;
                best = min(best, score);
            }
        }
        if (lane == last_lane) {
            free_end[pair] = best;
            global_d[pair] = score;
        }
        __syncwarp();
    }
}

template <int K>
cudaError_t launch_k(const uint32_t *texts, const int64_t *toff, const int32_t *tlen, const uint32_t *pats,
                     const int64_t *poff, const int32_t *plen, int32_t n, int32_t max_m, int32_t *fe, int32_t *gl,
                     int sms, cudaStream_t st) {
    const int threads = 256;
    const int64_t want = ((int64_t)n * 32 + threads - 1) / threads;
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)sms * 8));
    edit_distance_kernel<K><<<blocks, threads, 0, st>>>(texts, toff, tlen, pats, poff, plen, n, max_m, fe, gl);
    return cudaGetLastError();
}

}  // namespace
}  // namespace scrooge

using namespace scrooge;

extern "C" int scrooge_edit_distance(scrooge_ctx *c, const uint32_t *texts, const int64_t *text_offsets,
                                     const int32_t *text_lengths, const uint32_t *patterns,
                                     const int64_t *pattern_offsets, const int32_t *pattern_lengths, int32_t n_pairs,
                                     int32_t max_pattern_length, uint32_t flags, int32_t *free_end,
                                     int32_t *global_distance) {
    if (!c || n_pairs < 0) return SCROOGE_E_INVAL;
    if (!(flags & SCROOGE_DEVICE_PTRS)) return fail(c, SCROOGE_E_INVAL, "scrooge_edit_distance takes device pointers");
    if (max_pattern_length < 0 || max_pattern_length > SCROOGE_EDIT_DISTANCE_MAX_M)
        return fail(c, SCROOGE_E_INVAL, "max_pattern_length %d outside 0..%d", max_pattern_length,
                    SCROOGE_EDIT_DISTANCE_MAX_M);
    if (n_pairs == 0) return SCROOGE_OK;
    if (!texts || !text_offsets || !text_lengths || !patterns || !pattern_offsets || !pattern_lengths || !free_end ||
        !global_distance)
        return fail(c, SCROOGE_E_INVAL, "null pointer argument");
    const int words = std::max(1, (max_pattern_length + 63) / 64);
    const int K = words <= 32 ? 1 : (words <= 64 ? 2 : (words <= 128 ? 4 : 8));
    cudaError_t e;
    switch (K) {
        case 1: e = launch_k<1>(texts, text_offsets, text_lengths, patterns, pattern_offsets, pattern_lengths, n_pairs,
                                max_pattern_length, free_end, global_distance, c->sm_count, c->stream); break;
        case 2: e = launch_k<2>(texts, text_offsets, text_lengths, patterns, pattern_offsets, pattern_lengths, n_pairs,
                                max_pattern_length, free_end, global_distance, c->sm_count, c->stream); break;
        case 4: e = launch_k<4>(texts, text_offsets, text_lengths, patterns, pattern_offsets, pattern_lengths, n_pairs,
                                max_pattern_length, free_end, global_distance, c->sm_count, c->stream); break;
        default: e = launch_k<8>(texts, text_offsets, text_lengths, patterns, pattern_offsets, pattern_lengths, n_pairs,
                                 max_pattern_length, free_end, global_distance, c->sm_count, c->stream); break;
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "edit distance launch");
    if (flags & SCROOGE_SYNC) {
        if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return cuda_fail(c, e, "edit distance");
    }
    return SCROOGE_OK;
}
