// Windowed GenASM alignment kernel for sm_103a (Scrooge, arXiv 2208.09985).
//
// Work decomposition. A warp holds 32/G pairs; the G lanes of a pair split the
// W columns (text positions) of a window into G contiguous chunks of C = W/G
// columns. Lane l owns columns [(G-1-l)*C, (G-l)*C): lane 0 the highest, lane
// G-1 column 0. Algorithm 1 (Section 2.2.1) computes a row d from column n-1
// down to column 0, because entry R[i][d] needs R[i+1][d]; the lanes form a
// pipeline over rows: in step s lane l computes row d = s - l of its chunk,
// taking R[top+1][d] from lane l-1 (computed one step earlier) by a warp
// shuffle. Every lane keeps, for each of its columns, the part of the
// recurrence that comes from the previous row in registers,
//     X[i] = (R[i][d-1] << 1) & R[i+1][d-1] & (R[i+1][d-1] << 1),
// so a cell costs one shift of the new entry and two 3-input logic ops per
// 32-bit word:  R[i][d] = X[i] & ((R[i+1][d] << 1) | PM[text[i]]).
// Rows are built one after the other, so early termination (ET, Section
// 2.4.3) stops a window as soon as lane G-1 sees a 0 in the first bit of
// R[0][d]: at most G-1 extra rows are touched by the other lanes.
//
// Storage. With SENE (Section 2.4.1) only entries are stored; with DENT
// (Section 2.4.2) only columns 0..W-O (rounded up to whole lane chunks, so a
// lane either stores all its columns or none) and the words holding bits
// 0..W-O. A stored cell is one 4-, 8- or 16-byte vector store. Rows below
// `rcap` go to shared memory, deeper rows to a per-warp device scratch area;
// both use the layout [row][column][pair of the warp][word], so a step needs
// one row pointer and every column store has a compile-time offset. Without
// SENE the three GenASM edge vectors I, D, M of every cell are stored instead
// (ablation). DENT extended to rows (Supplementary Section 1): row d goes to
// row slot d mod `ring`, a cycle of at least W-O+G slots that always holds the
// rows d_opt-(W-O) .. d_opt the traceback reads (ring = k+1 keeps every row).
//
// Traceback (GenASM-TB, Section 2.2.2) runs on lane G-1 of each pair. Along
// the path every visited entry holds a 0 (Theorem 1), so when text[i] equals
// pattern[j] the match edge is always open: a whole run of matches is taken at
// once by comparing 32 packed bases with one XOR and a count of leading zeros.
// Only at a mismatch (or at the end of the text) are stored bits read, and
// substitution, insertion, deletion are tried in that order. The traceback
// stops after W-O text or pattern characters or at the end of the pattern
// window (Section 2.2.3), and the window slides by what it consumed.
//
// Bit order: bit j of a vector (j = 0 is the paper's most significant "first
// bit") is bit 31 - (j % 32) of word j / 32. "<< 1" moves bit j+1 into bit j.
// Bits j >= m of every entry are 0, which is exactly the shifted-in 0 of
// Algorithm 1 for a shorter pattern window.
#pragma once

#include <stdint.h>

#include "scrooge_internal.h"

namespace scrooge {
namespace kern {

constexpr uint32_t kFull = 0xffffffffu;
constexpr int kOpI = 1, kOpD = 2, kOpEq = 7, kOpX = 8;

// First `bits` bits set (MSB-first); bits <= 0 -> 0, bits >= 32 -> all.
__device__ __forceinline__ uint32_t prefix_mask(int bits) {
    return bits <= 0 ? 0u : (bits >= 32 ? kFull : (kFull << (32 - bits)));
}

// Slot of stored row `row` (0 <= row <= k) in a cyclic row store of `ring` slots. The host keeps
// ring >= (k + 1) / 2, so a row wraps at most once: one compare and subtract, no division.
__device__ __forceinline__ int ring_slot(int row, int ring) { return row >= ring ? row - ring : row; }

__device__ __forceinline__ uint2 load_block(const uint2 *seq, int64_t b, int64_t nblk) {
    return (b >= 0 && b < nblk) ? __ldg(seq + b) : make_uint2(0u, 0u);
}

// Bit planes of the 32 bases starting at base `pos` (bases past the end read 0).
__device__ __forceinline__ void load32(const uint2 *seq, int64_t nblk, int64_t pos, uint32_t &p0, uint32_t &p1) {
    const int64_t b = pos >> 5;
    const int r = (int)(pos & 31);
    const uint2 a = load_block(seq, b, nblk);
    const uint2 c = load_block(seq, b + 1, nblk);
    p0 = __funnelshift_l(c.x, a.x, r);
    p1 = __funnelshift_l(c.y, a.y, r);
}

template <int NW>
__device__ __forceinline__ void shl1(const uint32_t (&x)[NW], uint32_t (&y)[NW]) {
#pragma unroll
    for (int w = 0; w + 1 < NW; ++w) y[w] = __funnelshift_l(x[w + 1], x[w], 1);
    y[NW - 1] = x[NW - 1] + x[NW - 1];
}

// 32 bases of a staged window (NW+1 words per plane) starting at `pos`.
__device__ __forceinline__ uint32_t stage_ext(const uint32_t *plane, int pos) {
    const int w = pos >> 5;
    return __funnelshift_l(plane[w + 1], plane[w], pos & 31);
}

struct CigarOut {
    uint32_t *dst;
    int64_t cap;
    int32_t n;
    uint32_t cur;  // pending run (len << 4 | op), 0 = none
    int32_t edits;

    // Append `len` >= 0 operations `op`, merging with the pending run (branch-free).
    __device__ __forceinline__ void emit_maybe(int op, int len) {
        const bool any = len > 0;
        edits += (any && op != kOpEq) ? len : 0;
        const bool same = cur != 0u && (int)(cur & 15u) == op;
        const bool spill = any && cur != 0u && !same;
        if (spill && n < cap) __stcs(dst + n, cur);  // streaming: not read again by this kernel
        n += spill ? 1 : 0;
        cur = !any ? cur : (same ? cur + ((uint32_t)len << 4) : (((uint32_t)len << 4) | (uint32_t)op));
    }
    __device__ __forceinline__ void emit(int op, int len) { emit_maybe(op, len); }
    __device__ __forceinline__ void flush() {
        if (cur != 0u) {
            if (n < cap) __stcs(dst + n, cur);
            ++n;
        }
        cur = 0u;
    }
};

// Store / load one stored vector of SWP words (SWP = 1, 2 or 4; 4-, 8- or 16-byte aligned).
template <int SWP, int NW>
__device__ __forceinline__ void store_vec(uint32_t *p, const uint32_t (&v)[NW]) {
    if (SWP == 1) {
        *p = v[0];
    } else if (SWP == 2) {
        *reinterpret_cast<uint2 *>(p) = make_uint2(v[0], NW > 1 ? v[NW > 1 ? 1 : 0] : 0u);
    } else {
        *reinterpret_cast<uint4 *>(p) = make_uint4(v[0], v[NW > 1 ? 1 : 0], NW > 2 ? v[NW > 2 ? 2 : 0] : 0u,
                                                    NW > 3 ? v[NW > 3 ? 3 : 0] : 0u);
    }
}

__device__ __forceinline__ uint32_t bit_of(uint32_t word, int b) { return (word >> (31 - (b & 31))) & 1u; }

// Bits j and j+1 of a stored entry of SWP words, as (bit j) << 1 | bit j+1;
// a bit past the stored words reads 0. One vector load per entry.
template <int SWP>
__device__ __forceinline__ uint32_t entry_bits2(const uint32_t *e, int j) {
    if (SWP == 1) {
        const uint64_t q = (uint64_t)(*e) << 32;
        return (uint32_t)((q << j) >> 62);
    } else if (SWP == 2) {
        const uint2 v = *reinterpret_cast<const uint2 *>(e);
        const uint64_t q = ((uint64_t)v.x << 32) | v.y;
        return (uint32_t)((q << j) >> 62);
    } else {
        const uint4 v = *reinterpret_cast<const uint4 *>(e);
        const int w = j >> 5;
        const uint32_t a = w == 0 ? v.x : (w == 1 ? v.y : (w == 2 ? v.z : v.w));
        const uint32_t b = w == 0 ? v.y : (w == 1 ? v.z : (w == 2 ? v.w : 0u));
        const uint64_t q = ((uint64_t)a << 32) | b;
        return (uint32_t)((q << (j & 31)) >> 62);
    }
}

// Bookkeeping of one pair slot (the G lanes of a pair): its pair, cursors
// and statistics. Used by the banded kernel.
struct Slot {
    int pair, n, m, ti, pj;
    const uint2 *tseq, *pseq;
    int64_t tblk, pblk, next_static;
    bool active, exhausted, failed;
    int64_t st_rows, st_cells;
    int32_t st_windows;
    long long t_start;
};

__device__ __forceinline__ void slot_init(Slot &s, int64_t first_static, bool idle) {
    s.pair = s.n = s.m = s.ti = s.pj = 0;
    s.tseq = s.pseq = nullptr;
    s.tblk = s.pblk = 0;
    s.next_static = first_static;
    s.active = s.failed = false;
    s.exhausted = idle;  // a slot beyond slots_per_warp never takes a pair
    s.st_rows = s.st_cells = 0;
    s.st_windows = 0;
    s.t_start = 0;
}

// An idle slot takes its next pair: lane G-1 draws it from the device queue over
// `order` (persistent launch) or from a fixed stride over the input (plain
// launch) and shares it with the slot's lanes. Pairs with an empty pattern are
// finished at fetch time.
// Slots [lo, hi) of the order this launch serves (persistent launches may split them).
__device__ __forceinline__ void slot_range(const AlignParams &p, int64_t &lo, int64_t &hi) {
    lo = (p.queue && p.range_lo) ? *p.range_lo : 0;
    hi = (p.queue && p.range_hi) ? *p.range_hi : p.n_pairs;
}

template <int G>
__device__ __forceinline__ void slot_fetch(const AlignParams &p, Slot &s, CigarOut &out, int l, int g, int tbl,
                                           int64_t stride, int64_t q_lo, int64_t q_hi) {
    if (s.active || s.exhausted) return;
    int next = -1;
    if (l == G - 1) {
        for (;;) {
            int64_t sl;
            if (p.queue) {
                sl = q_lo + atomicAdd(p.queue, 1);
            } else {
                sl = s.next_static;
                s.next_static += stride;
            }
            if (sl >= q_hi) break;
            const int pr = p.order ? p.order[sl] : (int)sl;
            if (p.pat_len[pr] > 0) {
                next = pr;
                break;
            }
            p.edit_counts[pr] = 0;
            p.text_consumed[pr] = 0;
            p.cigar_lens[pr] = 0;
            if (p.st_windows) p.st_windows[pr] = 0;
            if (p.st_rows) p.st_rows[pr] = 0;
            if (p.st_cells) p.st_cells[pr] = 0;
            if (p.st_cycles) p.st_cycles[pr] = 0;
        }
    }
    const uint32_t gmask = (G == 32) ? kFull : (((1u << G) - 1u) << (g * G));
    next = __shfl_sync(gmask, next, tbl);
    if (next < 0) {
        s.exhausted = true;
        return;
    }
    s.pair = next;
    s.n = p.text_len[next];
    s.m = p.pat_len[next];
    s.tseq = reinterpret_cast<const uint2 *>(p.texts + (p.text_off[next] >> 4));
    s.pseq = reinterpret_cast<const uint2 *>(p.patterns + (p.pat_off[next] >> 4));
    s.tblk = (s.n + 31) >> 5;
    s.pblk = (s.m + 31) >> 5;
    s.ti = 0;
    s.pj = 0;
    s.failed = false;
    s.st_rows = 0;
    s.st_cells = 0;
    s.st_windows = 0;
    if (l == G - 1) {
        const int64_t c0 = p.cigar_off[next];
        out.dst = p.cigar + c0;
        out.cap = p.cigar_off[next + 1] - c0;
        out.n = 0;
        out.cur = 0u;
        out.edits = 0;
        s.t_start = clock64();
    }
    s.active = true;
}

// After a window: the traceback lane finishes its pair when the pattern is
// consumed (or a window failed), then the slot's lanes take over its cursors.
template <int G>
__device__ __forceinline__ void slot_window_done(const AlignParams &p, Slot &s, CigarOut &out, int l, int tbl) {
    if (s.active && l == G - 1 && (s.failed || s.pj >= s.m)) {
        s.active = false;
        out.flush();
        const int pair = s.pair;
        p.edit_counts[pair] = s.failed ? -1 : out.edits;
        p.text_consumed[pair] = s.failed ? 0 : s.ti;
        if (out.n > out.cap) atomicOr(p.status, 2);  // capacity too small for this pair
        p.cigar_lens[pair] = s.failed ? 0 : min(out.n, (int32_t)out.cap);
        if (p.st_windows) p.st_windows[pair] = s.st_windows;
        if (p.st_rows) p.st_rows[pair] = s.st_rows;
        if (p.st_cells) p.st_cells[pair] = s.st_cells;
        if (p.st_cycles) p.st_cycles[pair] = clock64() - s.t_start;
    }
    s.ti = __shfl_sync(kFull, s.ti, tbl);
    s.pj = __shfl_sync(kFull, s.pj, tbl);
    s.active = __shfl_sync(kFull, (int)s.active, tbl) != 0;
    __syncwarp();
}

// Full-width DC of the windows in `full_mask` (Algorithm 1 on NW words per
// entry, as in the full-width kernel), rows stored to `rows` (this lane's first
// column of row 0; [row][column][pair][NW words]); d_opt of those windows is set
// on their traceback lanes. Kept out of line: it is rare, and its registers
// must not count against the banded loop.
template <int G, int NW>
__device__ __noinline__ void full_width_dc(const uint2 *pseq, int64_t pblk, int pj, const uint2 *tseq, int64_t tblk,
                                           int ti, int nw, int mw, int k, int l, int tbl, uint32_t tbl_all,
                                           uint32_t full_mask, bool lane_stores, uint32_t *rows, int row_words,
                                           int &d_opt) {
    constexpr int C = 32 * NW / G;
    constexpr int PPW = 32 / G;
    const bool full = (full_mask >> tbl) & 1u;
    const int colbase = (G - 1 - l) * C;
    uint32_t P0[NW], P1[NW], mm[NW], T0, T1;
#pragma unroll
    for (int w = 0; w < NW; ++w) {
        load32(pseq, pblk, (int64_t)pj + 32 * w, P0[w], P1[w]);
        mm[w] = prefix_mask(mw - 32 * w);
    }
    load32(tseq, tblk, (int64_t)ti + colbase, T0, T1);
    const int real_cols = nw - colbase;
    uint32_t FX[C][NW];  // X of the next row
#pragma unroll
    for (int c = 0; c < C; ++c)
#pragma unroll
        for (int w = 0; w < NW; ++w) FX[c][w] = mm[w];
    uint32_t fdone = tbl_all & ~full_mask;
    uint32_t bot[NW];
#pragma unroll
    for (int w = 0; w < NW; ++w) bot[w] = 0u;
    for (int st = 0; fdone != tbl_all; ++st) {
        const int d = st - l;
        const bool ddone = (fdone >> tbl) & 1u;
        uint32_t pR[NW], pS[NW];
#pragma unroll
        for (int w = 0; w < NW; ++w) {
            const uint32_t v = __shfl_up_sync(kFull, bot[w], 1);
            pR[w] = (l == 0) ? prefix_mask(mw - d - 32 * w) : v;
        }
        bool found = false;
        if (!ddone && d >= 0 && d <= k) {
            shl1<NW>(pR, pS);
            uint32_t *rowp = rows + (int64_t)d * row_words;
#pragma unroll
            for (int c = C - 1; c >= 0; --c) {
                // PM[text[i]] from the pattern planes
                const uint32_t m0 = 0u - ((T0 >> (31 - c)) & 1u);
                const uint32_t m1 = 0u - ((T1 >> (31 - c)) & 1u);
                const bool real = c < real_cols;
                uint32_t R[NW], S[NW];
#pragma unroll
                for (int w = 0; w < NW; ++w) {
                    const uint32_t pm = real ? ((P0[w] ^ m0) | (P1[w] ^ m1)) : kFull;
                    R[w] = FX[c][w] & (pS[w] | pm);
                }
                shl1<NW>(R, S);
                if (lane_stores) store_vec<NW, NW>(rowp + c * NW * PPW, R);
#pragma unroll
                for (int w = 0; w < NW; ++w) {
                    FX[c][w] = S[w] & pR[w] & pS[w];
                    pR[w] = R[w];
                    pS[w] = S[w];
                }
            }
#pragma unroll
            for (int w = 0; w < NW; ++w) bot[w] = pR[w];
            found = (l == G - 1) && ((pR[0] >> 31) == 0u);
        }
        const uint32_t fm = __ballot_sync(kFull, found);
        const int dl = st - (G - 1);
        if (full && !ddone && ((fm >> tbl) & 1u) && d_opt < 0) d_opt = dl;
        fdone |= fm;
        if (dl >= k) fdone = tbl_all;
    }
}

template <int NW, int G, bool SENE, int SWP>
__global__ void __launch_bounds__(64, 6) align_kernel(const AlignParams p) {
    constexpr int WMAX = 32 * NW;
    constexpr int C = WMAX / G;
    constexpr int PPW = 32 / G;
    constexpr int NV = SENE ? 1 : 3;       // stored vectors per cell
    constexpr int CELL = NV * SWP;          // words per stored cell
    constexpr int COLW = PPW * CELL;        // words between two columns of one row
    static_assert(C * G == WMAX && C <= 32 && 32 % G == 0, "unsupported shape");
    static_assert(SWP == 1 || SWP == 2 || SWP == 4, "stored words");

    extern __shared__ __align__(16) uint32_t smem[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int g = lane / G;
    const int l = lane - g * G;
    const int tbl = g * G + G - 1;  // traceback lane of this pair (owns column 0)
    const int W = p.W, L = p.W - p.O, k = p.k;
    const int ncolp = p.ncol, rcap = p.rcap, ring = p.ring;  // ncolp: stored columns
    const int colbase = (G - 1 - l) * C;
    const bool lane_stores = colbase < ncolp;  // stored columns come in whole lane chunks
    uint32_t tbl_all = 0;                      // one bit per pair: its traceback lane
#pragma unroll
    for (int q = 0; q < PPW; ++q) tbl_all |= 1u << (q * G + G - 1);

    uint32_t *tab = smem + (int64_t)wib * p.smem_words_per_warp;
    uint32_t *stage = tab + p.table_words_per_warp + g * (4 * (NW + 1));
    const int64_t gw = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    uint32_t *spill = p.spill + gw * p.spill_words_per_pair;  // per warp, same interleaved layout

    // word 0 of column 0 of `row` of this pair (shared memory or scratch)
    const int rstride = p.rstride;
    auto row_base = [&](int row) -> uint32_t * {
        const int slot = ring_slot(row, ring);
        return slot < rcap ? tab + ((int64_t)slot * rstride + g) * CELL
                           : spill + ((int64_t)(slot - rcap) * rstride + g) * CELL;
    };

    // Each pair slot of the warp refills itself as soon as its pair is done:
    // from a fixed stride over the input order (plain launch) or from the
    // device work queue over `order` (persistent launch). Pairs with an empty
    // pattern are finished at fetch time.
    int64_t next_static = gw * PPW + g;
    int64_t q_lo, q_hi;
    slot_range(p, q_lo, q_hi);
    bool exhausted = p.slots_per_warp > 0 && g >= p.slots_per_warp, active = false;
    int pair = 0, n = 0, m = 0;
    const uint2 *tseq = nullptr, *pseq = nullptr;
    int64_t tblk = 0, pblk = 0;
    int ti = 0, pj = 0;
    CigarOut out;
    out.dst = nullptr;
    out.cap = 0;
    out.n = 0;
    out.cur = 0u;
    out.edits = 0;
    int64_t st_rows = 0, st_cells = 0;
    int32_t st_windows = 0;
    long long t_start = 0;
    bool failed = false;
    for (;;) {
        if (!active && !exhausted) {
            int next = -1;
            if (l == G - 1) {
                for (;;) {
                    int64_t sl;
                    if (p.queue) {
                        sl = q_lo + atomicAdd(p.queue, 1);
                    } else {
                        sl = next_static;
                        next_static += nwarps * PPW;
                    }
                    if (sl >= q_hi) break;
                    const int pr = p.order ? p.order[sl] : (int)sl;
                    if (p.pat_len[pr] > 0) {
                        next = pr;
                        break;
                    }
                    p.edit_counts[pr] = 0;
                    p.text_consumed[pr] = 0;
                    p.cigar_lens[pr] = 0;
                    if (p.st_windows) p.st_windows[pr] = 0;
                    if (p.st_rows) p.st_rows[pr] = 0;
                    if (p.st_cells) p.st_cells[pr] = 0;
                    if (p.st_cycles) p.st_cycles[pr] = 0;
                }
            }
            const uint32_t gmask = (G == 32) ? kFull : (((1u << G) - 1u) << (g * G));
            next = __shfl_sync(gmask, next, tbl);
            if (next < 0) {
                exhausted = true;
            } else {
                pair = next;
                n = p.text_len[pair];
                m = p.pat_len[pair];
                tseq = reinterpret_cast<const uint2 *>(p.texts + (p.text_off[pair] >> 4));
                pseq = reinterpret_cast<const uint2 *>(p.patterns + (p.pat_off[pair] >> 4));
                tblk = (n + 31) >> 5;
                pblk = (m + 31) >> 5;
                ti = 0;
                pj = 0;
                failed = false;
                st_rows = 0;
                st_cells = 0;
                st_windows = 0;
                if (l == G - 1) {
                    const int64_t c0 = p.cigar_off[pair];
                    out.dst = p.cigar + c0;
                    out.cap = p.cigar_off[pair + 1] - c0;
                    out.n = 0;
                    out.cur = 0u;
                    out.edits = 0;
                    t_start = clock64();
                }
                active = true;
            }
        }
        if (!__any_sync(kFull, active)) break;
        {
            const int nw = active ? min(W, n - ti) : 0;
            const int mw = active ? min(W, m - pj) : 0;

            // ---- window set-up: pattern planes, per-column masks PM[text[i]]
            uint32_t XA[C][NW];             // X (SENE) or the insertion edge I of the next row
            uint32_t XB[SENE ? 1 : C][NW];  // without SENE: R[i+1][d-1] of the next row
            uint32_t PMC[C][NW];
            {
                uint32_t P0[NW], P1[NW], mm[NW];
#pragma unroll
                for (int w = 0; w < NW; ++w) {
                    load32(pseq, active ? pblk : 0, pj + 32 * w, P0[w], P1[w]);
                    mm[w] = prefix_mask(mw - 32 * w);
                }
                uint32_t T0, T1;
                load32(tseq, active ? tblk : 0, ti + colbase, T0, T1);
                const int real_cols = nw - colbase;  // columns of this lane inside the text window
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    const uint32_t m0 = 0u - ((T0 >> (31 - c)) & 1u);
                    const uint32_t m1 = 0u - ((T1 >> (31 - c)) & 1u);
                    const bool real = c < real_cols;
#pragma unroll
                    for (int w = 0; w < NW; ++w) {
                        PMC[c][w] = real ? ((P0[w] ^ m0) | (P1[w] ^ m1)) : kFull;
                        XA[c][w] = mm[w];
                        if (!SENE) XB[SENE ? 0 : c][w] = kFull;
                    }
                }
                if (active && l == G - 1) {
#pragma unroll
                    for (int w = 0; w <= NW; ++w) {
                        uint32_t a, b;
                        load32(tseq, tblk, ti + 32 * w, a, b);
                        stage[w] = a;
                        stage[(NW + 1) + w] = b;
                        load32(pseq, pblk, pj + 32 * w, a, b);
                        stage[2 * (NW + 1) + w] = a;
                        stage[3 * (NW + 1) + w] = b;
                    }
                }
            }

            // ---- GenASM-DC, rows in a pipeline over the lanes of each pair
            uint32_t done_mask = __ballot_sync(kFull, l == G - 1 && !active);
            int d_opt = -1;
            uint32_t bottom[NW];
#pragma unroll
            for (int w = 0; w < NW; ++w) bottom[w] = 0u;
            for (int s = 0; done_mask != tbl_all; ++s) {
                const int d = s - l;
                const bool dc_done = (done_mask >> tbl) & 1u;
                uint32_t pR[NW], pS[NW];
#pragma unroll
                for (int w = 0; w < NW; ++w) {
                    const uint32_t v = __shfl_up_sync(kFull, bottom[w], 1);
                    // lane 0 starts from the right column R[n][d] = 1..1 << d
                    pR[w] = (l == 0) ? prefix_mask(mw - d - 32 * w) : v;
                }
                bool found = false;
                if (!dc_done && d >= 0 && d <= k) {
                    shl1<NW>(pR, pS);
                    uint32_t *rowp = row_base(d) + (int64_t)colbase * COLW;
#pragma unroll
                    for (int c = C - 1; c >= 0; --c) {
                        uint32_t R[NW], S[NW];
                        if (SENE) {
#pragma unroll
                            for (int w = 0; w < NW; ++w) R[w] = XA[c][w] & (pS[w] | PMC[c][w]);
                        } else {
                            // row 0 has no I/D/S edges: XA = mask, XB = all ones
                            uint32_t Dd[NW], Sd[NW];
#pragma unroll
                            for (int w = 0; w < NW; ++w) Dd[w] = XB[SENE ? 0 : c][w];
                            shl1<NW>(Dd, Sd);
#pragma unroll
                            for (int w = 0; w < NW; ++w) {
                                const uint32_t sdm = (d == 0) ? kFull : Sd[w];
                                R[w] = XA[c][w] & Dd[w] & sdm & (pS[w] | PMC[c][w]);
                            }
                        }
                        shl1<NW>(R, S);
                        if (lane_stores) {
                            if (SENE) {
                                store_vec<SWP, NW>(rowp + c * COLW, R);
                            } else if (d > 0) {
                                // GenASM's stored edges: I, D (S = D << 1) and M
                                uint32_t M[NW], Dd[NW];
#pragma unroll
                                for (int w = 0; w < NW; ++w) {
                                    M[w] = pS[w] | PMC[c][w];
                                    Dd[w] = XB[SENE ? 0 : c][w];
                                }
                                store_vec<SWP, NW>(rowp + c * COLW, XA[c]);
                                store_vec<SWP, NW>(rowp + c * COLW + SWP, Dd);
                                store_vec<SWP, NW>(rowp + c * COLW + 2 * SWP, M);
                            }
                        }
                        if (SENE) {
#pragma unroll
                            for (int w = 0; w < NW; ++w) XA[c][w] = S[w] & pR[w] & pS[w];
                        } else {
#pragma unroll
                            for (int w = 0; w < NW; ++w) {
                                XA[c][w] = S[w];                 // I of cell (i, d+1)
                                XB[SENE ? 0 : c][w] = pR[w];     // D of cell (i, d+1)
                            }
                        }
#pragma unroll
                        for (int w = 0; w < NW; ++w) {
                            pR[w] = R[w];
                            pS[w] = S[w];
                        }
                    }
#pragma unroll
                    for (int w = 0; w < NW; ++w) bottom[w] = pR[w];
                    found = (l == G - 1) && ((pR[0] >> 31) == 0u);
                }
                // one vote per step: which pairs reached the window start in this row
                const uint32_t fmask = __ballot_sync(kFull, found);
                const int dl = s - (G - 1);  // row finished by the traceback lane
                if (!dc_done && ((fmask >> tbl) & 1u) && d_opt < 0) d_opt = dl;
                if (p.et) done_mask |= fmask;
                if (dl >= k) done_mask = tbl_all;
            }

            __syncwarp();  // entries written by every lane are visible to the traceback lane

            // ---- GenASM-TB: all traceback lanes of the warp step together. One
            // step takes a run of matches (one XOR + CLZ over 32 packed bases)
            // and then, unless the window's traceback ends, one S/I/D edge read
            // from the stored entries; the code is branch-free so the lanes of
            // different pairs do not diverge.
            if (l == G - 1) {
                const bool tb_live = active && d_opt >= 0;
                if (active) st_windows += 1;
                if (active && d_opt < 0) failed = true;
                if (tb_live) {
                    st_rows += d_opt + 1;
                    st_cells += (int64_t)(d_opt + 1) * nw;
                }
                const uint32_t *T0s = stage, *T1s = stage + (NW + 1);
                const uint32_t *P0s = stage + 2 * (NW + 1), *P1s = stage + 3 * (NW + 1);
                // windows of up to 64 bases: the four planes in 64-bit registers. A
                // match run never reaches past the window, so the zeros shifted in
                // at the end are never compared.
                uint64_t qT0 = 0, qT1 = 0, qP0 = 0, qP1 = 0;
                if (NW <= 2) {
                    qT0 = ((uint64_t)T0s[0] << 32) | T0s[1];
                    qT1 = ((uint64_t)T1s[0] << 32) | T1s[1];
                    qP0 = ((uint64_t)P0s[0] << 32) | P0s[1];
                    qP1 = ((uint64_t)P1s[0] << 32) | P1s[1];
                }
                auto ext = [&](uint64_t q, const uint32_t *plane, int pos) -> uint32_t {
                    if (NW <= 2) return (uint32_t)((q << pos) >> 32);
                    return stage_ext(plane, pos);
                };
                int i = 0, j = 0, d = d_opt;
                bool going = tb_live && (j < mw && i < L && j < L);
                while (__any_sync(tbl_all, going)) {
                    if (going) {
                        const int lim = min(min(nw - i, mw - j), min(L - i, L - j));
                        const uint32_t x = (ext(qT0, T0s, i) ^ ext(qP0, P0s, j)) | (ext(qT1, T1s, i) ^ ext(qP1, P1s, j));
                        const int z = __clz(x);
                        const int run = min(z, lim);
                        out.emit_maybe(kOpEq, run);
                        i += run;
                        j += run;
                        const bool cont = j < mw && i < L && j < L;
                        // z == 32 with room left: keep matching in the next step
                        const bool edit = cont && !(z == 32 && run < lim);
                        if (edit && d <= 0) {  // no edge can leave row 0 here (Theorem 1)
                            atomicOr(p.status, 1);
                            failed = true;
                            going = false;
                        } else if (edit) {
                            const bool tx = i < nw;
                            const bool j1 = j + 1 < mw;  // bit j+1 exists (else it is the shifted-in 0)
                            const int lim_r = mw - (d - 1);  // bits < lim_r of the right column R[n][d-1] are 1
                            uint32_t bS, bI, bD;
                            if (SENE) {
                                // entries (i+1, d-1) and (i, d-1): shared memory or scratch
                                const int r = ring_slot(d - 1, ring);
                                const bool ld1 = tx && i + 1 < nw;
                                uint32_t e1 = 0u, e0 = 0u;
                                if (r < rcap) {
                                    const uint32_t *rp = tab + (r * rstride + g) * CELL + i * COLW;
                                    if (ld1) e1 = entry_bits2<SWP>(rp + COLW, j);
                                    if (tx) e0 = entry_bits2<SWP>(rp, j);
                                } else {
                                    const uint32_t *rp = spill + ((r - rcap) * rstride + g) * CELL + i * COLW;
                                    if (ld1) e1 = entry_bits2<SWP>(rp + COLW, j);
                                    if (tx) e0 = entry_bits2<SWP>(rp, j);
                                }
                                const uint32_t r1j = ld1 ? (e1 >> 1) : (j < lim_r ? 1u : 0u);
                                const uint32_t r1j1 = !j1 ? 0u : (ld1 ? (e1 & 1u) : (j + 1 < lim_r ? 1u : 0u));
                                const uint32_t r0j1 = !j1 ? 0u : (tx ? (e0 & 1u) : (j + 1 < lim_r ? 1u : 0u));
                                bS = tx ? r1j1 : 1u;
                                bI = r0j1;
                                bD = tx ? r1j : 1u;
                            } else {
                                // stored edge vectors of cell (i, d)
                                const uint32_t *rp = row_base(d) + (int64_t)i * COLW;
                                const uint32_t wDa = tx ? rp[SWP + (j >> 5)] : 0u;
                                const uint32_t wDb = (tx && j1) ? rp[SWP + ((j + 1) >> 5)] : 0u;
                                const uint32_t wI = tx ? rp[j >> 5] : 0u;
                                bS = tx ? (j1 ? bit_of(wDb, j + 1) : 0u) : 1u;
                                // at the right column, I = R[n][d-1] << 1
                                bI = tx ? bit_of(wI, j) : ((j1 && j + 1 < lim_r) ? 1u : 0u);
                                bD = tx ? bit_of(wDa, j) : 1u;
                            }
                            const bool tS = tx && bS == 0u;
                            const bool tI = !tS && bI == 0u;
                            const bool tD = !tS && !tI && tx && bD == 0u;
                            if (!(tS || tI || tD)) {
                                atomicOr(p.status, 1);
                                failed = true;
                                going = false;
                            } else {
                                out.emit(tS ? kOpX : (tI ? kOpI : kOpD), 1);
                                i += (tS || tD) ? 1 : 0;
                                j += (tS || tI) ? 1 : 0;
                                d -= 1;
                                going = j < mw && i < L && j < L;
                            }
                        } else {
                            going = cont;
                        }
                    }
                }
                if (tb_live) {
                    ti += i;
                    pj += j;
                }
            }
            if (active && l == G - 1) {
                if (failed || pj >= m) {
                    active = false;
                    out.flush();
                    p.edit_counts[pair] = failed ? -1 : out.edits;
                    p.text_consumed[pair] = failed ? 0 : ti;
                    if (out.n > out.cap) atomicOr(p.status, 2);  // capacity too small for this pair
                    p.cigar_lens[pair] = failed ? 0 : min(out.n, (int32_t)out.cap);
                    if (p.st_windows) p.st_windows[pair] = st_windows;
                    if (p.st_rows) p.st_rows[pair] = st_rows;
                    if (p.st_cells) p.st_cells[pair] = st_cells;
                    if (p.st_cycles) p.st_cycles[pair] = clock64() - t_start;
                }
            }
            ti = __shfl_sync(kFull, ti, tbl);
            pj = __shfl_sync(kFull, pj, tbl);
            active = __shfl_sync(kFull, (int)active, tbl) != 0;
            __syncwarp();
        }
    }
}

}  // namespace kern
}  // namespace scrooge
