// Banded GenASM alignment kernel for windows of 64 bases (Scrooge, arXiv
// 2208.09985), with its instantiations and launchers.
//
// Coordinates. The full-width kernel (align_kernel.cuh) keeps, for text
// column i, the W-bit vector R[i][d] indexed by the pattern position j. This
// kernel keeps only the 32 bits of a band around the main diagonal, indexed
// by k = j - i + 15, i.e. the diagonals j - i = -15..16, in one 32-bit word
// V[i][d] (bit k is bit 31 - k, as everywhere). In these coordinates the
// edges of Algorithm 1 (Section 2.2.1) read
//     match / substitution (i+1, j+1): V[i+1] bit k      (no shift)
//     deletion             (i+1, j)  : V[i+1] bit k - 1  (V >> 1)
//     insertion            (i, j+1)  : V[i]   bit k + 1  (V << 1)
// so a cell is
//     V[i][d] = X[i] & (V[i+1][d] | PMrel[i]),
//     X[i]    = V[i+1][d-1] & (V[i+1][d-1] >> 1) & (V[i][d-1] << 1),
// where PMrel[i] is the 32-bit window of PM[text[i]] starting at j = i - 15,
// and the bits shifted in at the band edges are 1 (no path there). The chain
// along a row is a single 3-input logic op per cell (the shifts act on the
// previous row), and a cell is one word instead of two.
//
// Exactness. A path of the GenASM DP (Theorem 1) that starts at (0, 0) and
// spends at most d edits keeps |j - i| <= d. Hence for d <= 15:
//   * bit j = 0 of R[0][d] is 0 in the band exactly when it is 0 in the full
//     table, so ET (Section 2.4.3) finds the same d_opt;
//   * every entry the traceback (Section 2.2.2) reads -- (i+1, j+1), (i, j+1),
//     (i+1, j) at row d-1 from a point reached after d_opt - d edits -- is 0
//     in the full table only if a path of at most d_opt edits from (0, 0) runs
//     through it, which stays inside the band; an entry the band does not hold
//     is therefore 1 in the full table too.
// So with d_opt <= 15 the band gives the same d_opt and the same traceback,
// bit for bit. A window with no d_opt <= 15 (about 0.3% of windows at 10%
// edits) is recomputed at full width (two words per cell, rows in a per-warp
// device area) by the lanes of its pair before the traceback.
//
// Windows of 65..128 bases use a band of 64 diagonals (j - i = -31..32) in two
// words per entry, exact for d_opt <= 31, with the same recurrence on 64-bit
// words and a four-word full-width fallback.
//
// The rest -- lanes per pair, the row pipeline over the lanes, rows below
// `rcap` in shared memory and deeper ones in device scratch, DENT columns,
// the traceback by runs of matches, the pair queue -- is as in the full-width
// kernel. ET is always on here.
#include "align_kernel.cuh"

namespace scrooge {
namespace kern {

// Band of 32 * BW diagonals in one (BW = 1) or two (BW = 2) 32-bit words per entry.
template <int BW>
struct BandT;
template <>
struct BandT<1> {
    using T = uint32_t;
};
template <>
struct BandT<2> {
    using T = uint64_t;
};
template <int BW>
constexpr int band_diag() { return 16 * BW - 1; }  // band bit of the main diagonal j == i
template <int BW>
constexpr int band_rows() { return 16 * BW; }      // rows d = 0..band_rows()-1 are exact

// First `bits` bits (MSB-first) of a band word set.
__device__ __forceinline__ uint32_t band_prefix(uint32_t, int bits) { return prefix_mask(bits); }
__device__ __forceinline__ uint64_t band_prefix(uint64_t, int bits) {
    return bits <= 0 ? 0ull : (bits >= 64 ? ~0ull : (~0ull << (64 - bits)));
}
// v >> 1 and v << 1 in band order with a 1 shifted in (no path beyond the band edge).
__device__ __forceinline__ uint32_t shr1_fill(uint32_t v) { return __funnelshift_r(v, kFull, 1); }
__device__ __forceinline__ uint64_t shr1_fill(uint64_t v) { return (v >> 1) | (1ull << 63); }
__device__ __forceinline__ uint32_t shl1_fill(uint32_t v) { return __funnelshift_l(kFull, v, 1); }
__device__ __forceinline__ uint64_t shl1_fill(uint64_t v) { return (v << 1) | 1ull; }
__device__ __forceinline__ void store_band(uint32_t *p, uint32_t v) { *p = v; }
__device__ __forceinline__ void store_band(uint32_t *p, uint64_t v) {
    *reinterpret_cast<uint2 *>(p) = make_uint2((uint32_t)(v >> 32), (uint32_t)v);
}
__device__ __forceinline__ uint64_t load_band64(const uint32_t *p) {
    const uint2 v = *reinterpret_cast<const uint2 *>(p);
    return ((uint64_t)v.x << 32) | v.y;
}

// resident blocks of two warps the register budget is sized for
template <int G, int NWW, int BW>
struct BandMinBlocks {
    static constexpr int value = BW == 2 ? 6 : (G == 8 ? 12 : (G == 4 ? 8 : 6));
};

// One window of one pair slot of a banded launch, as the DC and traceback routines see it.
struct BandWindow {
    const uint2 *tseq, *pseq;
    int64_t tblk, pblk;  // 0 for an idle slot
    int ti, pj, nw, mw;
    bool active;
};

// GenASM-DC of one window for the 32/G pairs of a warp (all 32 lanes take part). Band rows go to
// `tab` (rows < rcap, shared memory) and `spill` (deeper rows); the traceback lane of each pair
// stages its text and pattern at `stage` (4 planes x (2 BW + 1) words per pair); windows beyond
// the band are recomputed at full width into `fb`. On the traceback lane, d_opt gets the
// window's edit distance (-1: none <= k) and full whether the full-width rows hold it.
template <int G, int NWW, int BW>
__device__ __forceinline__ void band_window_dc(const AlignParams &p, const BandWindow &bw, int l, int g, int tbl,
                                               uint32_t tbl_all, uint32_t *tab, uint32_t *spill, uint32_t *fb,
                                               uint32_t *stage, int &d_opt_out, bool &full_out) {
    using T = typename BandT<BW>::T;
    constexpr int BITS = 32 * BW;
    constexpr int NW = NWW;  // words of a full-width entry (windows of up to 32 NW bases)
    constexpr int WMAX = 32 * NWW;
    constexpr int C = WMAX / G;
    constexpr int PPW = 32 / G;
    constexpr int COLW = PPW * BW;  // words between two columns of one stored band row
    constexpr int B0 = band_diag<BW>();
    const int k = p.k, ncolp = p.ncol, rcap = p.rcap, rstride = p.rstride;
    const int dmax = min(k, band_rows<BW>() - 1);  // deepest row the band computes
    const int colbase = (G - 1 - l) * C;
    const bool lane_stores = colbase < ncolp;
    const bool active = bw.active;
    const int nw = bw.nw, mw = bw.mw;
    auto band_row = [&](int row) -> uint32_t * {
        return row < rcap ? tab + (row * rstride + g) * BW : spill + ((row - rcap) * rstride + g) * BW;
    };

    // ---- window set-up: band pattern masks and row-0 masks of this lane's columns
    T XA[C];   // X of the next row (row 0: bits with j >= m_w cleared)
    T PMC[C];  // PMrel[text[i]]
    {
        uint32_t T0, T1;
        load32(bw.tseq, bw.tblk, (int64_t)bw.ti + colbase, T0, T1);
        const int real_cols = nw - colbase;
        if (BW == 1) {
            // pattern planes from pj + colbase - 16: column colbase + c starts c + 1 bits in
            uint32_t Pa0, Pa1, Pb0, Pb1;
            load32(bw.pseq, bw.pblk, (int64_t)bw.pj + colbase - 16, Pa0, Pa1);
            load32(bw.pseq, bw.pblk, (int64_t)bw.pj + colbase + 16, Pb0, Pb1);
#pragma unroll
            for (int c = 0; c < C; ++c) {
                const uint32_t m0 = 0u - ((T0 >> (31 - c)) & 1u);
                const uint32_t m1 = 0u - ((T1 >> (31 - c)) & 1u);
                const uint32_t w0 = __funnelshift_lc(Pb0, Pa0, c + 1);
                const uint32_t w1 = __funnelshift_lc(Pb1, Pa1, c + 1);
                PMC[c] = (T)(c < real_cols ? ((w0 ^ m0) | (w1 ^ m1)) : kFull);
                XA[c] = band_prefix(T(0), mw - (colbase + c) + B0);
            }
        } else {
            // pattern planes from pj + colbase - 32: column colbase + c starts c + 1 bits in
            uint32_t Q0[3], Q1[3];
#pragma unroll
            for (int w = 0; w < 3; ++w) load32(bw.pseq, bw.pblk, (int64_t)bw.pj + colbase - 32 + 32 * w, Q0[w], Q1[w]);
#pragma unroll
            for (int c = 0; c < C; ++c) {
                const uint32_t m0 = 0u - ((T0 >> (31 - c)) & 1u);
                const uint32_t m1 = 0u - ((T1 >> (31 - c)) & 1u);
                const uint32_t h = (__funnelshift_l(Q0[1], Q0[0], c + 1) ^ m0) | (__funnelshift_l(Q1[1], Q1[0], c + 1) ^ m1);
                const uint32_t o = (__funnelshift_l(Q0[2], Q0[1], c + 1) ^ m0) | (__funnelshift_l(Q1[2], Q1[1], c + 1) ^ m1);
                PMC[c] = c < real_cols ? (T)(((uint64_t)h << 32) | o) : ~T(0);
                XA[c] = band_prefix(T(0), mw - (colbase + c) + B0);
            }
        }
        if (active && l == G - 1) {
#pragma unroll
            for (int w = 0; w <= NW; ++w) {
                uint32_t a, b;
                load32(bw.tseq, bw.tblk, (int64_t)bw.ti + 32 * w, a, b);
                stage[w] = a;
                stage[(NW + 1) + w] = b;
                load32(bw.pseq, bw.pblk, (int64_t)bw.pj + 32 * w, a, b);
                stage[2 * (NW + 1) + w] = a;
                stage[3 * (NW + 1) + w] = b;
            }
        }
    }

    // ---- GenASM-DC in the band, rows in a pipeline over the lanes of each pair
    uint32_t done_mask = __ballot_sync(kFull, l == G - 1 && !active);
    int d_opt = -1;
    T bottom = T(0);
    for (int st = 0; done_mask != tbl_all; ++st) {
        const int d = st - l;
        const bool dc_done = (done_mask >> tbl) & 1u;
        T v;
        if (BW == 1) {
            v = (T)__shfl_up_sync(kFull, (uint32_t)bottom, 1);
        } else {
            const uint32_t hi = __shfl_up_sync(kFull, (uint32_t)((uint64_t)bottom >> 32), 1);
            const uint32_t lo = __shfl_up_sync(kFull, (uint32_t)bottom, 1);
            v = (T)(((uint64_t)hi << 32) | lo);
        }
        // lane 0 starts from column W_max, whose bits j < m_w - d are 1
        T pR = (l == 0) ? band_prefix(T(0), mw - d - WMAX + B0) : v;
        bool found = false;
        if (!dc_done && d >= 0 && d <= dmax) {
            uint32_t *rowp = band_row(d) + colbase * COLW;
#pragma unroll
            for (int c = C - 1; c >= 0; --c) {
                const T R = XA[c] & (pR | PMC[c]);
                if (lane_stores) store_band(rowp + c * COLW, R);
                // next row: S = V[i+1][d], D = V[i+1][d] >> 1, I = V[i][d] << 1 (1s shifted in)
                XA[c] = pR & shr1_fill(pR) & shl1_fill(R);
                pR = R;
            }
            bottom = pR;
            found = (l == G - 1) && (((pR >> (BITS - 1 - B0)) & T(1)) == T(0));
        }
        const uint32_t fmask = __ballot_sync(kFull, found);
        const int dl = st - (G - 1);  // row finished by the traceback lane
        if (!dc_done && ((fmask >> tbl) & 1u) && d_opt < 0) d_opt = dl;
        done_mask |= fmask;
        if (dl >= dmax) done_mask = tbl_all;
    }

    // ---- windows beyond the band: full-width DC (Algorithm 1 on NW words)
    const uint32_t full_mask = __ballot_sync(kFull, l == G - 1 && active && d_opt < 0 && k >= band_rows<BW>());
    const bool full = (full_mask >> tbl) & 1u;
    if (full_mask)
        full_width_dc<G, NW>(bw.pseq, bw.pblk, bw.pj, bw.tseq, bw.tblk, bw.ti, nw, mw, k, l, tbl, tbl_all, full_mask,
                             lane_stores, fb + ((int64_t)colbase * PPW + g) * NW, ncolp * PPW * NW, d_opt);
    d_opt_out = d_opt;
    full_out = full;
}

// GenASM-TB of one window, one lane per pair; every lane of `mask` calls it (the loop is warp
// uniform over those lanes). The pair's band rows are column-interleaved with the other pairs of
// a warp of G-lane pairs (pair index g) in `tab` / `spill`, its full-width rows in `fb`, its
// staged bases at `stage`. Emits the window's CIGAR runs, counts the window in the statistics and
// advances the cursors by what it consumed.
template <int G, int NWW, int BW>
__device__ __forceinline__ void band_window_tb(const AlignParams &p, uint32_t mask, bool active, int d_opt,
                                               bool full, int nw, int mw, const uint32_t *stage,
                                               const uint32_t *tab, const uint32_t *spill, const uint32_t *fb,
                                               int g, CigarOut &out, int &ti, int &pj, bool &failed,
                                               int64_t &st_rows, int64_t &st_cells, int32_t &st_windows) {
    constexpr int NW = NWW;
    constexpr int PPW = 32 / G;
    constexpr int COLW = PPW * BW;
    constexpr int B0 = band_diag<BW>();
    const int L = p.W - p.O, rcap = p.rcap, rstride = p.rstride;
    const int fb_row = p.ncol * PPW * NW;
    auto band_row = [&](int row) -> const uint32_t * {
        return row < rcap ? tab + (row * rstride + g) * BW : spill + ((row - rcap) * rstride + g) * BW;
    };
    const bool tb_live = active && d_opt >= 0;
    if (active) st_windows += 1;
    if (active && d_opt < 0) failed = true;
    if (tb_live) {
        st_rows += d_opt + 1;
        st_cells += (int64_t)(d_opt + 1) * nw;
    }
    const uint32_t *T0s = stage, *T1s = stage + (NW + 1);
    const uint32_t *P0s = stage + 2 * (NW + 1), *P1s = stage + 3 * (NW + 1);
    // windows of 64 bases: the four planes in 64-bit registers (a match run never reaches past
    // the window, so the zeros shifted in are never compared); wider windows read the stage
    uint64_t qT0 = 0, qT1 = 0, qP0 = 0, qP1 = 0;
    if (NW == 2) {
        qT0 = ((uint64_t)T0s[0] << 32) | T0s[1];
        qT1 = ((uint64_t)T1s[0] << 32) | T1s[1];
        qP0 = ((uint64_t)P0s[0] << 32) | P0s[1];
        qP1 = ((uint64_t)P1s[0] << 32) | P1s[1];
    }
    int i = 0, j = 0, d = d_opt;
    bool going = tb_live && (j < mw && i < L && j < L);
    while (__any_sync(mask, going)) {
        if (going) {
            const int lim = min(min(nw - i, mw - j), min(L - i, L - j));
            uint32_t x;
            if (NW == 2)
                x = (uint32_t)(((qT0 << i) ^ (qP0 << j)) >> 32) | (uint32_t)(((qT1 << i) ^ (qP1 << j)) >> 32);
            else
                x = (stage_ext(T0s, i) ^ stage_ext(P0s, j)) | (stage_ext(T1s, i) ^ stage_ext(P1s, j));
            const int z = __clz(x);
            const int run = min(z, lim);
            out.emit_maybe(kOpEq, run);
            i += run;
            j += run;
            const bool cont = j < mw && i < L && j < L;
            const bool edit = cont && !(z == 32 && run < lim);
            if (edit && d <= 0) {  // no edge can leave row 0 here (Theorem 1)
                atomicOr(p.status, 1);
                failed = true;
                going = false;
            } else if (edit) {
                const bool tx = i < nw;
                const bool j1 = j + 1 < mw;
                const int lim_r = mw - (d - 1);  // bits < lim_r of the right column R[n][d-1] are 1
                const int r = d - 1;
                const bool ld1 = tx && i + 1 < nw;
                // t1 = bits j, j+1 of entry (i+1, d-1); r0b = bit j+1 of entry (i, d-1)
                uint32_t t1, r0b;
                if (!full) {
                    const uint32_t *rp = band_row(r) + i * COLW;
                    const int kk = j - i + B0;  // band bit of (i, j); 0..2 B0 on the path
                    if (BW == 1) {
                        const uint32_t v1 = ld1 ? rp[COLW] : 0u;
                        const uint32_t v0 = tx ? rp[0] : 0u;
                        const uint64_t q1 = (1ull << 63) | ((uint64_t)v1 << 31);  // band bit kk-1 at position kk
                        t1 = (uint32_t)((q1 << kk) >> 62);
                        r0b = (uint32_t)((((uint64_t)v0 << 32) << (kk + 1)) >> 63);
                    } else {
                        const uint64_t v1 = ld1 ? load_band64(rp + COLW) : 0ull;
                        const uint64_t v0 = tx ? load_band64(rp) : 0ull;
                        const uint32_t lo = kk == 0 ? 1u : (uint32_t)((v1 >> (64 - kk)) & 1ull);  // bit kk-1
                        t1 = (lo << 1) | (uint32_t)((v1 >> (63 - kk)) & 1ull);
                        r0b = (uint32_t)((v0 >> (62 - kk)) & 1ull);
                    }
                } else {
                    const uint32_t *fp = fb + (int64_t)r * fb_row + (i * PPW + g) * NW;
                    t1 = ld1 ? entry_bits2<NW>(fp + PPW * NW, j) : 0u;
                    r0b = tx ? (entry_bits2<NW>(fp, j) & 1u) : 0u;
                }
                const uint32_t r1j = ld1 ? (t1 >> 1) : (j < lim_r ? 1u : 0u);
                const uint32_t r1j1 = !j1 ? 0u : (ld1 ? (t1 & 1u) : (j + 1 < lim_r ? 1u : 0u));
                const uint32_t r0j1 = !j1 ? 0u : (tx ? r0b : (j + 1 < lim_r ? 1u : 0u));
                const uint32_t bS = tx ? r1j1 : 1u;
                const uint32_t bI = r0j1;
                const uint32_t bD = tx ? r1j : 1u;
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

template <int G, int NWW, int BW>
__global__ void __launch_bounds__(64, (BandMinBlocks<G, NWW, BW>::value)) align_band_kernel(const AlignParams p) {
    constexpr int PPW = 32 / G;
    constexpr int NW = NWW;
    static_assert((32 * NWW / G) * G == 32 * NWW && 32 * NWW / G <= 32 && 32 % G == 0, "unsupported shape");

    extern __shared__ __align__(16) uint32_t smem[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int g = lane / G;
    const int l = lane - g * G;
    const int tbl = g * G + G - 1;  // traceback lane of this pair (owns column 0)
    const int W = p.W;
    uint32_t tbl_all = 0;
#pragma unroll
    for (int q = 0; q < PPW; ++q) tbl_all |= 1u << (q * G + G - 1);

    uint32_t *tab = smem + (int64_t)wib * p.smem_words_per_warp;
    uint32_t *stage = tab + p.table_words_per_warp + g * (4 * (NW + 1));
    const int64_t gw = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    uint32_t *spill = p.spill + gw * p.spill_words_per_pair;
    // full-width fallback rows: [row][column][pair][NW words]
    uint32_t *fb = p.fb ? p.fb + gw * p.fb_words_per_warp : nullptr;

    Slot s;
    slot_init(s, gw * PPW + g, p.slots_per_warp > 0 && g >= p.slots_per_warp);
    int64_t q_lo, q_hi;
    slot_range(p, q_lo, q_hi);
    CigarOut out;
    out.dst = nullptr;
    out.cap = 0;
    out.n = 0;
    out.cur = 0u;
    out.edits = 0;
    for (;;) {
        slot_fetch<G>(p, s, out, l, g, tbl, nwarps * PPW, q_lo, q_hi);
        if (!__any_sync(kFull, s.active)) break;
        BandWindow bw;
        bw.active = s.active;
        bw.nw = bw.active ? min(W, s.n - s.ti) : 0;
        bw.mw = bw.active ? min(W, s.m - s.pj) : 0;
        bw.tblk = bw.active ? s.tblk : 0;
        bw.pblk = bw.active ? s.pblk : 0;
        bw.tseq = s.tseq;
        bw.pseq = s.pseq;
        bw.ti = s.ti;
        bw.pj = s.pj;
        int d_opt;
        bool full;
        band_window_dc<G, NWW, BW>(p, bw, l, g, tbl, tbl_all, tab, spill, fb, stage, d_opt, full);
        __syncwarp();  // entries written by every lane are visible to the traceback lane
        if (l == G - 1)
            band_window_tb<G, NWW, BW>(p, tbl_all, bw.active, d_opt, full, bw.nw, bw.mw, stage, tab, spill, fb, g, out,
                                  s.ti, s.pj, s.failed, s.st_rows, s.st_cells, s.st_windows);
        slot_window_done<G>(p, s, out, l, tbl);
    }
}

// ---------------------------------------------------------------- warp-specialised banded kernel
//
// A block holds kWsDcWarps DC warps and one traceback warp. Each DC warp owns two sets of eight
// pair slots (4 lanes per pair) and alternates between them: while the traceback warp traces set
// A of every DC warp (32 pairs, one lane each), the DC warps compute the next window of set B.
// The hand-offs are mbarriers in shared memory: full[w][x] (the 32 lanes of DC warp w arrive when
// set x's rows and d_opt are written) and empty[w][x] (the traceback warp's 8 lanes for warp w
// arrive when set x is traced and its cursors advanced). Every wait is bounded; on a time-out the
// warp sets status bit 3 and returns as a whole.

constexpr int kWsDcWarps = 4;
constexpr int kWsSlotFree = 0, kWsSlotActive = 1, kWsSlotFresh = 2, kWsSlotDone = 3;

// One pair slot of a set, in shared memory: the DC warp refills it, the traceback warp advances it.
struct WsSlot {
    int64_t toff, poff;         // sequence offsets (bases)
    int64_t cig_base, cig_cap;  // the pair's CIGAR scratch
    int64_t st_rows, st_cells;
    long long t_start;
    int32_t pair, state, n, m, ti, pj, d_opt, full;
    int32_t cig_n, edits, st_windows, failed;
    uint32_t cig_cur, pad;
};

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_addr(bar))
                 : "memory");
}

// Wait for the completion of the phase of parity `parity`. limit == 0: up to 2^24 polls with
// mbarrier.try_wait (which may suspend the thread for a while between polls); limit > 0: up to
// `limit` polls with the non-suspending mbarrier.test_wait, so a wait that nothing completes ends
// after a bounded, short time. False when the polls ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity, int limit) {
    const uint32_t a = smem_addr(bar);
    if (limit > 0) {
        for (int it = 0; it < limit; ++it) {
            uint32_t ok;
            asm volatile(
                "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
                : "=r"(ok)
                : "r"(a), "r"(parity)
                : "memory");
            if (ok) return true;
        }
        return false;
    }
    for (int it = 0; it < (1 << 24); ++it) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(a), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

__global__ void __launch_bounds__(32 * (kWsDcWarps + 1), 3) align_ws_kernel(const AlignParams p) {
    constexpr int G = 4, PPW = 8;
    extern __shared__ __align__(16) uint32_t smem[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int set_words = p.smem_words_per_warp;  // rows + stage of one set
    WsSlot *slots = reinterpret_cast<WsSlot *>(smem + (int64_t)2 * kWsDcWarps * set_words);  // [w][x][g]
    int32_t *set_done = reinterpret_cast<int32_t *>(slots + 2 * kWsDcWarps * PPW);           // [w][x]
    uint64_t *bars = reinterpret_cast<uint64_t *>(set_done + 2 * kWsDcWarps);                // full[w][x], empty[w][x]
    uint64_t *full_bar = bars, *empty_bar = bars + 2 * kWsDcWarps;
    const int W = p.W;
    int64_t q_lo, q_hi;
    slot_range(p, q_lo, q_hi);

    if (threadIdx.x == 0) {
        for (int b = 0; b < 2 * kWsDcWarps; ++b) {
            mbar_init(full_bar + b, 32);
            mbar_init(empty_bar + b, PPW);
            set_done[b] = 0;
        }
    }
    for (int t = threadIdx.x; t < 2 * kWsDcWarps * PPW; t += blockDim.x) {
        slots[t].state = kWsSlotFree;
        slots[t].pair = -1;
        slots[t].toff = slots[t].poff = 0;
        slots[t].n = slots[t].m = slots[t].ti = slots[t].pj = 0;
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    __syncthreads();

    auto set_tab = [&](int w, int x) { return smem + (int64_t)(w * 2 + x) * set_words; };
    auto set_scratch = [&](uint32_t *base, int64_t words, int w, int x) -> uint32_t * {
        return base ? base + (((int64_t)blockIdx.x * kWsDcWarps + w) * 2 + x) * words : nullptr;
    };

    if (wib < kWsDcWarps) {
        // ------------------------------------------------------------ DC warp
        const int w = wib;
        const int g = lane / G, l = lane - g * G, tbl = g * G + G - 1;
        uint32_t tbl_all = 0;
#pragma unroll
        for (int q = 0; q < PPW; ++q) tbl_all |= 1u << (q * G + G - 1);
        int rounds[2] = {0, 0};
        bool fin[2] = {false, false};
        for (int r = 0; !(fin[0] && fin[1]); ++r) {
            const int x = r & 1;
            if (fin[x]) continue;
            const bool timed_out = rounds[x] > 0 && !mbar_wait(empty_bar + w * 2 + x, (rounds[x] - 1) & 1, p.wait_limit);
            if (__any_sync(kFull, timed_out)) {  // the whole warp leaves together
                if (lane == 0) atomicOr(p.status, 8);
                return;
            }
            WsSlot &sl = slots[(w * 2 + x) * PPW + g];
            // refill: the pair's traceback lane takes the next pair from the queue
            if (l == G - 1 && sl.state == kWsSlotFree) {
                int next = -1;
                for (;;) {
                    const int64_t q = q_lo + atomicAdd(p.queue, 1);
                    if (q >= q_hi) break;
                    const int pr = p.order ? p.order[q] : (int)q;
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
                if (next < 0) {
                    sl.state = kWsSlotDone;
                } else {
                    sl.pair = next;
                    sl.n = p.text_len[next];
                    sl.m = p.pat_len[next];
                    sl.toff = p.text_off[next];
                    sl.poff = p.pat_off[next];
                    sl.ti = 0;
                    sl.pj = 0;
                    sl.t_start = clock64();
                    sl.state = kWsSlotFresh;
                }
            }
            __syncwarp();
            const int state = sl.state;
            const bool active = state == kWsSlotActive || state == kWsSlotFresh;
            if (!__any_sync(kFull, active)) {
                if (lane == 0) set_done[w * 2 + x] = 1;
                __syncwarp();
                mbar_arrive(full_bar + w * 2 + x);
                fin[x] = true;
                ++rounds[x];
                continue;
            }
            BandWindow bw;
            bw.active = active;
            bw.tseq = reinterpret_cast<const uint2 *>(p.texts + (sl.toff >> 4));
            bw.pseq = reinterpret_cast<const uint2 *>(p.patterns + (sl.poff >> 4));
            bw.ti = sl.ti;
            bw.pj = sl.pj;
            bw.nw = active ? min(W, sl.n - sl.ti) : 0;
            bw.mw = active ? min(W, sl.m - sl.pj) : 0;
            bw.tblk = active ? (sl.n + 31) >> 5 : 0;
            bw.pblk = active ? (sl.m + 31) >> 5 : 0;
            uint32_t *tab = set_tab(w, x);
            uint32_t *stage = tab + p.table_words_per_warp + g * (4 * 3);
            int d_opt;
            bool full;
            band_window_dc<G, 2, 1>(p, bw, l, g, tbl, tbl_all, tab, set_scratch(p.spill, p.spill_words_per_pair, w, x),
                              set_scratch(p.fb, p.fb_words_per_warp, w, x), stage, d_opt, full);
            if (l == G - 1) {
                sl.d_opt = d_opt;
                sl.full = full ? 1 : 0;
            }
            __syncwarp();
            mbar_arrive(full_bar + w * 2 + x);  // every lane: its rows, stage and slot writes are released
            ++rounds[x];
        }
    } else {
        // ------------------------------------------------------------ traceback warp
        const int w = lane / PPW, g = lane % PPW;
        int rounds[2] = {0, 0};
        bool fin[2] = {false, false};
        for (int r = 0; !__all_sync(kFull, fin[0] && fin[1]); ++r) {
            const int x = r & 1;
            const bool waited = !fin[x];
            const bool timed_out = waited && !mbar_wait(full_bar + w * 2 + x, rounds[x] & 1, p.wait_limit);
            if (__any_sync(kFull, timed_out)) {  // the whole warp leaves together
                if (lane == 0) atomicOr(p.status, 8);
                return;
            }
            const bool set_fin = waited && set_done[w * 2 + x] != 0;
            WsSlot &sl = slots[(w * 2 + x) * PPW + g];
            const int state = waited ? sl.state : kWsSlotDone;
            const bool active = !set_fin && (state == kWsSlotActive || state == kWsSlotFresh);
            CigarOut out;
            int ti = 0, pj = 0, nw = 0, mw = 0, d_opt = -1;
            bool full = false, failed = false;
            int64_t st_rows = 0, st_cells = 0;
            int32_t st_windows = 0;
            if (active) {
                if (state == kWsSlotFresh) {
                    const int64_t c0 = p.cigar_off[sl.pair];
                    sl.cig_base = c0;
                    sl.cig_cap = p.cigar_off[sl.pair + 1] - c0;
                    sl.cig_n = 0;
                    sl.cig_cur = 0u;
                    sl.edits = 0;
                    sl.failed = 0;
                    sl.st_rows = 0;
                    sl.st_cells = 0;
                    sl.st_windows = 0;
                }
                out.dst = p.cigar + sl.cig_base;
                out.cap = sl.cig_cap;
                out.n = sl.cig_n;
                out.cur = sl.cig_cur;
                out.edits = sl.edits;
                ti = sl.ti;
                pj = sl.pj;
                nw = min(W, sl.n - ti);
                mw = min(W, sl.m - pj);
                d_opt = sl.d_opt;
                full = sl.full != 0;
                failed = sl.failed != 0;
                st_rows = sl.st_rows;
                st_cells = sl.st_cells;
                st_windows = sl.st_windows;
            } else {
                out.dst = nullptr;
                out.cap = 0;
                out.n = 0;
                out.cur = 0u;
                out.edits = 0;
            }
            const uint32_t *tab = set_tab(w, x);
            band_window_tb<G, 2, 1>(p, kFull, active, d_opt, full, nw, mw, tab + p.table_words_per_warp + g * (4 * 3), tab,
                              set_scratch(p.spill, p.spill_words_per_pair, w, x),
                              set_scratch(p.fb, p.fb_words_per_warp, w, x), g, out, ti, pj, failed, st_rows, st_cells,
                              st_windows);
            if (active) {
                if (failed || pj >= sl.m) {
                    out.flush();
                    const int pair = sl.pair;
                    p.edit_counts[pair] = failed ? -1 : out.edits;
                    p.text_consumed[pair] = failed ? 0 : ti;
                    if (out.n > out.cap) atomicOr(p.status, 2);
                    p.cigar_lens[pair] = failed ? 0 : min(out.n, (int32_t)out.cap);
                    if (p.st_windows) p.st_windows[pair] = st_windows;
                    if (p.st_rows) p.st_rows[pair] = st_rows;
                    if (p.st_cells) p.st_cells[pair] = st_cells;
                    if (p.st_cycles) p.st_cycles[pair] = clock64() - sl.t_start;
                    sl.state = kWsSlotFree;
                } else {
                    sl.ti = ti;
                    sl.pj = pj;
                    sl.cig_n = out.n;
                    sl.cig_cur = out.cur;
                    sl.edits = out.edits;
                    sl.failed = 0;
                    sl.st_rows = st_rows;
                    sl.st_cells = st_cells;
                    sl.st_windows = st_windows;
                    sl.state = kWsSlotActive;
                }
            }
            __syncwarp();
            if (waited && !set_fin) mbar_arrive(empty_bar + w * 2 + x);
            if (set_fin) fin[x] = true;
            if (waited) ++rounds[x];
        }
    }
}

cudaError_t launch_ws_kernel(const AlignParams &p, int blocks, size_t smem, cudaStream_t st) {
    align_ws_kernel<<<blocks, 32 * (kWsDcWarps + 1), smem, st>>>(p);
    return cudaGetLastError();
}

cudaError_t occupancy_ws_kernel(size_t smem, int *per_sm) {
    return occupancy_raising_smem(align_ws_kernel, 32 * (kWsDcWarps + 1), smem, per_sm);
}

template <int G, int NWW, int BW>
cudaError_t launch_g(const AlignParams &p, int wpb, int blocks, size_t smem, cudaStream_t st) {
    align_band_kernel<G, NWW, BW><<<blocks, 32 * wpb, smem, st>>>(p);
    return cudaGetLastError();
}

template <int G, int NWW, int BW>
cudaError_t occupancy_g(int wpb, size_t smem, int *per_sm) {
    return occupancy_raising_smem(align_band_kernel<G, NWW, BW>, 32 * wpb, smem, per_sm);
}

}  // namespace kern

// Instantiations: (window words, band words, lanes) = (2, 1, 2|4|8), (2, 2, 4|8), (4, 2, 8|16).
cudaError_t launch_align_band(const AlignParams &p, int nww, int bw, int lanes, int wpb, int blocks, size_t smem,
                              cudaStream_t st) {
    switch (nww * 1000 + bw * 100 + lanes) {
        case 2102: return kern::launch_g<2, 2, 1>(p, wpb, blocks, smem, st);
        case 2104: return kern::launch_g<4, 2, 1>(p, wpb, blocks, smem, st);
        case 2108: return kern::launch_g<8, 2, 1>(p, wpb, blocks, smem, st);
        case 2204: return kern::launch_g<4, 2, 2>(p, wpb, blocks, smem, st);
        case 2208: return kern::launch_g<8, 2, 2>(p, wpb, blocks, smem, st);
        case 4208: return kern::launch_g<8, 4, 2>(p, wpb, blocks, smem, st);
        case 4216: return kern::launch_g<16, 4, 2>(p, wpb, blocks, smem, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t occupancy_band(int nww, int bw, int lanes, int wpb, size_t smem, int *per_sm) {
    switch (nww * 1000 + bw * 100 + lanes) {
        case 2102: return kern::occupancy_g<2, 2, 1>(wpb, smem, per_sm);
        case 2104: return kern::occupancy_g<4, 2, 1>(wpb, smem, per_sm);
        case 2108: return kern::occupancy_g<8, 2, 1>(wpb, smem, per_sm);
        case 2204: return kern::occupancy_g<4, 2, 2>(wpb, smem, per_sm);
        case 2208: return kern::occupancy_g<8, 2, 2>(wpb, smem, per_sm);
        case 4208: return kern::occupancy_g<8, 4, 2>(wpb, smem, per_sm);
        case 4216: return kern::occupancy_g<16, 4, 2>(wpb, smem, per_sm);
        default: return cudaErrorInvalidValue;
    }
}

bool supported_band(int nww, int bw, int lanes) {
    if (nww == 2 && bw == 1) return lanes == 1 || lanes == 2 || lanes == 4 || lanes == 8;
    if (nww == 2 && bw == 2) return lanes == 4 || lanes == 8;
    return nww == 4 && bw == 2 && (lanes == 8 || lanes == 16);
}

cudaError_t launch_align_ws(const AlignParams &p, int blocks, size_t smem, cudaStream_t st) {
    return kern::launch_ws_kernel(p, blocks, smem, st);
}

cudaError_t occupancy_ws(size_t smem, int *per_sm) { return kern::occupancy_ws_kernel(smem, per_sm); }

size_t ws_meta_bytes() {
    return sizeof(kern::WsSlot) * 2 * kern::kWsDcWarps * 8 + sizeof(int32_t) * 2 * kern::kWsDcWarps +
           sizeof(uint64_t) * 4 * kern::kWsDcWarps + 16;
}

}  // namespace scrooge
