// Banded GenASM alignment kernel with one lane per pair, for windows of 33..64
// bases (Scrooge, arXiv 2208.09985).
//
// Each lane aligns its own pair: it computes every column of its window, so a
// warp holds 32 pairs and needs no shuffles between the lanes of a pair, no
// row pipeline over lanes (hence no rows past a window's edit distance), and
// runs the traceback on all 32 lanes.
//
// Recurrence (as in align_band.cu): the DP entry of text column i and row d
// is kept as the 32 diagonals j - i = -15..16 around the main diagonal,
// V[i][d] (bit k <-> pattern position j = i + k - 15, MSB first), and
//     V[i][d] = X[i] & (V[i+1][d] | PMrel[i]),
//     X[i]    = V[i+1][d-1] & (V[i+1][d-1] >> 1) & (V[i][d-1] << 1),
// with 1s shifted in at the band edges. It is exact for windows whose edit
// distance is at most 15 (see align_band.cu); the others are recomputed at
// full width (Algorithm 1 on two words, Section 2.2.1) by groups of 16, 8 or
// 4 lanes (one window per group), whichever takes all of the warp's pending
// windows: usually there is one, and the whole warp waits for it.
//
// Registers hold the whole window: X (the part of the next row that comes
// from the current one) and PMrel for all 64 columns, both in complement
// form (a set bit means reachable), where the band edges shift in 0s and the
// two shifts of a cell are plain shifts. A row is 64 cells of one 3-input
// logic op on its dependency chain and two shifts and one logic op off it.
// The row is a single unrolled block: a second inlined copy of it (even one
// never executed) measured 45% slower.
//
// Storage (SENE, Section 2.4.1; DENT, Section 2.4.2). Only entries of the
// columns 0..W-O are stored (W-O+1 of them where the kernel is compiled for
// that count, else rounded up to 8), one word per cell. The last
// `rcap` rows of each lane are kept in a cycle of row slots in shared memory
// laid out [slot][column][lane], so every access of a lane falls on its own
// bank whatever its column. A row that is about to be overwritten is copied
// to a per-warp device area first ([row][column][lane]) by one TMA bulk copy
// issued a row ahead; the traceback reads those rows from L2. Stored entries are in
// complement form; the traceback inverts what it reads. ET (Section 2.4.3)
// stops a lane at the first row that reaches the window start, so the slots
// then hold rows d_opt-rcap+1 .. d_opt: the rows the traceback (Section
// 2.2.2) reads first, and usually the only ones it reads.
//
// Pair state (cursors, CIGAR output, the window's bases) lives in a per-warp
// table in shared memory, [field][lane], so it does not hold registers during
// the DP.
// Idle lanes take their next pairs together: one atomic on the work queue per
// warp and refill.
#include "align_kernel.cuh"

namespace scrooge {
namespace kern {

constexpr int kLB0 = 15;         // band bit of the main diagonal j == i
constexpr int kLBandRows = 16;   // rows d < 16 are exact in the band
constexpr int kLFbLanes = 4;     // lanes per window of the full-width fallback
constexpr int kLFbWin = 32 / kLFbLanes;  // fallback windows per pass
constexpr int kLaneIdle = 0, kLaneActive = 1, kLaneDone = 2;

// Per-pair statistics, when asked for, accumulate in the caller's arrays directly (a pair stays on
// one lane), so the table holds none of them.
struct LaneTable {
    int64_t toff[32], poff[32], cbase[32];
    int32_t pair[32], n[32], m[32], ti[32], pj[32], ccap[32], cn[32], edits[32], state[32];
    uint32_t ccur[32];
    // the current window's 64 text and pattern bases (both bit planes), staged by the set-up for
    // the traceback
    uint64_t qT0[32], qT1[32], qP0[32], qP1[32];
};
static_assert(sizeof(LaneTable) == kLaneTableBytes, "lane table size");

// v >> 1 and v << 1 in band order with a 1 shifted in (no path beyond the band edge)
__device__ __forceinline__ uint32_t lane_shr1(uint32_t v) { return __funnelshift_r(v, kFull, 1); }
__device__ __forceinline__ uint32_t lane_shl1(uint32_t v) { return __funnelshift_l(kFull, v, 1); }

// Bulk copies from shared to global memory (TMA, asynchronous): a row slot goes to the device area
// in one instruction of one lane. The callers order them against the row stores with __syncwarp.
__device__ __forceinline__ void bulk_copy_s2g(uint32_t *gdst, const uint32_t *ssrc, uint32_t bytes) {
    // the evicted rows are read back within a window: keep them in L2 ahead of streaming data
    uint64_t policy;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(policy));
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group.L2::cache_hint [%0], [%1], %2, %3;" ::"l"(gdst),
                 "r"((uint32_t)__cvta_generic_to_shared(ssrc)), "r"(bytes), "l"(policy));
    asm volatile("cp.async.bulk.commit_group;");
}
// The copies issued so far have read their source (it may be overwritten).
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;"); }
// The copies issued so far are complete (their destination may be read).
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;"); }

__device__ __forceinline__ int64_t shfl64(int64_t v, int src) {
    const int lo = __shfl_sync(kFull, (int)(uint32_t)v, src);
    const int hi = __shfl_sync(kFull, (int)(uint32_t)((uint64_t)v >> 32), src);
    return (int64_t)(((uint64_t)(uint32_t)hi << 32) | (uint32_t)lo);
}

// Idle lanes take pairs until every lane is active or the work is exhausted:
// from the device queue over `order` (persistent launch; one atomic per warp and
// round) or from a fixed stride over the input (plain launch). Pairs with an
// empty pattern are finished here.
__device__ __forceinline__ void lane_fetch(const AlignParams &p, LaneTable &lt, int lane, int64_t q_lo, int64_t q_hi,
                                           int64_t &next_static, int64_t stride) {
    for (;;) {
        const bool need = lt.state[lane] == kLaneIdle;
        const uint32_t needm = __ballot_sync(kFull, need);
        if (!needm) return;
        int64_t sl = 0;
        if (p.queue) {
            const int leader = __ffs(needm) - 1;
            int base = 0;
            if (lane == leader) base = atomicAdd(p.queue, __popc(needm));
            base = __shfl_sync(kFull, base, leader);
            sl = q_lo + base + __popc(needm & ((1u << lane) - 1u));
        } else if (need) {
            sl = next_static;
            next_static += stride;
        }
        if (need) {
            if (sl >= q_hi) {
                lt.state[lane] = kLaneDone;
            } else {
                const int pr = p.order ? p.order[sl] : (int)sl;
                if (p.pat_len[pr] > 0) {
                    lt.pair[lane] = pr;
                    lt.n[lane] = p.text_len[pr];
                    lt.m[lane] = p.pat_len[pr];
                    lt.toff[lane] = p.text_off[pr];
                    lt.poff[lane] = p.pat_off[pr];
                    lt.ti[lane] = 0;
                    lt.pj[lane] = 0;
                    const int64_t c0 = p.cigar_off[pr];
                    lt.cbase[lane] = c0;
                    const int64_t cap = p.cigar_off[pr + 1] - c0;
                    lt.ccap[lane] = (int32_t)(cap < 0x7fffffff ? cap : 0x7fffffff);
                    lt.cn[lane] = 0;
                    lt.ccur[lane] = 0u;
                    lt.edits[lane] = 0;
                    if (p.st_windows) p.st_windows[pr] = 0;
                    if (p.st_rows) p.st_rows[pr] = 0;
                    if (p.st_cells) p.st_cells[pr] = 0;
                    if (p.st_cycles) p.st_cycles[pr] = -(int64_t)clock64();  // the finish adds its clock
                    lt.state[lane] = kLaneActive;
                } else {
                    p.edit_counts[pr] = 0;
                    p.text_consumed[pr] = 0;
                    p.cigar_lens[pr] = 0;
                    if (p.st_windows) p.st_windows[pr] = 0;
                    if (p.st_rows) p.st_rows[pr] = 0;
                    if (p.st_cells) p.st_cells[pr] = 0;
                    if (p.st_cycles) p.st_cycles[pr] = 0;
                }
            }
        }
        __syncwarp();
    }
}

// One band row of a lane's window, columns 63 down to 0, in complement form (a set bit means
// the entry is reachable: C = ~V). pC enters as the column right of the window and leaves as
// column 0. With the complement the band edges shift in 0s, so both shifts are plain shifts:
//     C[i][d] = CX[i] | (C[i+1][d] & CPM[i]),
//     CX[i]   = C[i+1][d-1] | (C[i+1][d-1] >> 1) | (C[i][d-1] << 1)   (the next row's part).
// Stores the stored columns to `rowp` (this lane's first word of the row slot) when `st`.
template <int NCOL>
__device__ __forceinline__ void lane_dc_row(uint32_t (&CX)[64], const uint32_t (&CPM)[64], uint32_t &pC, bool st,
                                            uint32_t *rowp) {
#pragma unroll
    for (int c = 63; c >= 0; --c) {
        const uint32_t C = CX[c] | (pC & CPM[c]);
        if (c < NCOL && st) rowp[c * 32] = C;
        // next row: S = C[i+1][d], D = C[i+1][d] >> 1, I = C[i][d] << 1
        CX[c] = pC | (pC >> 1) | (C << 1);
        pC = C;
    }
}

// GenASM-TB of the windows of the lanes with `part`, each lane on its own pair. Band rows
// come from the slot cycle (`ring`, rows above d_opt - rcap) or the evicted rows
// (`spill`), each pointer already at this lane's word; full-width rows of a fallback
// window (fbg >= 0) from its group in `fb`. Emits the CIGAR runs, advances the pair's
// cursors and statistics in the lane table, and finishes the pair when its pattern is
// consumed or the window failed.
template <int NCOL>
__device__ __forceinline__ void lane_window_tb(const AlignParams &p, LaneTable &lt, int lane, bool part, int d_opt,
                                               int fbg, int nw, int mw, const uint32_t *ring, const uint32_t *spill,
                                               const uint32_t *fb, int fbw, int rcap, bool stats) {
    constexpr int ROWW = NCOL * 32;
    const int L = p.W - p.O;
    const int fb_row = p.fb_ncol * fbw * 2;
    const int ti = part ? lt.ti[lane] : 0, pj = part ? lt.pj[lane] : 0;
    const int m = part ? lt.m[lane] : 0;
    // the window's 64 text and pattern bases in 64-bit registers (a match run never
    // reaches past the window, so the zeros beyond the sequence ends are never compared)
    uint64_t qT0 = 0, qT1 = 0, qP0 = 0, qP1 = 0;
    CigarOut out;
    out.dst = nullptr;
    out.cap = 0;
    out.n = 0;
    out.cur = 0u;
    out.edits = 0;
    if (part) {
        qT0 = lt.qT0[lane];
        qT1 = lt.qT1[lane];
        qP0 = lt.qP0[lane];
        qP1 = lt.qP1[lane];
        out.dst = p.cigar + lt.cbase[lane];
        out.cap = lt.ccap[lane];
        out.n = lt.cn[lane];
        out.cur = lt.ccur[lane];
        out.edits = lt.edits[lane];
    }
    const bool live = part && d_opt >= 0;
    bool failed = part && d_opt < 0;
    int i = 0, j = 0, d = d_opt;
    int rs = 0;  // slot of row d - 1 in the cycle
    if (live && fbg < 0 && d_opt >= 1) {
        rs = d_opt - 1;
        while (rs >= rcap) rs -= rcap;
    }
    const int ring_lo = d_opt - rcap;  // rows above this are in the slot cycle
    bool going = live && (j < mw && i < L && j < L);
    while (__any_sync(kFull, going)) {
        if (going) {
            const int lim = min(min(nw - i, mw - j), min(L - i, L - j));
            const uint32_t x =
                (uint32_t)(((qT0 << i) ^ (qP0 << j)) >> 32) | (uint32_t)(((qT1 << i) ^ (qP1 << j)) >> 32);
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
                if (fbg < 0) {
                    const int kk = j - i + kLB0;  // band bit of (i, j); 0..30 on the path
                    // stored in complement form; evicted rows were written by bulk copies, which do not
                    // pass through this SM's L1, so they are read from L2 (ld.global.cg)
                    uint32_t v1 = 0u, v0 = 0u;
                    if (r > ring_lo) {
                        const uint32_t *rp = ring + rs * ROWW + i * 32;
                        if (ld1) v1 = ~rp[32];
                        if (tx) v0 = ~rp[0];
                    } else {
                        const uint32_t *gp = spill + (int64_t)r * ROWW + i * 32;
                        if (ld1) v1 = ~__ldcg(gp + 32);
                        if (tx) v0 = ~__ldcg(gp);
                    }
                    const uint64_t q1 = (1ull << 63) | ((uint64_t)v1 << 31);  // band bit kk-1 at position kk
                    t1 = (uint32_t)((q1 << kk) >> 62);
                    r0b = (uint32_t)((((uint64_t)v0 << 32) << (kk + 1)) >> 63);
                } else {
                    const uint32_t *fp = fb + (int64_t)r * fb_row + (i * fbw + fbg) * 2;
                    t1 = ld1 ? entry_bits2<2>(fp + fbw * 2, j) : 0u;
                    r0b = tx ? (entry_bits2<2>(fp, j) & 1u) : 0u;
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
                    rs = rs == 0 ? rcap - 1 : rs - 1;
                    going = j < mw && i < L && j < L;
                }
            } else {
                going = cont;
            }
        }
    }
    if (!part) return;
    if (stats) {
        const int pair = lt.pair[lane];
        if (p.st_windows) p.st_windows[pair] += 1;
        if (live && p.st_rows) p.st_rows[pair] += d_opt + 1;
        if (live && p.st_cells) p.st_cells[pair] += (int64_t)(d_opt + 1) * nw;
    }
    const int nti = ti + (live ? i : 0), npj = pj + (live ? j : 0);
    if (failed || npj >= m) {
        out.flush();
        const int pair = lt.pair[lane];
        p.edit_counts[pair] = failed ? -1 : out.edits;
        p.text_consumed[pair] = failed ? 0 : nti;
        if (out.n > out.cap) atomicOr(p.status, 2);  // capacity too small for this pair
        p.cigar_lens[pair] = failed ? 0 : min(out.n, (int32_t)out.cap);
        if (p.st_cycles) p.st_cycles[pair] += (int64_t)clock64();
        lt.state[lane] = kLaneIdle;
    } else {
        lt.ti[lane] = nti;
        lt.pj[lane] = npj;
        lt.cn[lane] = out.n;
        lt.ccur[lane] = out.cur;
        lt.edits[lane] = out.edits;
    }
}

// Full-width DC (Algorithm 1 on two words) of the windows of the lanes in `take` (at most 32 / FG,
// lowest lanes first), each by a group of FG lanes; group g's rows go to window slot g of the
// fallback rows ([row][column][32 / FG slots][2 words]). Returns, on each lane of `take`, its
// window's edit distance (-1: none up to k).
template <int FG>
__device__ __forceinline__ int lane_fallback(const AlignParams &p, uint32_t take, int lane, int ti, int pj, int nw,
                                             int mw, int64_t tblk, int64_t pblk, const uint2 *tseq,
                                             const uint2 *pseq, uint32_t *fb) {
    constexpr int slots = 32 / FG;
    // lane FG-1 of every group
    constexpr uint32_t tb_lanes = FG == 16 ? 0x80008000u : (FG == 8 ? 0x80808080u : 0x88888888u);
    static_assert(FG == 4 || FG == 8 || FG == 16, "fallback groups of 4, 8 or 16 lanes");
    const int g = lane / FG, l = lane % FG;
    uint32_t x = take;
    for (int t = 0; t < g && x; ++t) x &= x - 1u;
    const int src = x ? __ffs(x) - 1 : -1;  // lane whose window group g computes
    const int sl = src >= 0 ? src : lane;
    const int f_ti = __shfl_sync(kFull, ti, sl), f_pj = __shfl_sync(kFull, pj, sl);
    const int f_nw = __shfl_sync(kFull, nw, sl), f_mw = __shfl_sync(kFull, mw, sl);
    const int64_t f_tblk = shfl64(tblk, sl), f_pblk = shfl64(pblk, sl);
    const uint2 *f_tseq = reinterpret_cast<const uint2 *>(shfl64((int64_t)(uintptr_t)tseq, sl));
    const uint2 *f_pseq = reinterpret_cast<const uint2 *>(shfl64((int64_t)(uintptr_t)pseq, sl));
    const uint32_t full_mask = __ballot_sync(kFull, l == FG - 1 && src >= 0);
    const int colbase = (FG - 1 - l) * (64 / FG);
    int dfb = -1;
    full_width_dc<FG, 2>(f_pseq, src >= 0 ? f_pblk : 0, f_pj, f_tseq, src >= 0 ? f_tblk : 0, f_ti, f_nw, f_mw, p.k, l,
                         g * FG + FG - 1, tb_lanes, full_mask, colbase < p.fb_ncol,
                         fb + ((int64_t)colbase * slots + g) * 2, p.fb_ncol * slots * 2, dfb);
    const bool mine = (take >> lane) & 1u;
    const int myg = __popc(take & ((1u << lane) - 1u));
    return __shfl_sync(kFull, dfb, (mine ? myg : 0) * FG + FG - 1);
}

template <int NCOL>
__global__ void __launch_bounds__(64, 4) align_lane_kernel(const AlignParams p) {
    constexpr int ROWW = NCOL * 32;  // words of one stored row of a warp
    extern __shared__ __align__(16) uint32_t smem[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    uint32_t *wsm = smem + (int64_t)wib * p.smem_words_per_warp;
    LaneTable &lt = *reinterpret_cast<LaneTable *>(wsm);
    uint32_t *ring = wsm + kLaneTableBytes / 4 + lane;  // row slot s, column c: ring[s * ROWW + c * 32]
    const int64_t gw = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    uint32_t *spill = p.spill + gw * p.spill_words_per_pair + lane;  // evicted row r: spill[r * ROWW + c * 32]
    uint32_t *fb = p.fb ? p.fb + gw * p.fb_words_per_warp : nullptr;
    const int W = p.W, k = p.k, rcap = p.rcap;
    const int dmax = min(k, kLBandRows - 1);  // deepest row the band computes
    const bool stats = p.st_windows || p.st_rows || p.st_cells || p.st_cycles;
    int64_t q_lo, q_hi;
    slot_range(p, q_lo, q_hi);
    int64_t next_static = gw * 32 + lane;
    lt.state[lane] = (p.slots_per_warp > 0 && lane >= p.slots_per_warp) ? kLaneDone : kLaneIdle;
    __syncwarp();

    for (;;) {
        lane_fetch(p, lt, lane, q_lo, q_hi, next_static, stride);
        const bool active = lt.state[lane] == kLaneActive;
        if (!__any_sync(kFull, active)) break;
        const int n = active ? lt.n[lane] : 0, m = active ? lt.m[lane] : 0;
        const int ti = active ? lt.ti[lane] : 0, pj = active ? lt.pj[lane] : 0;
        const int nw = active ? min(W, n - ti) : 0, mw = active ? min(W, m - pj) : 0;
        const int64_t tblk = active ? (n + 31) >> 5 : 0, pblk = active ? (m + 31) >> 5 : 0;
        const uint2 *tseq = reinterpret_cast<const uint2 *>(p.texts + (active ? lt.toff[lane] >> 4 : 0));
        const uint2 *pseq = reinterpret_cast<const uint2 *>(p.patterns + (active ? lt.poff[lane] >> 4 : 0));

        // ---- window set-up, in complement form: CX of row 0 and ~PMrel[text[i]] for the 64 columns
        uint32_t XA[64], PMC[64];
        {
            uint32_t Ta0, Ta1, Tb0, Tb1, Pa0, Pa1, Pb0, Pb1, Pc0, Pc1;
            load32(tseq, tblk, ti, Ta0, Ta1);
            load32(tseq, tblk, (int64_t)ti + 32, Tb0, Tb1);
            // pattern planes from pj - 16: column c's band starts c + 1 bases in
            load32(pseq, pblk, (int64_t)pj - 16, Pa0, Pa1);
            load32(pseq, pblk, (int64_t)pj + 16, Pb0, Pb1);
            load32(pseq, pblk, (int64_t)pj + 48, Pc0, Pc1);
            // row 0: bit k of column c is set iff k + c < m_w + 15 (pattern positions j < m_w)
            const uint32_t S0 = prefix_mask(mw + kLB0), S1 = prefix_mask(mw + kLB0 - 32),
                           S2 = prefix_mask(mw + kLB0 - 64);
#pragma unroll
            for (int c = 0; c < 64; ++c) {
                const uint32_t t0 = c < 32 ? Ta0 : Tb0, t1 = c < 32 ? Ta1 : Tb1;
                const uint32_t m0 = (uint32_t)((int32_t)(t0 << (c & 31)) >> 31);  // text base c, each plane
                const uint32_t m1 = (uint32_t)((int32_t)(t1 << (c & 31)) >> 31);
                const uint32_t w0 = c < 32 ? __funnelshift_lc(Pb0, Pa0, c + 1) : __funnelshift_lc(Pc0, Pb0, c - 31);
                const uint32_t w1 = c < 32 ? __funnelshift_lc(Pb1, Pa1, c + 1) : __funnelshift_lc(Pc1, Pb1, c - 31);
                PMC[c] = ~((w0 ^ m0) | (w1 ^ m1));  // bit j set: pattern base j equals text base c
                XA[c] = ~(c < 32 ? __funnelshift_l(S1, S0, c) : __funnelshift_l(S2, S1, c - 32));
            }
            // the window's bases for the traceback: text from ti, pattern from pj (64 each)
            lt.qT0[lane] = ((uint64_t)Ta0 << 32) | Tb0;
            lt.qT1[lane] = ((uint64_t)Ta1 << 32) | Tb1;
            lt.qP0[lane] = ((uint64_t)__funnelshift_l(Pb0, Pa0, 16) << 32) | __funnelshift_l(Pc0, Pb0, 16);
            lt.qP1[lane] = ((uint64_t)__funnelshift_l(Pb1, Pa1, 16) << 32) | __funnelshift_l(Pc1, Pb1, 16);
            if (__any_sync(kFull, nw < 64)) {
                // columns at or past the end of the text window match nothing
                const uint32_t v0 = ~prefix_mask(nw), v1 = ~prefix_mask(nw - 32);
#pragma unroll
                for (int c = 0; c < 64; ++c) PMC[c] &= ~(uint32_t)((int32_t)((c < 32 ? v0 : v1) << (c & 31)) >> 31);
            }
        }

        // ---- GenASM-DC in the band, row by row, each lane until its window's edit distance
        int d_opt = -1;
        bool busy = active;
        int slot = 0;  // row slot of row d
        // Before a row slot is reused its row goes to the device area ([row][column][lane], the slot's own
        // layout) by a bulk copy that lane 0 issues one row ahead, so the copy runs behind a row of
        // work; a lane whose pair is done copies a stale row, which its traceback never reads.
        uint32_t *ring_w = ring - lane, *spill_w = spill - lane;
        for (int d = 0; d <= dmax; ++d) {
            if (!__any_sync(kFull, busy)) break;
            if (d >= rcap) {
                if (rcap == 1) {
                    // one slot: row d - 1 is copied out just before row d overwrites it, once every
                    // lane's store of it is done and ordered before the copy's read
                    __syncwarp();
                    if (lane == 0) {
                        asm volatile("fence.proxy.async.shared::cta;");
                        bulk_copy_s2g(spill_w + (int64_t)(d - 1) * ROWW, ring_w, ROWW * 4);
                    }
                }
                if (lane == 0) bulk_wait_read();  // the slot of row d - rcap has been read
                __syncwarp();
            }
            if (rcap > 1 && d + 1 >= rcap && d + 1 <= dmax) {
                // the slot that row d + 1 takes holds row d + 1 - rcap, complete since an earlier row
                const int s1 = slot + 1 == rcap ? 0 : slot + 1;
                __syncwarp();
                if (lane == 0) {
                    asm volatile("fence.proxy.async.shared::cta;");
                    bulk_copy_s2g(spill_w + (int64_t)(d + 1 - rcap) * ROWW, ring_w + s1 * ROWW, ROWW * 4);
                }
            }
            // the column right of the window: bits j < m_w - d of R[n][d] are 1 (0 in complement)
            uint32_t pC = ~prefix_mask(mw - d - 64 + kLB0);
            uint32_t *rowp = ring + slot * ROWW;
            lane_dc_row<NCOL>(XA, PMC, pC, busy, rowp);
            if (busy && ((pC >> (31 - kLB0)) & 1u) != 0u) {
                d_opt = d;
                busy = false;
            }
            slot = slot + 1 == rcap ? 0 : slot + 1;
        }
        if (lane == 0) {
            bulk_wait_all();  // the evicted rows are in place before the traceback reads them
            asm volatile("fence.proxy.async.global;" ::: "memory");  // and visible to generic loads
        }
        __syncwarp();

        // ---- windows beyond the band: full-width DC by groups of lanes, 16 lanes per window when at
        // most 2 are pending (the usual case: one), 8 when at most 4, else 4 lanes per window for up
        // to 8 of them; a window beyond that waits (keeps its cursors) and is recomputed next round
        const uint32_t pend = __ballot_sync(kFull, active && d_opt < 0 && k >= kLBandRows);
        int fbg = -1, fbw = kLFbWin;
        bool wait = false;
        if (pend) {
            const int npend = __popc(pend);
            fbw = npend <= 32 / 16 ? 32 / 16 : (npend <= 32 / 8 ? 32 / 8 : kLFbWin);
            uint32_t take = 0, rest = pend;
            for (int t = 0; t < fbw && rest; ++t) {
                const uint32_t b = rest & (0u - rest);
                take |= b;
                rest ^= b;
            }
            const int got =
                fbw == 32 / 16 ? lane_fallback<16>(p, take, lane, ti, pj, nw, mw, tblk, pblk, tseq, pseq, fb)
                : fbw == 32 / 8 ? lane_fallback<8>(p, take, lane, ti, pj, nw, mw, tblk, pblk, tseq, pseq, fb)
                                : lane_fallback<kLFbLanes>(p, take, lane, ti, pj, nw, mw, tblk, pblk, tseq, pseq, fb);
            if ((take >> lane) & 1u) {
                d_opt = got;
                fbg = __popc(take & ((1u << lane) - 1u));
            }
            wait = ((rest >> lane) & 1u) != 0u;
        }

        // ---- GenASM-TB, every lane on its own pair
        lane_window_tb<NCOL>(p, lt, lane, active && !wait, d_opt, fbg, nw, mw, ring, spill, fb, fbw, rcap, stats);
        __syncwarp();
    }
}

template <int NCOL>
cudaError_t launch_nc(const AlignParams &p, int wpb, int blocks, size_t smem, cudaStream_t st) {
    align_lane_kernel<NCOL><<<blocks, 32 * wpb, smem, st>>>(p);
    return cudaGetLastError();
}

template <int NCOL>
cudaError_t occupancy_nc(int wpb, size_t smem, int *per_sm) {
    return occupancy_raising_smem(align_lane_kernel<NCOL>, 32 * wpb, smem, per_sm);
}

}  // namespace kern

cudaError_t launch_align_lane(const AlignParams &p, int wpb, int blocks, size_t smem, cudaStream_t st) {
    switch (p.ncol) {
#define SCROOGE_LANE_NCOL(n) \
    case n: return kern::launch_nc<n>(p, wpb, blocks, smem, st);
        SCROOGE_LANE_NCOLS
#undef SCROOGE_LANE_NCOL
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t occupancy_lane(int ncol, int wpb, size_t smem, int *per_sm) {
    switch (ncol) {
#define SCROOGE_LANE_NCOL(n) \
    case n: return kern::occupancy_nc<n>(wpb, smem, per_sm);
        SCROOGE_LANE_NCOLS
#undef SCROOGE_LANE_NCOL
        default: return cudaErrorInvalidValue;
    }
}

bool lane_ncol_supported(int ncol) {
    switch (ncol) {
#define SCROOGE_LANE_NCOL(n) \
    case n: return true;
        SCROOGE_LANE_NCOLS
#undef SCROOGE_LANE_NCOL
        default: return false;
    }
}

}  // namespace scrooge
