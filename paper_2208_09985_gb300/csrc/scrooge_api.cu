// C ABI of the library: contexts, argument checks, packing and launches.
// The operations are described in include/scrooge.h.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <thread>
#include <vector>

#include "scrooge_ctx.h"

namespace scrooge {

bool align_supported(int words, int lanes) {
    switch (words) {
        case 1: return lanes == 1 || lanes == 2 || lanes == 4;
        case 2: return lanes == 2 || lanes == 4 || lanes == 8;
        case 4: return lanes == 8 || lanes == 16;
        case 0: return supported_band(2, 1, lanes);
        case 3: return supported_band(4, 2, lanes);
        default: return false;
    }
}
}  // namespace scrooge


using namespace scrooge;

extern "C" {

int scrooge_create(scrooge_ctx **out, int cuda_device, void *cuda_stream) {
    if (!out) return SCROOGE_E_INVAL;
    *out = nullptr;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return SCROOGE_E_CUDA;
    }
    if (cuda_device < 0 || cuda_device >= ndev) return SCROOGE_E_INVAL;
    scrooge_ctx *c = new (std::nothrow) scrooge_ctx();
    if (!c) return SCROOGE_E_NOMEM;
    c->device = cuda_device;
    c->stream = (cudaStream_t)cuda_stream;
    if ((e = cudaSetDevice(cuda_device)) != cudaSuccess) {
        delete c;
        return SCROOGE_E_CUDA;
    }
    cudaDeviceProp prop;
    if ((e = cudaGetDeviceProperties(&prop, cuda_device)) != cudaSuccess) {
        delete c;
        return SCROOGE_E_CUDA;
    }
    c->sm_count = prop.multiProcessorCount;
    c->smem_optin = prop.sharedMemPerBlockOptin;
    *out = c;
    return SCROOGE_OK;
}

int scrooge_destroy(scrooge_ctx *c) {
    if (!c) return SCROOGE_OK;
    cudaSetDevice(c->device);
    DevBuf *all[] = {&c->spill,   &c->status,  &c->in_text, &c->in_pat,   &c->in_toff,  &c->in_tlen,
                     &c->in_poff,   &c->in_plen, &c->out_ec,  &c->out_tc,   &c->out_cig,  &c->out_off,
                     &c->scr_runs,  &c->scr_off, &c->scr_len, &c->scr_cap,  &c->scan_tmp, &c->queue,
                     &c->model,     &c->grad,    &c->adam_m1, &c->adam_m2,  &c->loss,     &c->l_feat,
                     &c->l_pred,    &c->l_key,   &c->l_order, &c->l_tmp,    &c->t_rows,   &c->fallback, &c->spill2,
                     &c->spill3,    &c->fallback2, &c->fallback3, &c->split_bounds, &c->out_cig_parts[0],
                     &c->out_cig_parts[1], &c->out_cig_parts[2]};
    if (c->graph) cudaGraphExecDestroy(c->graph);
    if (c->stream2) cudaStreamDestroy(c->stream2);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    if (c->ev_join3) cudaEventDestroy(c->ev_join3);
    if (c->stream3) cudaStreamDestroy(c->stream3);
    if (c->split_copy) cudaStreamDestroy(c->split_copy);
    if (c->split_a) cudaStreamDestroy(c->split_a);
    if (c->split_b) cudaStreamDestroy(c->split_b);
    for (cudaEvent_t ev : c->split_ev)
        if (ev) cudaEventDestroy(ev);
    for (DevBuf *b : all) release(*b);
    delete c;
    return SCROOGE_OK;
}

const char *scrooge_last_error(const scrooge_ctx *c) { return c ? c->err.c_str() : "no context"; }

int scrooge_set_stream(scrooge_ctx *c, void *cuda_stream) {
    if (!c) return SCROOGE_E_INVAL;
    c->stream = (cudaStream_t)cuda_stream;
    return SCROOGE_OK;
}

int scrooge_set_wait_limit(scrooge_ctx *c, int32_t polls) {
    if (!c || polls < 0) return SCROOGE_E_INVAL;
    c->wait_limit = polls;
    return SCROOGE_OK;
}

int scrooge_set_host_overlap(scrooge_ctx *c, int32_t on) {
    if (!c) return SCROOGE_E_INVAL;
    c->host_split = on != 0;
    return SCROOGE_OK;
}

int32_t scrooge_get_host_overlap(const scrooge_ctx *c) { return c ? (c->host_split ? 1 : 0) : -1; }

int scrooge_debug_fail_next_allocs(scrooge_ctx *c, int32_t count) {
    if (!c || count < 0) return SCROOGE_E_INVAL;
    c->fail_allocs = count;
    return SCROOGE_OK;
}

int64_t scrooge_packed_words(int64_t n_bases) {
    if (n_bases < 0) return -1;
    return ((n_bases + 63) / 64) * 4;
}

int scrooge_pack_2bit(const uint8_t *seqs, const int64_t *offsets, int32_t n_seqs, int ascii, uint32_t *packed,
                      int64_t packed_words, int64_t *packed_offsets, int32_t *lengths) {
    if (n_seqs < 0 || (n_seqs > 0 && (!seqs || !offsets || !packed || !packed_offsets || !lengths)))
        return SCROOGE_E_INVAL;
    std::vector<int64_t> wstart((size_t)n_seqs + 1, 0);
    for (int32_t s = 0; s < n_seqs; ++s) {
        const int64_t len = offsets[s + 1] - offsets[s];
        if (len < 0 || len > INT32_MAX) return SCROOGE_E_INVAL;
        wstart[s + 1] = wstart[s] + scrooge_packed_words(len);
    }
    if (wstart[n_seqs] > packed_words) return SCROOGE_E_INVAL;
    uint8_t code_of[256];
    memset(code_of, 255, sizeof code_of);
    if (ascii) {
        const char *a = "ACGT", *b = "acgt";
        for (int x = 0; x < 4; ++x) code_of[(uint8_t)a[x]] = code_of[(uint8_t)b[x]] = (uint8_t)x;
    } else {
        for (int x = 0; x < 4; ++x) code_of[x] = (uint8_t)x;
    }
    int bad = 0;
    auto work = [&](int32_t lo, int32_t hi, int *badflag) {
        for (int32_t s = lo; s < hi; ++s) {
            const uint8_t *q = seqs + offsets[s];
            const int64_t len = offsets[s + 1] - offsets[s];
            uint32_t *dst = packed + wstart[s];
            const int64_t nw = wstart[s + 1] - wstart[s];
            for (int64_t blk = 0; blk < nw / 2; ++blk) {
                uint32_t p0 = 0, p1 = 0;
                for (int t = 0; t < 32; ++t) {
                    const int64_t pos = blk * 32 + t;
                    if (pos >= len) break;
                    const uint8_t c = code_of[q[pos]];
                    if (c > 3) {
                        *badflag = 1;
                        return;
                    }
                    p0 |= (uint32_t)(c & 1u) << (31 - t);
                    p1 |= (uint32_t)((c >> 1) & 1u) << (31 - t);
                }
                dst[2 * blk] = p0;
                dst[2 * blk + 1] = p1;
            }
            packed_offsets[s] = wstart[s] * 16;
            lengths[s] = (int32_t)len;
        }
    };
    const int64_t total = offsets[n_seqs] - offsets[0];
    unsigned nth = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    if (total < (1 << 22) || n_seqs < 64) nth = 1;
    std::vector<std::thread> th;
    std::vector<int> bads(nth, 0);
    const int32_t per = (n_seqs + (int32_t)nth - 1) / (int32_t)nth;
    for (unsigned t = 0; t < nth; ++t) {
        const int32_t lo = (int32_t)t * per, hi = std::min(n_seqs, lo + per);
        if (lo >= hi) break;
        if (nth == 1) work(lo, hi, &bads[t]);
        else th.emplace_back(work, lo, hi, &bads[t]);
    }
    for (auto &x : th) x.join();
    for (int b : bads) bad |= b;
    return bad ? SCROOGE_E_INVAL : SCROOGE_OK;
}

int scrooge_set_kernel_config(scrooge_ctx *c, int32_t words, int32_t lanes, int32_t rows, int32_t wpb) {
    if (!c) return SCROOGE_E_INVAL;
    const int ix = kcfg_index(words);
    if (ix < 0 || !align_supported(words, lanes) || rows < 1 || rows > 129 || wpb < 1 || wpb > 2)
        return fail(c, SCROOGE_E_INVAL, "unsupported kernel config words=%d lanes=%d rows=%d warps=%d", words,
                    lanes, rows, wpb);
    c->kcfg[ix] = {lanes, rows, wpb};
    return SCROOGE_OK;
}

int scrooge_get_kernel_config(const scrooge_ctx *c, int32_t words, int32_t *lanes, int32_t *rows, int32_t *wpb) {
    if (!c) return SCROOGE_E_INVAL;
    const int ix = kcfg_index(words);
    if (ix < 0) return SCROOGE_E_INVAL;
    if (lanes) *lanes = c->kcfg[ix].lanes;
    if (rows) *rows = c->kcfg[ix].rows;
    if (wpb) *wpb = c->kcfg[ix].wpb;
    return SCROOGE_OK;
}

int scrooge_set_bucket_config(scrooge_ctx *c, int32_t bucket, int32_t kind, int32_t lanes, int32_t rows,
                              int32_t wpb) {
    if (!c) return SCROOGE_E_INVAL;
    const bool ok_kind = kind == 0 ? align_supported(0, lanes) : (kind == 1 && align_supported(2, lanes));
    if (bucket < 0 || bucket > 1 || !ok_kind || rows < 1 || rows > 129 || wpb < 1 || wpb > 2)
        return fail(c, SCROOGE_E_INVAL, "unsupported bucket config bucket=%d kind=%d lanes=%d rows=%d warps=%d", bucket,
                    kind, lanes, rows, wpb);
    c->bucket_kind[bucket] = kind;
    c->bucket_cfg[bucket] = {lanes, rows, wpb};
    return SCROOGE_OK;
}

int scrooge_get_bucket_config(const scrooge_ctx *c, int32_t bucket, int32_t *kind, int32_t *lanes, int32_t *rows,
                              int32_t *wpb) {
    if (!c || bucket < 0 || bucket > 1) return SCROOGE_E_INVAL;
    if (kind) *kind = c->bucket_kind[bucket];
    if (lanes) *lanes = c->bucket_cfg[bucket].lanes;
    if (rows) *rows = c->bucket_cfg[bucket].rows;
    if (wpb) *wpb = c->bucket_cfg[bucket].wpb;
    return SCROOGE_OK;
}

int scrooge_set_learned_order(scrooge_ctx *c, int32_t on) {
    if (!c || (on != 0 && on != 1)) return SCROOGE_E_INVAL;
    c->learned_order_on = on != 0;
    return SCROOGE_OK;
}

int32_t scrooge_get_learned_order(const scrooge_ctx *c) { return c ? (c->learned_order_on ? 1 : 0) : -1; }

int scrooge_set_heavy_class(scrooge_ctx *c, int32_t load_class) {
    if (!c || load_class < 0 || load_class > 16) return SCROOGE_E_INVAL;
    c->heavy_class = load_class;
    return SCROOGE_OK;
}

int32_t scrooge_get_heavy_class(const scrooge_ctx *c) { return c ? c->heavy_class : -1; }

int scrooge_set_long_class(scrooge_ctx *c, int32_t work_class) {
    if (!c || work_class < 0 || work_class > 16) return SCROOGE_E_INVAL;
    c->long_class = work_class;
    return SCROOGE_OK;
}

int32_t scrooge_get_long_class(const scrooge_ctx *c) { return c ? c->long_class : -1; }

int scrooge_last_launch_shape(const scrooge_ctx *c, int64_t *shape, int32_t n) {
    if (!c || !shape || n < 1) return SCROOGE_E_INVAL;
    memcpy(shape, c->last_shape, sizeof(int64_t) * (size_t)std::min(n, 13));
    return SCROOGE_OK;
}

int scrooge_set_timing_events(scrooge_ctx *c, void *start, void *stop) {
    if (!c || (!start) != (!stop)) return SCROOGE_E_INVAL;
    c->t_start = (cudaEvent_t)start;
    c->t_stop = (cudaEvent_t)stop;
    return SCROOGE_OK;
}

int32_t scrooge_last_kernel_count(const scrooge_ctx *c) { return c ? c->last_kernels : -1; }

int scrooge_set_order(scrooge_ctx *c, const int32_t *order, int32_t n_pairs) {
    if (!c || n_pairs < 0 || (order && n_pairs == 0)) return SCROOGE_E_INVAL;
    c->order = order;
    c->order_n = order ? n_pairs : 0;
    return SCROOGE_OK;
}

int scrooge_set_stats(scrooge_ctx *c, int32_t *windows, int64_t *rows, int64_t *cells, int64_t *cycles) {
    if (!c) return SCROOGE_E_INVAL;
    c->st_windows = windows;
    c->st_rows = rows;
    c->st_cells = cells;
    c->st_cycles = cycles;
    return SCROOGE_OK;
}

}  // extern "C"

namespace {

// One alignment-kernel launch: which kernel, its shape and its parameters.
struct LaunchPlan {
    bool band = false, sene = true, ws = false, lane = false;
    int words = 0, nww = 2, bw = 1, G = 0, wpb = 1, blocks = 0;
    size_t smem = 0;
    TableShape ts{};
    AlignParams p{};
};

// Plan of the banded kernel with one lane per pair (windows of 33..64 bases, 32-diagonal band).
int make_lane_plan(scrooge_ctx *c, const AlignParams &base, uint32_t flags, DevBuf &spill, DevBuf &fallback,
                   const KernelConfig &kc, LaunchPlan &out) {
    const int W = base.W, O = base.O, k = base.k, L = W - O;
    const bool dent = !(flags & SCROOGE_NO_DENT);
    AlignParams p = base;
    // stored columns: 0..W-O with DENT (exactly, where the kernel is compiled for that count, else
    // rounded up to 8), else all W
    const int want = dent ? std::min(L + 1, W) : W;
    const int ncol = lane_ncol_supported(want) ? want : std::min(64, ((want + 7) / 8) * 8);
    p.et = 1;
    p.sene = 1;
    p.ncol = ncol;
    p.sw = 1;
    p.rstride = ncol * 32;
    p.ring = k + 1;
    const int rows_needed = std::min(k, band_rows_for(1) - 1) + 1;
    int rcap = std::min(kc.rows, rows_needed);
    int wpb = kc.wpb;
    auto warp_words = [&](int rows) { return (int64_t)kLaneTableBytes / 4 + (int64_t)rows * ncol * 32; };
    while (rcap > 1 && (size_t)wpb * warp_words(rcap) * 4 > c->smem_optin) --rcap;
    while (wpb > 1 && (size_t)wpb * warp_words(rcap) * 4 > c->smem_optin) --wpb;
    p.rcap = rcap;
    p.table_words_per_warp = (int32_t)(rcap * ncol * 32);
    p.smem_words_per_warp = (int32_t)warp_words(rcap);
    const size_t smem = (size_t)wpb * p.smem_words_per_warp * 4;
    int per_sm = 0;
    cudaError_t e = occupancy_lane(ncol, wpb, smem, &per_sm);
    if (e != cudaSuccess) return cuda_fail(c, e, "occupancy query");
    if (per_sm < 1) return fail(c, SCROOGE_E_INVAL, "kernel config does not fit on an SM (smem %zu B)", smem);
    const int64_t warps = ((int64_t)p.n_pairs + 31) / 32;
    const int64_t want_blocks = (warps + wpb - 1) / wpb;
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(want_blocks, (int64_t)per_sm * c->sm_count));
    p.slots_per_warp = 0;
    // rows evicted from the slot cycle: 0 .. rows_needed - 1 - rcap
    p.spill_words_per_pair = (int64_t)std::max(0, rows_needed - rcap) * ncol * 32;  // per warp
    int rc;
    if ((rc = ensure(c, spill, (size_t)blocks * wpb * (size_t)std::max<int64_t>(p.spill_words_per_pair, 4) * 4,
                     "DP row scratch")))
        return rc;
    p.spill = (uint32_t *)spill.p;
    p.fb = nullptr;
    p.fb_words_per_warp = 0;
    p.fb_ncol = table_shape(W, O, 2, 4, dent, true).ncol;  // full-width fallback: 4 lanes per window
    p.fb_words_per_warp = band_fallback_words(k, p.fb_ncol, 8, 2, 1);
    if (p.fb_words_per_warp > 0) {
        if ((rc = ensure(c, fallback, (size_t)blocks * wpb * (size_t)p.fb_words_per_warp * 4,
                         "full-width fallback scratch")))
            return rc;
        p.fb = (uint32_t *)fallback.p;
    }
    TableShape ts;
    ts.ncol = ncol;
    ts.swp = 1;
    ts.nv = 1;
    out.band = true;
    out.lane = true;
    out.nww = 2;
    out.bw = 1;
    out.ws = false;
    out.sene = true;
    out.words = 2;
    out.G = 1;
    out.wpb = wpb;
    out.blocks = blocks;
    out.smem = smem;
    out.ts = ts;
    out.p = p;
    return SCROOGE_OK;
}

// Shape of the kernel a call with these flags uses (banded or full width), sized for the device
// and the context's kernel settings; sizes the row scratch in `spill` (and the banded kernel's
// fallback area). Queue, order and status are set by the caller.
// slots > 0: a launch with that many pair slots per warp, one warp per block and three blocks per SM.
int make_plan(scrooge_ctx *c, const AlignParams &base, bool band, uint32_t flags, DevBuf &spill, DevBuf &fallback,
              int slots, LaunchPlan &out, const KernelConfig *settings = nullptr) {
    const int W = base.W, O = base.O, k = base.k;
    // the banded kernels: window words nww (their full-width fallback and staged bases), band words bw
    const int nww = W > 64 ? 4 : 2;
    const int bw = (W > 64 || (flags & SCROOGE_WIDE_BAND)) ? 2 : 1;
    const int words = band ? nww : words_for(W);
    const bool sene = !(flags & SCROOGE_NO_SENE);
    const bool dent = !(flags & SCROOGE_NO_DENT);
    const KernelConfig kc = settings ? *settings : c->kcfg[kcfg_index(band ? band_slot_for(W) : words)];
    // warp-specialised blocks: 64-base bands, persistent, four lanes per pair, not the long-pair launch
    const bool ws = band && nww == 2 && bw == 1 && slots == 0 && (flags & SCROOGE_WARP_SPECIALIZED) &&
                    (flags & SCROOGE_PERSISTENT);
    int G = ws ? 4 : kc.lanes;
    auto supported = [&](int lanes, int swp) {
        return words == 1 ? supported_w32(lanes, sene, swp)
                          : (words == 2 ? supported_w64(lanes, sene, swp) : supported_w128(lanes, sene, swp));
    };
    if (band && !supported_band(nww, bw, G)) G = nww == 2 ? 4 : 8;
    if (band && G == 1 && slots > 0) G = 4;  // a pair of its own per warp: the lanes of one pair share it
    // one lane per pair (align_lane.cu): stored columns rounded to 8, not to a lane chunk
    if (band && G == 1) return make_lane_plan(c, base, flags, spill, fallback, kc, out);
    TableShape ts = table_shape(W, O, words, G, dent, sene);
    if (band) ts.swp = bw;  // one band of bw 32-bit words per stored entry
    if (!band && !supported(G, ts.swp)) {  // the edge-storing ablation exists for the default lane count only
        G = words == 1 ? 2 : (words == 2 ? 4 : 8);
        ts = table_shape(W, O, words, G, dent, sene);
        if (!supported(G, ts.swp)) return fail(c, SCROOGE_E_INVAL, "no kernel for this W/O/flags combination");
    }
    AlignParams p = base;
    const int PPW = 32 / G, chunk = 32 * words / G;
    p.et = (flags & SCROOGE_NO_ET) ? 0 : 1;
    p.sene = sene ? 1 : 0;
    p.ncol = ts.ncol;
    p.sw = ts.swp;
    p.rstride = row_stride_cells(ts, PPW, chunk);
    // full-width kernels: rows in a cycle (DENT extended to rows) with SENE, DENT and ET. The banded
    // kernels keep all k+1 rows of their rare full-width fallback: the slot arithmetic in their
    // traceback loop cost more than the memory it saves.
    p.ring = band ? k + 1 : ext_dent_ring(W, O, k, G, sene && dent && p.et && !(flags & SCROOGE_NO_EXT_DENT));
    // rows the kernel may store: the band's rows (banded kernels), or the full-width row slots
    const int rows_needed = band ? std::min(k, band_rows_for(bw) - 1) + 1 : p.ring;
    int rcap = std::min(kc.rows, rows_needed);
    const int stage = stage_words_per_warp(words, PPW);
    int wpb = slots > 0 ? 1 : kc.wpb;
    // keep the block's shared memory within the opt-in limit (a warp-specialised block holds 8 sets)
    const int sets = ws ? kWsSets : wpb;
    const size_t meta = ws ? ws_meta_bytes() : 0;
    while (rcap > 1 && (size_t)sets * (table_words_per_warp(rcap, ts, PPW, chunk) + stage) * 4 + meta > c->smem_optin)
        --rcap;
    while (!ws && wpb > 1 && (size_t)wpb * (table_words_per_warp(rcap, ts, PPW, chunk) + stage) * 4 > c->smem_optin)
        --wpb;
    p.rcap = rcap;
    p.table_words_per_warp = (int32_t)table_words_per_warp(rcap, ts, PPW, chunk);
    p.smem_words_per_warp = p.table_words_per_warp + stage;
    const size_t smem = (size_t)(ws ? kWsSets : wpb) * p.smem_words_per_warp * 4 + meta;
    int per_sm = 0;
    cudaError_t e = ws ? occupancy_ws(smem, &per_sm)
                  : band ? occupancy_band(nww, bw, G, wpb, smem, &per_sm)
                         : (words == 1 ? occupancy_w32(G, sene, ts.swp, wpb, smem, &per_sm)
                                       : (words == 2 ? occupancy_w64(G, sene, ts.swp, wpb, smem, &per_sm)
                                                     : occupancy_w128(G, sene, ts.swp, wpb, smem, &per_sm)));
    if (e != cudaSuccess) return cuda_fail(c, e, "occupancy query");
    if (per_sm < 1) return fail(c, SCROOGE_E_INVAL, "kernel config does not fit on an SM (smem %zu B)", smem);
    const int64_t groups = ((int64_t)p.n_pairs + PPW - 1) / PPW;
    const int64_t want_blocks = ws ? (groups + kWsSets - 1) / kWsSets : (groups + wpb - 1) / wpb;
    int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(want_blocks, (int64_t)per_sm * c->sm_count));
    if (slots > 0) blocks = (int)std::min<int64_t>((int64_t)per_sm * c->sm_count, 3LL * c->sm_count);
    p.slots_per_warp = slots;
    const int spill_rows = std::max(0, rows_needed - rcap);
    p.spill_words_per_pair = table_words_per_warp(spill_rows, ts, PPW, chunk);  // per warp
    const size_t spill_bytes = (size_t)blocks * sets * (size_t)std::max<int64_t>(p.spill_words_per_pair, 4) * 4;
    int rc;
    if ((rc = ensure(c, spill, spill_bytes, "DP row scratch"))) return rc;
    p.spill = (uint32_t *)spill.p;
    p.fb = nullptr;
    p.fb_words_per_warp = 0;
    if (band) {
        p.fb_words_per_warp = band_fallback_words(k, ts.ncol, PPW, nww, bw);
        if (p.fb_words_per_warp > 0) {
            if ((rc = ensure(c, fallback, (size_t)blocks * sets * (size_t)p.fb_words_per_warp * 4,
                             "full-width fallback scratch")))
                return rc;
            p.fb = (uint32_t *)fallback.p;
        }
    }
    out.band = band;
    out.nww = nww;
    out.bw = bw;
    out.ws = ws;
    out.sene = sene;
    out.words = words;
    out.G = G;
    out.wpb = wpb;
    out.blocks = blocks;
    out.smem = smem;
    out.ts = ts;
    out.p = p;
    return SCROOGE_OK;
}

cudaError_t launch_plan(const LaunchPlan &lp, cudaStream_t st) {
    if (lp.ws) return launch_align_ws(lp.p, lp.blocks, lp.smem, st);
    if (lp.lane) return launch_align_lane(lp.p, lp.wpb, lp.blocks, lp.smem, st);
    if (lp.band) return launch_align_band(lp.p, lp.nww, lp.bw, lp.G, lp.wpb, lp.blocks, lp.smem, st);
    switch (lp.words) {
        case 1: return launch_align_w32(lp.p, lp.G, lp.sene, lp.ts.swp, lp.wpb, lp.blocks, lp.smem, st);
        case 2: return launch_align_w64(lp.p, lp.G, lp.sene, lp.ts.swp, lp.wpb, lp.blocks, lp.smem, st);
        default: return launch_align_w128(lp.p, lp.G, lp.sene, lp.ts.swp, lp.wpb, lp.blocks, lp.smem, st);
    }
}

constexpr int kMaxParts = 4;

// Layout of a host-pointer batch: every pair's offsets must be >= 0 multiples of 64 bases and its
// lengths >= 0. Gives the packed words of the text and pattern arrays that the pairs [0, ends[i])
// reach, for each of the `nparts` ascending part ends (the last is n), and the CIGAR scratch runs
// (n + m + 1 per pair). Large batches are checked by several host threads. Returns the first pair
// that breaks the layout, or -1.
struct HostLayout {
    int64_t text_upto[kMaxParts] = {}, pat_upto[kMaxParts] = {}, runs = 0;
};

int32_t host_layout(const int64_t *to, const int32_t *tl, const int64_t *po, const int32_t *pl, int32_t n,
                    const int32_t *ends, int nparts, HostLayout &out) {
    // per chunk of pairs: the words each part's pairs in the chunk reach, the runs, the first bad pair
    struct Part {
        int64_t text[kMaxParts] = {}, pat[kMaxParts] = {}, runs = 0;
        int32_t bad = -1;
    };
    auto run = [&](int32_t lo, int32_t hi, Part &r) {
        int pi = 0;
        for (int32_t q = lo; q < hi; ++q) {
            while (q >= ends[pi]) ++pi;
            const int64_t x = to[q], y = po[q];
            const int32_t u = tl[q], v = pl[q];
            if (x < 0 || y < 0 || (x & 63) || (y & 63) || u < 0 || v < 0) {
                r.bad = q;
                return;
            }
            r.text[pi] = std::max(r.text[pi], x / 16 + scrooge_packed_words(u));
            r.pat[pi] = std::max(r.pat[pi], y / 16 + scrooge_packed_words(v));
            r.runs += (int64_t)u + v + 1;
        }
    };
    const unsigned hw = std::thread::hardware_concurrency();
    int nt = n >= 65536 ? (int)std::min(8u, std::max(1u, hw)) : 1;
    std::vector<Part> rs(nt);
    if (nt > 1) {
        std::vector<std::thread> th;
        try {
            for (int t = 0; t < nt; ++t)
                th.emplace_back(run, (int32_t)((int64_t)n * t / nt), (int32_t)((int64_t)n * (t + 1) / nt),
                                std::ref(rs[t]));
        } catch (...) {  // no threads: check on this one
            for (auto &x : th) x.join();
            th.clear();
            nt = 1;
            rs.assign(1, Part());
        }
        for (auto &x : th) x.join();
    }
    if (nt == 1) run(0, n, rs[0]);
    out = HostLayout();
    for (int t = 0; t < nt; ++t) {
        if (rs[t].bad >= 0) return rs[t].bad;  // chunks are in pair order: the first bad chunk holds the first bad pair
        for (int i = 0; i < nparts; ++i) {
            out.text_upto[i] = std::max(out.text_upto[i], rs[t].text[i]);
            out.pat_upto[i] = std::max(out.pat_upto[i], rs[t].pat[i]);
        }
        out.runs += rs[t].runs;
    }
    for (int i = 1; i < nparts; ++i) {  // words reached by every pair before the end of part i
        out.text_upto[i] = std::max(out.text_upto[i], out.text_upto[i - 1]);
        out.pat_upto[i] = std::max(out.pat_upto[i], out.pat_upto[i - 1]);
    }
    return -1;
}

constexpr int32_t kHostSplitMinPairs = 8192;

// Host-pointer persistent calls on large batches, in K = 2..4 parts of the pair range, each of at
// least a wave of the kernel's pair slots where the batch allows. Part i's sequences are copied
// while the parts before it run, and its outputs
// are gathered and copied back while the parts after it run, so only the first part's input copy
// and the last part's output copy are exposed. One kernel launch per part over its range of the
// persistent queue; parts alternate between two kernel streams, each with its own row scratch, so
// that part i + 1's blocks take the SMs that part i's blocks free. Each part's run offsets are
// scanned, gathered and rebased by the previous parts' total on the device. Same results as the
// one-launch path (the kernels align each pair independently).
int align_host_split(scrooge_ctx *c, const uint32_t *texts, const int64_t *text_offsets, const int32_t *text_lengths,
                     const uint32_t *patterns, const int64_t *pattern_offsets, const int32_t *pattern_lengths,
                     int32_t n_pairs, int32_t W, int32_t O, int32_t k, uint32_t flags, int32_t *edit_counts,
                     int32_t *text_consumed, uint32_t *cigar, int64_t cigar_capacity, int64_t *cigar_offsets) {
    const size_t np = (size_t)n_pairs;
    cudaError_t e;
    int rc;
    AlignParams p;
    memset(&p, 0, sizeof p);
    p.n_pairs = n_pairs;
    p.W = W;
    p.O = O;
    p.k = k;
    const bool band = use_band(W, flags);
    // parts of at least a wave of pair slots each, so that a part's launch fills the GPU
    LaunchPlan shape_plan;
    if ((rc = make_plan(c, p, band, flags, c->spill, c->fallback, 0, shape_plan))) return rc;
    const int64_t slots = (int64_t)shape_plan.blocks * shape_plan.wpb * (32 / shape_plan.G);
    const int K = (int)std::max<int64_t>(2, std::min<int64_t>(kMaxParts, n_pairs / std::max<int64_t>(slots, 1)));
    int32_t start[kMaxParts + 1];
    for (int i = 0; i <= K; ++i) start[i] = (int32_t)((int64_t)n_pairs * i / K);
    // layout check; the words of both sequence arrays that the parts up to each one need (prefixes)
    HostLayout lay;
    const int32_t bad =
        host_layout(text_offsets, text_lengths, pattern_offsets, pattern_lengths, n_pairs, start + 1, K, lay);
    if (bad >= 0)
        return fail(c, SCROOGE_E_INVAL, "pair %d: offsets must be >= 0 multiples of 64, lengths >= 0", bad);
    const int64_t text_words = lay.text_upto[K - 1], pat_words = lay.pat_upto[K - 1], scratch_runs = lay.runs;
    if ((rc = ensure(c, c->scr_off, (np + 1) * 8, "CIGAR scratch offsets")) ||
        (rc = ensure(c, c->scr_len, np * 4, "CIGAR run counts")) ||
        (rc = ensure(c, c->scan_tmp, (size_t)scan_temp_words((int64_t)np + 1) * 8, "scan scratch")) ||
        (rc = ensure(c, c->in_text, text_words * 4, "texts")) || (rc = ensure(c, c->in_pat, pat_words * 4, "patterns")) ||
        (rc = ensure(c, c->in_toff, np * 8, "text offsets")) || (rc = ensure(c, c->in_tlen, np * 4, "text lengths")) ||
        (rc = ensure(c, c->in_poff, np * 8, "pattern offsets")) ||
        (rc = ensure(c, c->in_plen, np * 4, "pattern lengths")) || (rc = ensure(c, c->out_ec, np * 4, "edit counts")) ||
        (rc = ensure(c, c->out_tc, np * 4, "text consumed")) ||
        (rc = ensure(c, c->out_off, (np + kMaxParts) * 8, "cigar offsets")) ||
        (rc = ensure(c, c->scr_cap, (np + 1) * 8, "CIGAR capacities")) ||
        (rc = ensure(c, c->scr_runs, (size_t)std::max<int64_t>(scratch_runs, 1) * 4, "CIGAR run scratch")) ||
        (rc = ensure(c, c->status, 64, "status")) || (rc = ensure(c, c->queue, 256, "work queues")) ||
        (rc = ensure(c, c->split_bounds, 2 * kMaxParts * 8, "range bounds")))
        return rc;
    if ((!c->split_copy && (e = cudaStreamCreateWithFlags(&c->split_copy, cudaStreamNonBlocking)) != cudaSuccess) ||
        (!c->split_a && (e = cudaStreamCreateWithFlags(&c->split_a, cudaStreamNonBlocking)) != cudaSuccess) ||
        (!c->split_b && (e = cudaStreamCreateWithFlags(&c->split_b, cudaStreamNonBlocking)) != cudaSuccess))
        return cuda_fail(c, e, "split streams");
    for (cudaEvent_t &ev : c->split_ev)
        if (!ev && (e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess)
            return cuda_fail(c, e, "split events");
    cudaStream_t st = c->stream, cs = c->split_copy, ks[2] = {c->split_a, c->split_b};
    cudaEvent_t ev_start = c->split_ev[0], ev_ready = c->split_ev[1], *ev_in = c->split_ev + 2,
                *ev_k = c->split_ev + 2 + kMaxParts, *ev_g = c->split_ev + 2 + 2 * kMaxParts;
    p.texts = (const uint32_t *)c->in_text.p;
    p.patterns = (const uint32_t *)c->in_pat.p;
    p.text_off = (const int64_t *)c->in_toff.p;
    p.text_len = (const int32_t *)c->in_tlen.p;
    p.pat_off = (const int64_t *)c->in_poff.p;
    p.pat_len = (const int32_t *)c->in_plen.p;
    p.edit_counts = (int32_t *)c->out_ec.p;
    p.text_consumed = (int32_t *)c->out_tc.p;
    p.cigar = (uint32_t *)c->scr_runs.p;
    p.cigar_off = (const int64_t *)c->scr_off.p;
    p.cigar_lens = (int32_t *)c->scr_len.p;
    p.st_windows = c->st_windows;
    p.st_rows = c->st_rows;
    p.st_cells = c->st_cells;
    p.st_cycles = c->st_cycles;
    LaunchPlan plans[2];
    if ((rc = make_plan(c, p, band, flags, c->spill, c->fallback, 0, plans[0])) ||
        (rc = make_plan(c, p, band, flags, c->spill2, c->fallback3, 0, plans[1])))
        return rc;
    {
        const LaunchPlan &pa = plans[0];
        const TableShape &ts = pa.ts;
        const int64_t shape[13] = {pa.band ? 0 : pa.words, pa.G, pa.p.rcap, pa.wpb, (int64_t)pa.smem, pa.blocks,
                                   pa.p.ncol, ts.swp, pa.p.table_words_per_warp * 4LL, pa.p.spill_words_per_pair * 4,
                                   pa.p.fb_words_per_warp * 4, 32 / pa.G, pa.p.ring};
        memcpy(c->last_shape, shape, sizeof shape);
    }
    // kernels: an alignment launch, a scan and a gather per part, and a rebase per part after the first
    c->last_kernels = 3 * K - 1;
    for (int i = 0; i < K; ++i) c->last_kernels += scan_kernel_count(start[i + 1] - start[i]);
    int64_t bounds_h[2 * kMaxParts];
    for (int i = 0; i < K; ++i) {
        bounds_h[2 * i] = start[i];
        bounds_h[2 * i + 1] = start[i + 1];
    }
    struct Copy {
        void *d;
        const void *h;
        size_t b;
    };
    // inputs: the per-pair arrays, then each part's new sequence words (prefixes of the arrays)
    if ((e = cudaEventRecord(ev_start, st)) != cudaSuccess || (e = cudaStreamWaitEvent(cs, ev_start, 0)) != cudaSuccess)
        return cuda_fail(c, e, "stream fork");
    const Copy per_pair[] = {{c->in_toff.p, text_offsets, np * 8},
                             {c->in_tlen.p, text_lengths, np * 4},
                             {c->in_poff.p, pattern_offsets, np * 8},
                             {c->in_plen.p, pattern_lengths, np * 4}};
    for (const Copy &x : per_pair)
        if ((e = cudaMemcpyAsync(x.d, x.h, x.b, cudaMemcpyHostToDevice, cs)) != cudaSuccess)
            return cuda_fail(c, e, "host-to-device copy");
    for (int i = 0; i < K; ++i) {
        const int64_t t0 = i ? lay.text_upto[i - 1] : 0, p0 = i ? lay.pat_upto[i - 1] : 0;
        const Copy seq[] = {{(uint32_t *)c->in_text.p + t0, texts + t0, (size_t)(lay.text_upto[i] - t0) * 4},
                            {(uint32_t *)c->in_pat.p + p0, patterns + p0, (size_t)(lay.pat_upto[i] - p0) * 4}};
        for (const Copy &x : seq)
            if (x.b && (e = cudaMemcpyAsync(x.d, x.h, x.b, cudaMemcpyHostToDevice, cs)) != cudaSuccess)
                return cuda_fail(c, e, "host-to-device copy");
        if ((e = cudaEventRecord(ev_in[i], cs)) != cudaSuccess) return cuda_fail(c, e, "event");
    }
    // run scratch layout and resets, once the per-pair arrays are in (they precede part 0's words)
    if ((e = cudaMemcpyAsync(c->split_bounds.p, bounds_h, sizeof(int64_t) * 2 * K, cudaMemcpyHostToDevice, st)) !=
            cudaSuccess ||
        (e = cudaStreamWaitEvent(st, ev_in[0], 0)) != cudaSuccess ||
        (e = launch_capacity(p.text_len, p.pat_len, n_pairs, (int64_t *)c->scr_cap.p, st)) != cudaSuccess ||
        (e = exclusive_scan(c->scr_cap.p, 1, n_pairs, (int64_t *)c->scr_off.p, (int64_t *)c->scan_tmp.p, st)) !=
            cudaSuccess ||
        (e = cudaMemsetAsync(c->status.p, 0, 4, st)) != cudaSuccess ||
        (e = cudaMemsetAsync(c->queue.p, 0, 256, st)) != cudaSuccess || (e = cudaEventRecord(ev_ready, st)) != cudaSuccess)
        return cuda_fail(c, e, "CIGAR scratch layout");
    // the parts' kernels, alternating between two streams (part i + 2 after part i)
    const int64_t *bounds = (const int64_t *)c->split_bounds.p;
    for (int i = 0; i < K; ++i) {
        LaunchPlan lp = plans[i & 1];
        lp.p.status = (int32_t *)c->status.p;
        lp.p.wait_limit = c->wait_limit;
        lp.p.order = nullptr;
        lp.p.queue = (int32_t *)c->queue.p + 16 * i;
        lp.p.range_lo = bounds + 2 * i;
        lp.p.range_hi = bounds + 2 * i + 1;
        cudaStream_t s = ks[i & 1];
        if ((e = cudaStreamWaitEvent(s, ev_in[i], 0)) != cudaSuccess || (e = cudaStreamWaitEvent(s, ev_ready, 0)) != cudaSuccess)
            return cuda_fail(c, e, "stream wait");
        if ((e = launch_plan(lp, s)) != cudaSuccess) return cuda_fail(c, e, "alignment kernel launch");
        if ((e = cudaEventRecord(ev_k[i], s)) != cudaSuccess) return cuda_fail(c, e, "event");
    }
    // each part's outputs, in order, while the later parts run: run offsets from 0 (into out_off
    // at start + i), gather below the capacity left, rebase by the previous part's end, copy back
    int64_t base = 0;  // runs of the parts before this one
    int32_t status_h = 0;
    for (int i = 0; i < K; ++i) {
        const int32_t lo = start[i], ni = start[i + 1] - start[i];
        int64_t *off_i = (int64_t *)c->out_off.p + lo + i;  // ni + 1 entries
        int64_t total_i = 0;
        if ((e = cudaStreamWaitEvent(st, ev_k[i], 0)) != cudaSuccess ||
            (e = exclusive_scan(p.cigar_lens + lo, 0, ni, off_i, (int64_t *)c->scan_tmp.p, st)) != cudaSuccess ||
            (e = cudaMemcpyAsync(&total_i, off_i + ni, 8, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
            (e = cudaStreamSynchronize(st)) != cudaSuccess)
            return cuda_fail(c, e, "CIGAR offsets");
        const int64_t keep_i = std::max<int64_t>(0, std::min(total_i, cigar_capacity - base));
        DevBuf &dense = i ? c->out_cig_parts[i - 1] : c->out_cig;
        if (keep_i > 0) {
            if ((rc = ensure(c, dense, (size_t)keep_i * 4, "cigar"))) return rc;
            if ((e = launch_compact(p.cigar, p.cigar_off + lo, p.cigar_lens + lo, off_i, ni, (uint32_t *)dense.p,
                                    keep_i, c->sm_count, st)) != cudaSuccess)
                return cuda_fail(c, e, "CIGAR gather");
        }
        if (i && (e = launch_add_base(off_i, (int64_t)ni + 1, off_i - 1, st)) != cudaSuccess)  // previous part's end
            return cuda_fail(c, e, "CIGAR offsets");
        if ((e = cudaEventRecord(ev_g[i], st)) != cudaSuccess || (e = cudaStreamWaitEvent(cs, ev_g[i], 0)) != cudaSuccess)
            return cuda_fail(c, e, "event");
        const bool last = i == K - 1;
        const Copy out[] = {{edit_counts + lo, p.edit_counts + lo, (size_t)ni * 4},
                            {text_consumed + lo, p.text_consumed + lo, (size_t)ni * 4},
                            {cigar_offsets + lo, off_i, ((size_t)ni + (last ? 1 : 0)) * 8},
                            {cigar + base, dense.p, (size_t)keep_i * 4},
                            {&status_h, c->status.p, last ? 4u : 0u}};
        for (const Copy &x : out)  // host destination in d, device source in h
            if (x.b && (e = cudaMemcpyAsync(x.d, x.h, x.b, cudaMemcpyDeviceToHost, cs)) != cudaSuccess)
                return cuda_fail(c, e, "device-to-host copy");
        base += total_i;
    }
    if ((e = cudaStreamSynchronize(cs)) != cudaSuccess || (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return cuda_fail(c, e, "stream synchronise");
    if (status_h & 8) return fail(c, SCROOGE_E_TIMEOUT, "a bounded device wait gave up (status %d)", status_h);
    if (status_h != 0) return fail(c, SCROOGE_E_INTERNAL, "kernel status %d", status_h);
    if (base > cigar_capacity)
        return fail(c, SCROOGE_E_CAPACITY, "CIGAR needs %lld runs, capacity %lld", (long long)base,
                    (long long)cigar_capacity);
    return SCROOGE_OK;
}

}  // namespace

extern "C" {

int scrooge_align_batch(scrooge_ctx *c, const uint32_t *texts, const int64_t *text_offsets,
                        const int32_t *text_lengths, const uint32_t *patterns, const int64_t *pattern_offsets,
                        const int32_t *pattern_lengths, int32_t n_pairs, int32_t W, int32_t O, int32_t k,
                        uint32_t flags, int32_t *edit_counts, int32_t *text_consumed, uint32_t *cigar,
                        int64_t cigar_capacity, int64_t *cigar_offsets) {
    if (!c) return SCROOGE_E_INVAL;
    c->err.clear();
    if (n_pairs < 0) return fail(c, SCROOGE_E_INVAL, "n_pairs < 0");
    if (W < 1 || W > 128) return fail(c, SCROOGE_E_INVAL, "W=%d outside 1..128", W);
    if (O < 0 || O >= W) return fail(c, SCROOGE_E_INVAL, "O=%d outside 0..W-1", O);
    if (k < 0 || k > W) return fail(c, SCROOGE_E_INVAL, "k=%d outside 0..W", k);
    if (cigar_capacity < 0) return fail(c, SCROOGE_E_INVAL, "cigar_capacity < 0");
    if (flags & SCROOGE_LEARNED) flags |= SCROOGE_PERSISTENT;
    if ((flags & SCROOGE_LEARNED) && !c->model_ready)
        return fail(c, SCROOGE_E_NOMODEL, "SCROOGE_LEARNED needs a model (scrooge_model_set or scrooge_model_train)");
    // the autotuner found that the model's order does not pay on this workload: input order
    if ((flags & SCROOGE_LEARNED) && !c->learned_order_on) flags &= ~(uint32_t)SCROOGE_LEARNED;
    if (!cigar_offsets) return fail(c, SCROOGE_E_INVAL, "null cigar_offsets");
    const bool dev = (flags & SCROOGE_DEVICE_PTRS) != 0;
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
    cudaStream_t st = c->stream;
    if (n_pairs == 0) {
        if (dev) {
            if ((e = cudaMemsetAsync(cigar_offsets, 0, 8, st)) != cudaSuccess) return cuda_fail(c, e, "memset");
            if ((flags & SCROOGE_SYNC) && (e = cudaStreamSynchronize(st)) != cudaSuccess)
                return cuda_fail(c, e, "stream synchronise");
        } else {
            cigar_offsets[0] = 0;
        }
        return SCROOGE_OK;
    }
    if (!texts || !text_offsets || !text_lengths || !patterns || !pattern_offsets || !pattern_lengths ||
        !edit_counts || !text_consumed || (cigar_capacity > 0 && !cigar))
        return fail(c, SCROOGE_E_INVAL, "null pointer argument");
    // host pointers, persistent launch in input order: parts, copies under the kernels
    if (!dev && c->host_split && (flags & SCROOGE_PERSISTENT) &&
        !(flags & (SCROOGE_LEARNED | SCROOGE_WARP_SPECIALIZED)) && n_pairs >= kHostSplitMinPairs &&
        !(c->order && c->order_n == n_pairs))
        return align_host_split(c, texts, text_offsets, text_lengths, patterns, pattern_offsets, pattern_lengths,
                                n_pairs, W, O, k, flags, edit_counts, text_consumed, cigar, cigar_capacity,
                                cigar_offsets);
    int rc;
    const size_t np = (size_t)n_pairs;

    AlignParams p;
    memset(&p, 0, sizeof p);
    p.n_pairs = n_pairs;
    p.W = W;
    p.O = O;
    p.k = k;
    int64_t scratch_runs = 0;
    if ((rc = ensure(c, c->scr_off, (np + 1) * 8, "CIGAR scratch offsets")) ||
        (rc = ensure(c, c->scr_len, np * 4, "CIGAR run counts")) ||
        (rc = ensure(c, c->scan_tmp, (size_t)scan_temp_words((int64_t)np + 1) * 8, "scan scratch")))
        return rc;
    if (dev) {
        p.texts = texts;
        p.text_off = text_offsets;
        p.text_len = text_lengths;
        p.patterns = patterns;
        p.pat_off = pattern_offsets;
        p.pat_len = pattern_lengths;
        p.edit_counts = edit_counts;
        p.text_consumed = text_consumed;
        // size the run scratch from the device-resident lengths
        int64_t *cap = (int64_t *)c->scr_len.p;  // reused below for the run counts
        if ((rc = ensure(c, c->scr_cap, np * 8, "CIGAR capacities"))) return rc;
        cap = (int64_t *)c->scr_cap.p;
        if ((e = launch_capacity(text_lengths, pattern_lengths, n_pairs, cap, st)) != cudaSuccess ||
            (e = exclusive_scan(cap, 1, n_pairs, (int64_t *)c->scr_off.p, (int64_t *)c->scan_tmp.p, st)) != cudaSuccess)
            return cuda_fail(c, e, "CIGAR scratch layout");
        if ((e = cudaMemcpyAsync(&scratch_runs, (int64_t *)c->scr_off.p + n_pairs, 8, cudaMemcpyDeviceToHost, st)) !=
                cudaSuccess ||
            (e = cudaStreamSynchronize(st)) != cudaSuccess)
            return cuda_fail(c, e, "CIGAR scratch size");
    } else {
        // host pointers: check the layout, then stage everything on the device (the run scratch
        // offsets are laid out on the device from the copied lengths, as for device pointers)
        HostLayout lay;
        const int32_t bad =
            host_layout(text_offsets, text_lengths, pattern_offsets, pattern_lengths, n_pairs, &n_pairs, 1, lay);
        if (bad >= 0)
            return fail(c, SCROOGE_E_INVAL, "pair %d: offsets must be >= 0 multiples of 64, lengths >= 0", bad);
        const int64_t text_words = lay.text_upto[0], pat_words = lay.pat_upto[0];
        scratch_runs = lay.runs;
        if ((rc = ensure(c, c->in_text, text_words * 4, "texts")) ||
            (rc = ensure(c, c->in_pat, pat_words * 4, "patterns")) ||
            (rc = ensure(c, c->in_toff, np * 8, "text offsets")) ||
            (rc = ensure(c, c->in_tlen, np * 4, "text lengths")) ||
            (rc = ensure(c, c->in_poff, np * 8, "pattern offsets")) ||
            (rc = ensure(c, c->in_plen, np * 4, "pattern lengths")) ||
            (rc = ensure(c, c->out_ec, np * 4, "edit counts")) || (rc = ensure(c, c->out_tc, np * 4, "text consumed")) ||
            (rc = ensure(c, c->out_off, (np + 1) * 8, "cigar offsets")) ||
            (rc = ensure(c, c->scr_cap, np * 8, "CIGAR capacities")))
            return rc;
        struct {
            void *d;
            const void *h;
            size_t b;
        } cp[] = {{c->in_text.p, texts, (size_t)text_words * 4}, {c->in_pat.p, patterns, (size_t)pat_words * 4},
                  {c->in_toff.p, text_offsets, np * 8},          {c->in_tlen.p, text_lengths, np * 4},
                  {c->in_poff.p, pattern_offsets, np * 8},       {c->in_plen.p, pattern_lengths, np * 4}};
        for (auto &x : cp)
            if (x.b && (e = cudaMemcpyAsync(x.d, x.h, x.b, cudaMemcpyHostToDevice, st)) != cudaSuccess)
                return cuda_fail(c, e, "host-to-device copy");
        if ((e = launch_capacity((const int32_t *)c->in_tlen.p, (const int32_t *)c->in_plen.p, n_pairs,
                                 (int64_t *)c->scr_cap.p, st)) != cudaSuccess ||
            (e = exclusive_scan(c->scr_cap.p, 1, n_pairs, (int64_t *)c->scr_off.p, (int64_t *)c->scan_tmp.p, st)) !=
                cudaSuccess)
            return cuda_fail(c, e, "CIGAR scratch layout");
        p.texts = (const uint32_t *)c->in_text.p;
        p.patterns = (const uint32_t *)c->in_pat.p;
        p.text_off = (const int64_t *)c->in_toff.p;
        p.text_len = (const int32_t *)c->in_tlen.p;
        p.pat_off = (const int64_t *)c->in_poff.p;
        p.pat_len = (const int32_t *)c->in_plen.p;
        p.edit_counts = (int32_t *)c->out_ec.p;
        p.text_consumed = (int32_t *)c->out_tc.p;
    }
    if ((rc = ensure(c, c->scr_runs, (size_t)std::max<int64_t>(scratch_runs, 1) * 4, "CIGAR run scratch"))) return rc;
    p.cigar = (uint32_t *)c->scr_runs.p;
    p.cigar_off = (const int64_t *)c->scr_off.p;
    p.cigar_lens = (int32_t *)c->scr_len.p;

    p.st_windows = c->st_windows;
    p.st_rows = c->st_rows;
    p.st_cells = c->st_cells;
    p.st_cycles = c->st_cycles;
    // kernel shape(s): the kernel the call uses, and with SCROOGE_LEARNED on band-sized windows
    // the full-width kernel for the pairs the ordering puts in the heavy load classes
    const bool band = use_band(W, flags);
    // Learned launches on band-sized windows split the order (see the bucket key in learn.cu):
    //   [0, start of key 128)    long pairs, one pair per warp, banded kernel, high-priority stream;
    //   [.., start of key 192)   heavy pairs, full-width kernel, the context stream;
    //   [.., n_pairs)            the rest, banded kernel, low-priority stream.
    const bool learned_split = band && (flags & SCROOGE_LEARNED) && (c->heavy_class < 16 || c->long_class < 16);
    const bool use_heavy = learned_split && c->heavy_class < 16;
    const bool use_long = learned_split && c->long_class < 16;
    LaunchPlan plan, heavy, lng;
    // learned launches on band-sized windows take their kernel and settings per load bucket
    const bool per_bucket = band && (flags & SCROOGE_LEARNED);
    if (per_bucket) {
        const bool rest_band = c->bucket_kind[1] == 0;
        if ((rc = make_plan(c, p, rest_band, rest_band ? flags : (flags | SCROOGE_NO_BAND), c->spill, c->fallback, 0,
                            plan, &c->bucket_cfg[1])))
            return rc;
    } else if ((rc = make_plan(c, p, band, flags, c->spill, c->fallback, 0, plan))) {
        return rc;
    }
    if (use_heavy) {
        const bool heavy_band = c->bucket_kind[0] == 0;
        if ((rc = make_plan(c, p, heavy_band, heavy_band ? flags : (flags | SCROOGE_NO_BAND), c->spill2, c->fallback3,
                            0, heavy, &c->bucket_cfg[0])))
            return rc;
    }
    if (use_long && (rc = make_plan(c, p, true, flags, c->spill3, c->fallback2, 1, lng))) return rc;
    if ((rc = ensure(c, c->status, 64, "status"))) return rc;
    if ((flags & SCROOGE_PERSISTENT) && (rc = ensure(c, c->queue, 256, "work queues"))) return rc;
    for (LaunchPlan *lp : {&plan, &heavy, &lng}) {
        lp->p.status = (int32_t *)c->status.p;
        lp->p.wait_limit = c->wait_limit;
        if (flags & SCROOGE_PERSISTENT) {
            lp->p.queue = (int32_t *)c->queue.p + (lp == &heavy ? 16 : (lp == &lng ? 32 : 0));
            lp->p.order = (c->order && c->order_n == n_pairs) ? c->order : nullptr;
        }
    }
    if (flags & SCROOGE_LEARNED) {
        // buffers of the ordering pipeline must exist before any capture
        const size_t npp = (size_t)std::max(n_pairs, 1);
        if ((rc = ensure(c, c->l_feat, npp * kFeatures * 4, "features")) ||
            (rc = ensure(c, c->l_pred, npp * 4, "predictions")) || (rc = ensure(c, c->l_key, npp, "bucket keys")) ||
            (rc = ensure(c, c->l_order, npp * 4, "pair order")) ||
            (rc = ensure(c, c->l_tmp, (size_t)sort_temp_words(n_pairs) * 8, "sort scratch")))
            return rc;
        plan.p.order = heavy.p.order = lng.p.order = (const int32_t *)c->l_order.p;
    }
    if (learned_split) {
        const int64_t *k128 = learned_bucket_start((int64_t *)c->l_tmp.p, n_pairs, 128);
        const int64_t *k192 = learned_bucket_start((int64_t *)c->l_tmp.p, n_pairs, 192);
        lng.p.range_hi = k128;
        heavy.p.range_lo = k128;
        heavy.p.range_hi = k192;
        plan.p.range_lo = k192;
        // stream priorities order the block scheduler: long pairs first, then the heavy kernel, then the
        // banded one, whatever order the launches (or graph nodes) reach it in
        int prio_least = 0, prio_greatest = 0;
        cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest);
        if (!c->stream2 && ((e = cudaStreamCreateWithPriority(&c->stream2, cudaStreamNonBlocking, prio_least)) !=
                                cudaSuccess ||
                            (e = cudaStreamCreateWithPriority(&c->stream3, cudaStreamNonBlocking, prio_greatest)) !=
                                cudaSuccess ||
                            (e = cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming)) != cudaSuccess ||
                            (e = cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming)) != cudaSuccess ||
                            (e = cudaEventCreateWithFlags(&c->ev_join3, cudaEventDisableTiming)) != cudaSuccess))
            return cuda_fail(c, e, "second stream");
    }
    {
        const TableShape &ts = plan.ts;
        const int64_t shape[13] = {plan.band ? 0 : plan.words, plan.G, plan.p.rcap, plan.wpb, (int64_t)plan.smem,
                                   plan.blocks, plan.p.ncol, ts.swp, plan.p.table_words_per_warp * 4LL,
                                   plan.p.spill_words_per_pair * 4, plan.p.fb_words_per_warp * 4, 32 / plan.G,
                                   plan.p.ring};
        memcpy(c->last_shape, shape, sizeof shape);
    }
    int64_t *dense_off = dev ? cigar_offsets : (int64_t *)c->out_off.p;
    c->last_kernels = 1 + scan_kernel_count(n_pairs) + 1;  // alignment, CIGAR offsets, gather
    if (learned_split) c->last_kernels += 2;
    if (flags & SCROOGE_LEARNED) c->last_kernels += learned_kernel_count(n_pairs);
    // everything from the status reset to the CIGAR offsets, on `st`
    auto enqueue = [&]() -> int {
        if ((e = cudaMemsetAsync(plan.p.status, 0, 4, st)) != cudaSuccess) return cuda_fail(c, e, "status reset");
        if (plan.p.queue && (e = cudaMemsetAsync(c->queue.p, 0, 256, st)) != cudaSuccess)
            return cuda_fail(c, e, "queue reset");
        if (flags & SCROOGE_LEARNED) {
            const int lrc = learned_order(c, p.texts, p.text_off, p.text_len, p.patterns, p.pat_off, p.pat_len,
                                          n_pairs);
            if (lrc) return lrc;
        }
        const bool timed = c->t_start && c->t_stop && !(flags & SCROOGE_GRAPH);
        if (timed) cudaEventRecord(c->t_start, st);
        if (learned_split) {
            // three launches over disjoint ranges of the order; an empty range costs one short launch
            if ((e = cudaEventRecord(c->ev_fork, st)) != cudaSuccess ||
                (e = cudaStreamWaitEvent(c->stream2, c->ev_fork, 0)) != cudaSuccess ||
                (e = cudaStreamWaitEvent(c->stream3, c->ev_fork, 0)) != cudaSuccess)
                return cuda_fail(c, e, "stream fork");
            if (use_long && (e = launch_plan(lng, c->stream3)) != cudaSuccess)
                return cuda_fail(c, e, "alignment kernel launch");
            if (use_heavy && (e = launch_plan(heavy, st)) != cudaSuccess)
                return cuda_fail(c, e, "alignment kernel launch");
            if ((e = launch_plan(plan, c->stream2)) != cudaSuccess) return cuda_fail(c, e, "alignment kernel launch");
            if ((e = cudaEventRecord(c->ev_join, c->stream2)) != cudaSuccess ||
                (e = cudaEventRecord(c->ev_join3, c->stream3)) != cudaSuccess ||
                (e = cudaStreamWaitEvent(st, c->ev_join, 0)) != cudaSuccess ||
                (e = cudaStreamWaitEvent(st, c->ev_join3, 0)) != cudaSuccess)
                return cuda_fail(c, e, "stream join");
        } else if ((e = launch_plan(plan, st)) != cudaSuccess) {
            return cuda_fail(c, e, "alignment kernel launch");
        }
        if (timed) cudaEventRecord(c->t_stop, st);
        // dense CIGAR: prefix sums of the run counts (the gather follows)
        if ((e = exclusive_scan(p.cigar_lens, 0, n_pairs, dense_off, (int64_t *)c->scan_tmp.p, st)) != cudaSuccess)
            return cuda_fail(c, e, "CIGAR offsets");
        if (dev && (e = launch_compact(p.cigar, p.cigar_off, p.cigar_lens, dense_off, n_pairs, cigar, cigar_capacity,
                                       c->sm_count, st)) != cudaSuccess)
            return cuda_fail(c, e, "CIGAR gather");
        return SCROOGE_OK;
    };
    if (flags & SCROOGE_GRAPH) {
        // one captured graph per distinct call; replayed while the call repeats
        const unsigned long long key[28] = {(unsigned long long)(uintptr_t)p.texts, (unsigned long long)(uintptr_t)p.text_off,
            (unsigned long long)(uintptr_t)p.text_len, (unsigned long long)(uintptr_t)p.patterns,
            (unsigned long long)(uintptr_t)p.pat_off, (unsigned long long)(uintptr_t)p.pat_len,
            (unsigned long long)(uintptr_t)p.edit_counts, (unsigned long long)(uintptr_t)p.text_consumed,
            (unsigned long long)(uintptr_t)p.cigar, (unsigned long long)(uintptr_t)p.cigar_off,
            (unsigned long long)(uintptr_t)dense_off, (unsigned long long)(uintptr_t)(dev ? cigar : nullptr),
            (unsigned long long)cigar_capacity, (unsigned long long)n_pairs,
            ((unsigned long long)W << 32) | ((unsigned long long)O << 16) | (unsigned long long)k,
            (unsigned long long)flags, (unsigned long long)(uintptr_t)plan.p.spill,
            (unsigned long long)(uintptr_t)plan.p.order, (unsigned long long)(uintptr_t)st,
            ((unsigned long long)plan.G << 32) | (unsigned long long)plan.p.rcap,
            ((unsigned long long)plan.wpb << 32) | (unsigned long long)plan.blocks,
            (unsigned long long)(uintptr_t)c->st_rows, (unsigned long long)(uintptr_t)c->st_cells,
            (unsigned long long)(uintptr_t)c->st_windows, (unsigned long long)(uintptr_t)plan.p.fb,
            (unsigned long long)band | ((unsigned long long)(uint32_t)c->wait_limit << 8) |
                ((unsigned long long)plan.band << 40) | ((unsigned long long)plan.lane << 41) |
                ((unsigned long long)heavy.band << 42) | ((unsigned long long)heavy.lane << 43),
            use_heavy ? (((unsigned long long)heavy.G << 48) | ((unsigned long long)heavy.p.rcap << 32) |
                         ((unsigned long long)heavy.wpb << 24) | (unsigned long long)heavy.blocks)
                      : 0ull,
            learned_split ? (((unsigned long long)(uintptr_t)heavy.p.spill) ^ ((unsigned long long)c->heavy_class << 56) ^
                             ((unsigned long long)c->long_class << 48) ^ ((unsigned long long)(uintptr_t)lng.p.spill))
                          : 0ull};
        if (!c->graph || memcmp(key, c->graph_key, sizeof key) != 0) {
            if (c->graph) {
                cudaGraphExecDestroy(c->graph);
                c->graph = nullptr;
            }
            cudaGraph_t g = nullptr;
            if ((e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
                return cuda_fail(c, e, "stream capture (the stream must not be the legacy default stream)");
            const int erc = enqueue();
            cudaError_t ee = cudaStreamEndCapture(st, &g);
            if (erc) {
                if (g) cudaGraphDestroy(g);
                return erc;
            }
            if (ee != cudaSuccess) return cuda_fail(c, ee, "stream capture");
            ee = cudaGraphInstantiate(&c->graph, g, 0);
            cudaGraphDestroy(g);
            if (ee != cudaSuccess) {
                c->graph = nullptr;
                return cuda_fail(c, ee, "graph instantiation");
            }
            memcpy(c->graph_key, key, sizeof key);
        }
        if ((e = cudaGraphLaunch(c->graph, st)) != cudaSuccess) return cuda_fail(c, e, "graph launch");
    } else {
        if ((rc = enqueue())) return rc;
    }
    int32_t status_h = 0;
    if (dev) {
        if (!(flags & SCROOGE_SYNC)) return SCROOGE_OK;
        int64_t total = 0;
        if ((e = cudaMemcpyAsync(&status_h, plan.p.status, 4, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
            (e = cudaMemcpyAsync(&total, dense_off + n_pairs, 8, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
            (e = cudaStreamSynchronize(st)) != cudaSuccess)
            return cuda_fail(c, e, "stream synchronise");
        if (status_h & 8)
            return fail(c, SCROOGE_E_TIMEOUT, "a bounded device wait gave up (status %d)", status_h);
        if (status_h != 0) return fail(c, SCROOGE_E_INTERNAL, "kernel status %d", status_h);
        if (total > cigar_capacity)
            return fail(c, SCROOGE_E_CAPACITY, "CIGAR needs %lld runs, capacity %lld", (long long)total,
                        (long long)cigar_capacity);
        return SCROOGE_OK;
    }
    // host pointers: learn the total, gather into a device buffer, copy back
    if ((e = cudaMemcpyAsync(cigar_offsets, dense_off, (np + 1) * 8, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(&status_h, plan.p.status, 4, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return cuda_fail(c, e, "CIGAR offsets copy");
    if (status_h & 8)
        return fail(c, SCROOGE_E_TIMEOUT, "a bounded device wait gave up (status %d)", status_h);
    if (status_h != 0) return fail(c, SCROOGE_E_INTERNAL, "kernel status %d", status_h);
    const int64_t total = cigar_offsets[np];
    const int64_t keep = std::min(total, cigar_capacity);
    if ((rc = ensure(c, c->out_cig, (size_t)std::max<int64_t>(keep, 1) * 4, "cigar"))) return rc;
    if ((e = launch_compact(p.cigar, p.cigar_off, p.cigar_lens, dense_off, n_pairs, (uint32_t *)c->out_cig.p, keep,
                            c->sm_count, st)) != cudaSuccess)
        return cuda_fail(c, e, "CIGAR gather");
    struct {
        void *h;
        const void *d;
        size_t b;
    } cp[] = {{edit_counts, p.edit_counts, np * 4}, {text_consumed, p.text_consumed, np * 4},
              {cigar, c->out_cig.p, (size_t)keep * 4}};
    for (auto &x : cp)
        if (x.b && (e = cudaMemcpyAsync(x.h, x.d, x.b, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
            return cuda_fail(c, e, "device-to-host copy");
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(c, e, "stream synchronise");
    if (total > cigar_capacity)
        return fail(c, SCROOGE_E_CAPACITY, "CIGAR needs %lld runs, capacity %lld", (long long)total,
                    (long long)cigar_capacity);
    return SCROOGE_OK;
}

int scrooge_autotune(scrooge_ctx *c, const uint32_t *texts, const int64_t *text_offsets, const int32_t *text_lengths,
                     const uint32_t *patterns, const int64_t *pattern_offsets, const int32_t *pattern_lengths,
                     int32_t n_pairs, int32_t W, int32_t O, int32_t k, uint32_t flags, int32_t *edit_counts,
                     int32_t *text_consumed, uint32_t *cigar, int64_t cigar_capacity, int64_t *cigar_offsets,
                     int32_t repeats, int32_t *results, int32_t max_results, int32_t *n_results) {
    if (!c || n_pairs < 1 || repeats < 1) return SCROOGE_E_INVAL;
    if (W < 1 || W > 128) return fail(c, SCROOGE_E_INVAL, "W=%d outside 1..128", W);
    const int words = words_for(W);
    const int ix = kcfg_index(use_band(W, flags) ? band_slot_for(W) : words);
    const KernelConfig saved = c->kcfg[ix];
    const int32_t saved_class = c->heavy_class;
    const int lanes_opts[5][4] = {{1, 2, 4, 0}, {2, 4, 8, 0}, {8, 16, 0, 0}, {1, 2, 4, 8}, {8, 16, 0, 0}};
    const int rows_opts[] = {1, 2, 3, 4, 6, 8, 10, 12, 16, 20};
    const int wpb_opts[] = {1, 2};
    const int classes[] = {16, 15, 14, 13, 12, 11, 10, 0};
    const bool tune_classes = (flags & SCROOGE_LEARNED) && use_band(W, flags);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return fail(c, SCROOGE_E_CUDA, "cudaEventCreate failed");
    int nres = 0, rc = SCROOGE_OK;
    const uint32_t fl = (flags | SCROOGE_DEVICE_PTRS) & ~(uint32_t)SCROOGE_SYNC;
    // the kernel settings sweep times launches that use those settings: with SCROOGE_LEARNED on
    // band-sized windows (whose launches take the per-bucket settings) a persistent launch in input order
    uint32_t fl_run = fl;
    auto call = [&]() {
        return scrooge_align_batch(c, texts, text_offsets, text_lengths, patterns, pattern_offsets, pattern_lengths,
                                   n_pairs, W, O, k, fl_run, edit_counts, text_consumed, cigar, cigar_capacity,
                                   cigar_offsets);
    };
    // one untimed run, then the fastest of `reps` timed runs (CUDA events on the context stream)
    auto time_it = [&](int reps, float &tmin) -> int {
        tmin = -1.f;
        int r = call();
        for (int i = 0; i < reps && r == SCROOGE_OK; ++i) {
            cudaEventRecord(e0, c->stream);
            r = call();
            cudaEventRecord(e1, c->stream);
            if (cudaEventSynchronize(e1) != cudaSuccess) return fail(c, SCROOGE_E_CUDA, "event sync failed");
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (tmin < 0.f || ms < tmin) tmin = ms;
        }
        return r;
    };
    auto record = [&](int a, int b, int w, float ms, int kind) {
        if (results && nres < max_results) {
            int32_t *r = results + 5 * nres;
            r[0] = a;
            r[1] = b;
            r[2] = w;
            r[3] = (int32_t)(ms * 1000.f);
            r[4] = kind;
        }
        ++nres;
    };
    // learned launches on band-sized windows: which load classes go to the full-width kernel
    // A split must beat "no split" (class 16) by 10% to be chosen: the class times of one sample
    // vary with its hardest pairs, and a marginal split can cost more on the next batch.
    auto sweep_classes = [&]() -> int {
        float best_t = -1.f, t_none = -1.f;
        int best_class = c->heavy_class;
        for (int hc : classes) {
            c->heavy_class = hc;
            float t;
            const int r = time_it(std::max(repeats, 3), t);
            if (r != SCROOGE_OK) return r;
            record(0, hc, 0, t, 2);
            if (hc == 16) t_none = t;
            if (best_t < 0.f || t < best_t) {
                best_t = t;
                best_class = hc;
            }
        }
        if (best_class != 16 && t_none > 0.f && best_t > 0.9f * t_none) best_class = 16;
        c->heavy_class = best_class;
        return SCROOGE_OK;
    };
    if (tune_classes) rc = sweep_classes();
    float best = -1.f;
    KernelConfig best_cfg = saved;
    if (tune_classes) fl_run = (fl & ~(uint32_t)SCROOGE_LEARNED) | SCROOGE_PERSISTENT;
    for (int li = 0; li < 4 && rc == SCROOGE_OK; ++li) {
        const int lanes = lanes_opts[ix][li];
        if (!lanes) continue;
        for (int rows : rows_opts) {
            for (int wpb : wpb_opts) {
                c->kcfg[ix] = {lanes, rows, wpb};
                float t;
                if ((rc = time_it(repeats, t)) != SCROOGE_OK) break;
                record(lanes, rows, wpb, t, 1);
                if (best < 0.f || t < best) {
                    best = t;
                    best_cfg = c->kcfg[ix];
                }
            }
            if (rc != SCROOGE_OK) break;
        }
    }
    c->kcfg[ix] = rc == SCROOGE_OK ? best_cfg : saved;
    fl_run = fl;
    if (rc == SCROOGE_OK && tune_classes) rc = sweep_classes();  // again, with the chosen settings
    if (rc != SCROOGE_OK) c->heavy_class = saved_class;
    // learned launches: kernel and settings per load bucket (the rest, then the heavy pairs if the
    // order splits them off), each chosen with the other fixed, by the time of the whole call
    const int32_t saved_kind[2] = {c->bucket_kind[0], c->bucket_kind[1]};
    const KernelConfig saved_bcfg[2] = {c->bucket_cfg[0], c->bucket_cfg[1]};
    const bool saved_order = c->learned_order_on;
    if (rc == SCROOGE_OK && tune_classes) {
        c->learned_order_on = true;
        if (ix == kcfg_index(0)) {  // 64-base windows: the rest starts from the tuned banded settings
            c->bucket_kind[1] = 0;
            c->bucket_cfg[1] = c->kcfg[ix];
        }
        const int band_lanes[] = {1, 2, 4, 8}, full_lanes[] = {2, 4, 8}, bucket_rows[] = {2, 4, 8};
        for (int b = 1; b >= 0 && rc == SCROOGE_OK; --b) {
            if (b == 0 && c->heavy_class >= 16) break;  // no heavy bucket
            float bbest = -1.f;
            int bkind = c->bucket_kind[b];
            KernelConfig bcfg = c->bucket_cfg[b];
            for (int kind = 0; kind < 2 && rc == SCROOGE_OK; ++kind) {
                const int *lanes = kind == 0 ? band_lanes : full_lanes;
                const int nl = kind == 0 ? 4 : 3;
                for (int li = 0; li < nl && rc == SCROOGE_OK; ++li) {
                    if (ix != kcfg_index(0) && kind == 0 && lanes[li] == 1) continue;  // lane kernel: 64-base windows
                    for (int rows : bucket_rows) {
                        for (int wpb = 1; wpb <= 2; ++wpb) {
                            c->bucket_kind[b] = kind;
                            c->bucket_cfg[b] = {lanes[li], rows, wpb};
                            float t;
                            if ((rc = time_it(repeats, t)) != SCROOGE_OK) break;
                            record(b * 1000 + kind * 100 + lanes[li], rows, wpb, t, 3);
                            if (bbest < 0.f || t < bbest) {
                                bbest = t;
                                bkind = kind;
                                bcfg = c->bucket_cfg[b];
                            }
                        }
                        if (rc != SCROOGE_OK) break;
                    }
                }
            }
            c->bucket_kind[b] = bkind;
            c->bucket_cfg[b] = bcfg;
        }
        // the long pairs' own launch (one pair per warp, scrooge_set_long_class): kept only if it is at
        // least 5% faster than none
        if (rc == SCROOGE_OK) {
            const int32_t saved_long = c->long_class;
            float t_off = -1.f, best_t = -1.f;
            int best_lc = 16;
            for (int lc : {16, 14, 13, 12}) {
                c->long_class = lc;
                float t;
                if ((rc = time_it(std::max(repeats, 3), t)) != SCROOGE_OK) break;
                record(0, lc, 1, t, 5);
                if (lc == 16) t_off = t;
                if (best_t < 0.f || t < best_t) {
                    best_t = t;
                    best_lc = lc;
                }
            }
            c->long_class = rc != SCROOGE_OK ? saved_long
                                             : ((best_lc != 16 && best_t <= 0.95f * t_off) ? best_lc : 16);
        }
        // does the model's order pay for itself on this workload? keep it only if it is at least 2%
        // faster than the persistent launch in input order (which SCROOGE_LEARNED then falls back to)
        if (rc == SCROOGE_OK) {
            float t_model, t_input;
            if ((rc = time_it(std::max(repeats, 3), t_model)) == SCROOGE_OK) {
                c->learned_order_on = false;
                rc = time_it(std::max(repeats, 3), t_input);
                record(1, 0, 0, t_model, 4);
                record(0, 0, 0, t_input, 4);
                c->learned_order_on = rc == SCROOGE_OK && t_model <= 0.98f * t_input;
            }
        }
    }
    if (rc != SCROOGE_OK) {
        for (int b = 0; b < 2; ++b) {
            c->bucket_kind[b] = saved_kind[b];
            c->bucket_cfg[b] = saved_bcfg[b];
        }
        c->learned_order_on = saved_order;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (n_results) *n_results = std::min(nres, max_results);
    return rc;
}

}  // extern "C"
