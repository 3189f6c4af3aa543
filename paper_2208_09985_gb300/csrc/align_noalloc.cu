// scrooge_align_batch_noalloc: the alignment kernel run without any device
// allocation, for callers that cannot call cudaMalloc.
//
// The only scratch the kernel needs beyond its inputs and outputs is the area
// for DP rows that do not fit in shared memory, plus one status word. Here both
// live in file-scope __device__ arrays of a fixed size, so every GPU that loads
// the library holds them (16 MiB + 256 B) until the process exits. Host code
// must not use the arrays' names as device addresses: the first call on each
// device looks their addresses up with cudaGetSymbolAddress (with that device
// current) and caches them.
#include <mutex>

#include "../../include/scrooge.h"
#include "align_kernel.cuh"

namespace scrooge {
namespace {

constexpr int64_t kNoAllocRowWords = 4 * 1024 * 1024;  // 16 MiB of DP-row scratch
constexpr int kMaxDevices = 64;

static __device__ __align__(256) uint32_t g_noalloc_rows[kNoAllocRowWords];
static __device__ __align__(256) int32_t g_noalloc_status[64];

struct NoAllocDevice {
    bool ready;
    uint32_t *rows;
    int32_t *status;
    int sm_count;
    size_t smem_optin;
};

std::mutex g_noalloc_mu;
NoAllocDevice g_noalloc_dev[kMaxDevices];

// Fixed kernel shapes per bitvector width (words 1, 2, 4): lanes per pair,
// rows in shared memory, warps per block.
struct Shape {
    int lanes, rows, wpb;
};
constexpr Shape kShapes[3] = {{2, 16, 2}, {4, 12, 2}, {8, 12, 2}};

template <int NW, int G, int SWP>
cudaError_t prepare_kernel(size_t smem_optin) {
    return cudaFuncSetAttribute(kern::align_kernel<NW, G, true, SWP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem_optin);
}

// One-time set-up of the current device: symbol addresses and kernel attributes.
int setup_device(int dev, NoAllocDevice **out) {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    NoAllocDevice &d = g_noalloc_dev[dev];
    if (!d.ready) {
        void *rows = nullptr, *status = nullptr;
        if (cudaGetSymbolAddress(&rows, g_noalloc_rows) != cudaSuccess ||
            cudaGetSymbolAddress(&status, g_noalloc_status) != cudaSuccess) {
            cudaGetLastError();
            return SCROOGE_E_CUDA;
        }
        int sms = 0, optin = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
            cudaGetLastError();
            return SCROOGE_E_CUDA;
        }
        if (prepare_kernel<1, 2, 1>(optin) != cudaSuccess || prepare_kernel<2, 4, 1>(optin) != cudaSuccess ||
            prepare_kernel<2, 4, 2>(optin) != cudaSuccess || prepare_kernel<4, 8, 1>(optin) != cudaSuccess ||
            prepare_kernel<4, 8, 2>(optin) != cudaSuccess || prepare_kernel<4, 8, 4>(optin) != cudaSuccess) {
            cudaGetLastError();
            return SCROOGE_E_CUDA;
        }
        d.rows = static_cast<uint32_t *>(rows);
        d.status = static_cast<int32_t *>(status);
        d.sm_count = sms;
        d.smem_optin = (size_t)optin;
        d.ready = true;
    }
    *out = &d;
    return SCROOGE_OK;
}

template <int NW, int G, int SWP>
cudaError_t launch(const AlignParams &p, int wpb, int blocks, size_t smem, cudaStream_t s, int *per_sm) {
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, kern::align_kernel<NW, G, true, SWP>,
                                                                  32 * wpb, smem);
    if (e != cudaSuccess || blocks <= 0) return e;
    kern::align_kernel<NW, G, true, SWP><<<blocks, 32 * wpb, smem, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_any(int words, int swp, const AlignParams &p, int wpb, int blocks, size_t smem, cudaStream_t s,
                       int *per_sm) {
    if (words == 1) return launch<1, 2, 1>(p, wpb, blocks, smem, s, per_sm);
    if (words == 2) return swp == 1 ? launch<2, 4, 1>(p, wpb, blocks, smem, s, per_sm)
                                    : launch<2, 4, 2>(p, wpb, blocks, smem, s, per_sm);
    return swp == 1 ? launch<4, 8, 1>(p, wpb, blocks, smem, s, per_sm)
                    : (swp == 2 ? launch<4, 8, 2>(p, wpb, blocks, smem, s, per_sm)
                                : launch<4, 8, 4>(p, wpb, blocks, smem, s, per_sm));
}

}  // namespace
}  // namespace scrooge

using namespace scrooge;

extern "C" int scrooge_align_batch_noalloc(const uint32_t *texts, const int64_t *text_offsets,
                                           const int32_t *text_lengths, const uint32_t *patterns,
                                           const int64_t *pattern_offsets, const int32_t *pattern_lengths,
                                           int32_t n_pairs, int32_t W, int32_t O, int32_t k, uint32_t flags,
                                           int32_t *edit_counts, int32_t *text_consumed, uint32_t *cigar,
                                           const int64_t *cigar_offsets, int32_t *cigar_lens, int32_t *status,
                                           void *cuda_stream) {
    if (n_pairs < 0 || W < 1 || W > 128 || O < 0 || O >= W || k < 0 || k > W) return SCROOGE_E_INVAL;
    if (flags & ~(uint32_t)(SCROOGE_SYNC | SCROOGE_NO_DENT | SCROOGE_NO_ET | SCROOGE_NO_EXT_DENT | SCROOGE_DEVICE_PTRS))
        return SCROOGE_E_INVAL;
    if (n_pairs == 0) return SCROOGE_OK;
    if (!texts || !text_offsets || !text_lengths || !patterns || !pattern_offsets || !pattern_lengths ||
        !edit_counts || !text_consumed || !cigar || !cigar_offsets || !cigar_lens)
        return SCROOGE_E_INVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return SCROOGE_E_CUDA;
    }
    NoAllocDevice *d = nullptr;
    int rc = setup_device(dev, &d);
    if (rc != SCROOGE_OK) return rc;
    cudaStream_t st = (cudaStream_t)cuda_stream;

    const int words = W <= 32 ? 1 : (W <= 64 ? 2 : 4);
    const Shape sh = kShapes[words == 1 ? 0 : (words == 2 ? 1 : 2)];
    const int PPW = 32 / sh.lanes;
    const bool dent = !(flags & SCROOGE_NO_DENT);
    const TableShape ts = table_shape(W, O, words, sh.lanes, dent, true);
    AlignParams p;
    memset(&p, 0, sizeof p);
    p.texts = texts;
    p.text_off = text_offsets;
    p.text_len = text_lengths;
    p.patterns = patterns;
    p.pat_off = pattern_offsets;
    p.pat_len = pattern_lengths;
    p.n_pairs = n_pairs;
    p.W = W;
    p.O = O;
    p.k = k;
    p.et = (flags & SCROOGE_NO_ET) ? 0 : 1;
    p.sene = 1;
    p.ncol = ts.ncol;
    p.sw = ts.swp;
    p.rstride = row_stride_cells(ts, PPW, 32 * words / sh.lanes);
    // DENT extended to rows: W-O+G row slots per window instead of k+1 (with DENT and ET)
    p.ring = ext_dent_ring(W, O, k, sh.lanes, dent && p.et && !(flags & SCROOGE_NO_EXT_DENT));
    int rcap = std::min(sh.rows, (int)p.ring);
    const int stage = stage_words_per_warp(words, PPW);
    while (rcap > 1 && (size_t)sh.wpb * (table_words_per_warp(rcap, ts, PPW, 32 * words / sh.lanes) + stage) * 4 > d->smem_optin) --rcap;
    p.rcap = rcap;
    p.table_words_per_warp = (int32_t)table_words_per_warp(rcap, ts, PPW, 32 * words / sh.lanes);
    p.smem_words_per_warp = p.table_words_per_warp + stage;
    const size_t smem = (size_t)sh.wpb * p.smem_words_per_warp * 4;
    p.spill_words_per_pair = table_words_per_warp(std::max(0, p.ring - rcap), ts, PPW, 32 * words / sh.lanes);  // per warp
    // the static row scratch bounds how many warps may be resident
    const int64_t words_per_block = (int64_t)sh.wpb * std::max<int64_t>(p.spill_words_per_pair, 4);
    const int64_t fit_blocks = kNoAllocRowWords / words_per_block;
    if (fit_blocks < 1) return SCROOGE_E_INVAL;  // this W/O/k needs more than the static scratch holds
    p.spill = d->rows;
    p.status = d->status;
    p.cigar = cigar;
    p.cigar_off = cigar_offsets;
    p.cigar_lens = cigar_lens;
    p.edit_counts = edit_counts;
    p.text_consumed = text_consumed;

    // the status word keeps the last call's value: clear it first
    if (cudaMemsetAsync(d->status, 0, sizeof(int32_t), st) != cudaSuccess) return SCROOGE_E_CUDA;
    const int64_t want = ((int64_t)n_pairs + (int64_t)PPW * sh.wpb - 1) / ((int64_t)PPW * sh.wpb);
    int per_sm = 0;
    cudaError_t e;
    // first query occupancy (blocks = 0 launches nothing), then launch
    e = launch_any(words, ts.swp, p, sh.wpb, 0, smem, st, &per_sm);
    if (e != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        return SCROOGE_E_CUDA;
    }
    const int blocks = (int)std::max<int64_t>(
        1, std::min<int64_t>(std::min<int64_t>(want, (int64_t)per_sm * d->sm_count), fit_blocks));
    int dummy = 0;
    e = launch_any(words, ts.swp, p, sh.wpb, blocks, smem, st, &dummy);
    if (e != cudaSuccess) return SCROOGE_E_CUDA;
    if (status && cudaMemcpyAsync(status, d->status, sizeof(int32_t), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return SCROOGE_E_CUDA;
    if ((flags & SCROOGE_SYNC) && cudaStreamSynchronize(st) != cudaSuccess) return SCROOGE_E_CUDA;
    return SCROOGE_OK;
}
