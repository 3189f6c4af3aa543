// The library context (opaque to callers) and host-side helpers shared by the
// C-ABI translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>

#include <string>

#include "../../include/scrooge.h"
#include "scrooge_internal.h"

namespace scrooge {

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

struct KernelConfig {
    int lanes, rows, wpb;
};

}  // namespace scrooge

struct scrooge_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int sm_count = 0;
    size_t smem_optin = 0;
    std::string err;
    // full-width kernels of 1, 2, 4 words, then the banded kernels of 64- and 128-base windows
    // (autotuned on GB300)
    scrooge::KernelConfig kcfg[5] = {{2, 8, 2}, {4, 4, 2}, {8, 8, 2}, {1, 4, 1}, {8, 6, 2}};
    int fail_allocs = 0;  // testing hook: fail the next N device allocations
    int32_t wait_limit = 0;  // polls per bounded device wait (0: the kernel's default bound)
    scrooge::DevBuf spill, status, fallback, spill2, spill3, fallback2, fallback3;
    // learned launches: pairs in load classes >= heavy_class run on the full-width kernel, pairs in
    // work classes >= long_class one per warp on stream3 (16: none); the banded kernel runs the rest
    // on stream2
    int32_t heavy_class = 16, long_class = 16;
    // kernel settings of the learned launches per load bucket: 0 = the heavy pairs, 1 = the rest;
    // kind 0 = banded kernel, 1 = full-width kernel (see scrooge_set_bucket_config)
    int32_t bucket_kind[2] = {1, 0};
    scrooge::KernelConfig bucket_cfg[2] = {{4, 4, 2}, {1, 4, 1}};
    bool learned_order_on = true;  // SCROOGE_LEARNED orders by the model (else input order)
    cudaStream_t stream2 = nullptr, stream3 = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_join3 = nullptr;
    scrooge::DevBuf in_text, in_pat, in_toff, in_tlen, in_poff, in_plen;
    scrooge::DevBuf out_ec, out_tc, out_cig, out_off;
    scrooge::DevBuf scr_runs, scr_off, scr_len, scr_cap, scan_tmp;
    scrooge::DevBuf queue;
    const int32_t *order = nullptr;  // pair order of persistent launches (device), or input order
    int32_t order_n = 0;
    int32_t *st_windows = nullptr;
    int64_t *st_rows = nullptr, *st_cells = nullptr, *st_cycles = nullptr;
    // learned ordering
    scrooge::DevBuf model, grad, adam_m1, adam_m2, loss;
    bool model_ready = false;
    scrooge::DevBuf l_feat, l_pred, l_key, l_order, l_tmp, t_rows;
    // optional events recorded around the alignment kernel (not in graph mode)
    cudaEvent_t t_start = nullptr, t_stop = nullptr;
    int32_t last_kernels = 0;  // kernels launched by the last alignment call
    int64_t last_shape[13] = {0};  // launch shape of the last alignment call (scrooge_last_launch_shape)
    // host-pointer persistent calls in parts (align_host_split): copy stream, two kernel streams,
    // events, range bounds, the dense CIGAR of the parts after the first (which uses out_cig)
    bool host_split = true;
    cudaStream_t split_copy = nullptr, split_a = nullptr, split_b = nullptr;
    cudaEvent_t split_ev[16] = {};
    scrooge::DevBuf split_bounds, out_cig_parts[3];
    // CUDA graph of the learned pipeline, keyed by the call it was captured for
    cudaGraphExec_t graph = nullptr;
    unsigned long long graph_key[28] = {0};
};

namespace scrooge {

inline int fail(scrooge_ctx *c, int code, const char *fmt, ...) {
    if (c) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        c->err = buf;
    }
    return code;
}

inline int cuda_fail(scrooge_ctx *c, cudaError_t e, const char *what) {
    return fail(c, SCROOGE_E_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// settings slots: 1, 2, 4 = the full-width kernels of that many words; 0 = the banded kernel of
// 33..64-base windows; 3 = the banded kernel of 65..128-base windows
inline int kcfg_index(int words) {
    return words == 1 ? 0 : (words == 2 ? 1 : (words == 4 ? 2 : (words == 0 ? 3 : (words == 3 ? 4 : -1))));
}

// Grow a device buffer to at least `bytes` (contents are not kept).
inline int ensure(scrooge_ctx *c, DevBuf &b, size_t bytes, const char *what) {
    if (bytes == 0) bytes = 16;
    if (b.bytes >= bytes) return SCROOGE_OK;
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
    if (c->fail_allocs > 0) {
        c->fail_allocs -= 1;
        return fail(c, SCROOGE_E_NOMEM, "device allocation of %zu bytes for %s failed (injected)", bytes, what);
    }
    size_t sz = bytes + bytes / 8;  // some headroom for growing batches
    cudaError_t e = cudaMalloc(&b.p, sz);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(c, SCROOGE_E_NOMEM, "device allocation of %zu bytes for %s failed: %s", sz, what,
                    cudaGetErrorString(e));
    }
    b.bytes = sz;
    return SCROOGE_OK;
}

inline void release(DevBuf &b) {
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
}

inline int words_for(int W) { return W <= 32 ? 1 : (W <= 64 ? 2 : 4); }

// The banded kernels serve windows of 33..128 bases with SENE and ET on.
inline bool use_band(int W, uint32_t flags) {
    return W > 32 && W <= 128 && !(flags & (SCROOGE_NO_SENE | SCROOGE_NO_ET | SCROOGE_NO_BAND));
}

// the settings slot of the banded kernel for windows of W bases
inline int band_slot_for(int W) { return W > 64 ? 3 : 0; }

// Order of the pairs by predicted load (learn_api.cu): features, MLP, bucket
// keys, stable sort; writes ctx->l_order. Device pointers; asynchronous.
int learned_order(scrooge_ctx *c, const uint32_t *texts, const int64_t *text_off, const int32_t *text_len,
                  const uint32_t *patterns, const int64_t *pat_off, const int32_t *pat_len, int32_t n_pairs);

}  // namespace scrooge
