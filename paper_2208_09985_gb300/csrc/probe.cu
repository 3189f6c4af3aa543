// Throughput probe of the integer logic pipe (LOP3 and funnel shifts), the pipe the
// alignment kernels are bound by. It measures the denominator of their roofline on the
// device it runs on: every thread runs 8 independent chains, each step one 3-input
// logic op and one funnel shift, so the pipe, not latency, sets the rate. Each block
// reads the SM clock around its loop; the per-SM rate is the ops an SM's blocks
// executed over the span of that SM's clock readings, which needs no knowledge of
// the clock frequency.
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "scrooge_ctx.h"

namespace scrooge {
namespace kern {

constexpr int kProbeChains = 8;
constexpr int kProbeUnroll = 16;
constexpr int kProbeThreads = 256;

__device__ __forceinline__ uint32_t lop3_xor3(uint32_t a, uint32_t b, uint32_t c) {
    uint32_t r;
    asm volatile("lop3.b32 %0, %1, %2, %3, 0x96;" : "=r"(r) : "r"(a), "r"(b), "r"(c));
    return r;
}

__device__ __forceinline__ uint32_t shf_l(uint32_t lo, uint32_t hi, uint32_t s) {
    uint32_t r;
    asm volatile("shf.l.wrap.b32 %0, %1, %2, %3;" : "=r"(r) : "r"(lo), "r"(hi), "r"(s));
    return r;
}

// rec[block] = {smid, clock at start, clock at end}; sink keeps the chains alive.
__global__ void __launch_bounds__(kProbeThreads) logic_probe_kernel(int iters, uint32_t seed, long long *rec,
                                                                    uint32_t *sink) {
    uint32_t x[kProbeChains], y[kProbeChains];
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) {
        x[c] = seed ^ (threadIdx.x * 2654435761u) ^ (uint32_t)c;
        y[c] = (seed >> 3) + blockIdx.x + 17u * (uint32_t)c;
    }
    __syncthreads();
    const long long t0 = clock64();
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kProbeUnroll; ++u) {
#pragma unroll
            for (int c = 0; c < kProbeChains; ++c) {
                x[c] = lop3_xor3(x[c], y[c], 0x9e3779b9u);
                y[c] = shf_l(y[c], x[c], 5);
            }
        }
    }
    __syncthreads();
    const long long t1 = clock64();
    uint32_t acc = 0;
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) acc ^= x[c] ^ y[c];
    if (acc == 0x12345678u) sink[0] = acc;  // practically never taken; keeps the chains live
    if (threadIdx.x == 0) {
        uint32_t smid;
        asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
        rec[3 * blockIdx.x + 0] = smid;
        rec[3 * blockIdx.x + 1] = t0;
        rec[3 * blockIdx.x + 2] = t1;
    }
}

}  // namespace kern
}  // namespace scrooge

using namespace scrooge;

extern "C" int scrooge_logic_peak(scrooge_ctx *c, int32_t iterations, double *ops_per_s, double *ops_per_clk_per_sm) {
    if (!c || iterations < 1 || iterations > (1 << 20)) return SCROOGE_E_INVAL;
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
    int per_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern::logic_probe_kernel, kern::kProbeThreads,
                                                           0)) != cudaSuccess)
        return cuda_fail(c, e, "occupancy query");
    if (per_sm < 1) return fail(c, SCROOGE_E_INTERNAL, "probe kernel does not fit on an SM");
    const int blocks = per_sm * c->sm_count;  // one full wave
    long long *rec = nullptr;
    uint32_t *sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = SCROOGE_OK;
    std::vector<long long> h((size_t)blocks * 3);
    float ms = 0.f;
    if ((e = cudaMalloc(&rec, sizeof(long long) * 3 * (size_t)blocks)) != cudaSuccess ||
        (e = cudaMalloc(&sink, 16)) != cudaSuccess || (e = cudaEventCreate(&e0)) != cudaSuccess ||
        (e = cudaEventCreate(&e1)) != cudaSuccess) {
        rc = cuda_fail(c, e, "probe set-up");
        goto done;
    }
    // one warm-up launch, then the timed one
    for (int rep = 0; rep < 2 && rc == SCROOGE_OK; ++rep) {
        if (rep == 1) cudaEventRecord(e0, c->stream);
        kern::logic_probe_kernel<<<blocks, kern::kProbeThreads, 0, c->stream>>>(rep == 0 ? 1 : iterations, 0x2545f491u,
                                                                               rec, sink);
        if ((e = cudaGetLastError()) != cudaSuccess) rc = cuda_fail(c, e, "probe launch");
        if (rep == 1) cudaEventRecord(e1, c->stream);
    }
    if (rc == SCROOGE_OK && ((e = cudaEventSynchronize(e1)) != cudaSuccess ||
                             (e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess ||
                             (e = cudaMemcpy(h.data(), rec, h.size() * sizeof(long long), cudaMemcpyDeviceToHost)) !=
                                 cudaSuccess))
        rc = cuda_fail(c, e, "probe read-back");
    if (rc == SCROOGE_OK) {
        const double ops_per_block =
            2.0 * kern::kProbeChains * kern::kProbeUnroll * (double)iterations * kern::kProbeThreads;
        if (ops_per_s) *ops_per_s = ops_per_block * blocks / (ms * 1e-3);
        // per SM: the ops of its blocks over the span of its clock readings; median over SMs
        std::vector<long long> lo(1024, -1), hi(1024, -1);
        std::vector<int> nb(1024, 0);
        for (int b = 0; b < blocks; ++b) {
            const long long sm = h[3 * b];
            if (sm < 0 || sm >= 1024) continue;
            lo[sm] = lo[sm] < 0 ? h[3 * b + 1] : std::min(lo[sm], h[3 * b + 1]);
            hi[sm] = std::max(hi[sm], h[3 * b + 2]);
            nb[sm] += 1;
        }
        std::vector<double> rate;
        for (int sm = 0; sm < 1024; ++sm)
            if (nb[sm] > 0 && hi[sm] > lo[sm]) rate.push_back(ops_per_block * nb[sm] / (double)(hi[sm] - lo[sm]));
        std::sort(rate.begin(), rate.end());
        if (ops_per_clk_per_sm) *ops_per_clk_per_sm = rate.empty() ? 0.0 : rate[rate.size() / 2];
    }
done:
    if (rec) cudaFree(rec);
    if (sink) cudaFree(sink);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return rc;
}
