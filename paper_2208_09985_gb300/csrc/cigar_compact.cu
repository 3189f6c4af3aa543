// Dense CIGAR output: per-pair scratch capacities, exclusive prefix sums and
// the gather of every pair's runs into one contiguous array in pair order.
#include <algorithm>

#include "scrooge_internal.h"

namespace scrooge {
namespace {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

// scratch run capacity of pair p: every run holds at least one operation, and
// a pair makes at most m + n operations
__global__ void capacity_kernel(const int32_t *text_len, const int32_t *pat_len, int32_t n, int64_t *cap) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n) cap[p] = (int64_t)text_len[p] + (int64_t)pat_len[p] + 1;
}

// v[i] += *base for i < n (the base is a device value, e.g. an earlier scan's total)
__global__ void add_base_kernel(int64_t *v, int64_t n, const int64_t *base) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) v[i] += *base;
}

__device__ __forceinline__ int64_t warp_incl_scan(int64_t v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

// Exclusive scan of one tile of kScanTile values; the tile total goes to sums.
// `in` may be int32 (wide = 0) or int64 (wide = 1).
__global__ void __launch_bounds__(kScanThreads) scan_tile_kernel(const void *in, int wide, int64_t n, int64_t *out,
                                                                 int64_t *sums) {
    __shared__ int64_t warp_tot[kScanThreads / 32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int64_t v[kScanItems];
    int64_t run = 0;
#pragma unroll
    for (int t = 0; t < kScanItems; ++t) {
        const int64_t i = base + t;
        int64_t x = 0;
        if (i < n) x = wide ? static_cast<const int64_t *>(in)[i] : (int64_t) static_cast<const int32_t *>(in)[i];
        v[t] = run;
        run += x;
    }
    const int64_t incl = warp_incl_scan(run);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 31) warp_tot[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        const int64_t t = warp_incl_scan(warp_tot[lane]);
        warp_tot[lane] = t;
    }
    __syncthreads();
    const int64_t before = (incl - run) + (wid > 0 ? warp_tot[wid - 1] : 0);
#pragma unroll
    for (int t = 0; t < kScanItems; ++t) {
        const int64_t i = base + t;
        if (i < n) out[i] = before + v[t];
    }
    if (threadIdx.x == kScanThreads - 1) sums[blockIdx.x] = before + run;
}

__global__ void add_tile_offsets(int64_t *out, int64_t n, const int64_t *tile_off) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] += tile_off[i / kScanTile];
}

// out[n] = out[n-1] + last input (the total)
__global__ void total_kernel(const void *in, int wide, int64_t n, int64_t *out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        const int64_t last = n > 0 ? (wide ? static_cast<const int64_t *>(in)[n - 1]
                                           : (int64_t) static_cast<const int32_t *>(in)[n - 1])
                                   : 0;
        out[n] = n > 0 ? out[n - 1] + last : 0;
    }
}

// One warp per pair: copy its runs from the scratch layout to the dense layout,
// only if they fit entirely below `capacity`.
__global__ void compact_kernel(const uint32_t *scratch, const int64_t *scratch_off, const int32_t *lens,
                               const int64_t *dense_off, int32_t n, uint32_t *dense, int64_t capacity) {
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t p = warp; p < n; p += nwarps) {
        const int32_t len = lens[p];
        const int64_t dst = dense_off[p];
        if (len <= 0 || dst + len > capacity) continue;
        const uint32_t *src = scratch + scratch_off[p];
        for (int32_t r = lane; r < len; r += 32) dense[dst + r] = src[r];
    }
}

}  // namespace

// Exclusive prefix sums with a total: out[0..n] (n+1 entries). `tmp` must hold
// scan_temp_words(n) int64 values.
int64_t scan_temp_words(int64_t n) {
    int64_t words = 0;
    while (n > kScanTile) {
        const int64_t tiles = (n + kScanTile - 1) / kScanTile;
        words += 2 * tiles + 2;
        n = tiles;
    }
    return words + 2;
}

int scan_kernel_count(int64_t n) {
    if (n <= 0) return 0;
    const int64_t tiles = (n + kScanTile - 1) / kScanTile;
    return 1 + (tiles > 1 ? scan_kernel_count(tiles) + 1 : 0) + 1;
}

cudaError_t exclusive_scan(const void *in, int wide, int64_t n, int64_t *out, int64_t *tmp, cudaStream_t s) {
    if (n <= 0) return cudaMemsetAsync(out, 0, sizeof(int64_t), s);
    const int64_t tiles = (n + kScanTile - 1) / kScanTile;
    int64_t *sums = tmp;
    scan_tile_kernel<<<(unsigned)tiles, kScanThreads, 0, s>>>(in, wide, n, out, sums);
    if (tiles > 1) {
        int64_t *sum_off = tmp + tiles + 1;
        cudaError_t e = exclusive_scan(sums, 1, tiles, sum_off, sum_off + tiles + 1, s);
        if (e != cudaSuccess) return e;
        add_tile_offsets<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(out, n, sum_off);
    }
    total_kernel<<<1, 32, 0, s>>>(in, wide, n, out);
    return cudaGetLastError();
}

cudaError_t launch_add_base(int64_t *v, int64_t n, const int64_t *base, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    add_base_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(v, n, base);
    return cudaGetLastError();
}

cudaError_t launch_capacity(const int32_t *text_len, const int32_t *pat_len, int32_t n, int64_t *cap,
                            cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    capacity_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(text_len, pat_len, n, cap);
    return cudaGetLastError();
}

cudaError_t launch_compact(const uint32_t *scratch, const int64_t *scratch_off, const int32_t *lens,
                           const int64_t *dense_off, int32_t n, uint32_t *dense, int64_t capacity, int sm_count,
                           cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int64_t warps = n;
    const int64_t blocks = std::min<int64_t>((warps * 32 + 255) / 256, (int64_t)sm_count * 8);
    compact_kernel<<<(unsigned)blocks, 256, 0, s>>>(scratch, scratch_off, lens, dense_off, n, dense, capacity);
    return cudaGetLastError();
}

}  // namespace scrooge
