// Learned pair ordering: per-pair features, a small MLP (inference and
// training), bucket keys and a stable counting sort. None of it touches the
// alignment arithmetic: the MLP only decides the order in which pairs are
// handed to the persistent alignment kernel, so results are identical with or
// without it.
#include <math.h>

#include <algorithm>

#include "scrooge_internal.h"

namespace scrooge {
namespace {

constexpr int kK = 12;         // k-mer length of the shared k-mer features
constexpr int kBand = 64;      // text positions searched on each side of the expected one
constexpr int kSamples = 128;  // at most this many pattern k-mers per pair

__device__ __forceinline__ uint2 blk(const uint2 *seq, int64_t b, int64_t nblk) {
    return (b >= 0 && b < nblk) ? __ldg(seq + b) : make_uint2(0u, 0u);
}

// bit planes of the 32 bases starting at `pos` (>= 0)
__device__ __forceinline__ void planes32(const uint2 *seq, int64_t nblk, int64_t pos, uint32_t &p0, uint32_t &p1) {
    const int64_t b = pos >> 5;
    const int r = (int)(pos & 31);
    const uint2 a = blk(seq, b, nblk), c = blk(seq, b + 1, nblk);
    p0 = __funnelshift_l(c.x, a.x, r);
    p1 = __funnelshift_l(c.y, a.y, r);
}

// Eight lanes per pair (kFeatLanes). Features (all float32):
//   0: log2(m + 1)             1: log2(n + 1)           2: (n - m) / max(m, 1)
//   3: fraction of sampled pattern 12-mers found in the text within +-64 of
//      the same position (anchored start)
//   4: spread (standard deviation / 64) of the offsets text - pattern of the hits
//   5: fraction of hits within +-16 of the mean offset
constexpr int kFeatLanes = 8;  // lanes per pair in features_kernel

// Nearest text position of a sampled pattern k-mer, bit-parallel: bit u of
// the candidate mask (MSB-first, in 32-bit words) says whether the k-mer
// occurs at text position lo + u; all 12 k-mer bases are tested against 160
// candidates with shifted words of the text planes. Returns the offset
// (lo + u) - q of the match nearest to q, the lower one on a tie, or 0x7fff.
__device__ __forceinline__ int nearest_kmer(const uint2 *ts, int64_t tb, int n, uint32_t a0, uint32_t a1, int q) {
    const int lo = max(0, q - kBand), hi = min(n - kK, q + kBand);
    if (hi < lo) return 0x7fff;
    uint32_t T0[6], T1[6], M[5];
#pragma unroll
    for (int w = 0; w < 6; ++w) planes32(ts, tb, (int64_t)lo + 32 * w, T0[w], T1[w]);
#pragma unroll
    for (int w = 0; w < 5; ++w) M[w] = 0xffffffffu;
#pragma unroll
    for (int c = 0; c < kK; ++c) {
        const uint32_t k0 = 0u - ((a0 >> (31 - c)) & 1u), k1 = 0u - ((a1 >> (31 - c)) & 1u);
#pragma unroll
        for (int w = 0; w < 5; ++w) {
            const uint32_t x0 = __funnelshift_l(T0[w + 1], T0[w], c);
            const uint32_t x1 = __funnelshift_l(T1[w + 1], T1[w], c);
            M[w] &= ~((x0 ^ k0) | (x1 ^ k1));
        }
    }
    const int ncand = hi - lo + 1, u0 = q - lo;
#pragma unroll
    for (int w = 0; w < 5; ++w) {
        const int keep = ncand - 32 * w;
        M[w] &= keep <= 0 ? 0u : (keep >= 32 ? 0xffffffffu : (0xffffffffu << (32 - keep)));
    }
    // first candidate at or after u0, last one before u0
    const int wf = u0 >> 5, bf = u0 & 31;
    const int wb = (u0 - 1) >> 5, bb = (u0 - 1) & 31;
    int uf = 1 << 20, ub = -(1 << 20);
#pragma unroll
    for (int w = 4; w >= 0; --w) {
        const uint32_t v = w > wf ? M[w] : (w == wf ? (M[w] & (0xffffffffu >> bf)) : 0u);
        if (v) uf = 32 * w + __clz(v);
    }
    if (u0 > 0) {
#pragma unroll
        for (int w = 0; w < 5; ++w) {
            const uint32_t v = w < wb ? M[w] : (w == wb ? (M[w] & (0xffffffffu << (31 - bb))) : 0u);
            if (v) ub = 32 * w + 31 - (__ffs(v) - 1);
        }
    }
    const bool hf = uf < (1 << 20), hb = ub > -(1 << 20);
    if (!hf && !hb) return 0x7fff;
    if (hb && (!hf || u0 - ub <= uf - u0)) return ub - u0;
    return uf - u0;
}

__global__ void __launch_bounds__(256) features_kernel(const uint32_t *texts, const int64_t *text_off,
                                                       const int32_t *text_len, const uint32_t *patterns,
                                                       const int64_t *pat_off, const int32_t *pat_len, int32_t n_pairs,
                                                       float *feat) {
    constexpr int GPB = 256 / kFeatLanes;  // pair groups per block
    __shared__ int16_t delta_s[GPB][kSamples];
    const int lane = threadIdx.x & (kFeatLanes - 1), gib = threadIdx.x / kFeatLanes;
    const uint32_t gmask = 0xffu << (kFeatLanes * ((threadIdx.x & 31) / kFeatLanes));
    const int64_t group = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / kFeatLanes;
    const int64_t ngroups = ((int64_t)gridDim.x * blockDim.x) / kFeatLanes;
    for (int64_t p = group; p < n_pairs; p += ngroups) {
        const int n = text_len[p], m = pat_len[p];
        const uint2 *ts = reinterpret_cast<const uint2 *>(texts + (text_off[p] >> 4));
        const uint2 *ps = reinterpret_cast<const uint2 *>(patterns + (pat_off[p] >> 4));
        const int64_t tb = (n + 31) >> 5, pb = (m + 31) >> 5;
        const int nsamp_max = m >= kK ? m - kK + 1 : 0;
        const int stride = max(16, (nsamp_max + kSamples - 1) / kSamples);
        const int nsamp = nsamp_max > 0 ? min(kSamples, (nsamp_max + stride - 1) / stride) : 0;
        int hits = 0;
        float sum = 0.f, sum2 = 0.f;
        for (int s = lane; s < nsamp; s += kFeatLanes) {
            const int q = s * stride;
            uint32_t a0, a1;
            planes32(ps, pb, q, a0, a1);
            const int best = nearest_kmer(ts, tb, n, a0, a1, q);
            delta_s[gib][s] = (int16_t)best;
            if (best != 0x7fff) {
                hits += 1;
                sum += (float)best;
                sum2 += (float)best * (float)best;
            }
        }
#pragma unroll
        for (int o = kFeatLanes / 2; o > 0; o >>= 1) {
            hits += __shfl_xor_sync(gmask, hits, o, kFeatLanes);
            sum += __shfl_xor_sync(gmask, sum, o, kFeatLanes);
            sum2 += __shfl_xor_sync(gmask, sum2, o, kFeatLanes);
        }
        const float mean = hits > 0 ? sum / hits : 0.f;
        __syncwarp(gmask);
        int near = 0;
        for (int s = lane; s < nsamp; s += kFeatLanes) {
            const int dlt = delta_s[gib][s];
            if (dlt != 0x7fff && fabsf((float)dlt - mean) <= 16.f) near += 1;
        }
#pragma unroll
        for (int o = kFeatLanes / 2; o > 0; o >>= 1) near += __shfl_xor_sync(gmask, near, o, kFeatLanes);
        __syncwarp(gmask);
        if (lane == 0) {
            float *f = feat + p * kFeatures;
            f[0] = log2f((float)m + 1.f);
            f[1] = log2f((float)n + 1.f);
            f[2] = (float)(n - m) / (float)max(m, 1);
            f[3] = nsamp > 0 ? (float)hits / (float)nsamp : 0.f;
            const float var = hits > 0 ? fmaxf(sum2 / hits - mean * mean, 0.f) : 0.f;
            f[4] = sqrtf(var) / 64.f;
            f[5] = hits > 0 ? (float)near / (float)hits : 0.f;
        }
    }
}

// Model parameter layout (floats): W1[H][F] b1[H] W2[H][H] b2[H] w3[H] b3 mu[F] sd[F]
constexpr int kH = kHidden, kF = kFeatures;
constexpr int oW1 = 0, ob1 = oW1 + kH * kF, oW2 = ob1 + kH, ob2 = oW2 + kH * kH, ow3 = ob2 + kH, ob3 = ow3 + kH,
              omu = ob3 + 1, osd = omu + kF;
static_assert(osd + kF == kModelFloats, "model layout");

// One thread per pair; the model lives in shared memory.
__global__ void __launch_bounds__(128) mlp_forward_kernel(const float *model, const float *feat, int32_t n,
                                                          float *pred) {
    __shared__ float w[kModelFloats];
    for (int i = threadIdx.x; i < kModelFloats; i += blockDim.x) w[i] = model[i];
    __syncthreads();
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    float x[kF];
#pragma unroll
    for (int f = 0; f < kF; ++f) x[f] = (feat[p * kF + f] - w[omu + f]) / w[osd + f];
    float h1[kH];
#pragma unroll
    for (int o = 0; o < kH; ++o) {
        float a = w[ob1 + o];
#pragma unroll
        for (int f = 0; f < kF; ++f) a = fmaf(w[oW1 + o * kF + f], x[f], a);
        h1[o] = fmaxf(a, 0.f);
    }
    float y = w[ob3];
    for (int o = 0; o < kH; ++o) {
        float a = w[ob2 + o];
#pragma unroll
        for (int i = 0; i < kH; ++i) a = fmaf(w[oW2 + o * kH + i], h1[i], a);
        y = fmaf(w[ow3 + o], fmaxf(a, 0.f), y);
    }
    pred[p] = y;
}

// Gradient of the mean squared error over samples [0, n) (targets t) into
// grad (zeroed by the caller), accumulated with atomics; loss_sum gets the sum
// of squared errors. Blocks of kH threads, thread o owns hidden unit o.
__global__ void __launch_bounds__(kH) mlp_grad_kernel(const float *model, const float *feat, const float *target,
                                                      const int32_t *rows, int32_t n, float inv_n, float *grad,
                                                      float *loss_sum) {
    __shared__ float w[kModelFloats];
    __shared__ float h1s[kH], d2s[kH], xs[kF], red[kH];
    for (int i = threadIdx.x; i < kModelFloats; i += blockDim.x) w[i] = model[i];
    __syncthreads();
    const int o = threadIdx.x;
    float gW2[kH];
#pragma unroll
    for (int i = 0; i < kH; ++i) gW2[i] = 0.f;
    float gW1[kF];
#pragma unroll
    for (int f = 0; f < kF; ++f) gW1[f] = 0.f;
    float gb1 = 0.f, gb2 = 0.f, gw3 = 0.f, gb3 = 0.f, loss = 0.f;
    for (int64_t q = blockIdx.x; q < n; q += gridDim.x) {
        const int64_t s = rows ? rows[q] : q;
        if (o < kF) xs[o] = (feat[s * kF + o] - w[omu + o]) / w[osd + o];
        __syncthreads();
        float a1 = w[ob1 + o];
#pragma unroll
        for (int f = 0; f < kF; ++f) a1 = fmaf(w[oW1 + o * kF + f], xs[f], a1);
        const float h1 = fmaxf(a1, 0.f);
        h1s[o] = h1;
        __syncthreads();
        float a2 = w[ob2 + o];
#pragma unroll 8
        for (int i = 0; i < kH; ++i) a2 = fmaf(w[oW2 + o * kH + i], h1s[i], a2);
        const float h2 = fmaxf(a2, 0.f);
        red[o] = w[ow3 + o] * h2;
        __syncthreads();
        for (int st = kH / 2; st > 0; st >>= 1) {
            if (o < st) red[o] += red[o + st];
            __syncthreads();
        }
        const float y = red[0] + w[ob3];
        const float err = y - target[s];
        const float dy = 2.f * err * inv_n;
        if (o == 0) {
            loss += err * err;
            gb3 += dy;
        }
        gw3 += dy * h2;
        const float d2 = a2 > 0.f ? dy * w[ow3 + o] : 0.f;
        d2s[o] = d2;
        gb2 += d2;
#pragma unroll
        for (int i = 0; i < kH; ++i) gW2[i] = fmaf(d2, h1s[i], gW2[i]);
        __syncthreads();
        // dh1[o] = sum_j W2[j][o] d2[j]
        float dh1 = 0.f;
#pragma unroll 8
        for (int j = 0; j < kH; ++j) dh1 = fmaf(w[oW2 + j * kH + o], d2s[j], dh1);
        const float d1 = a1 > 0.f ? dh1 : 0.f;
        gb1 += d1;
#pragma unroll
        for (int f = 0; f < kF; ++f) gW1[f] = fmaf(d1, xs[f], gW1[f]);
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < kH; ++i) atomicAdd(grad + oW2 + o * kH + i, gW2[i]);
#pragma unroll
    for (int f = 0; f < kF; ++f) atomicAdd(grad + oW1 + o * kF + f, gW1[f]);
    atomicAdd(grad + ob1 + o, gb1);
    atomicAdd(grad + ob2 + o, gb2);
    atomicAdd(grad + ow3 + o, gw3);
    if (o == 0) {
        atomicAdd(grad + ob3, gb3);
        atomicAdd(loss_sum, loss);
    }
}

// Mean and standard deviation of each feature column into the model's mu, sd
// (one warp per feature; a zero spread becomes 1 so the input stays finite).
__global__ void feature_stats_kernel(const float *feat, int32_t n, float *model) {
    const int f = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (f >= kF) return;
    double s1 = 0.0, s2 = 0.0;
    for (int64_t p = lane; p < n; p += 32) {
        const double v = feat[p * kF + f];
        s1 += v;
        s2 += v * v;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    }
    if (lane == 0) {
        const double mean = n > 0 ? s1 / n : 0.0;
        const double var = n > 0 ? s2 / n - mean * mean : 0.0;
        model[omu + f] = (float)mean;
        model[osd + f] = var > 1e-12 ? (float)sqrt(var) : 1.f;
    }
}

// Adam step on the trainable part of the model (everything but mu, sd).
__global__ void adam_kernel(float *model, const float *grad, float *m1, float *m2, int32_t n_params, float lr,
                            float beta1, float beta2, float eps, float bc1, float bc2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_params) return;
    const float gr = grad[i];
    const float a = beta1 * m1[i] + (1.f - beta1) * gr;
    const float b = beta2 * m2[i] + (1.f - beta2) * gr * gr;
    m1[i] = a;
    m2[i] = b;
    model[i] -= lr * (a / bc1) / (sqrtf(b / bc2) + eps);
}

// Bucket key of each pair from the predicted per-window load (log1p of the
// mean DP rows per window) and the pattern length. 8-bit key, sorted ascending
// (a stable sort keeps input order inside a bucket):
//   bit 7     0 for the long pairs (work class >= long_class): they go first;
//   bit 6     0 for the heavy pairs (load class >= heavy_class): they go next;
//   bits 0-5  length class, eighths of an octave below the batch's longest pattern: the longest
//             pairs first (the windows of a pair are sequential, so the longest chains must start
//             first; on the measured batches ordering by predicted load inside this key gained
//             nothing over length alone).
// rows = predicted mean DP rows per window, load class = floor(4 log2(rows + 1)) in 0..15,
// work class = floor(log2((m + 1)(rows + 1))) - 6 in 0..15.
// The longest pattern of the batch (one block).
__global__ void __launch_bounds__(1024) max_len_kernel(const int32_t *pat_len, int32_t n, int32_t *out) {
    __shared__ int32_t wmax[32];
    int32_t v = 0;
    for (int64_t p = threadIdx.x; p < n; p += blockDim.x) v = max(v, pat_len[p]);
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        v = threadIdx.x < (blockDim.x >> 5) ? wmax[threadIdx.x] : 0;
        for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (threadIdx.x == 0) *out = v;
    }
}

__global__ void bucket_key_kernel(const float *pred, const int32_t *pat_len, int32_t n, int heavy_class,
                                  int long_class, const int32_t *max_len, uint8_t *key) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const float rows = fmaxf(expm1f(pred[p]), 0.f);
    int load = (int)floorf(log2f(rows + 1.f) * 4.f);
    load = max(0, min(15, load));
    int work = (int)floorf(log2f(((float)pat_len[p] + 1.f) * (rows + 1.f))) - 6;
    work = max(0, min(15, work));
    const int shortp = work >= long_class ? 0 : 1;
    const int light = load >= heavy_class ? 0 : 1;
    // length class: eighths of an octave below the batch's longest pattern (longest first)
    int lc = (int)floorf((log2f((float)*max_len + 1.f) - log2f((float)pat_len[p] + 1.f)) * 8.f);
    lc = max(0, min(63, lc));
    key[p] = (uint8_t)((shortp << 7) | (light << 6) | lc);
}

constexpr int kSortTile = 2048;  // elements per block of the counting sort

__global__ void __launch_bounds__(256) key_hist_kernel(const uint8_t *key, int32_t n, int32_t *counts, int nblocks) {
    __shared__ int32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
    for (int i = threadIdx.x; i < kSortTile; i += blockDim.x) {
        const int64_t p = base + i;
        if (p < n) atomicAdd(&h[key[p]], 1);
    }
    __syncthreads();
    counts[(int64_t)threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];  // bucket-major
}

// One warp per tile, 32 elements per round in input order: stable.
__global__ void __launch_bounds__(32) key_scatter_kernel(const uint8_t *key, int32_t n, const int64_t *offsets,
                                                         int nblocks, int32_t *order) {
    __shared__ int64_t next[256];
    const int lane = threadIdx.x;
    for (int b = lane; b < 256; b += 32) next[b] = offsets[(int64_t)b * nblocks + blockIdx.x];
    __syncwarp();
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
    for (int r = 0; r < kSortTile; r += 32) {
        const int64_t p = base + r + lane;
        const bool ok = p < n;
        const int k = ok ? key[p] : 256 + lane;  // out-of-range lanes never match
        const uint32_t same = __match_any_sync(0xffffffffu, k);
        const int rank = __popc(same & ((1u << lane) - 1u));
        if (ok) order[next[k] + rank] = (int32_t)p;
        __syncwarp();
        if (ok && rank == 0) next[k] += __popc(same);
        __syncwarp();
    }
}

}  // namespace

cudaError_t launch_features(const uint32_t *texts, const int64_t *text_off, const int32_t *text_len,
                            const uint32_t *patterns, const int64_t *pat_off, const int32_t *pat_len, int32_t n,
                            float *feat, int sm_count, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int64_t blocks = std::min<int64_t>(((int64_t)n * kFeatLanes + 255) / 256, (int64_t)sm_count * 16);
    features_kernel<<<(unsigned)blocks, 256, 0, s>>>(texts, text_off, text_len, patterns, pat_off, pat_len, n, feat);
    return cudaGetLastError();
}

cudaError_t launch_mlp_forward(const float *model, const float *feat, int32_t n, float *pred, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    mlp_forward_kernel<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(model, feat, n, pred);
    return cudaGetLastError();
}

cudaError_t launch_mlp_grad(const float *model, const float *feat, const float *target, const int32_t *rows,
                            int32_t n, float *grad, float *loss_sum, int sm_count, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(grad, 0, sizeof(float) * kModelFloats, s);
    if (e != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(loss_sum, 0, sizeof(float), s)) != cudaSuccess) return e;
    if (n <= 0) return cudaSuccess;
    const int blocks = (int)std::min<int64_t>(n, (int64_t)sm_count * 4);
    mlp_grad_kernel<<<blocks, kH, 0, s>>>(model, feat, target, rows, n, 1.f / (float)n, grad, loss_sum);
    return cudaGetLastError();
}

cudaError_t launch_adam(float *model, const float *grad, float *m1, float *m2, float lr, int step, cudaStream_t s) {
    const float b1 = 0.9f, b2 = 0.999f;
    const int n = kModelFloats - 2 * kF;  // mu and sd stay fixed
    adam_kernel<<<(n + 255) / 256, 256, 0, s>>>(model, grad, m1, m2, n, lr, b1, b2, 1e-8f,
                                                1.f - powf(b1, (float)step), 1.f - powf(b2, (float)step));
    return cudaGetLastError();
}

cudaError_t launch_feature_stats(const float *feat, int32_t n, float *model, cudaStream_t s) {
    feature_stats_kernel<<<1, 32 * kF, 0, s>>>(feat, n, model);
    return cudaGetLastError();
}

int learned_kernel_count(int32_t n) {
    if (n <= 0) return 0;
    const int64_t nb = ((int64_t)n + kSortTile - 1) / kSortTile;
    return 2 /* features, MLP */ + 1 /* longest pattern */ + 1 /* keys */ + 1 /* histogram */ +
           scan_kernel_count(256 * nb) + 1 /* scatter */;
}

int64_t sort_temp_words(int32_t n) {
    const int64_t nb = ((int64_t)n + kSortTile - 1) / kSortTile;
    return 256 * nb * 3 + scan_temp_words(256 * nb) + 8;
}

const int64_t *learned_bucket_start(const int64_t *tmp, int32_t n, int key) {
    const int64_t nb = ((int64_t)n + kSortTile - 1) / kSortTile;
    return tmp + 256 * nb + (int64_t)key * nb;  // bucket-major exclusive offsets, tile 0 of the bucket
}

cudaError_t launch_learned_order(const float *pred, const int32_t *pat_len, int32_t n, int heavy_class, int long_class,
                                 uint8_t *key, int32_t *order, int64_t *tmp, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int nb = (int)(((int64_t)n + kSortTile - 1) / kSortTile);
    int32_t *counts = reinterpret_cast<int32_t *>(tmp);       // 256 * nb int32
    int64_t *offsets = tmp + 256 * (int64_t)nb;               // 256 * nb + 1 int64
    int64_t *scan_tmp = offsets + 256 * (int64_t)nb + 8;
    int32_t *max_len = reinterpret_cast<int32_t *>(tmp + sort_temp_words(n) - 2);  // past the scan's scratch
    max_len_kernel<<<1, 1024, 0, s>>>(pat_len, n, max_len);
    bucket_key_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(pred, pat_len, n, heavy_class, long_class, max_len,
                                                                  key);
    key_hist_kernel<<<nb, 256, 0, s>>>(key, n, counts, nb);
    cudaError_t e = exclusive_scan(counts, 0, 256 * (int64_t)nb, offsets, scan_tmp, s);
    if (e != cudaSuccess) return e;
    key_scatter_kernel<<<nb, 32, 0, s>>>(key, n, offsets, nb, order);
    return cudaGetLastError();
}

}  // namespace scrooge
