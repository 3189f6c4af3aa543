// C ABI of the learned pair ordering: features, MLP parameters, inference,
// gradients and training. The operations are described in include/scrooge.h.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "scrooge_ctx.h"

using namespace scrooge;

namespace {

// splitmix64: seeded, reproducible initialisation and shuffling
struct SplitMix {
    uint64_t s;
    uint64_t next() {
        uint64_t z = (s += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    }
    double uniform() { return (next() >> 11) * (1.0 / 9007199254740992.0); }
};

constexpr int kH = kHidden, kF = kFeatures;
constexpr int oW1 = 0, ob1 = oW1 + kH * kF, oW2 = ob1 + kH, ob2 = oW2 + kH * kH, ow3 = ob2 + kH, ob3 = ow3 + kH,
              omu = ob3 + 1, osd = omu + kF;

int model_buffers(scrooge_ctx *c) {
    int rc;
    if ((rc = ensure(c, c->model, kModelFloats * 4, "model")) || (rc = ensure(c, c->grad, kModelFloats * 4, "gradient")) ||
        (rc = ensure(c, c->adam_m1, kModelFloats * 4, "Adam moments")) ||
        (rc = ensure(c, c->adam_m2, kModelFloats * 4, "Adam moments")))
        return rc;
    return SCROOGE_OK;
}

}  // namespace

namespace scrooge {

int learned_order(scrooge_ctx *c, const uint32_t *texts, const int64_t *text_off, const int32_t *text_len,
                  const uint32_t *patterns, const int64_t *pat_off, const int32_t *pat_len, int32_t n) {
    if (!c->model_ready) return fail(c, SCROOGE_E_NOMODEL, "no model loaded or trained");
    int rc;
    const size_t np = (size_t)std::max(n, 1);
    if ((rc = ensure(c, c->l_feat, np * kF * 4, "features")) || (rc = ensure(c, c->l_pred, np * 4, "predictions")) ||
        (rc = ensure(c, c->l_key, np, "bucket keys")) || (rc = ensure(c, c->l_order, np * 4, "pair order")) ||
        (rc = ensure(c, c->l_tmp, (size_t)sort_temp_words(n) * 8, "sort scratch")))
        return rc;
    cudaError_t e;
    if ((e = launch_features(texts, text_off, text_len, patterns, pat_off, pat_len, n, (float *)c->l_feat.p,
                             c->sm_count, c->stream)) != cudaSuccess ||
        (e = launch_mlp_forward((const float *)c->model.p, (const float *)c->l_feat.p, n, (float *)c->l_pred.p,
                                c->stream)) != cudaSuccess ||
        (e = launch_learned_order((const float *)c->l_pred.p, pat_len, n, c->heavy_class, c->long_class,
                                  (uint8_t *)c->l_key.p,
                                  (int32_t *)c->l_order.p, (int64_t *)c->l_tmp.p, c->stream)) != cudaSuccess)
        return cuda_fail(c, e, "learned ordering");
    return SCROOGE_OK;
}

}  // namespace scrooge

extern "C" {

int32_t scrooge_model_floats(void) { return kModelFloats; }

int scrooge_model_set(scrooge_ctx *c, const float *params, int32_t n) {
    if (!c || !params || n != kModelFloats) return SCROOGE_E_INVAL;
    int rc = model_buffers(c);
    if (rc) return rc;
    for (int f = 0; f < kF; ++f)
        if (!(params[osd + f] > 0.f)) return fail(c, SCROOGE_E_INVAL, "feature scale %d must be > 0", f);
    cudaError_t e = cudaMemcpy(c->model.p, params, kModelFloats * 4, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(c, e, "model upload");
    c->model_ready = true;
    return SCROOGE_OK;
}

int scrooge_model_get(scrooge_ctx *c, float *params, int32_t n) {
    if (!c || !params || n != kModelFloats) return SCROOGE_E_INVAL;
    if (!c->model_ready) return fail(c, SCROOGE_E_NOMODEL, "no model loaded or trained");
    cudaError_t e = cudaMemcpy(params, c->model.p, kModelFloats * 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "model download");
    return SCROOGE_OK;
}

int scrooge_features(scrooge_ctx *c, const uint32_t *texts, const int64_t *text_offsets, const int32_t *text_lengths,
                     const uint32_t *patterns, const int64_t *pattern_offsets, const int32_t *pattern_lengths,
                     int32_t n_pairs, float *features) {
    if (!c || n_pairs < 0) return SCROOGE_E_INVAL;
    if (n_pairs == 0) return SCROOGE_OK;
    if (!texts || !text_offsets || !text_lengths || !patterns || !pattern_offsets || !pattern_lengths || !features)
        return fail(c, SCROOGE_E_INVAL, "null pointer argument");
    cudaError_t e = launch_features(texts, text_offsets, text_lengths, patterns, pattern_offsets, pattern_lengths,
                                    n_pairs, features, c->sm_count, c->stream);
    return e == cudaSuccess ? SCROOGE_OK : cuda_fail(c, e, "features");
}

int scrooge_model_predict(scrooge_ctx *c, const float *features, int32_t n, float *pred) {
    if (!c || n < 0 || (n > 0 && (!features || !pred))) return SCROOGE_E_INVAL;
    if (!c->model_ready) return fail(c, SCROOGE_E_NOMODEL, "no model loaded or trained");
    cudaError_t e = launch_mlp_forward((const float *)c->model.p, features, n, pred, c->stream);
    return e == cudaSuccess ? SCROOGE_OK : cuda_fail(c, e, "model inference");
}

int scrooge_model_grad(scrooge_ctx *c, const float *features, const float *targets, int32_t n, float *grad,
                       float *loss) {
    if (!c || n < 1 || !features || !targets || !grad) return SCROOGE_E_INVAL;
    if (!c->model_ready) return fail(c, SCROOGE_E_NOMODEL, "no model loaded or trained");
    int rc = ensure(c, c->loss, 64, "loss");
    if (rc) return rc;
    cudaError_t e = launch_mlp_grad((const float *)c->model.p, features, targets, nullptr, n, grad,
                                    (float *)c->loss.p, c->sm_count, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "model gradient");
    float sse = 0.f;
    if ((e = cudaMemcpyAsync(&sse, c->loss.p, 4, cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess ||
        (e = cudaStreamSynchronize(c->stream)) != cudaSuccess)
        return cuda_fail(c, e, "model gradient");
    if (loss) *loss = sse / (float)n;
    return SCROOGE_OK;
}

int scrooge_model_train(scrooge_ctx *c, const float *features, const float *targets, int32_t n, int32_t epochs,
                        int32_t batch, float lr, uint64_t seed, float *loss_history) {
    if (!c || n < 1 || epochs < 1 || batch < 1 || !(lr > 0.f) || !features || !targets) return SCROOGE_E_INVAL;
    int rc = model_buffers(c);
    if (rc) return rc;
    const int32_t nb = (n + batch - 1) / batch;
    if ((rc = ensure(c, c->t_rows, (size_t)n * 4, "shuffle")) || (rc = ensure(c, c->loss, (size_t)nb * 4 + 64, "loss")))
        return rc;
    cudaStream_t st = c->stream;
    cudaError_t e;
    // initial parameters: uniform(+-sqrt(6 / fan_in)) weights, zero biases,
    // output bias at the mean target; feature scaling from the training set
    SplitMix rng{seed};
    std::vector<float> w(kModelFloats, 0.f);
    const double a1 = sqrt(6.0 / kF), a2 = sqrt(6.0 / kH);
    for (int i = 0; i < kH * kF; ++i) w[oW1 + i] = (float)((2.0 * rng.uniform() - 1.0) * a1);
    for (int i = 0; i < kH * kH; ++i) w[oW2 + i] = (float)((2.0 * rng.uniform() - 1.0) * a2);
    for (int i = 0; i < kH; ++i) w[ow3 + i] = (float)((2.0 * rng.uniform() - 1.0) * a2 * 0.1);
    {
        std::vector<float> t((size_t)n);
        if ((e = cudaMemcpyAsync(t.data(), targets, (size_t)n * 4, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
            (e = cudaStreamSynchronize(st)) != cudaSuccess)
            return cuda_fail(c, e, "targets");
        double mean = 0.0;
        for (float v : t) mean += v;
        w[ob3] = (float)(mean / n);
    }
    for (int f = 0; f < kF; ++f) w[osd + f] = 1.f;
    if ((e = cudaMemcpyAsync(c->model.p, w.data(), kModelFloats * 4, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
        (e = launch_feature_stats(features, n, (float *)c->model.p, st)) != cudaSuccess ||
        (e = cudaMemsetAsync(c->adam_m1.p, 0, kModelFloats * 4, st)) != cudaSuccess ||
        (e = cudaMemsetAsync(c->adam_m2.p, 0, kModelFloats * 4, st)) != cudaSuccess)
        return cuda_fail(c, e, "model initialisation");
    std::vector<int32_t> perm((size_t)n);
    for (int32_t i = 0; i < n; ++i) perm[i] = i;
    std::vector<float> bl((size_t)nb);
    int step = 0;
    for (int ep = 0; ep < epochs; ++ep) {
        for (int32_t i = n - 1; i > 0; --i) std::swap(perm[i], perm[(int32_t)(rng.next() % (uint64_t)(i + 1))]);
        if ((e = cudaMemcpyAsync(c->t_rows.p, perm.data(), (size_t)n * 4, cudaMemcpyHostToDevice, st)) != cudaSuccess)
            return cuda_fail(c, e, "shuffle upload");
        for (int32_t b = 0; b < nb; ++b) {
            const int32_t lo = b * batch, cnt = std::min(batch, n - lo);
            if ((e = launch_mlp_grad((const float *)c->model.p, features, targets, (const int32_t *)c->t_rows.p + lo,
                                     cnt, (float *)c->grad.p, (float *)c->loss.p + b, c->sm_count, st)) != cudaSuccess ||
                (e = launch_adam((float *)c->model.p, (const float *)c->grad.p, (float *)c->adam_m1.p,
                                 (float *)c->adam_m2.p, lr, ++step, st)) != cudaSuccess)
                return cuda_fail(c, e, "training step");
        }
        if ((e = cudaMemcpyAsync(bl.data(), c->loss.p, (size_t)nb * 4, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
            (e = cudaStreamSynchronize(st)) != cudaSuccess)
            return cuda_fail(c, e, "loss download");
        double sse = 0.0;
        for (float v : bl) sse += v;
        if (loss_history) loss_history[ep] = (float)(sse / n);
    }
    c->model_ready = true;
    return SCROOGE_OK;
}

int scrooge_learned_order(scrooge_ctx *c, const uint32_t *texts, const int64_t *text_offsets,
                          const int32_t *text_lengths, const uint32_t *patterns, const int64_t *pattern_offsets,
                          const int32_t *pattern_lengths, int32_t n_pairs, int32_t *order) {
    if (!c || n_pairs < 0 || (n_pairs > 0 && !order)) return SCROOGE_E_INVAL;
    if (n_pairs == 0) return SCROOGE_OK;
    int rc = learned_order(c, texts, text_offsets, text_lengths, patterns, pattern_offsets, pattern_lengths, n_pairs);
    if (rc) return rc;
    cudaError_t e = cudaMemcpyAsync(order, c->l_order.p, (size_t)n_pairs * 4, cudaMemcpyDeviceToDevice, c->stream);
    return e == cudaSuccess ? SCROOGE_OK : cuda_fail(c, e, "order copy");
}

}  // extern "C"
