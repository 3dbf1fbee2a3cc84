// Learned sample widths: a small MLP predicts each front's largest HSS rank
// before sampling (no counterpart in the paper, which grows the width
// adaptively; the adaptive loop stays as the fallback).
//
//   features (6):  log(1 + |B|), tree level, kappa h, p, mean and variance of
//                  c over the box's elements
//   network:       xh = (x - mu) / sd; h1 = relu(W1 xh + b1);
//                  h2 = relu(W2 h1 + b2); h3 = relu(W3 h2 + b3); y = W4 h3 + b4
//   target:        (log(1 + k) - tmu) / tsd, mean squared error, Adam
//
// Training runs in FP32 with one fused forward + backward kernel per tile of
// 32 samples (per-tile gradient partials, reduced over tiles in a fixed
// order by the Adam kernel: deterministic).  Inference runs on BF16 weights
// and activations with FP32 accumulation.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.h"
#include "prof.h"

namespace hssnd {
namespace {

constexpr int NF = HSS_RANK_FEATURES, NH = HSS_RANK_HIDDEN;
constexpr int OW1 = 0, OB1 = OW1 + NH * NF, OW2 = OB1 + NH, OB2 = OW2 + NH * NH, OW3 = OB2 + NH,
              OB3 = OW3 + NH * NH, OW4 = OB3 + NH, OB4 = OW4 + NH, NP = OB4 + 1;
static_assert(NP == HSS_RANK_NPARAMS, "parameter layout");
constexpr int TS = 32;          // samples per tile
constexpr int LD = NH + 1;      // padded row of the shared-memory matrices (conflict-free columns)

struct Norm {
    float mu[NF], sd[NF], tmu, tsd;
};

// Shared-memory image of one tile: W2, W3 (padded), activations, deltas.
struct TileSmem {
    float W2[NH * LD], W3[NH * LD];
    float xh[TS][NF];
    float h1[TS][LD], h2[TS][LD], h3[TS][LD];
    float d[TS][LD];            // delta of the current layer
    float y[TS], dy[TS];
};

__device__ void load_weights(const float *__restrict__ th, TileSmem &S) {
    for (int e = threadIdx.x; e < NH * NH; e += blockDim.x) {
        const int j = e / NH, i = e % NH;
        S.W2[j * LD + i] = th[OW2 + e];
        S.W3[j * LD + i] = th[OW3 + e];
    }
}

// Fused forward and backward pass over tile blockIdx.x of a minibatch
// (sample k of the batch is row idx[k] of feat).  64 threads: thread j owns
// hidden unit j.  Writes the tile's gradient partial (NP floats) and its sum
// of squared residuals.
__global__ void __launch_bounds__(NH) k_mlp_train_tile(const float *__restrict__ th, const float *__restrict__ feat,
                                                       const float *__restrict__ target, const int *__restrict__ idx,
                                                       int nb, Norm nm, float gscale, float *__restrict__ partial,
                                                       float *__restrict__ lossp) {
    extern __shared__ __align__(16) unsigned char smraw[];
    TileSmem &S = *reinterpret_cast<TileSmem *>(smraw);
    const int j = threadIdx.x;
    const int s0 = blockIdx.x * TS;
    const int ns = min(TS, nb - s0);
    load_weights(th, S);
    for (int e = j; e < TS * NF; e += NH) {
        const int s = e / NF, i = e % NF;
        float v = 0.f;
        if (s < ns) v = (feat[(long)idx[s0 + s] * NF + i] - nm.mu[i]) / nm.sd[i];
        S.xh[s][i] = v;
    }
    __syncthreads();
    // ---- forward
    float w1[NF];
#pragma unroll
    for (int i = 0; i < NF; ++i) w1[i] = th[OW1 + j * NF + i];
    const float b1 = th[OB1 + j], b2 = th[OB2 + j], b3 = th[OB3 + j], w4 = th[OW4 + j];
    for (int s = 0; s < TS; ++s) {
        float z = b1;
#pragma unroll
        for (int i = 0; i < NF; ++i) z = fmaf(w1[i], S.xh[s][i], z);
        S.h1[s][j] = fmaxf(z, 0.f);
    }
    __syncthreads();
    for (int s = 0; s < TS; ++s) {
        float z = b2;
        for (int i = 0; i < NH; ++i) z = fmaf(S.W2[j * LD + i], S.h1[s][i], z);
        S.h2[s][j] = fmaxf(z, 0.f);
    }
    __syncthreads();
    for (int s = 0; s < TS; ++s) {
        float z = b3;
        for (int i = 0; i < NH; ++i) z = fmaf(S.W3[j * LD + i], S.h2[s][i], z);
        S.h3[s][j] = fmaxf(z, 0.f);
    }
    __syncthreads();
    if (j < TS) {
        float yv = th[OB4];
        for (int i = 0; i < NH; ++i) yv = fmaf(th[OW4 + i], S.h3[j][i], yv);
        float r = 0.f;
        if (j < ns) r = yv - (target[idx[s0 + j]] - nm.tmu) / nm.tsd;
        S.y[j] = yv;
        S.dy[j] = gscale * 2.f * r;
        S.d[j][NH] = r * r;   // scratch column for the loss
    }
    __syncthreads();
    if (j == 0) {
        float l = 0.f;
        for (int s = 0; s < TS; ++s) l += S.d[s][NH];
        lossp[blockIdx.x] = l;
    }
    float *gp = partial + (long)blockIdx.x * NP;
    // ---- output layer
    {
        float gw = 0.f;
        for (int s = 0; s < TS; ++s) gw = fmaf(S.dy[s], S.h3[s][j], gw);
        gp[OW4 + j] = gw;
        if (j == 0) {
            float gb = 0.f;
            for (int s = 0; s < TS; ++s) gb += S.dy[s];
            gp[OB4] = gb;
        }
    }
    __syncthreads();
    for (int s = 0; s < TS; ++s) S.d[s][j] = S.h3[s][j] > 0.f ? S.dy[s] * w4 : 0.f;   // delta of layer 3
    __syncthreads();
    // ---- layer 3: gW3[j][i] = sum_s d3[s][j] h2[s][i]
    {
        float gb = 0.f;
        for (int s = 0; s < TS; ++s) gb += S.d[s][j];
        gp[OB3 + j] = gb;
        for (int i = 0; i < NH; ++i) {
            float g = 0.f;
            for (int s = 0; s < TS; ++s) g = fmaf(S.d[s][j], S.h2[s][i], g);
            gp[OW3 + j * NH + i] = g;
        }
    }
    // delta of layer 2 for unit j: sum_k W3[k][j] d3[s][k], masked
    float d2v[TS];
    for (int s = 0; s < TS; ++s) {
        float a = 0.f;
        for (int k = 0; k < NH; ++k) a = fmaf(S.W3[k * LD + j], S.d[s][k], a);
        d2v[s] = S.h2[s][j] > 0.f ? a : 0.f;
    }
    __syncthreads();
    for (int s = 0; s < TS; ++s) S.d[s][j] = d2v[s];
    __syncthreads();
    // ---- layer 2
    {
        float gb = 0.f;
        for (int s = 0; s < TS; ++s) gb += S.d[s][j];
        gp[OB2 + j] = gb;
        for (int i = 0; i < NH; ++i) {
            float g = 0.f;
            for (int s = 0; s < TS; ++s) g = fmaf(S.d[s][j], S.h1[s][i], g);
            gp[OW2 + j * NH + i] = g;
        }
    }
    float d1v[TS];
    for (int s = 0; s < TS; ++s) {
        float a = 0.f;
        for (int k = 0; k < NH; ++k) a = fmaf(S.W2[k * LD + j], S.d[s][k], a);
        d1v[s] = S.h1[s][j] > 0.f ? a : 0.f;
    }
    // ---- layer 1
    {
        float gb = 0.f;
        for (int s = 0; s < TS; ++s) gb += d1v[s];
        gp[OB1 + j] = gb;
#pragma unroll
        for (int i = 0; i < NF; ++i) {
            float g = 0.f;
            for (int s = 0; s < TS; ++s) g = fmaf(d1v[s], S.xh[s][i], g);
            gp[OW1 + j * NF + i] = g;
        }
    }
}

// grad[p] = sum over tiles of the partials (fixed order); with lr > 0 also
// one Adam step on parameter p (step counted from 1).
__global__ void k_mlp_reduce_adam(const float *__restrict__ partial, int ntiles, float *__restrict__ grad,
                                  float *__restrict__ th, float *__restrict__ m, float *__restrict__ v, float lr,
                                  float c1, float c2) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= NP) return;
    float g = 0.f;
    for (int t = 0; t < ntiles; ++t) g += partial[(long)t * NP + p];
    if (grad) grad[p] = g;
    if (lr > 0.f) {
        const float mm = 0.9f * m[p] + 0.1f * g;
        const float vv = 0.999f * v[p] + 0.001f * g * g;
        m[p] = mm;
        v[p] = vv;
        th[p] -= lr * (mm / c1) / (sqrtf(vv / c2) + 1e-8f);
    }
}

__global__ void k_to_bf16(const float *__restrict__ th, __nv_bfloat16 *__restrict__ out) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < NP) out[p] = __float2bfloat16_rn(th[p]);
}

// BF16 inference: weights, standardised features and activations rounded to
// BF16, products accumulated in FP32.  pred[k] = tmu + tsd * y (log(1 + k)
// units); r[k] = the sample width for the prediction (a multiple of 8 that
// covers the predicted rank plus the oversampling, within [16, rmax]).
__global__ void __launch_bounds__(NH) k_mlp_infer_bf16(const __nv_bfloat16 *__restrict__ wb,
                                                       const float *__restrict__ feat, int n, Norm nm,
                                                       int oversample, int rmax, float *__restrict__ pred,
                                                       int *__restrict__ rout) {
    __shared__ __nv_bfloat16 W2[NH * LD], W3[NH * LD];
    __shared__ __nv_bfloat16 xh[TS][NF], h1[TS][LD], h2[TS][LD], h3[TS][LD];
    const int j = threadIdx.x, s0 = blockIdx.x * TS, ns = min(TS, n - s0);
    for (int e = j; e < NH * NH; e += NH) {
        W2[(e / NH) * LD + e % NH] = wb[OW2 + e];
        W3[(e / NH) * LD + e % NH] = wb[OW3 + e];
    }
    for (int e = j; e < TS * NF; e += NH) {
        const int s = e / NF, i = e % NF;
        xh[s][i] = __float2bfloat16_rn(s < ns ? (feat[(long)(s0 + s) * NF + i] - nm.mu[i]) / nm.sd[i] : 0.f);
    }
    __syncthreads();
    for (int s = 0; s < TS; ++s) {
        float z = __bfloat162float(wb[OB1 + j]);
        for (int i = 0; i < NF; ++i) z = fmaf(__bfloat162float(wb[OW1 + j * NF + i]), __bfloat162float(xh[s][i]), z);
        h1[s][j] = __float2bfloat16_rn(fmaxf(z, 0.f));
    }
    __syncthreads();
    for (int s = 0; s < TS; ++s) {
        float z = __bfloat162float(wb[OB2 + j]);
        for (int i = 0; i < NH; ++i) z = fmaf(__bfloat162float(W2[j * LD + i]), __bfloat162float(h1[s][i]), z);
        h2[s][j] = __float2bfloat16_rn(fmaxf(z, 0.f));
    }
    __syncthreads();
    for (int s = 0; s < TS; ++s) {
        float z = __bfloat162float(wb[OB3 + j]);
        for (int i = 0; i < NH; ++i) z = fmaf(__bfloat162float(W3[j * LD + i]), __bfloat162float(h2[s][i]), z);
        h3[s][j] = __float2bfloat16_rn(fmaxf(z, 0.f));
    }
    __syncthreads();
    if (j < ns) {
        float y = __bfloat162float(wb[OB4]);
        for (int i = 0; i < NH; ++i) y = fmaf(__bfloat162float(wb[OW4 + i]), __bfloat162float(h3[j][i]), y);
        const float lk = nm.tmu + nm.tsd * y;
        pred[s0 + j] = lk;
        if (rout) {
            const float k = fmaxf(expm1f(lk), 0.f);
            int r = (int)ceilf((k + (float)oversample) / 8.f) * 8;
            rout[s0 + j] = min(max(r, 16), rmax);
        }
    }
}

}  // namespace
}  // namespace hssnd

struct hss_rank_model {
    hssnd::DevBuf theta, m, v, bf, partial, grad, lossp;
    long partial_tiles = 0;
    hssnd::Norm norm{};
    int step = 0;
    bool bf_fresh = false;
};

namespace hssnd {
namespace {

int ensure_tiles(hss_rank_model *M, long tiles) {
    if (tiles <= M->partial_tiles) return HSS_OK;
    int rc;
    if ((rc = M->partial.alloc(sizeof(float) * tiles * NP)) || (rc = M->lossp.alloc(sizeof(float) * tiles)))
        return rc;
    M->partial_tiles = tiles;
    return HSS_OK;
}

// One fused pass over n samples (rows idx of feat): gradient partials and
// squared residuals; then the reduction (and an Adam step when lr > 0).
int train_pass(hss_rank_model *M, const float *feat, const float *target, const int *idx, int n, float lr,
               float *loss_out, cudaStream_t s) {
    const int tiles = cdiv(n, TS);
    int rc;
    if ((rc = ensure_tiles(M, tiles))) return rc;
    HSS_SMEM(k_mlp_train_tile, sizeof(TileSmem));
    {
        HSS_PROF("mlp_train_tile", s);
        k_mlp_train_tile<<<tiles, NH, sizeof(TileSmem), s>>>(M->theta.as<float>(), feat, target, idx, n, M->norm,
                                                             1.f / (float)n, M->partial.as<float>(),
                                                             M->lossp.as<float>());
    }
    float c1 = 1.f, c2 = 1.f;
    if (lr > 0.f) {
        ++M->step;
        c1 = 1.f - powf(0.9f, (float)M->step);
        c2 = 1.f - powf(0.999f, (float)M->step);
    }
    {
        HSS_PROF("mlp_reduce_adam", s);
        k_mlp_reduce_adam<<<cdiv(NP, 256), 256, 0, s>>>(M->partial.as<float>(), tiles, M->grad.as<float>(),
                                                        M->theta.as<float>(), M->m.as<float>(), M->v.as<float>(), lr,
                                                        c1, c2);
    }
    HSS_CHECK_LAUNCH("mlp train pass");
    M->bf_fresh = false;
    if (loss_out) {
        std::vector<float> lp(tiles);
        HSS_CUDA(cudaMemcpyAsync(lp.data(), M->lossp.p, sizeof(float) * tiles, cudaMemcpyDeviceToHost, s));
        HSS_CUDA(cudaStreamSynchronize(s));
        double l = 0.0;
        for (float x : lp) l += x;
        *loss_out = (float)(l / n);
    }
    return HSS_OK;
}

}  // namespace
}  // namespace hssnd

using namespace hssnd;

extern "C" int hss_rank_model_create(uint64_t seed, hss_rank_model **out) {
    if (!out) {
        set_error("hss_rank_model_create: null argument");
        return HSS_EINVAL;
    }
    *out = nullptr;
    auto *M = new hss_rank_model();
    // He initialisation from the counter hash: uniform in [-a, a] with a = sqrt(6 / fan_in); biases 0
    std::vector<float> th(NP, 0.f);
    auto fill = [&](int off, int rows, int fan_in) {
        const float a = std::sqrt(6.f / (float)fan_in);
        for (int e = 0; e < rows * fan_in; ++e) {
            const uint64_t h = splitmix64(seed ^ ((uint64_t)(off + e) * 0x9E3779B97F4A7C15ULL));
            const float u = (float)((h >> 11) * (1.0 / 9007199254740992.0));
            th[off + e] = (2.f * u - 1.f) * a;
        }
    };
    fill(OW1, NH, NF);
    fill(OW2, NH, NH);
    fill(OW3, NH, NH);
    fill(OW4, 1, NH);
    for (int i = 0; i < NF; ++i) {
        M->norm.mu[i] = 0.f;
        M->norm.sd[i] = 1.f;
    }
    M->norm.tmu = 0.f;
    M->norm.tsd = 1.f;
    int rc;
    if ((rc = M->theta.alloc(sizeof(float) * NP)) || (rc = M->m.alloc(sizeof(float) * NP)) ||
        (rc = M->v.alloc(sizeof(float) * NP)) || (rc = M->grad.alloc(sizeof(float) * NP)) ||
        (rc = M->bf.alloc(sizeof(__nv_bfloat16) * NP))) {
        delete M;
        return rc;
    }
    if (cudaMemcpy(M->theta.p, th.data(), sizeof(float) * NP, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(M->m.p, 0, sizeof(float) * NP) != cudaSuccess ||
        cudaMemset(M->v.p, 0, sizeof(float) * NP) != cudaSuccess) {
        delete M;
        return cuda_fail(cudaGetLastError(), "hss_rank_model_create");
    }
    *out = M;
    return HSS_OK;
}

extern "C" void hss_rank_model_destroy(hss_rank_model *m) { delete m; }

extern "C" int hss_rank_model_get(const hss_rank_model *M, float *params, float *norm) {
    if (!M) {
        set_error("hss_rank_model_get: null model");
        return HSS_EINVAL;
    }
    if (params) HSS_CUDA(cudaMemcpy(params, M->theta.p, sizeof(float) * NP, cudaMemcpyDeviceToHost));
    if (norm) {
        for (int i = 0; i < NF; ++i) {
            norm[i] = M->norm.mu[i];
            norm[NF + i] = M->norm.sd[i];
        }
        norm[2 * NF] = M->norm.tmu;
        norm[2 * NF + 1] = M->norm.tsd;
    }
    return HSS_OK;
}

extern "C" int hss_rank_model_set(hss_rank_model *M, const float *params, const float *norm) {
    if (!M) {
        set_error("hss_rank_model_set: null model");
        return HSS_EINVAL;
    }
    if (norm) {
        for (int i = 0; i < NF; ++i) {
            if (!(norm[NF + i] > 0.f)) {
                set_error("hss_rank_model_set: standard deviations must be positive");
                return HSS_EINVAL;
            }
            M->norm.mu[i] = norm[i];
            M->norm.sd[i] = norm[NF + i];
        }
        if (!(norm[2 * NF + 1] > 0.f)) {
            set_error("hss_rank_model_set: standard deviations must be positive");
            return HSS_EINVAL;
        }
        M->norm.tmu = norm[2 * NF];
        M->norm.tsd = norm[2 * NF + 1];
    }
    if (params) {
        HSS_CUDA(cudaMemcpy(M->theta.p, params, sizeof(float) * NP, cudaMemcpyHostToDevice));
        HSS_CUDA(cudaMemset(M->m.p, 0, sizeof(float) * NP));
        HSS_CUDA(cudaMemset(M->v.p, 0, sizeof(float) * NP));
        M->step = 0;
        M->bf_fresh = false;
    }
    return HSS_OK;
}

extern "C" int hss_rank_model_fit_norm(hss_rank_model *M, int n, const float *feat, const float *target,
                                       void *stream) {
    if (!M || !feat || !target || n < 1) {
        set_error("hss_rank_model_fit_norm: invalid argument");
        return HSS_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<float> X((size_t)n * NF), t(n);
    HSS_CUDA(cudaMemcpyAsync(X.data(), feat, sizeof(float) * X.size(), cudaMemcpyDeviceToHost, s));
    HSS_CUDA(cudaMemcpyAsync(t.data(), target, sizeof(float) * n, cudaMemcpyDeviceToHost, s));
    HSS_CUDA(cudaStreamSynchronize(s));
    // mean and population standard deviation (1 where it is zero)
    for (int i = 0; i < NF; ++i) {
        double mu = 0.0, var = 0.0;
        for (int k = 0; k < n; ++k) mu += X[(size_t)k * NF + i];
        mu /= n;
        for (int k = 0; k < n; ++k) var += (X[(size_t)k * NF + i] - mu) * (X[(size_t)k * NF + i] - mu);
        var /= n;
        M->norm.mu[i] = (float)mu;
        M->norm.sd[i] = var > 0.0 ? (float)std::sqrt(var) : 1.f;
    }
    double mu = 0.0, var = 0.0;
    for (int k = 0; k < n; ++k) mu += t[k];
    mu /= n;
    for (int k = 0; k < n; ++k) var += (t[k] - mu) * (t[k] - mu);
    var /= n;
    M->norm.tmu = (float)mu;
    M->norm.tsd = var > 0.0 ? (float)std::sqrt(var) : 1.f;
    return HSS_OK;
}

extern "C" int hss_rank_model_loss_grad(hss_rank_model *M, int n, const float *feat, const float *target,
                                        float *loss, float *grad, void *stream) {
    if (!M || !feat || !target || n < 1) {
        set_error("hss_rank_model_loss_grad: invalid argument");
        return HSS_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<int> idx(n);
    for (int k = 0; k < n; ++k) idx[k] = k;
    DevBuf d_idx;
    int rc;
    if ((rc = upload(d_idx, idx, s)) || (rc = train_pass(M, feat, target, d_idx.as<int>(), n, 0.f, loss, s)))
        return rc;
    if (grad) {
        HSS_CUDA(cudaMemcpyAsync(grad, M->grad.p, sizeof(float) * NP, cudaMemcpyDeviceToHost, s));
        HSS_CUDA(cudaStreamSynchronize(s));
    }
    return HSS_OK;
}

extern "C" int hss_rank_model_train(hss_rank_model *M, int n, const float *feat, const float *target, int epochs,
                                    int batch, float lr, uint64_t seed, float *final_loss, void *stream) {
    if (!M || !feat || !target || n < 1 || epochs < 0 || batch < 1 || !(lr > 0.f)) {
        set_error("hss_rank_model_train: invalid argument");
        return HSS_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<int> order(n);
    DevBuf d_idx;
    int rc;
    if ((rc = d_idx.alloc(sizeof(int) * (size_t)n * std::max(epochs, 1)))) return rc;
    // per epoch a permutation of the samples (Fisher-Yates driven by the counter hash)
    std::vector<int> all((size_t)n * std::max(epochs, 1));
    for (int e = 0; e < epochs; ++e) {
        for (int k = 0; k < n; ++k) order[k] = k;
        for (int k = n - 1; k > 0; --k) {
            const uint64_t h = splitmix64(seed ^ ((uint64_t)e << 32) ^ (uint64_t)k);
            std::swap(order[k], order[(int)(h % (uint64_t)(k + 1))]);
        }
        std::copy(order.begin(), order.end(), all.begin() + (size_t)e * n);
    }
    if (epochs > 0)
        HSS_CUDA(cudaMemcpyAsync(d_idx.p, all.data(), sizeof(int) * all.size(), cudaMemcpyHostToDevice, s));
    for (int e = 0; e < epochs; ++e)
        for (int b0 = 0; b0 < n; b0 += batch) {
            const int nb = std::min(batch, n - b0);
            if ((rc = train_pass(M, feat, target, d_idx.as<int>() + (size_t)e * n + b0, nb, lr, nullptr, s)))
                return rc;
        }
    if (final_loss) return hss_rank_model_loss_grad(M, n, feat, target, final_loss, nullptr, stream);
    HSS_CUDA(cudaStreamSynchronize(s));
    return HSS_OK;
}

extern "C" int hss_rank_model_predict(hss_rank_model *M, int n, const float *feat, int oversample, int rmax,
                                      float *pred, int *r, void *stream) {
    if (!M || !feat || !pred || n < 0 || oversample < 0 || rmax < 16) {
        set_error("hss_rank_model_predict: invalid argument");
        return HSS_EINVAL;
    }
    if (n == 0) return HSS_OK;
    cudaStream_t s = (cudaStream_t)stream;
    if (!M->bf_fresh) {
        HSS_PROF("mlp_to_bf16", s);
        k_to_bf16<<<cdiv(NP, 256), 256, 0, s>>>(M->theta.as<float>(), M->bf.as<__nv_bfloat16>());
        M->bf_fresh = true;
    }
    {
        HSS_PROF("mlp_infer_bf16", s);
        k_mlp_infer_bf16<<<cdiv(n, TS), NH, 0, s>>>(M->bf.as<__nv_bfloat16>(), feat, n, M->norm, oversample, rmax,
                                                    pred, r);
    }
    HSS_CHECK_LAUNCH("mlp inference");
    return HSS_OK;
}

extern "C" int hss_rank_features(const hss_tree *t, const double *c_elem, double kappa_h, float *feat) {
    if (!t || !feat) {
        set_error("hss_rank_features: null argument");
        return HSS_EINVAL;
    }
    const int bs = t->bs;
    for (int b = 0; b < t->nbox; ++b) {
        const int e0 = t->pos0[b] / bs, e1 = t->pos1[b] / bs;
        double mu = 1.0, var = 0.0;
        if (c_elem && e1 > e0) {
            mu = 0.0;
            for (int q = e0; q < e1; ++q) mu += c_elem[t->dfs_elem[q]];
            mu /= (e1 - e0);
            for (int q = e0; q < e1; ++q) var += (c_elem[t->dfs_elem[q]] - mu) * (c_elem[t->dfs_elem[q]] - mu);
            var /= (e1 - e0);
        }
        float *f = feat + (size_t)b * NF;
        f[0] = (float)std::log1p((double)t->nb[b]);
        f[1] = (float)t->level[b];
        f[2] = (float)kappa_h;
        f[3] = (float)t->p;
        f[4] = (float)mu;
        f[5] = (float)var;
    }
    return HSS_OK;
}
