// Latency predictor (Sec. 7.1, with a small MLP standing in for the paper's
// decision tree): forward, backward and Adam kernels in FP32.
//
// Network 12 -> 64 -> 64 -> 1: h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2),
// y = W3 h2 + b3, relu'(0) = 0.  Parameters in one flat vector: W1 [64x12
// row-major], b1 [64], W2 [64x64], b2 [64], W3 [64], b3 [1] (5057 values).
// Inputs are z-scored inside the kernels with the stored mean and inverse
// standard deviation: x = (raw - mean) * inv_std.  Training minimises the
// mean squared error (1/n) sum (y - t)^2 with Adam (Kingma & Ba).
//
// A training step is two launches.  Pass 1 (one thread per sample, parameters
// staged in shared memory) runs the forward pass and back-propagates the
// deltas, storing each sample's layer inputs and deltas in a structure-of-
// arrays record.  Pass 2 (one thread per parameter) sums that parameter's
// gradient over the samples in sample order and applies the Adam update, so
// every step is deterministic and independent of the launch shape.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/camelot.h"

camelot_status camelot_internal_fail(camelot_status st, const char* msg);

namespace {

constexpr int kIn = CAMELOT_PRED_FEATURES, kH = 64;
constexpr int kNP = kH * kIn + kH + kH * kH + kH + kH + 1;
static_assert(kNP == CAMELOT_PRED_PARAMS, "parameter count");
constexpr int kOffB1 = kH * kIn, kOffW2 = kOffB1 + kH, kOffB2 = kOffW2 + kH * kH,
              kOffW3 = kOffB2 + kH, kOffB3 = kOffW3 + kH;
// Record rows (each row holds one value per sample, n samples wide).
constexpr int kRX = 0, kRH1 = kIn, kRH2 = kRH1 + kH, kRD1 = kRH2 + kH, kRD2 = kRD1 + kH,
              kRDY = kRD2 + kH, kRR = kRDY + 1, kRec = kRR + 1;   // 270 rows
constexpr uint32_t kMaxTrainBatch = 65536;
constexpr int kSampleThreads = 128;

struct Norm {
    float mean[kIn];
    float inv_std[kIn];
};

__device__ __forceinline__ void stage_params(const float* __restrict__ g, float* s) {
    for (int i = threadIdx.x; i < kNP; i += blockDim.x) s[i] = g[i];
    __syncthreads();
}

__device__ __forceinline__ void load_x(const float* __restrict__ X, uint32_t row, const Norm& nm, float (&x)[kIn]) {
#pragma unroll
    for (int k = 0; k < kIn; ++k) x[k] = (X[(size_t)row * kIn + k] - nm.mean[k]) * nm.inv_std[k];
}

__device__ __forceinline__ void layer1(const float* th, const float (&x)[kIn], float (&h1)[kH]) {
#pragma unroll
    for (int j = 0; j < kH; ++j) {
        float s = th[kOffB1 + j];
#pragma unroll
        for (int k = 0; k < kIn; ++k) s = fmaf(th[j * kIn + k], x[k], s);
        h1[j] = s > 0.f ? s : 0.f;
    }
}

__device__ __forceinline__ float layer2_unit(const float* th, const float (&h1)[kH], int j) {
    float s = th[kOffB2 + j];
#pragma unroll
    for (int k = 0; k < kH; ++k) s = fmaf(th[kOffW2 + j * kH + k], h1[k], s);
    return s > 0.f ? s : 0.f;
}

__global__ void __launch_bounds__(kSampleThreads) pred_forward_kernel(const float* __restrict__ theta, Norm nm,
                                                                      const float* __restrict__ X, uint32_t n,
                                                                      float* __restrict__ y) {
    __shared__ float th[kNP];
    stage_params(theta, th);
    const uint32_t q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    float x[kIn], h1[kH];
    load_x(X, q, nm, x);
    layer1(th, x, h1);
    float out = th[kOffB3];
    for (int j = 0; j < kH; ++j) out = fmaf(th[kOffW3 + j], layer2_unit(th, h1, j), out);
    y[q] = out;
}

// Pass 1.  Sample q of the minibatch is row idx[q] of X and t (row q when idx
// is null).  rec is [kRec][n].
__global__ void __launch_bounds__(kSampleThreads) pred_backward_kernel(const float* __restrict__ theta, Norm nm,
                                                                       const float* __restrict__ X,
                                                                       const float* __restrict__ t,
                                                                       const uint32_t* __restrict__ idx,
                                                                       uint32_t n, float* __restrict__ rec) {
    __shared__ float th[kNP];
    stage_params(theta, th);
    const uint32_t q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const uint32_t row = idx ? idx[q] : q;
    float x[kIn], h1[kH], h2[kH];
    load_x(X, row, nm, x);
    layer1(th, x, h1);
    float y = th[kOffB3];
    for (int j = 0; j < kH; ++j) {
        h2[j] = layer2_unit(th, h1, j);
        y = fmaf(th[kOffW3 + j], h2[j], y);
    }
    const float r = y - t[row];
    const float dy = 2.f * r / (float)n;
#pragma unroll
    for (int k = 0; k < kIn; ++k) rec[(size_t)(kRX + k) * n + q] = x[k];
    for (int j = 0; j < kH; ++j) {
        rec[(size_t)(kRH1 + j) * n + q] = h1[j];
        rec[(size_t)(kRH2 + j) * n + q] = h2[j];
    }
    // delta of layer-2 pre-activations (h2 > 0 exactly where a2 > 0)
#pragma unroll
    for (int j = 0; j < kH; ++j) {
        h2[j] = h2[j] > 0.f ? dy * th[kOffW3 + j] : 0.f;
        rec[(size_t)(kRD2 + j) * n + q] = h2[j];
    }
    // delta of layer-1 pre-activations: (W2^T da2) masked by relu'
    for (int k = 0; k < kH; ++k) {
        float s = 0.f;
#pragma unroll
        for (int j = 0; j < kH; ++j) s = fmaf(th[kOffW2 + j * kH + k], h2[j], s);
        rec[(size_t)(kRD1 + k) * n + q] = h1[k] > 0.f ? s : 0.f;
    }
    rec[(size_t)kRDY * n + q] = dy;
    rec[(size_t)kRR * n + q] = r;
}

// Pass 2.  Gradient of parameter i = sum over samples of (delta of its output
// unit) x (its input, 1 for a bias).  Writes the gradient to grad_out and,
// when do_adam, updates theta, m, v.  Thread 0 also writes the loss.
__global__ void __launch_bounds__(256) pred_grad_adam_kernel(float* __restrict__ theta, float* __restrict__ m,
                                                             float* __restrict__ v, const float* __restrict__ rec,
                                                             uint32_t n, float* __restrict__ grad_out,
                                                             float* __restrict__ loss_out, int do_adam, float lr,
                                                             float b1, float b2, float eps, float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0 && loss_out) {
        const float* R = rec + (size_t)kRR * n;
        float s = 0.f;
        for (uint32_t q = 0; q < n; ++q) s = fmaf(R[q], R[q], s);
        *loss_out = s / (float)n;
    }
    if (i >= kNP) return;
    int drow, irow = -1;
    if (i < kOffB1) { drow = kRD1 + i / kIn; irow = kRX + i % kIn; }
    else if (i < kOffW2) { drow = kRD1 + (i - kOffB1); }
    else if (i < kOffB2) { drow = kRD2 + (i - kOffW2) / kH; irow = kRH1 + (i - kOffW2) % kH; }
    else if (i < kOffW3) { drow = kRD2 + (i - kOffB2); }
    else if (i < kOffB3) { drow = kRDY; irow = kRH2 + (i - kOffW3); }
    else { drow = kRDY; }
    const float* D = rec + (size_t)drow * n;
    float g = 0.f;
    if (irow < 0) {
        for (uint32_t q = 0; q < n; ++q) g += D[q];
    } else {
        const float* I = rec + (size_t)irow * n;
        for (uint32_t q = 0; q < n; ++q) g = fmaf(D[q], I[q], g);
    }
    if (grad_out) grad_out[i] = g;
    if (!do_adam) return;
    const float mi = b1 * m[i] + (1.f - b1) * g;
    const float vi = b2 * v[i] + (1.f - b2) * (g * g);
    m[i] = mi;
    v[i] = vi;
    theta[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

}  // namespace

struct camelot_predictor {
    float* theta = nullptr;   // device [kNP]
    float* m = nullptr;       // Adam first moment
    float* v = nullptr;       // Adam second moment
    float* rec = nullptr;     // device [kRec][kMaxTrainBatch]
    Norm norm{};
    long long step = 0;
};

#define PTRY(expr)                                                                               \
    do {                                                                                         \
        if ((expr) != cudaSuccess) return camelot_internal_fail(CAMELOT_ECUDA, #expr " failed"); \
    } while (0)

extern "C" camelot_status camelot_predictor_destroy(camelot_predictor* p) {
    if (!p) return camelot_internal_fail(CAMELOT_EINVAL, "null predictor");
    cudaFree(p->theta);
    cudaFree(p->m);
    cudaFree(p->v);
    cudaFree(p->rec);
    delete p;
    return CAMELOT_OK;
}

extern "C" camelot_status camelot_predictor_set_params(camelot_predictor* p, const float* params) {
    if (!p || !params) return camelot_internal_fail(CAMELOT_EINVAL, "null argument");
    PTRY(cudaMemcpy(p->theta, params, kNP * sizeof(float), cudaMemcpyHostToDevice));
    PTRY(cudaMemset(p->m, 0, kNP * sizeof(float)));
    PTRY(cudaMemset(p->v, 0, kNP * sizeof(float)));
    p->step = 0;
    return CAMELOT_OK;
}

extern "C" camelot_status camelot_predictor_create(const float* init_params, camelot_predictor** out) {
    if (!init_params || !out) return camelot_internal_fail(CAMELOT_EINVAL, "null argument");
    auto* p = new camelot_predictor();
    for (int k = 0; k < kIn; ++k) {
        p->norm.mean[k] = 0.f;
        p->norm.inv_std[k] = 1.f;
    }
    if (cudaMalloc(&p->theta, kNP * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&p->m, kNP * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&p->v, kNP * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&p->rec, (size_t)kRec * kMaxTrainBatch * sizeof(float)) != cudaSuccess) {
        camelot_predictor_destroy(p);
        return camelot_internal_fail(CAMELOT_ENOMEM, "predictor device allocation failed");
    }
    const camelot_status st = camelot_predictor_set_params(p, init_params);
    if (st != CAMELOT_OK) {
        camelot_predictor_destroy(p);
        return st;
    }
    *out = p;
    return CAMELOT_OK;
}

extern "C" camelot_status camelot_predictor_set_norm(camelot_predictor* p, const float* mean, const float* inv_std) {
    if (!p || !mean || !inv_std) return camelot_internal_fail(CAMELOT_EINVAL, "null argument");
    memcpy(p->norm.mean, mean, sizeof p->norm.mean);
    memcpy(p->norm.inv_std, inv_std, sizeof p->norm.inv_std);
    return CAMELOT_OK;
}

extern "C" camelot_status camelot_predictor_get_params(camelot_predictor* p, float* out) {
    if (!p || !out) return camelot_internal_fail(CAMELOT_EINVAL, "null argument");
    PTRY(cudaMemcpy(out, p->theta, kNP * sizeof(float), cudaMemcpyDeviceToHost));
    return CAMELOT_OK;
}

extern "C" camelot_status camelot_predictor_forward(camelot_predictor* p, const float* X, uint32_t n, float* y,
                                                    void* stream) {
    if (!p || !X || !y || n == 0) return camelot_internal_fail(CAMELOT_EINVAL, "null argument or n == 0");
    const unsigned blocks = (n + kSampleThreads - 1) / kSampleThreads;
    pred_forward_kernel<<<blocks, kSampleThreads, 0, (cudaStream_t)stream>>>(p->theta, p->norm, X, n, y);
    PTRY(cudaGetLastError());
    return CAMELOT_OK;
}

static camelot_status grad_step(camelot_predictor* p, const float* X, const float* t, const uint32_t* idx,
                                uint32_t n, float* grad, float* loss, bool adam, float lr, cudaStream_t s) {
    if (!p || !X || !t) return camelot_internal_fail(CAMELOT_EINVAL, "null argument");
    if (n == 0 || n > kMaxTrainBatch) return camelot_internal_fail(CAMELOT_EINVAL, "n must be in 1..65536");
    pred_backward_kernel<<<(n + kSampleThreads - 1) / kSampleThreads, kSampleThreads, 0, s>>>(
        p->theta, p->norm, X, t, idx, n, p->rec);
    PTRY(cudaGetLastError());
    const double b1 = 0.9, b2 = 0.999;
    float c1 = 1.f, c2 = 1.f;
    if (adam) {
        p->step += 1;
        c1 = (float)(1.0 - std::pow(b1, (double)p->step));
        c2 = (float)(1.0 - std::pow(b2, (double)p->step));
    }
    pred_grad_adam_kernel<<<(kNP + 255) / 256, 256, 0, s>>>(p->theta, p->m, p->v, p->rec, n, grad, loss,
                                                           adam ? 1 : 0, lr, (float)b1, (float)b2, 1e-8f, c1,
                                                           c2);
    PTRY(cudaGetLastError());
    return CAMELOT_OK;
}

extern "C" camelot_status camelot_predictor_grad(camelot_predictor* p, const float* X, const float* t,
                                                 const uint32_t* idx, uint32_t n, float* grad, float* loss,
                                                 void* stream) {
    if (!grad) return camelot_internal_fail(CAMELOT_EINVAL, "null gradient buffer");
    return grad_step(p, X, t, idx, n, grad, loss, false, 0.f, (cudaStream_t)stream);
}

extern "C" camelot_status camelot_predictor_train_step(camelot_predictor* p, const float* X, const float* t,
                                                       const uint32_t* idx, uint32_t n, float lr, float* loss,
                                                       void* stream) {
    if (!(lr > 0.f)) return camelot_internal_fail(CAMELOT_EINVAL, "lr must be positive");
    return grad_step(p, X, t, idx, n, nullptr, loss, true, lr, (cudaStream_t)stream);
}

// ---------------------------------------------------------------------------
// The predictor inside the allocator: features, table conversion, and the
// predicted camelot_profile (Sec. 7.1-7.2).
// ---------------------------------------------------------------------------
static bool cost_ok(const camelot_stage_cost& c) {
    return c.flop_per_query >= 0.0 && c.bytes_per_batch >= 0.0 && c.bytes_per_query >= 0.0 && c.mem_bytes >= 0.0 &&
           c.bytes_per_batch + c.bytes_per_query > 0.0;
}

static void feature_row(const camelot_stage_cost& c, int s, int b, int p, int co, double g, float* x) {
    const double F = (double)b * c.flop_per_query;
    const double Y = c.bytes_per_batch + (double)b * c.bytes_per_query;
    (void)s;
    const double v[kIn] = {(double)c.stage_id, (double)b, (double)p, F, Y, F / Y, (double)co, co > 0 ? g : 0.0,
                           co > 0 ? 1.0 : 0.0, (double)(p + co), std::log2((double)b), 1.0 / (double)p};
    for (int k = 0; k < kIn; ++k) x[k] = (float)v[k];
}

extern "C" camelot_status camelot_predictor_features(const camelot_stage_cost* costs, int n_stages, uint32_t n,
                                                     const int32_t* stage, const int32_t* batch, const int32_t* sms,
                                                     const int32_t* co_sms, const double* co_gbs, float* X) {
    if (!costs || !stage || !batch || !sms || !co_sms || !co_gbs || !X)
        return camelot_internal_fail(CAMELOT_EINVAL, "null argument");
    if (n_stages < 1) return camelot_internal_fail(CAMELOT_EINVAL, "n_stages must be >= 1");
    for (int i = 0; i < n_stages; ++i)
        if (!cost_ok(costs[i])) return camelot_internal_fail(CAMELOT_EINVAL, "negative or empty stage cost");
    for (uint32_t r = 0; r < n; ++r) {
        if (stage[r] < 0 || stage[r] >= n_stages || batch[r] < 1 || sms[r] < 1 || co_sms[r] < 0)
            return camelot_internal_fail(CAMELOT_EINVAL, "stage index, batch, SMs or co-runner SMs out of range");
        feature_row(costs[stage[r]], stage[r], batch[r], sms[r], co_sms[r], co_gbs[r], X + (size_t)r * kIn);
    }
    return CAMELOT_OK;
}

extern "C" camelot_status camelot_profile_from_latency(const camelot_stage_cost* costs, int n_stages,
                                                       const int32_t* batch_sizes, int n_batches, int n_levels,
                                                       const double* lat_s, double* thr, double* bw, double* dur,
                                                       double* mem) {
    if (!costs || !batch_sizes || !lat_s || !thr || !bw || !dur || !mem)
        return camelot_internal_fail(CAMELOT_EINVAL, "null argument");
    if (n_stages < 1 || n_batches < 1 || n_levels < 1)
        return camelot_internal_fail(CAMELOT_EINVAL, "empty table");
    for (int i = 0; i < n_stages; ++i)
        if (!cost_ok(costs[i])) return camelot_internal_fail(CAMELOT_EINVAL, "negative or empty stage cost");
    for (int b = 0; b < n_batches; ++b) {
        if (batch_sizes[b] < 1) return camelot_internal_fail(CAMELOT_EINVAL, "batch size < 1");
        const double B = (double)batch_sizes[b];
        for (int i = 0; i < n_stages; ++i) {
            const double Y = costs[i].bytes_per_batch + B * costs[i].bytes_per_query;
            mem[(size_t)b * n_stages + i] = costs[i].mem_bytes;
            for (int l = 0; l < n_levels; ++l) {
                const size_t k = ((size_t)b * n_stages + i) * n_levels + l;
                const double d = lat_s[k];
                if (!(d > 0.0) || !std::isfinite(d))
                    return camelot_internal_fail(CAMELOT_EINVAL, "latencies must be positive and finite");
                dur[k] = d;
                thr[k] = B / d;
                bw[k] = Y / d / 1e9;
            }
        }
    }
    return CAMELOT_OK;
}

extern "C" camelot_status camelot_profile_predict(camelot_predictor* p, const camelot_stage_cost* costs,
                                                  int n_stages, const int32_t* batch_sizes, int n_batches, int unit,
                                                  int n_levels, int32_t co_sms, double co_gbs, double* thr,
                                                  double* bw, double* dur, double* mem) {
    if (!p || !costs || !batch_sizes) return camelot_internal_fail(CAMELOT_EINVAL, "null argument");
    if (n_stages < 1 || n_batches < 1 || n_levels < 1 || unit < 1 || co_sms < 0)
        return camelot_internal_fail(CAMELOT_EINVAL, "empty table, unit < 1 or co_sms < 0");
    const size_t rows = (size_t)n_batches * n_stages * n_levels;
    // X and y live in the predictor's record scratch (kRec x kMaxTrainBatch floats)
    if (rows > kMaxTrainBatch) return camelot_internal_fail(CAMELOT_EINVAL, "more than 65536 table rows");
    std::vector<float> X(rows * kIn), y(rows);
    for (int b = 0; b < n_batches; ++b) {
        if (batch_sizes[b] < 1) return camelot_internal_fail(CAMELOT_EINVAL, "batch size < 1");
        for (int i = 0; i < n_stages; ++i) {
            if (!cost_ok(costs[i])) return camelot_internal_fail(CAMELOT_EINVAL, "negative or empty stage cost");
            for (int l = 0; l < n_levels; ++l) {
                const size_t r = ((size_t)b * n_stages + i) * n_levels + l;
                feature_row(costs[i], i, batch_sizes[b], (l + 1) * unit, co_sms, co_gbs, X.data() + r * kIn);
            }
        }
    }
    float* dX = p->rec;
    float* dy = p->rec + rows * kIn;
    PTRY(cudaMemcpy(dX, X.data(), X.size() * sizeof(float), cudaMemcpyHostToDevice));
    camelot_status st = camelot_predictor_forward(p, dX, (uint32_t)rows, dy, nullptr);
    if (st != CAMELOT_OK) return st;
    PTRY(cudaMemcpy(y.data(), dy, rows * sizeof(float), cudaMemcpyDeviceToHost));
    std::vector<double> lat(rows);
    for (size_t r = 0; r < rows; ++r) lat[r] = std::exp((double)y[r]) * 1e-6;   // log(us) -> s
    return camelot_profile_from_latency(costs, n_stages, batch_sizes, n_batches, n_levels, lat.data(), thr, bw,
                                        dur, mem);
}
