// Prepare-time kernels: per-tensor e4m3 quantisation of FP32 weights into the
// tiled, swizzled layout of the tensor-core layers.  s_w = max|W| / 448 (f32);
// code = e4m3(w / s_w), rounded to nearest even and saturated to +-448, the
// OCP FP8 E4M3 format.
#include <cuda_fp8.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>

#include "../../include/camelot.h"

camelot_status camelot_internal_fail(camelot_status st, const char* msg);

namespace {

// max |w| over n values; non-negative floats order like their bit patterns
__global__ void absmax_kernel(const float* __restrict__ w, size_t n, unsigned int* out) {
    float m = 0.f;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        m = fmaxf(m, fabsf(w[i]));
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));
}

// One byte of the tiled layout per thread: tile (mt, kb) of 128 rows x 128
// codes at ((mt * KB) + kb) * 16 KB, row r's 16-byte piece j at r * 128 +
// (j ^ (r % 8)) * 16; rows >= N are zero.
__global__ void quantize_tile_e4m3_kernel(const float* __restrict__ w, int N, int K, int Npad, float scale,
                                          uint8_t* __restrict__ out) {
    const size_t total = (size_t)Npad * K;
    const int KB = K / 128;
    for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < total;
         p += (size_t)gridDim.x * blockDim.x) {
        const size_t tile = p >> 14;
        const int mt = (int)(tile / KB), kb = (int)(tile % KB);
        const int within = (int)(p & 16383);
        const int r = within >> 7, pos = within & 127;
        const int j = (pos >> 4) ^ (r & 7), b = pos & 15;
        const int row = mt * 128 + r, k = kb * 128 + j * 16 + b;
        uint8_t code = 0;
        if (row < N)
            code = (uint8_t)__nv_cvt_float_to_fp8(__fdiv_rn(w[(size_t)row * K + k], scale), __NV_SATFINITE,
                                                  __NV_E4M3);
        out[p] = code;
    }
}

}  // namespace

// Quantise device weights w [N][K] (f32, finite, not all zero) into a new
// device buffer of Npad x K codes in the tiled layout; *scale receives s_w.
camelot_status camelot_internal_quantize_e4m3(const float* w, int N, int K, int Npad, void** out, float* scale) {
    // a private stream: prepare never waits for a running pipeline's kernel
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess)
        return camelot_internal_fail(CAMELOT_ECUDA, "stream creation failed");
    unsigned int* d_max = nullptr;
    void* q = nullptr;
    camelot_status rc = CAMELOT_OK;
    unsigned int bits = 0;
    if (cudaMalloc(&d_max, sizeof(unsigned int)) != cudaSuccess ||
        cudaMalloc(&q, (size_t)Npad * K) != cudaSuccess) {
        rc = camelot_internal_fail(CAMELOT_ENOMEM, "quantisation allocation failed");
    } else {
        cudaMemsetAsync(d_max, 0, sizeof(unsigned int), st);
        absmax_kernel<<<592, 256, 0, st>>>(w, (size_t)N * K, d_max);
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpyAsync(&bits, d_max, sizeof bits, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            rc = camelot_internal_fail(CAMELOT_ECUDA, "weight absmax failed");
    }
    float amax = 0.f;
    memcpy(&amax, &bits, sizeof amax);
    if (rc == CAMELOT_OK && (!(amax > 0.f) || !std::isfinite(amax)))
        rc = camelot_internal_fail(CAMELOT_EINVAL, "FP8 weights must be finite and not all zero");
    const float s = amax / 448.0f;
    if (rc == CAMELOT_OK) {
        quantize_tile_e4m3_kernel<<<1184, 256, 0, st>>>(w, N, K, Npad, s, (uint8_t*)q);
        if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess)
            rc = camelot_internal_fail(CAMELOT_ECUDA, "weight quantisation failed");
    }
    if (d_max) cudaFree(d_max);
    cudaStreamDestroy(st);
    if (rc != CAMELOT_OK) {
        if (q) cudaFree(q);
        return rc;
    }
    *out = q;
    *scale = s;
    return CAMELOT_OK;
}

extern "C" camelot_status camelot_fp8_scale(const float* x, size_t n, void* stream, float* scale) {
    if (!x || !scale || n == 0) return camelot_internal_fail(CAMELOT_EINVAL, "null argument or n = 0");
    cudaStream_t st = (cudaStream_t)stream;
    unsigned int* d_max = nullptr;
    if (cudaMalloc(&d_max, sizeof(unsigned int)) != cudaSuccess)
        return camelot_internal_fail(CAMELOT_ENOMEM, "result word allocation failed");
    unsigned int bits = 0;
    camelot_status rc = CAMELOT_OK;
    if (cudaMemsetAsync(d_max, 0, sizeof(unsigned int), st) != cudaSuccess) rc = CAMELOT_ECUDA;
    if (rc == CAMELOT_OK) {
        absmax_kernel<<<592, 256, 0, st>>>(x, n, d_max);
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpyAsync(&bits, d_max, sizeof bits, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            rc = CAMELOT_ECUDA;
    }
    cudaFree(d_max);
    if (rc != CAMELOT_OK) return camelot_internal_fail(rc, "activation absmax failed");
    float amax = 0.f;
    memcpy(&amax, &bits, sizeof amax);
    if (!(amax > 0.f) || !std::isfinite(amax))
        return camelot_internal_fail(CAMELOT_EINVAL, "calibration values must be finite and not all zero");
    *scale = amax / 448.0f;
    return CAMELOT_OK;
}
