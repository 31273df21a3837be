// Profiling harness of the allocator's inputs (Sec. 7.1): timed repeated
// launches of one stage under an SM quota, and a bandwidth-hog co-runner that
// streams a large FP32 copy on SMs the stage does not use, so that stage
// latency can be measured under memory contention (Sec. 4.2, Sec. 7.2).
#include <cuda_runtime.h>

#include <chrono>
#include <cstring>
#include <thread>
#include <vector>

#include "../../include/camelot.h"
#include "device_sync.cuh"

camelot_status camelot_internal_fail(camelot_status st, const char* msg);
int camelot_internal_sm_count();

using namespace camelot;

namespace {

constexpr int kCoThreads = 512;
constexpr int kCoSmem = 120 * 1024;   // leaves no room for a stage CTA (216 KB) on the same SM

// Host-mapped words the co-runner shares with the host.
struct alignas(128) CoFlags {
    volatile unsigned long long stop;   // host -> device
    unsigned long long pad0[15];
    unsigned long long passes;          // device -> host: full passes completed
    unsigned long long timed_out;       // device -> host: stopped by its own deadline
    unsigned long long pad1[14];
    unsigned long long started[256];    // device -> host: CTA b is resident
};

// Copy src -> dst (n4 16-byte words) over and over.  Thread 0 of each CTA
// checks the host's stop word and the deadline between passes; the loop also
// ends after max_passes.  The dynamic shared memory only reserves the SM.
__global__ void __launch_bounds__(kCoThreads) corunner_kernel(const float4* __restrict__ src, float4* __restrict__ dst,
                                                              size_t n4, CoFlags* fl, long long max_passes,
                                                              long long max_ns) {
    extern __shared__ float4 reserve[];
    __shared__ int quit;
    const uint64_t t0 = gtime();
    if (threadIdx.x == 0) {
        reserve[0] = make_float4(0.f, 0.f, 0.f, 0.f);
        st_release_sys(&fl->started[blockIdx.x], 1ull);
    }
    long long pass = 0;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (; pass < max_passes; ++pass) {
        // eight independent 16-byte loads in flight per thread
        size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
        for (; i + 7 * stride < n4; i += 8 * stride) {
            float4 v[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) v[k] = __ldcs(src + i + k * stride);
#pragma unroll
            for (int k = 0; k < 8; ++k) __stcs(dst + i + k * stride, v[k]);
        }
        for (; i < n4; i += stride) __stcs(dst + i, __ldcs(src + i));
        if (threadIdx.x == 0) {
            const bool late = gtime() - t0 > (uint64_t)max_ns;
            quit = (ld_acquire_sys(&fl->stop) != 0) || late;
            if (late && blockIdx.x == 0) fl->timed_out = 1;
        }
        __syncthreads();
        const int q = quit;
        __syncthreads();
        if (q) {
            ++pass;
            break;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) st_release_sys(&fl->passes, (unsigned long long)pass);
}

}  // namespace

struct camelot_corunner {
    cudaStream_t stream = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CoFlags* flags = nullptr;   // pinned, mapped
    size_t bytes = 0;
    int ctas = 0;
};

static void corunner_free(camelot_corunner* c) {
    if (c->e0) cudaEventDestroy(c->e0);
    if (c->e1) cudaEventDestroy(c->e1);
    if (c->stream) cudaStreamDestroy(c->stream);
    if (c->flags) cudaFreeHost(c->flags);
    delete c;
}

extern "C" camelot_status camelot_corunner_start(const void* src, void* dst, size_t bytes, int n_ctas,
                                                 int64_t max_ns, camelot_corunner** out) {
    if (!src || !dst || !out) return camelot_internal_fail(CAMELOT_EINVAL, "null argument");
    if (bytes < 16 || ((uintptr_t)src | (uintptr_t)dst) % 16)
        return camelot_internal_fail(CAMELOT_EINVAL, "buffers must be 16-byte aligned and >= 16 bytes");
    if (n_ctas < 1 || n_ctas > camelot_internal_sm_count() || n_ctas > 256)
        return camelot_internal_fail(CAMELOT_EINVAL, "n_ctas outside 1..min(SM count, 256)");
    if (max_ns <= 0) return camelot_internal_fail(CAMELOT_EINVAL, "max_ns must be positive");
    auto* c = new camelot_corunner();
    c->bytes = bytes / 16 * 16;
    c->ctas = n_ctas;
    if (cudaFuncSetAttribute(corunner_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kCoSmem) != cudaSuccess ||
        cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&c->e0) != cudaSuccess || cudaEventCreate(&c->e1) != cudaSuccess ||
        cudaHostAlloc((void**)&c->flags, sizeof(CoFlags), cudaHostAllocMapped) != cudaSuccess) {
        corunner_free(c);
        return camelot_internal_fail(CAMELOT_ENOMEM, "co-runner setup failed");
    }
    memset((void*)c->flags, 0, sizeof(CoFlags));
    CoFlags* dflags = nullptr;
    if (cudaHostGetDevicePointer((void**)&dflags, (void*)c->flags, 0) != cudaSuccess) {
        corunner_free(c);
        return camelot_internal_fail(CAMELOT_ECUDA, "cudaHostGetDevicePointer failed");
    }
    cudaEventRecord(c->e0, c->stream);
    corunner_kernel<<<n_ctas, kCoThreads, kCoSmem, c->stream>>>((const float4*)src, (float4*)dst, c->bytes / 16,
                                                                dflags, 1ll << 40, (long long)max_ns);
    if (cudaGetLastError() != cudaSuccess) {
        cudaStreamSynchronize(c->stream);
        corunner_free(c);
        return camelot_internal_fail(CAMELOT_ECUDA, "co-runner launch failed");
    }
    cudaEventRecord(c->e1, c->stream);
    // Wait (bounded, 5 s) until every CTA is resident, so the SMs it holds are
    // taken before the caller launches the stage it measures.
    const auto t_end = std::chrono::steady_clock::now() + std::chrono::seconds(5);
    for (;;) {
        int up = 0;
        for (int b = 0; b < n_ctas; ++b) up += (int)(((volatile unsigned long long*)c->flags->started)[b] != 0);
        if (up == n_ctas) break;
        if (std::chrono::steady_clock::now() > t_end) {
            c->flags->stop = 1;
            cudaStreamSynchronize(c->stream);
            corunner_free(c);
            return camelot_internal_fail(CAMELOT_ETIMEDOUT, "co-runner CTAs did not all become resident");
        }
        std::this_thread::yield();
    }
    *out = c;
    return CAMELOT_OK;
}

extern "C" camelot_status camelot_corunner_stop(camelot_corunner* c, double* gbytes_per_s) {
    if (!c) return camelot_internal_fail(CAMELOT_EINVAL, "null co-runner");
    c->flags->stop = 1;
    __sync_synchronize();
    const cudaError_t e = cudaStreamSynchronize(c->stream);
    float ms = 0.f;
    if (e == cudaSuccess) cudaEventElapsedTime(&ms, c->e0, c->e1);
    const double passes = (double)((volatile unsigned long long&)c->flags->passes);
    const bool timed_out = ((volatile unsigned long long&)c->flags->timed_out) != 0;
    if (gbytes_per_s) *gbytes_per_s = ms > 0.f ? 2.0 * (double)c->bytes * passes / (ms * 1e-3) / 1e9 : 0.0;
    corunner_free(c);
    if (e != cudaSuccess) return camelot_internal_fail(CAMELOT_ECUDA, "co-runner kernel failed");
    if (timed_out) return camelot_internal_fail(CAMELOT_ETIMEDOUT, "co-runner stopped at its own deadline");
    return CAMELOT_OK;
}

extern "C" camelot_status camelot_stage_time(const camelot_stage* st, int n_ctas, const void* in, uint32_t n,
                                             void* out, int32_t* out_idx, float* out_val, float* out_logits,
                                             void* scratch, size_t scratch_bytes, void* stream, uint32_t runs,
                                             float* ms_out) {
    if (!ms_out || runs == 0 || runs > 65536) return camelot_internal_fail(CAMELOT_EINVAL, "runs must be in 1..65536");
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<cudaEvent_t> ev(runs + 1, nullptr);
    camelot_status st_out = CAMELOT_OK;
    for (auto& e : ev)
        if (cudaEventCreate(&e) != cudaSuccess) st_out = CAMELOT_ECUDA;
    if (st_out == CAMELOT_OK) {
        cudaEventRecord(ev[0], s);
        for (uint32_t r = 0; r < runs && st_out == CAMELOT_OK; ++r) {
            st_out = camelot_stage_launch(st, n_ctas, in, n, out, out_idx, out_val, out_logits, scratch,
                                          scratch_bytes, stream);
            cudaEventRecord(ev[r + 1], s);
        }
        if (st_out == CAMELOT_OK) {
            if (cudaEventSynchronize(ev[runs]) != cudaSuccess) {
                st_out = camelot_internal_fail(CAMELOT_ECUDA, "stage launch failed");
            } else {
                for (uint32_t r = 0; r < runs; ++r) cudaEventElapsedTime(&ms_out[r], ev[r], ev[r + 1]);
            }
        } else {
            cudaStreamSynchronize(s);
        }
    } else {
        st_out = camelot_internal_fail(CAMELOT_ECUDA, "cudaEventCreate failed");
    }
    for (auto& e : ev)
        if (e) cudaEventDestroy(e);
    return st_out;
}
