// camelot_stage_launch_noalloc: the direct stage launch without any device
// allocation by the caller or by the library.
//
// Some callers of this library cannot allocate device memory when they run a
// stage: a host application whose memory manager owns the whole device pool
// (a foreign cudaMalloc may fail, fragment the pool or break its accounting),
// serving loops that must not take the latency and implicit device-wide
// synchronisation a cudaMalloc/cudaFree can cost in the middle of a request,
// and embedded plug-ins that are only handed input and output buffers.  For
// them the scratch memory the stage needs lives in one file-scope device
// array of fixed size, created when the library is loaded on each GPU and
// kept until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/camelot.h"
#include "device_sync.cuh"
#include "stage_params.h"
#include "stage_dispatch.cuh"

namespace camelot {

// Largest scratch the allocation-free launch can use (per device).
constexpr size_t kNoAllocScratchBytes = size_t(16) << 20;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Same device code as the ordinary direct launch; the stage parameters (laid
// out for this batch size) travel by value, so nothing is staged in memory.
__global__ void __launch_bounds__(kThreads, 1)
    stage_direct_noalloc_kernel(const StageParams sp, RowRef in, int n, RowRef out, int32_t* idx,
                                float* val, RowRef logits, char* base, size_t header,
                                long long limit_ns) {
    extern __shared__ float4 smem4[];
    Ctl* ctl = reinterpret_cast<Ctl*>(base);
    GroupSync* gs = reinterpret_cast<GroupSync*>(base + ((sizeof(Ctl) + 255) / 256) * 256);
    StageCtx cx{(int)blockIdx.x, (int)gridDim.x, gs, ctl, (uint64_t)limit_ns, 0u, base + header,
                reinterpret_cast<float*>(smem4)};
    FinalOut fo{idx, val, logits};
    // the stages that stream by bulk copies set their mbarriers up first
    if (sp.kind == KIND_NORM_POOL2_BF16) pool_setup(reinterpret_cast<float*>(smem4));
    else if (sp.kind == KIND_STREAM_SYNTH) stream_setup(reinterpret_cast<float*>(smem4));
    else if (sp.kind == KIND_MLP_FP32) mlp_setup(reinterpret_cast<float*>(smem4));
    stage_body<kAllKinds & ~(kind_bit(KIND_GEMM_BF16) | kind_bit(KIND_GEMM_FP8))>(cx, sp, in, n, out, fo);

    // The caller holds no handle on the error word in the static array, so a
    // failed call marks its outputs instead: the last CTA to finish (the
    // others have fenced their writes before counting themselves out) looks
    // at the error word and, if a wait gave up, overwrites every output with
    // the failure pattern (indices -1; every other output byte 0xFF, which is
    // NaN in f32, bf16 and e4m3).
    __shared__ int s_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(&ctl->exited[0].v, 1ull) == (unsigned long long)(gridDim.x - 1);
        __threadfence();
    }
    __syncthreads();
    if (!s_last || !has_error(ctl)) return;
    if (sp.top_k > 0) {
        const size_t k = (size_t)n * (size_t)sp.res_k;
        for (size_t i = threadIdx.x; i < k; i += blockDim.x) {
            idx[i] = -1;
            val[i] = __int_as_float(-1);
        }
        if (logits.base != nullptr)
            for (size_t i = threadIdx.x; i < (size_t)n * logits.stride; i += blockDim.x) logits.base[i] = (char)0xFF;
    } else {
        for (size_t i = threadIdx.x; i < (size_t)n * out.stride; i += blockDim.x) out.base[i] = (char)0xFF;
    }
}

}  // namespace camelot

using namespace camelot;

const StageParams* camelot_internal_stage_params(const camelot_stage* st);
size_t camelot_internal_layout_scratch(StageParams& sp, int B);
int camelot_internal_sm_count();
camelot_status camelot_internal_fail(camelot_status st, const char* msg);

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Once per device, with that device current: the device address of the
// static scratch array (its host-side name is only a stand-in) and the
// kernel's shared-memory limit.
camelot_status setup_device(int dev, char** addr) {
    std::lock_guard<std::mutex> g(g_setup_mu);
    if (dev < 0 || dev >= kMaxDevices)
        return camelot_internal_fail(CAMELOT_EINVAL, "device index out of range for the static scratch");
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return camelot_internal_fail(CAMELOT_ECUDA, "cudaGetSymbolAddress of the static scratch failed");
        e = cudaFuncSetAttribute((const void*)stage_direct_noalloc_kernel,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
        if (e != cudaSuccess)
            return camelot_internal_fail(CAMELOT_ECUDA, "shared-memory attribute of the kernel failed");
        g_scratch_addr[dev] = p;
    }
    *addr = (char*)g_scratch_addr[dev];
    return CAMELOT_OK;
}
}  // namespace

extern "C" camelot_status camelot_stage_launch_noalloc(const camelot_stage* st, int n_ctas,
                                                       const void* in, uint32_t n, void* out,
                                                       int32_t* out_idx, float* out_val,
                                                       float* out_logits, void* stream) {
    if (!st) return camelot_internal_fail(CAMELOT_EINVAL, "null stage");
    StageParams sp = *camelot_internal_stage_params(st);
    if (is_tensor_kind(sp.kind))
        return camelot_internal_fail(CAMELOT_EINVAL, "tensor-core stages need camelot_stage_launch");
    if (n == 0 || (int)n > sp.max_batch)
        return camelot_internal_fail(CAMELOT_EINVAL, "n outside 1..max_batch");
    if (n_ctas < 1 || n_ctas > camelot_internal_sm_count())
        return camelot_internal_fail(CAMELOT_EINVAL, "n_ctas outside 1..SM count");
    if (!in) return camelot_internal_fail(CAMELOT_EINVAL, "null input");
    if (sp.top_k == 0 && !out) return camelot_internal_fail(CAMELOT_EINVAL, "intermediate stage needs `out`");
    if (sp.top_k > 0 && (!out_idx || !out_val))
        return camelot_internal_fail(CAMELOT_EINVAL, "final stage needs out_idx and out_val");
    const size_t header = ((sizeof(Ctl) + 255) / 256) * 256 + ((sizeof(GroupSync) + 255) / 256) * 256;
    const size_t body = camelot_internal_layout_scratch(sp, (int)n);   // laid out for this n
    if (header + body > kNoAllocScratchBytes)
        return camelot_internal_fail(
            CAMELOT_EINVAL, "batch needs more scratch than the 16 MiB static buffer; use "
                            "camelot_stage_launch with caller scratch or a smaller batch");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return camelot_internal_fail(CAMELOT_ECUDA, "cudaGetDevice failed");
    char* base = nullptr;
    camelot_status cs = setup_device(dev, &base);
    if (cs != CAMELOT_OK) return cs;
    cudaStream_t s = (cudaStream_t)stream;
    // the barrier counters and the error word must start at zero; the rest of
    // the buffer is written before it is read
    if (cudaMemsetAsync(base, 0, header, s) != cudaSuccess)
        return camelot_internal_fail(CAMELOT_ECUDA, "clearing the static scratch header failed");
    RowRef rin{(char*)in, 0, ~0ull, sp.in_row_bytes};
    RowRef rout{(char*)out, 0, ~0ull, sp.out_row_bytes};
    RowRef rlog{(char*)out_logits, 0, ~0ull, sp.out_width * sizeof(float)};
    int nn = (int)n;
    long long limit = 2000000000ll;
    size_t hdr = header;
    void* args[] = {&sp, &rin, &nn, &rout, &out_idx, &out_val, &rlog, &base, &hdr, &limit};
    cudaError_t e = cudaLaunchCooperativeKernel((const void*)stage_direct_noalloc_kernel, dim3(n_ctas),
                                                dim3(kThreads), args, kSmemBytes, s);
    if (e != cudaSuccess) return camelot_internal_fail(CAMELOT_ECUDA, cudaGetErrorString(e));
    return CAMELOT_OK;
}
