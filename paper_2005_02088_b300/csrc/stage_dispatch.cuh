// Dispatch of a stage body on its kind.
#pragma once
#include "gemm_bf16.cuh"
#include "stages.cuh"

namespace camelot {

static __device__ bool stage_body(const StageCtx& cx, const StageParams& P, RowRef in, int n, RowRef out,
                                  const FinalOut& fo) {
    switch (P.kind) {
        case KIND_NORMALIZE_U8: normalize_body(cx, P, in, n, out); return true;
        case KIND_NORM_POOL2_BF16: normpool_body(cx, P, in, n, out); return true;
        case KIND_MLP_FP32: return mlp_body(cx, P, in, n, out, fo);
        case KIND_GEMM_BF16:
        case KIND_GEMM_FP8: return gemm_body(cx, P, in, n, out, fo);
        case KIND_NORMALIZE_U8_E4M3: normalize_e4m3_body(cx, P, in, n, out); return true;
        case KIND_EMBED_GATHER: embed_body(cx, P, in, n, out); return true;
        default: return false;
    }
}

}  // namespace camelot
