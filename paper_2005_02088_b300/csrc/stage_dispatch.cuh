// Dispatch of a stage body on its kind.  KINDS is a bit set of the kinds a
// kernel instantiation carries (bit k = kind k): each pipeline launches the
// instantiation holding just its own kinds, so the compiler lays out and
// allocates registers for those bodies only.
#pragma once
#include "artifact.cuh"
#include "gemm_bf16.cuh"
#include "stages.cuh"

namespace camelot {

__host__ __device__ constexpr uint32_t kind_bit(int k) { return 1u << k; }
constexpr uint32_t kAllKinds = kind_bit(KIND_NORMALIZE_U8) | kind_bit(KIND_NORM_POOL2_BF16) |
                               kind_bit(KIND_MLP_FP32) | kind_bit(KIND_GEMM_BF16) | kind_bit(KIND_GEMM_FP8) |
                               kind_bit(KIND_NORMALIZE_U8_E4M3) | kind_bit(KIND_EMBED_GATHER) |
                               kind_bit(KIND_COMPUTE_SYNTH) | kind_bit(KIND_STREAM_SYNTH);

template <uint32_t KINDS>
static __device__ bool stage_body(const StageCtx& cx, const StageParams& P, RowRef in, int n, RowRef out,
                                  const FinalOut& fo) {
    switch (P.kind) {
        case KIND_NORMALIZE_U8:
            if constexpr ((KINDS & kind_bit(KIND_NORMALIZE_U8)) != 0) { normalize_body(cx, P, in, n, out); return true; }
            break;
        case KIND_NORM_POOL2_BF16:
            if constexpr ((KINDS & kind_bit(KIND_NORM_POOL2_BF16)) != 0) { normpool_body(cx, P, in, n, out); return true; }
            break;
        case KIND_MLP_FP32:
            if constexpr ((KINDS & kind_bit(KIND_MLP_FP32)) != 0) return mlp_body(cx, P, in, n, out, fo);
            break;
        case KIND_GEMM_BF16:
        case KIND_GEMM_FP8:
            if constexpr ((KINDS & (kind_bit(KIND_GEMM_BF16) | kind_bit(KIND_GEMM_FP8))) != 0)
                return gemm_body(cx, P, in, n, out, fo);
            break;
        case KIND_NORMALIZE_U8_E4M3:
            if constexpr ((KINDS & kind_bit(KIND_NORMALIZE_U8_E4M3)) != 0) { normalize_e4m3_body(cx, P, in, n, out); return true; }
            break;
        case KIND_EMBED_GATHER:
            if constexpr ((KINDS & kind_bit(KIND_EMBED_GATHER)) != 0) { embed_body(cx, P, in, n, out); return true; }
            break;
        case KIND_COMPUTE_SYNTH:
            if constexpr ((KINDS & kind_bit(KIND_COMPUTE_SYNTH)) != 0) return compute_synth_body(cx, P, in, n, out, fo);
            break;
        case KIND_STREAM_SYNTH:
            if constexpr ((KINDS & kind_bit(KIND_STREAM_SYNTH)) != 0) return stream_synth_body(cx, P, in, n, out, fo);
            break;
        default:
            break;
    }
    return false;
}

}  // namespace camelot
