// Artifact stages (the c_i, m_i and p_i of Sec. 2.3 and Sec. 8.5): tunable
// compute, memory or host-link intensity, defined in binary32.
#pragma once
#include "gemm_bf16.cuh"
#include "stages.cuh"
#include "tc_ptx.cuh"

namespace camelot {

// ---------------------------------------------------------------------------
// Artifact stages (the c_i, m_i and p_i of Sec. 2.3 and Sec. 8.5): tunable
// compute, memory or host-link intensity.  An intermediate stage writes its
// f32 rows to `out`; a final one writes them to the instance's scratch and
// takes their top-k.
// ---------------------------------------------------------------------------
// COMPUTE_SYNTH: y <- fma(y, 127/128, x / 128), P.H steps from y = 0, per
// value; every thread runs four independent chains (one float4).
static __device__ bool compute_synth_body(const StageCtx& cx, const StageParams& P, RowRef in, int n,
                                          RowRef out, const FinalOut& fo) {
    const int W4 = P.W / 4, steps = P.H;
    const bool fin = P.top_k > 0;
    const RowRef y = fin ? RowRef{cx.scratch + P.layer[0].h_off, 0, ~0ull, (size_t)P.W * 4} : out;
    const int total = n * W4;
    for (int e = cx.rank * kThreads + threadIdx.x; e < total; e += cx.nctas * kThreads) {
        const int q = e / W4, c = e - q * W4;
        const float4 x = __ldcs(reinterpret_cast<const float4*>(in.row(q)) + c);
        const float b0 = x.x * 0.0078125f, b1 = x.y * 0.0078125f, b2 = x.z * 0.0078125f, b3 = x.w * 0.0078125f;
        float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
#pragma unroll 8
        for (int i = 0; i < steps; ++i) {
            a0 = __fmaf_rn(a0, 0.9921875f, b0);
            a1 = __fmaf_rn(a1, 0.9921875f, b1);
            a2 = __fmaf_rn(a2, 0.9921875f, b2);
            a3 = __fmaf_rn(a3, 0.9921875f, b3);
        }
        __stcg(reinterpret_cast<float4*>(y.row(q)) + c, make_float4(a0, a1, a2, a3));
    }
    if (!fin) return true;
    if (!group_barrier(cx.gs, cx.nctas, cx.ctl, cx.limit_ns, cx.where)) return false;
    topk_rows(cx, y, n, P.W, P.top_k, fo);
    return true;
}

// STREAM_SYNTH over a table in pinned host memory (the p_i): y_j = x_j + sum
// over the query's P.H table windows, added in window order.  Each CTA first
// works out the window start of every query of the batch (shared memory), so
// the table loads depend on nothing in flight; 16 loads of 16 bytes are in
// flight per thread.
static __device__ bool stream_synth_loads(const StageCtx& cx, const StageParams& P, RowRef in, int n,
                                         RowRef out, const FinalOut& fo) {
    const int W4 = P.W / 4, terms = P.H;
    const uint32_t starts = (uint32_t)P.C;
    const float4* T = reinterpret_cast<const float4*>(P.layer[0].w);
    const bool fin = P.top_k > 0;
    const RowRef y = fin ? RowRef{cx.scratch + P.layer[0].h_off, 0, ~0ull, (size_t)P.W * 4} : out;
    uint32_t* wstart = reinterpret_cast<uint32_t*>(cx.smem);     // [n] window index per query
    for (int q = threadIdx.x; q < n; q += kThreads) {
        const uint32_t bits = __float_as_uint(*reinterpret_cast<const float*>(in.row(q)));
        const uint32_t h = (uint32_t)(((unsigned long long)bits * 0x9E3779B97F4A7C15ull) >> 32);
        wstart[q] = h % starts;
    }
    __syncthreads();
    const int total = n * W4;
    constexpr int U = 16;
    for (int e = cx.rank * kThreads + threadIdx.x; e < total; e += cx.nctas * kThreads) {
        const int q = e / W4, c = e - q * W4;
        const float4* tw = T + (size_t)wstart[q] * W4 + c;
        float4 acc = __ldcs(reinterpret_cast<const float4*>(in.row(q)) + c);
        for (int r0 = 0; r0 < terms; r0 += U) {
            float4 t[U];
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (r0 + u < terms) t[u] = __ldcs(tw + (size_t)(r0 + u) * W4);
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (r0 + u < terms) {
                    acc.x += t[u].x;
                    acc.y += t[u].y;
                    acc.z += t[u].z;
                    acc.w += t[u].w;
                }
            }
        }
        __stcg(reinterpret_cast<float4*>(y.row(q)) + c, acc);
    }
    if (!fin) return true;
    if (!group_barrier(cx.gs, cx.nctas, cx.ctl, cx.limit_ns, cx.where)) return false;
    topk_rows(cx, y, n, P.W, P.top_k, fo);
    return true;
}


// STREAM_SYNTH over a table in device memory (the m_i).  A query's windows are
// one contiguous run of P.H rows of W floats; each CTA takes whole queries
// (q = rank, rank + CTAs, ...) and streams their runs through a 4 x 32 KB
// shared-memory ring with bulk copies (L2 evict-first: the table is read once
// per query), every thread adding its columns row after row, so the sum keeps
// the window order.  Bulk copies rather than loads because a stream of 16-byte
// loads from 256 threads reaches only ~18 GB/s per SM here.
constexpr int kStreamStages = 4;
constexpr uint32_t kStreamChunk = 32 * 1024;

// The ring's mbarriers and their completed fill counts (after the ring),
// initialised once per kernel launch by stream_setup; calls continue the
// counts, so the barriers are never re-initialised in use.
__device__ __forceinline__ char* stream_base(float* smem) {
    return reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(smem) + 1023) & ~static_cast<uintptr_t>(1023));
}
__device__ __forceinline__ uint64_t* stream_bars(float* smem) {
    return reinterpret_cast<uint64_t*>(stream_base(smem) + kStreamStages * kStreamChunk);
}
__device__ __forceinline__ uint32_t* stream_fills(float* smem) {
    return reinterpret_cast<uint32_t*>(stream_bars(smem) + kStreamStages);
}
__device__ __forceinline__ void stream_setup(float* smem) {
    if (threadIdx.x < kStreamStages) {
        mbar_init(&stream_bars(smem)[threadIdx.x], 1);
        stream_fills(smem)[threadIdx.x] = 0u;
    }
    if (threadIdx.x == 0) mbar_fence_init();
    __syncthreads();
}

static __device__ bool stream_synth_bulk(const StageCtx& cx, const StageParams& P, RowRef in, int n,
                                         RowRef out, const FinalOut& fo) {
    const int W = P.W, W4 = W / 4, terms = P.H;
    const uint32_t starts = (uint32_t)P.C;
    const float* T = P.layer[0].w;
    const bool fin = P.top_k > 0;
    const RowRef y = fin ? RowRef{cx.scratch + P.layer[0].h_off, 0, ~0ull, (size_t)W * 4} : out;
    char* base = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(cx.smem) + 1023) & ~static_cast<uintptr_t>(1023));
    float* ring = reinterpret_cast<float*>(base);
    uint64_t* full = stream_bars(cx.smem);
    uint32_t* sfill = stream_fills(cx.smem);
    uint32_t* wstart = sfill + kStreamStages;
    const int crows = max(1, (int)(kStreamChunk / ((uint32_t)W * 4)));   // table rows per chunk
    const int nch = (terms + crows - 1) / crows;                        // chunks per query
    const int myq = cx.rank < n ? (n - cx.rank + cx.nctas - 1) / cx.nctas : 0;
    const int total = myq * nch;
    for (int i = threadIdx.x; i < myq; i += kThreads) {
        const uint32_t bits = __float_as_uint(*reinterpret_cast<const float*>(in.row(cx.rank + i * cx.nctas)));
        const uint32_t h = (uint32_t)(((unsigned long long)bits * 0x9E3779B97F4A7C15ull) >> 32);
        wstart[i] = h % starts;
    }
    __syncthreads();
    const uint64_t pol = l2_policy_evict_first();
    auto issue = [&](int g) {
        const int i = g / nch, c = g - i * nch;
        const int r0 = c * crows, nr = min(crows, terms - r0);
        const uint32_t bytes = (uint32_t)nr * (uint32_t)W * 4u;
        const int s = g % kStreamStages;
        mbar_arrive_expect_tx(&full[s], bytes);
        bulk_load_hint(ring + (size_t)s * (kStreamChunk / 4), T + ((size_t)wstart[i] + r0) * W, bytes, &full[s], pol);
    };
    if (threadIdx.x == 0)
        for (int g = 0; g < min(kStreamStages, total); ++g) issue(g);
    constexpr int kMaxCols = 8;                  // float4 columns per thread (W <= 8192)
    for (int i = 0; i < myq; ++i) {
        const int q = cx.rank + i * cx.nctas;
        float4 acc[kMaxCols];
        const float4* xr = reinterpret_cast<const float4*>(in.row(q));
#pragma unroll
        for (int k = 0; k < kMaxCols; ++k) {
            const int c4 = threadIdx.x + k * kThreads;
            acc[k] = c4 < W4 ? __ldcs(xr + c4) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        for (int c = 0; c < nch; ++c) {
            const int g = i * nch + c, s = g % kStreamStages;
            if (!mbar_wait_bounded(&full[s], (sfill[s] + (uint32_t)(g / kStreamStages)) & 1u, cx, 7)) return false;
            const float4* rows = reinterpret_cast<const float4*>(ring + (size_t)s * (kStreamChunk / 4));
            const int nr = min(crows, terms - c * crows);
            for (int r = 0; r < nr; ++r) {
#pragma unroll
                for (int k = 0; k < kMaxCols; ++k) {
                    const int c4 = threadIdx.x + k * kThreads;
                    if (c4 < W4) {
                        const float4 t = rows[(size_t)r * W4 + c4];
                        acc[k].x += t.x;
                        acc[k].y += t.y;
                        acc[k].z += t.z;
                        acc[k].w += t.w;
                    }
                }
            }
            __syncthreads();                     // the slot has been read by every thread
            if (threadIdx.x == 0 && g + kStreamStages < total) issue(g + kStreamStages);
        }
        float4* yr = reinterpret_cast<float4*>(y.row(q));
#pragma unroll
        for (int k = 0; k < kMaxCols; ++k) {
            const int c4 = threadIdx.x + k * kThreads;
            if (c4 < W4) __stcg(yr + c4, acc[k]);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0)
        for (int sl = 0; sl < kStreamStages; ++sl)
            sfill[sl] += (uint32_t)(total + kStreamStages - 1 - sl) / kStreamStages;
    __syncthreads();
    if (!fin) return true;
    if (!group_barrier(cx.gs, cx.nctas, cx.ctl, cx.limit_ns, cx.where)) return false;
    topk_rows(cx, y, n, W, P.top_k, fo);
    return true;
}

// The table's location (layer[0].act: 1 = pinned host memory) picks the path.
static __device__ bool stream_synth_body(const StageCtx& cx, const StageParams& P, RowRef in, int n,
                                         RowRef out, const FinalOut& fo) {
    if (P.layer[0].act == 1 || P.W > 8192) return stream_synth_loads(cx, P, in, n, out, fo);
    return stream_synth_bulk(cx, P, in, n, out, fo);
}

}  // namespace camelot
