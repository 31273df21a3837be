// Stage bodies of the synthetic microservices (stand-ins for the Sec. 3 suite).
//
// A body runs on the p CTAs of one stage instance (the SM quota p_i of Table 2)
// over one batch of n rows.  CTAs split the work by their rank in the instance
// and meet at group barriers between dependent phases.  The decomposition of
// every floating-point reduction is fixed by the stage (chunk sizes chosen when
// the stage is prepared), never by p, so the result of a query is bit-identical
// whatever the SM quota, the number of instances or the batch it travels in.
#pragma once
#include <cuda_fp8.h>
#include <cuda_bf16.h>
#include <cstdint>

#include "device_sync.cuh"
#include "stage_params.h"
#include "tc_ptx.cuh"

namespace camelot {

struct StageCtx {
    int rank;          // CTA rank inside the instance
    int nctas;         // CTAs (SMs) of the instance
    GroupSync* gs;
    Ctl* ctl;
    uint64_t limit_ns;
    uint32_t where;    // stage index, for error reports
    char* scratch;     // the instance's scratch memory
    float* smem;       // dynamic shared memory of this CTA
    bool defer_topk = false;   // a final GEMM stage leaves its top-k merge to the pipeline's leader
};

struct FinalOut {
    int32_t* idx;      // [n][top_k]
    float* val;        // [n][top_k]
    RowRef logits;     // final layer output rows (base == nullptr: not wanted)
};

// Bounded wait on an mbarrier phase; records an error and returns false.
// These waits hand work between the warps of one CTA every few hundred
// nanoseconds, so they spin on try_wait (which parks the thread in hardware
// until the phase flips or a short time passes) with no sleep; the deadline,
// the iteration cap and the pipeline's error word are checked every 256
// attempts.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, const StageCtx& cx,
                                                  uint32_t where) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t deadline = gtime() + cx.limit_ns;
    const uint64_t cap = cx.limit_ns / 16 + 4000000ull;
    for (uint64_t it = 1;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 255) == 0 && (it > cap || gtime() > deadline || has_error(cx.ctl))) {
            record_error(cx.ctl, DEV_ERR_GROUP_BARRIER, 400 + 10 * cx.where + where);
            return false;
        }
    }
}


// 16-byte global -> shared copy that bypasses L1 and completes asynchronously;
// one commit group per weight quad, waited for per lane.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }
// Same, reading `src_bytes` (0 or 16) bytes and zero-filling the rest.
__device__ __forceinline__ void cp_async16_zfill(void* smem, const void* gmem, unsigned src_bytes) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(s), "l"(gmem), "r"(src_bytes)
                 : "memory");
}

__device__ __forceinline__ float apply_act(float v, int act) {
    if (act == ACT_RELU) return v > 0.f ? v : 0.f;
    if (act == ACT_GELU) return 0.5f * v * (1.f + erff(v * 0.70710678118654752f));
    return v;
}

// ---------------------------------------------------------------------------
// NORMALIZE_U8: y = (x - 127.5) / 64, u8 -> f32, row layout unchanged.  Exact in
// FP32 (x - 127.5 is a half-integer below 256, and 1/64 is a power of two).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float norm_u8(uint32_t b) {
    return (static_cast<float>(b) - 127.5f) * 0.015625f;
}

static __device__ void normalize_body(const StageCtx& cx, const StageParams& P, RowRef in, int n,
                               RowRef out) {
    const uint64_t chunks = P.in_row_bytes / 16;     // 16 input bytes -> 64 output bytes
    const uint64_t total = (uint64_t)n * chunks;
    const uint64_t stride = (uint64_t)cx.nctas * kThreads;
    constexpr int U = 4;                               // loads in flight per thread
    for (uint64_t base = (uint64_t)cx.rank * kThreads + threadIdx.x; base < total;
         base += stride * U) {
        uint4 v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint64_t e = base + u * stride;
            if (e < total) {
                const uint64_t q = e / chunks, c = e - q * chunks;
                v[u] = __ldcs(reinterpret_cast<const uint4*>(in.row(q)) + c);   // read once
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint64_t e = base + u * stride;
            if (e < total) {
                const uint64_t q = e / chunks, c = e - q * chunks;
                float4* o = reinterpret_cast<float4*>(out.row(q)) + 4 * c;
                const uint32_t w[4] = {v[u].x, v[u].y, v[u].z, v[u].w};
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    __stcg(o + j, make_float4(norm_u8(w[j] & 0xff), norm_u8((w[j] >> 8) & 0xff),
                                              norm_u8((w[j] >> 16) & 0xff), norm_u8(w[j] >> 24)));
            }
        }
    }
}

// Embedding gather of the text-tagging microservice: out row t of query q =
// E[tok] (bf16, D columns) for 0 <= tok < V, zero otherwise.  One warp takes
// 8 consecutive token rows at a time: lanes 0-7 read the 8 token IDs, then
// every lane loads its 16-byte pieces of all 8 table rows (up to 16 loads in
// flight, 64 pieces of each row per round) before storing them.
static __device__ void embed_body(const StageCtx& cx, const StageParams& P, RowRef in, int n, RowRef out) {
    const int V = P.H, D = P.W, T = P.rows;
    const uint4* E = reinterpret_cast<const uint4*>(P.layer[0].w);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int pieces = D / 8;                       // 16-byte pieces per row
    const int rows = n * T;
    const int groups = (rows + 7) / 8;
    const size_t rowb = (size_t)D * 2;
    for (int g = cx.rank * kWarps + warp; g < groups; g += cx.nctas * kWarps) {
        const int r0 = g * 8;
        int q = 0, t = 0, tk = -1;
        if (lane < 8 && r0 + lane < rows) {
            q = (r0 + lane) / T;
            t = r0 + lane - q * T;
            tk = reinterpret_cast<const int32_t*>(in.row(q))[t];
        }
        for (int pb = 0; pb < pieces; pb += 64) {
            uint4 v[8][2];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int tok = __shfl_sync(0xffffffffu, tk, k);
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    const int p = pb + 32 * i + lane;
                    v[k][i] = make_uint4(0u, 0u, 0u, 0u);
                    if (p < pieces && tok >= 0 && tok < V) v[k][i] = __ldg(E + (size_t)tok * pieces + p);
                }
            }
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int r = r0 + k;
                const int qk = __shfl_sync(0xffffffffu, q, k), tt = __shfl_sync(0xffffffffu, t, k);
                if (r >= rows) break;
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    const int p = pb + 32 * i + lane;
                    if (p < pieces) {
                        char* dst = P.out_tiled ? out.base + tiled_offset(r, (size_t)p * 16, rowb, P.out_tile_h)
                                                : out.row(qk) + (size_t)tt * rowb + (size_t)p * 16;
                        __stcg(reinterpret_cast<uint4*>(dst), v[k][i]);
                    }
                }
            }
        }
    }
}

// FP8 arm of the normalisation stage: the code of 128 y, y = (x - 127.5) / 64,
// i.e. e4m3(2 x - 255) (exact in f32, then rounded to nearest even e4m3).  The
// next stage reads the codes with scale 1/128.  16 input bytes -> 16 codes.
static __device__ void normalize_e4m3_body(const StageCtx& cx, const StageParams& P, RowRef in, int n,
                                           RowRef out) {
    const uint64_t chunks = P.in_row_bytes / 16;
    const uint64_t total = (uint64_t)n * chunks;
    const uint64_t stride = (uint64_t)cx.nctas * kThreads;
    constexpr int U = 4;
    for (uint64_t base = (uint64_t)cx.rank * kThreads + threadIdx.x; base < total;
         base += stride * U) {
        uint4 v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint64_t e = base + u * stride;
            if (e < total) {
                const uint64_t q = e / chunks, c = e - q * chunks;
                v[u] = __ldcs(reinterpret_cast<const uint4*>(in.row(q)) + c);
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint64_t e = base + u * stride;
            if (e < total) {
                const uint64_t q = e / chunks, c = e - q * chunks;
                const uint32_t w[4] = {v[u].x, v[u].y, v[u].z, v[u].w};
                uint32_t o[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    uint32_t packed = 0;
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
                        const float y128 = ((float)((w[j] >> (8 * b)) & 0xffu) - 127.5f) * 2.0f;
                        packed |= (uint32_t)__nv_cvt_float_to_fp8(y128, __NV_SATFINITE, __NV_E4M3) << (8 * b);
                    }
                    o[j] = packed;
                }
                const uint4 w4 = make_uint4(o[0], o[1], o[2], o[3]);
                if (P.out_tiled)
                    __stcg(reinterpret_cast<uint4*>(out.base + tiled_offset((int)q, c * 16, P.out_row_bytes, P.out_tile_h)), w4);
                else
                    __stcg(reinterpret_cast<uint4*>(out.row(q)) + c, w4);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// NORM_POOL2_BF16: 2x2 mean, normalise, round to bf16.  The FP32 value is exact
// (an integer sum <= 1020, times 1/4, minus 127.5, times 1/64), so the bf16
// result is the round-to-nearest-even of the exact value.
// Work is cut into groups of G consecutive output rows of one query (2G input
// rows, contiguous in the image).  Each warp streams its groups into two
// shared-memory buffers with one bulk copy per group (the copy engine moves
// far more per SM than 16-byte loads do), the next group's copy in flight
// while the current one is computed, and each lane produces four consecutive
// outputs (8 bytes) at a time (3-channel images: 12 outputs from three 8-byte
// loads per input row, so the byte-wise shared-memory reads do not bound it).
// Output value m of an output row reads input
// bytes i0 = 2 m - (m mod C) and i0 + C of the row pair (pixels 2w and 2w + 1,
// channel c, with m = w C + c).
// ---------------------------------------------------------------------------
constexpr int kPoolBufBytes = 12 * 1024;   // per warp and buffer: 2 x 8 warps x 12 KB = 192 KB

// The pool stage's 16 mbarriers (one per warp and buffer) and their completed
// fill counts, after the buffers.  Initialised once per kernel launch by
// pool_setup; every later call continues the counts, so the wait parities
// stay right across batches (mbarriers are never re-initialised in use).
__device__ __forceinline__ uint64_t* pool_bars(float* smem) {
    return reinterpret_cast<uint64_t*>(reinterpret_cast<uint8_t*>(smem) + kWarps * 2 * kPoolBufBytes);
}
__device__ __forceinline__ uint32_t* pool_fills(float* smem) {
    return reinterpret_cast<uint32_t*>(pool_bars(smem) + 2 * kWarps);
}
__device__ __forceinline__ void pool_setup(float* smem) {
    if (threadIdx.x < 2 * kWarps) {
        mbar_init(&pool_bars(smem)[threadIdx.x], 1);
        pool_fills(smem)[threadIdx.x] = 0u;
    }
    if (threadIdx.x == 0) mbar_fence_init();
    __syncthreads();
}

// (sum / 4 - 127.5) / 64 = sum / 256 - 510 / 256 for an integer sum of four
// bytes (<= 1020): the float of sum comes from its bits under the exponent of
// 2^23 (0x4B000000 | sum is 2^23 + sum exactly; subtracting 2^23 is exact), and
// the fused multiply-add is exact too (the result needs at most 18 bits), so
// the value is the exact one, as (float(sum) * 0.25 - 127.5) * 0.015625 is.
__device__ __forceinline__ float pooled_value(uint32_t sum) {
    const float f = __uint_as_float(0x4B000000u | sum) - 8388608.0f;
    return fmaf(f, 0.00390625f, -1.9921875f);
}

static __device__ void normpool_body(const StageCtx& cx, const StageParams& P, RowRef in, int n,
                                     RowRef out) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int Ho = P.H / 2, WC = P.W * P.C, C = P.C;
    const int pair_bytes = 2 * WC;                 // a multiple of 16, at most 8192
    const int out_vals = (P.W / 2) * C;            // a multiple of 4
    const int P4 = out_vals / 4;                   // 4-value items per output row
    const int G = min(8, kPoolBufBytes / pair_bytes);
    const int gpq = (Ho + G - 1) / G;              // groups per query
    const int groups = n * gpq;
    const int d128 = 128 % C;                      // channel step between a lane's items (32 x 4 values)
    const bool rgb4 = C == 3 && (P.W / 2) % 4 == 0;    // the 3-channel path below
    uint8_t* buf = reinterpret_cast<uint8_t*>(cx.smem) + warp * 2 * kPoolBufBytes;
    // device-resident contiguous rows (traces, direct launches): one bulk copy
    // per group (its 2G input rows are contiguous) into the warp's buffer,
    // completion on that buffer's mbarrier; rows of the query ring, which may
    // live in pinned host memory: cp.async
    const bool bulk = in.mask == ~0ull;
    uint64_t* bar = pool_bars(cx.smem) + warp * 2;
    uint32_t* fills = pool_fills(cx.smem) + warp * 2;
    const uint64_t pol = l2_policy_evict_first();          // each image is read once
    auto issue = [&](int g, int b) {
        const int q = g / gpq, ho0 = (g - q * gpq) * G;
        const uint32_t bytes = (uint32_t)(min(G, Ho - ho0) * pair_bytes);
        const char* src = in.row(q) + (size_t)ho0 * pair_bytes;
        if (bulk) {
            if (lane == 0) {
                mbar_arrive_expect_tx(&bar[b], bytes);
                bulk_load_hint(buf + b * kPoolBufBytes, src, bytes, &bar[b], pol);
            }
        } else {
            for (int i = lane; i < (int)(bytes / 16); i += 32)
                cp_async16(buf + b * kPoolBufBytes + 16 * i, reinterpret_cast<const uint4*>(src) + i);
            cp_async_commit();
        }
    };
    const int gstride = cx.nctas * kWarps;
    int cur = 0;
    uint32_t uses[2] = {fills[0], fills[1]};                // completed fills of each buffer (all calls)
    int g = cx.rank * kWarps + warp;
    if (g < groups) issue(g, 0);
    for (; g < groups; g += gstride, cur ^= 1) {
        if (g + gstride < groups) {
            issue(g + gstride, cur ^ 1);
            if (!bulk) cp_async_wait<1>();
        } else if (!bulk) {
            cp_async_wait<0>();
        }
        if (bulk) {
            if (!mbar_wait_bounded(&bar[cur], uses[cur] & 1u, cx, 8)) return;
            ++uses[cur];
        }
        __syncwarp();
        const uint8_t* sm = buf + cur * kPoolBufBytes;
        const int q = g / gpq, ho0 = (g - q * gpq) * G;
        if (rgb4) {
            // 3 channels, output width a multiple of 4: a lane takes 4 output
            // pixels (12 values), reading their 24 input bytes of each row with
            // three 8-byte loads and storing three 8-byte runs
            const int k4 = (P.W / 2) / 4;                       // items per output row
            const int items = min(G, Ho - ho0) * k4;
#pragma unroll 2
            for (int it = lane; it < items; it += 32) {
                const int r = it / k4, k = it - r * k4;
                const uint2* a0 = reinterpret_cast<const uint2*>(sm + r * pair_bytes + 24 * k);
                const uint2* a1 = reinterpret_cast<const uint2*>(sm + r * pair_bytes + WC + 24 * k);
                uint32_t w0[6], w1[6];
#pragma unroll
                for (int t = 0; t < 3; ++t) {
                    const uint2 u0 = a0[t], u1 = a1[t];
                    w0[2 * t] = u0.x; w0[2 * t + 1] = u0.y;
                    w1[2 * t] = u1.x; w1[2 * t + 1] = u1.y;
                }
                auto byte = [](const uint32_t (&w)[6], int o) { return (w[o >> 2] >> (8 * (o & 3))) & 0xffu; };
                uint32_t packed[6];
#pragma unroll
                for (int v = 0; v < 12; v += 2) {
                    float y2[2];
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int j = (v + h) / 3, cch = (v + h) % 3;   // output pixel, channel
                        const int o = 6 * j + cch;                      // pixel 2j, then 2j + 1 at + 3
                        const uint32_t sum = byte(w0, o) + byte(w0, o + 3) + byte(w1, o) + byte(w1, o + 3);
                        y2[h] = pooled_value(sum);
                    }
                    const __nv_bfloat162 pr = __floats2bfloat162_rn(y2[0], y2[1]);
                    packed[v / 2] = *reinterpret_cast<const uint32_t*>(&pr);
                }
                const size_t b0 = ((size_t)(ho0 + r) * out_vals + 12 * k) * 2;   // byte in the output row
#pragma unroll
                for (int t = 0; t < 3; ++t) {
                    const size_t bt = b0 + 8 * t;
                    char* dst = P.out_tiled ? out.base + tiled_offset(q, bt, P.out_row_bytes, P.out_tile_h)
                                            : out.row(q) + bt;
                    __stcg(reinterpret_cast<uint2*>(dst), make_uint2(packed[2 * t], packed[2 * t + 1]));
                }
            }
            __syncwarp();
            continue;
        }
        const int items = min(G, Ho - ho0) * P4;
        int r = lane / P4, i = lane - r * P4;      // output row in the group, item in the row
        int c = (4 * i) % C;                       // channel of the item's first value
        for (int it = lane; it < items; it += 32) {
            const uint8_t* r0 = sm + r * pair_bytes;
            const uint8_t* r1 = r0 + WC;
            const int m0 = 4 * i;
            float y[4];
            int cc = c;
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const int i0 = 2 * (m0 + t) - cc;
                const uint32_t s = (uint32_t)r0[i0] + r0[i0 + C] + r1[i0] + r1[i0 + C];
                y[t] = (static_cast<float>(s) * 0.25f - 127.5f) * 0.015625f;
                cc = cc + 1 == C ? 0 : cc + 1;
            }
            const __nv_bfloat162 lo = __floats2bfloat162_rn(y[0], y[1]);
            const __nv_bfloat162 hi = __floats2bfloat162_rn(y[2], y[3]);
            const uint2 v = make_uint2(*reinterpret_cast<const uint32_t*>(&lo),
                                       *reinterpret_cast<const uint32_t*>(&hi));
            const size_t b = ((size_t)(ho0 + r) * out_vals + m0) * 2;   // byte in the query's output row
            char* dst = P.out_tiled ? out.base + tiled_offset(q, b, P.out_row_bytes, P.out_tile_h)
                                    : out.row(q) + b;
            __stcg(reinterpret_cast<uint2*>(dst), v);
            // next item of this lane: 32 items on (rows of out_vals values are
            // whole multiples of C, so only the in-row step moves the channel)
            i += 32;
            while (i >= P4) { i -= P4; ++r; }
            c += d128;
            if (c >= C) c -= C;
        }
        __syncwarp();
    }
    if (bulk && lane == 0) {
        fills[0] = uses[0];
        fills[1] = uses[1];
    }
}

// ---------------------------------------------------------------------------
// FP32 dense layers (MLP_FP32).
// Task layer: y[q][j] = act(sum_k W[j][k] x[q][k]).  The K axis is cut into
// fixed chunks of KC, and chunks into fixed groups of 8 (one per warp).  CTA
// task (query group of 16, neuron block, chunk group g): warp w accumulates
// chunk 8g+w for the block's outputs, each in ascending k with FMA; the 8 chunk
// partials are added in chunk order in shared memory and stored as the group
// partial P[g][q][j]; the reduce phase adds the groups in ascending order.  Each
// lane owns NL neurons of the block (lane, lane+32, ...).  The packed weights are
// block-major, [Npad/64][K/4][64][4] (64-neuron blocks, k-quads inside), so a
// warp's chunk of one block is one contiguous run of 1 KB per k-quad.  It
// streams into the warp's ring of kMRing slots of kMQuads quads by bulk copies
// (mbarrier completion): the copy engine takes in ~200 GB/s per SM where
// 16-byte cp.async requests from the warps reach ~36 GB/s.  The query
// activations are broadcast from the warp's copy of the chunk.  Blocks are 128
// neurons (NL = 4: two 64-neuron halves per slot); when an instance has more
// CTAs than such tasks, 64-neuron blocks (NL = 2) double the tasks.  Either way
// every output sums the same chunks in the same order, so the block width, like
// the SM quota, leaves the results unchanged.
// ---------------------------------------------------------------------------
constexpr int kMXs = kQGroup * kMaxKC / 4;           // float4 per warp: the query chunk
constexpr int kMSlot = 2 * kMQuads * 64;             // float4 per ring slot (two 64-neuron halves)
constexpr int kMWarp = kMXs + kMRing * kMSlot;       // float4 per warp
static_assert(kWarps * kMWarp * 16 + kWarps * kMRing * 12 <= (int)kSmemBytes, "FP32 layer smem");

// The ring's mbarriers (one per warp and slot) and their completed fills,
// after the warps' areas; initialised once per kernel launch by mlp_setup,
// continued by every later call (never re-initialised in use).
__device__ __forceinline__ uint64_t* mlp_bars(float* smem) {
    return reinterpret_cast<uint64_t*>(reinterpret_cast<float4*>(smem) + kWarps * kMWarp);
}
__device__ __forceinline__ uint32_t* mlp_fills(float* smem) {
    return reinterpret_cast<uint32_t*>(mlp_bars(smem) + kWarps * kMRing);
}
__device__ __forceinline__ void mlp_setup(float* smem) {
    if (threadIdx.x < kWarps * kMRing) {
        mbar_init(&mlp_bars(smem)[threadIdx.x], 1);
        mlp_fills(smem)[threadIdx.x] = 0u;
    }
    if (threadIdx.x == 0) mbar_fence_init();
    __syncthreads();
}

template <int NL>
static __device__ void dense_tasks_nl(const StageCtx& cx, const LayerParams& L, RowRef x, int n,
                                      float* Pbuf) {
    constexpr int NB = 32 * NL;                        // neurons per task
    constexpr int NH = NL / 2;                         // 64-neuron halves per task
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float4* xs = reinterpret_cast<float4*>(cx.smem) + warp * kMWarp;
    float4* ring = xs + kMXs;
    uint64_t* bar = mlp_bars(cx.smem) + warp * kMRing;
    uint32_t* fills = mlp_fills(cx.smem) + warp * kMRing;
    uint32_t uses[kMRing];                             // completed fills of each slot (all calls)
#pragma unroll
    for (int s = 0; s < kMRing; ++s) uses[s] = fills[s];
    bool ok = true;                                    // false once a ring wait gave up (error recorded)
    const int QG = (n + kQGroup - 1) / kQGroup, NBLK = L.Npad / NB;
    const int G = (L.C + kWarps - 1) / kWarps;         // chunk groups
    const int ntask = QG * NBLK * G;
    const int KQ = L.K >> 2;
    const float4* wp = reinterpret_cast<const float4*>(L.w);
    for (int t = cx.rank; t < ntask; t += cx.nctas) {
        const int g = t % G;
        const int r = t / G;
        const int nb = r % NBLK, qg = r / NBLK;
        const int c = g * kWarps + warp;               // this warp's chunk
        float acc[kQGroup][NL];
#pragma unroll
        for (int q = 0; q < kQGroup; ++q)
#pragma unroll
            for (int i = 0; i < NL; ++i) acc[q][i] = 0.f;
        if (c < L.C && ok) {
            const int k0 = c * L.KC;
            const int kq_n = min(L.KC, L.K - k0) >> 2;
            const int F = (kq_n + kMQuads - 1) / kMQuads;   // ring fills of this chunk
            // half h of the block: quads k0/4 .. of 64-neuron block nb NH + h
            const float4* wq = wp + ((size_t)nb * NH * KQ + (k0 >> 2)) * 64;
            const uint64_t pol = l2_policy_evict_last();   // every batch re-reads the weights
            auto issue = [&](int j) {   // lane 0: fill j of the chunk into slot j mod kMRing
                const int q0 = j * kMQuads, nq = min(kMQuads, kq_n - q0);
                const int s = j % kMRing;
                mbar_arrive_expect_tx(&bar[s], (uint32_t)(NH * nq * 1024));
#pragma unroll
                for (int h = 0; h < NH; ++h)
                    bulk_load_hint(ring + s * kMSlot + h * kMQuads * 64, wq + ((size_t)h * KQ + q0) * 64,
                                   (uint32_t)(nq * 1024), &bar[s], pol);
            };
            // the query chunk (zero rows past the batch) by cp.async, the first
            // ring fills by bulk copies
            for (int e = lane; e < kQGroup * kq_n; e += 32) {
                const int q = e / kq_n, kq = e - q * kq_n;
                const int gq = qg * kQGroup + q;
                const float4* src = reinterpret_cast<const float4*>(x.row(gq < n ? gq : 0)) +
                                    (k0 >> 2) + kq;
                cp_async16_zfill(xs + q * (kMaxKC / 4) + kq, src, gq < n ? 16u : 0u);
            }
            cp_async_commit();
            if (lane == 0)
                for (int j = 0; j < min(kMRing, F); ++j) issue(j);
            cp_async_wait<0>();
            __syncwarp();                               // every lane's part of the query chunk
            for (int j = 0; j < F && ok; ++j) {
                const int s = j % kMRing;
                if (!mbar_wait_bounded(&bar[s], uses[s] & 1u, cx, 9)) {
                    ok = false;
                    break;
                }
                ++uses[s];
                const int q0 = j * kMQuads, nq = min(kMQuads, kq_n - q0);
                for (int qq = 0; qq < nq; ++qq) {
                    const int kq = q0 + qq;
                    const float4* wv = ring + s * kMSlot + qq * 64 + lane;
                    float4 a[NL];
#pragma unroll
                    for (int i = 0; i < NL; ++i) a[i] = wv[(i >> 1) * kMQuads * 64 + 32 * (i & 1)];
#pragma unroll
                    for (int q = 0; q < kQGroup; ++q) {
                        const float4 xv = xs[q * (kMaxKC / 4) + kq];
#pragma unroll
                        for (int i = 0; i < NL; ++i) {
                            acc[q][i] = fmaf(xv.x, a[i].x, acc[q][i]);
                            acc[q][i] = fmaf(xv.y, a[i].y, acc[q][i]);
                            acc[q][i] = fmaf(xv.z, a[i].z, acc[q][i]);
                            acc[q][i] = fmaf(xv.w, a[i].w, acc[q][i]);
                        }
                    }
                }
                __syncwarp();                           // every lane is done with slot s
                if (lane == 0 && j + kMRing < F) issue(j + kMRing);
            }
            // a fill issued but not consumed (only after a failed wait) is
            // waited for, boundedly, so that no copy lands in a reused slot
            if (!ok)
                for (int j = 0; j < min(kMRing, F); ++j) {
                    const int s = j % kMRing;
                    (void)mbar_wait_bounded(&bar[s], uses[s] & 1u, cx, 9);
                }
        }
        // the warp's chunk partial [16][NB] goes to its (now free) query area
        static_assert(kQGroup * kNBlock <= 4 * kMXs, "partial does not fit");
        __syncwarp();
        float* part = reinterpret_cast<float*>(xs);
#pragma unroll
        for (int q = 0; q < kQGroup; ++q)
#pragma unroll
            for (int i = 0; i < NL; ++i) part[q * NB + 32 * i + lane] = acc[q][i];
        __syncthreads();
        // group partial = chunk partials added in warp (= chunk) order
        for (int o = threadIdx.x; o < kQGroup * NB; o += kThreads) {
            const int q = o / NB, j = o - q * NB;
            const int gq = qg * kQGroup + q;
            float sum = 0.f;
#pragma unroll
            for (int w = 0; w < kWarps; ++w)
                sum += reinterpret_cast<const float*>(cx.smem)[w * kMWarp * 4 + q * NB + j];
            if (gq < n) __stcg(Pbuf + ((size_t)g * n + gq) * L.Npad + nb * NB + j, sum);
        }
        __syncthreads();
    }
    if (lane == 0)
#pragma unroll
        for (int s = 0; s < kMRing; ++s) fills[s] = uses[s];
    __syncwarp();
}

static __device__ void dense_tasks(const StageCtx& cx, const LayerParams& L, RowRef x, int n,
                                   float* Pbuf) {
    // half-width blocks when they shorten the slowest CTA's work: their 2T
    // tasks take fewer rounds over the instance's CTAs than twice the rounds
    // of the T full tasks
    const int QG = (n + kQGroup - 1) / kQGroup;
    const int G = (L.C + kWarps - 1) / kWarps;
    const int T = QG * (L.Npad / kNBlock) * G;
    const int rounds = (T + cx.nctas - 1) / cx.nctas, rounds2 = (2 * T + cx.nctas - 1) / cx.nctas;
    if (rounds2 < 2 * rounds) dense_tasks_nl<2>(cx, L, x, n, Pbuf);
    else dense_tasks_nl<4>(cx, L, x, n, Pbuf);
}

// Reduction over the G chunk groups, in ascending group order; each thread
// owns outputs and issues its group loads eight at a time.
static __device__ void dense_reduce(const StageCtx& cx, const LayerParams& L, int n, const float* Pbuf,
                             RowRef out) {
    const int total = n * L.N;
    const int G = (L.C + kWarps - 1) / kWarps;
    const size_t gstride = (size_t)n * L.Npad;
    for (int e = cx.rank * kThreads + threadIdx.x; e < total; e += cx.nctas * kThreads) {
        const int q = e / L.N, j = e - q * L.N;
        const float* p = Pbuf + (size_t)q * L.Npad + j;
        float s = 0.f;
        int g = 0;
        for (; g + 8 <= G; g += 8) {
            float v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = __ldcg(p + (size_t)(g + u) * gstride);
#pragma unroll
            for (int u = 0; u < 8; ++u) s += v[u];
        }
        for (; g < G; ++g) s += __ldcg(p + (size_t)g * gstride);
        __stcg(reinterpret_cast<float*>(out.row(q)) + j, apply_act(s, L.act));
    }
}

// Warp-wide best of (value, index) under "larger value, then smaller index".
__device__ __forceinline__ void warp_best(float& v, int& i) {
#pragma unroll
    for (int off = 16; off; off >>= 1) {
        const float ov = __shfl_xor_sync(0xffffffffu, v, off);
        const int oi = __shfl_xor_sync(0xffffffffu, i, off);
        if (ov > v || (ov == v && oi < i)) { v = ov; i = oi; }
    }
}

// Head layer (last layer of a final stage, N <= 32): one warp per query.  Lane
// l accumulates k-quads l, l+32, ... in ascending order for all N outputs;
// the 32 lane partials of each output are then summed by an xor butterfly,
// which builds the same addition tree in every lane.  Lane j keeps output j;
// the top-k follows by repeated warp-wide best.
static __device__ void dense_head(const StageCtx& cx, const LayerParams& L, RowRef x, int n, int top_k,
                           const FinalOut& fo) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int KQ = L.K >> 2;
    for (int q = cx.rank * kWarps + warp; q < n; q += cx.nctas * kWarps) {
        float acc[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) acc[j] = 0.f;
        const float4* xr = reinterpret_cast<const float4*>(x.row(q));
        for (int kq = lane; kq < KQ; kq += 32) {
            const float4 xv = __ldcg(xr + kq);
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                if (j < L.N) {
                    const float4 wv = __ldg(reinterpret_cast<const float4*>(L.w + (size_t)j * L.K) + kq);
                    acc[j] = fmaf(xv.x, wv.x, acc[j]);
                    acc[j] = fmaf(xv.y, wv.y, acc[j]);
                    acc[j] = fmaf(xv.z, wv.z, acc[j]);
                    acc[j] = fmaf(xv.w, wv.w, acc[j]);
                }
            }
        }
        float mine = 0.f;
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            if (j < L.N) {
                float v = acc[j];
#pragma unroll
                for (int off = 16; off; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
                if (lane == j) mine = v;
            }
        }
        mine = apply_act(mine, L.act);
        if (fo.logits.base != nullptr && lane < L.N)
            reinterpret_cast<float*>(fo.logits.row(q))[lane] = mine;
        float cand = lane < L.N ? mine : -INFINITY;
        for (int r = 0; r < top_k; ++r) {
            float bv = cand;
            int bi = lane < L.N ? lane : 0x7fffffff;
            warp_best(bv, bi);
            if (lane == 0) {
                fo.idx[(size_t)q * top_k + r] = bi;
                fo.val[(size_t)q * top_k + r] = bv;
            }
            if (lane == bi) cand = -INFINITY;
        }
    }
}

// Top-k of each row (value descending, index ascending on ties).  A CTA takes
// several rows at once, each with wpr warps (all 8 warps on one row when the
// CTA has only one row to do, one warp per row when it has 8 or more): every
// warp scans a segment of its row (8 loads in flight per lane, insertion into
// the lane's sorted top-k) and reduces its lanes to the segment's top-k, and
// the row's first warp merges the segment lists.  The result does not depend
// on the split (the order is total).  The logits row is copied on the way
// when wanted.
static __device__ void topk_rows(const StageCtx& cx, RowRef z, int n, int N, int k, const FinalOut& fo) {
    __shared__ float s_v[kWarps][kMaxTopK];
    __shared__ int s_i[kWarps][kMaxTopK];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int rpc = (n + cx.nctas - 1) / cx.nctas;            // rows per CTA
    int wpr = kWarps;                                          // warps per row
    while (wpr > 1 && wpr * rpc > kWarps) wpr >>= 1;
    const int at_once = kWarps / wpr;
    const int slot = warp / wpr, sw = warp - slot * wpr;       // row slot, warp within the row
    const int seg = (N + wpr - 1) / wpr;
    for (int q0 = cx.rank * at_once; q0 < n; q0 += cx.nctas * at_once) {
        const int q = q0 + slot;
        if (q < n) {
            float bv[kMaxTopK];
            int bi[kMaxTopK];
#pragma unroll
            for (int r = 0; r < kMaxTopK; ++r) { bv[r] = -INFINITY; bi[r] = 0x7fffffff; }
            const float* zr = reinterpret_cast<const float*>(z.row(q));
            const int jb = sw * seg, je = min(N, jb + seg);
            for (int j0 = jb + lane; j0 < je; j0 += 32 * 8) {
                float vv[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) vv[u] = j0 + 32 * u < je ? __ldcg(zr + j0 + 32 * u) : 0.f;
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int j = j0 + 32 * u;
                    if (j >= je) break;
                    const float v = vv[u];
                    if (fo.logits.base != nullptr) reinterpret_cast<float*>(fo.logits.row(q))[j] = v;
                    // insert (v, j) into the lane's top kMaxTopK (a superset of its
                    // top k; indexes known at compile time keep the list in
                    // registers): j grows along the lane's scan, so ties keep the
                    // earlier index first
                    if (v > bv[kMaxTopK - 1] || bi[kMaxTopK - 1] == 0x7fffffff) {
                        float cv = v;
                        int ci = j;
#pragma unroll
                        for (int r = 0; r < kMaxTopK; ++r) {
                            if (cv > bv[r] || bi[r] == 0x7fffffff) {
                                const float tv = bv[r];
                                const int ti = bi[r];
                                bv[r] = cv; bi[r] = ci; cv = tv; ci = ti;
                            }
                        }
                    }
                }
            }
            // the segment's top-k: k rounds of warp-wide best, the winning lane pops its head
            for (int r = 0; r < k; ++r) {
                float v = bv[0];
                int i = bi[0];
                warp_best(v, i);
                if (lane == 0) {
                    s_v[warp][r] = v;
                    s_i[warp][r] = i;
                }
                if (bi[0] == i) {
#pragma unroll
                    for (int t = 0; t + 1 < kMaxTopK; ++t) { bv[t] = bv[t + 1]; bi[t] = bi[t + 1]; }
                    bv[kMaxTopK - 1] = -INFINITY;
                    bi[kMaxTopK - 1] = 0x7fffffff;
                }
            }
        }
        __syncthreads();
        if (q < n && sw == 0) {
            // the row's wpr k candidates (warp slot * wpr + c / k, rank c % k),
            // c = lane and lane + 32: each lane keeps its two in order, the
            // better first; empty entries carry index 0x7fffffff and lose
            // every comparison
            float cv[2] = {-INFINITY, -INFINITY};
            int ci[2] = {0x7fffffff, 0x7fffffff};
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int c = lane + 32 * h;
                if (c < wpr * k && s_i[warp + c / k][c % k] != 0x7fffffff) {
                    cv[h] = s_v[warp + c / k][c % k];
                    ci[h] = s_i[warp + c / k][c % k];
                }
            }
            if (cv[1] > cv[0] || (cv[1] == cv[0] && ci[1] < ci[0])) {
                const float tv = cv[0];
                const int ti = ci[0];
                cv[0] = cv[1]; ci[0] = ci[1]; cv[1] = tv; ci[1] = ti;
            }
            for (int r = 0; r < k; ++r) {
                float v = cv[0];
                int i = ci[0];
                warp_best(v, i);
                if (lane == 0) {
                    fo.idx[(size_t)q * k + r] = i;
                    fo.val[(size_t)q * k + r] = v;
                }
                if (ci[0] == i) {
                    cv[0] = cv[1]; ci[0] = ci[1];
                    cv[1] = -INFINITY; ci[1] = 0x7fffffff;
                }
            }
        }
        __syncthreads();
    }
}

// Token-level final stage: the argmax (lowest index among equal maxima) of
// each of the T rows of every query; the tags of the first res_k rows go to
// the result arrays, all T tags (int32) to the logits rows when wanted.
static __device__ void token_argmax(const StageCtx& cx, RowRef z, int n, int T, int N, int res_k,
                                    const FinalOut& fo) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int r = cx.rank * kWarps + warp; r < n * T; r += cx.nctas * kWarps) {
        const float* zr = reinterpret_cast<const float*>(z.row(r));
        float bv = -INFINITY;
        int bi = 0x7fffffff;
        for (int j = lane; j < N; j += 32) {
            const float v = __ldcg(zr + j);
            if (v > bv || bi == 0x7fffffff) { bv = v; bi = j; }
        }
        warp_best(bv, bi);
        if (lane == 0) {
            const int q = r / T, t = r - q * T;
            if (t < res_k) {
                fo.idx[(size_t)q * res_k + t] = bi;
                fo.val[(size_t)q * res_k + t] = bv;
            }
            if (fo.logits.base != nullptr) reinterpret_cast<int32_t*>(fo.logits.row(q))[t] = bi;
        }
    }
}

// The whole FP32 MLP stage.  Returns false if a group barrier failed.
static __device__ bool mlp_body(const StageCtx& cx, const StageParams& P, RowRef in, int n, RowRef out,
                         const FinalOut& fo) {
    RowRef x = in;
    for (int l = 0; l < P.n_layers; ++l) {
        const LayerParams& L = P.layer[l];
        const bool last = (l == P.n_layers - 1);
        if (L.head) {
            dense_head(cx, L, x, n, P.top_k, fo);
            return true;
        }
        float* Pbuf = reinterpret_cast<float*>(cx.scratch + L.p_off);
        dense_tasks(cx, L, x, n, Pbuf);
        if (!group_barrier(cx.gs, cx.nctas, cx.ctl, cx.limit_ns, cx.where)) return false;
        RowRef dst = (last && P.top_k == 0)
                         ? out
                         : RowRef{cx.scratch + L.h_off, 0, ~0ull, (size_t)L.N * sizeof(float)};
        dense_reduce(cx, L, n, Pbuf, dst);
        if (!group_barrier(cx.gs, cx.nctas, cx.ctl, cx.limit_ns, cx.where)) return false;
        x = dst;
        if (last && P.top_k > 0) topk_rows(cx, x, n, L.N, P.top_k, fo);
    }
    return true;
}

}  // namespace camelot
