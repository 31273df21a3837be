// GEMM_BF16 stage body: dense layers on the 5th-generation tensor cores.
//
// Each layer computes y[q][m] = act(sum_k W[m][k] x[q][k]) for a batch of at
// most 32 queries.  The batch is small, so the operands are swapped: the
// weights are the M = 128 operand (128 x 64 tiles streamed by TMA through a
// shared-memory ring with the 128-byte swizzle) and the queries are the N = 32
// operand (a K-chunk of all queries, staged with cp.async in the same swizzled
// layout into a double buffer and reused by every weight tile of the chunk).
// The CTA's warps specialise: one streams weight tiles, one stages query
// chunks, one thread issues tcgen05.mma (M=128, N=32, K=16) into one of two
// TMEM accumulators, four warps drain the other accumulator.  A unit is
// (K-chunk, 128-row tile); chunk partials are added in chunk order, so the
// result is the same whatever the number of CTAs.
#pragma once
#include <cuda_bf16.h>

#include "device_sync.cuh"
#include "stage_params.h"
#include "stages.cuh"
#include "tc_ptx.cuh"

namespace camelot {

constexpr int kGemmStages = 4;                   // weight-tile ring depth
constexpr int kGemmN = 32;                       // queries per MMA (N)
constexpr int kGemmMaxKC = 1024;                 // largest K-chunk (elements)
constexpr uint32_t kATileBytes = 128 * 64 * 2;   // one 128 x 64 bf16 weight tile
constexpr uint32_t kBTileBytes = kGemmN * 64 * 2;
constexpr uint32_t kBChunkBytes = (kGemmMaxKC / 64) * kBTileBytes;   // 64 KB
constexpr uint32_t kTmemCols = 64;               // two 32-column accumulators

// Warp roles inside a CTA running tensor-core layers.
constexpr int kWarpTma = 0;     // weight tiles, TMA
constexpr int kWarpMma = 1;     // tcgen05.mma issue (one thread)
constexpr int kWarpB = 2;       // query chunks, cp.async into the double buffer
constexpr int kWarpEpi0 = 4;    // warps 4..7 read the accumulators

struct GemmSmem {
    char* a_ring;          // kGemmStages x 16 KB weight tiles
    char* b_buf;           // 2 x 64 KB query chunks
    uint64_t* full;        // [kGemmStages] weight tile landed
    uint64_t* empty;       // [kGemmStages] MMAs reading the tile are done
    uint64_t* bfull;       // [2] query chunk staged (32 arrivals: warp kWarpB)
    uint64_t* bempty;      // [2] MMAs reading the chunk are done
    uint64_t* tfull;       // [2] accumulator complete
    uint64_t* tfree;       // [2] accumulator read out (4 arrivals: epilogue warps)
    uint32_t* tmem_slot;   // TMEM base address written by tcgen05.alloc
    uint32_t* ring_it;     // weight tiles so far (all launches of this CTA)
    uint32_t* b_it;        // query chunks staged so far
    uint32_t* acc_it;      // units finished so far
};

__device__ __forceinline__ GemmSmem gemm_smem(float* smem) {
    char* base = reinterpret_cast<char*>(
        (reinterpret_cast<uintptr_t>(smem) + 1023) & ~static_cast<uintptr_t>(1023));
    GemmSmem g;
    g.a_ring = base;
    g.b_buf = base + kGemmStages * kATileBytes;
    uint64_t* bars = reinterpret_cast<uint64_t*>(g.b_buf + 2 * kBChunkBytes);
    g.full = bars;
    g.empty = g.full + kGemmStages;
    g.bfull = g.empty + kGemmStages;
    g.bempty = g.bfull + 2;
    g.tfull = g.bempty + 2;
    g.tfree = g.tfull + 2;
    g.tmem_slot = reinterpret_cast<uint32_t*>(g.tfree + 2);
    g.ring_it = g.tmem_slot + 1;
    g.b_it = g.ring_it + 1;
    g.acc_it = g.b_it + 1;
    return g;
}

// Once per launch by every CTA that runs GEMM_BF16 work: barriers and TMEM.
__device__ __forceinline__ void gemm_setup(float* smem) {
    GemmSmem g = gemm_smem(smem);
    if (threadIdx.x == 0) {
        for (int s = 0; s < kGemmStages; ++s) {
            mbar_init(&g.full[s], 1);
            mbar_init(&g.empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&g.bfull[b], 32);
            mbar_init(&g.bempty[b], 1);
            mbar_init(&g.tfull[b], 1);
            mbar_init(&g.tfree[b], 4);
        }
        *g.ring_it = 0;
        *g.b_it = 0;
        *g.acc_it = 0;
        mbar_fence_init();
    }
    if (threadIdx.x < 32) {
        tmem_alloc(g.tmem_slot, kTmemCols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
}

__device__ __forceinline__ void gemm_teardown(float* smem) {
    GemmSmem g = gemm_smem(smem);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (threadIdx.x < 32) tmem_dealloc(*g.tmem_slot, kTmemCols);
}

// Bounded wait on an mbarrier phase; records an error and returns false.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, const StageCtx& cx,
                                                  uint32_t where) {
    if (mbar_try_wait(bar, parity)) return true;
    Backoff bo(cx.limit_ns);
    while (!mbar_try_wait(bar, parity)) {
        if (has_error(cx.ctl) || !bo.step()) {
            record_error(cx.ctl, DEV_ERR_GROUP_BARRIER, 400 + 10 * cx.where + where);
            return false;
        }
    }
    return true;
}

// Output of one layer: bf16 rows (hidden / next stage) or f32 rows (logits).
struct LayerOut {
    RowRef rows;
    int f32;
};

__device__ __forceinline__ void store_out(const LayerOut& o, int q, int m, float v) {
    if (o.f32) reinterpret_cast<float*>(o.rows.row(q))[m] = v;
    else reinterpret_cast<__nv_bfloat16*>(o.rows.row(q))[m] = __float2bfloat16_rn(v);
}

// One layer.  Work units u = (chunk c, 128-row tile mt) in chunk-major order
// (u = c * MT + mt); CTA r takes the contiguous units [r U / p, (r+1) U / p),
// so consecutive units share their query chunk.  Every unit accumulates the
// same K range in the same MMA order whichever CTA runs it.
static __device__ bool gemm_layer_tasks(const StageCtx& cx, const LayerParams& L, RowRef x, int n,
                                        float* Pbuf, const LayerOut& direct) {
    const GemmSmem g = gemm_smem(cx.smem);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int MT = L.Npad / 128;
    const int U = MT * L.C;
    const int u0 = (int)((long long)cx.rank * U / cx.nctas);
    const int u1 = (int)((long long)(cx.rank + 1) * U / cx.nctas);
    const uint32_t ring0 = *g.ring_it, b0 = *g.b_it, a0 = *g.acc_it;
    const uint32_t tmem = *g.tmem_slot;
    auto chunk_kb = [&](int c) { return min(L.KC, L.K - c * L.KC) / 64; };

    if (u0 < u1) {
        if (warp == kWarpTma && lane == 0) {
            // weight tiles of every unit, in order, through the ring
            uint32_t gi = ring0;
            for (int u = u0; u < u1; ++u) {
                const int c = u / MT, mt = u - c * MT;
                const int nkb = chunk_kb(c);
                for (int kb = 0; kb < nkb; ++kb, ++gi) {
                    const int s = gi % kGemmStages;
                    if (gi >= ring0 + kGemmStages || gi >= (uint32_t)kGemmStages) {
                        if (gi >= (uint32_t)kGemmStages &&
                            !mbar_wait_bounded(&g.empty[s], ((gi / kGemmStages) - 1) & 1, cx, 1))
                            goto done;
                    }
                    mbar_arrive_expect_tx(&g.full[s], kATileBytes);
                    tma_load_2d(g.a_ring + s * kATileBytes, &L.tmap, &g.full[s], c * L.KC + kb * 64,
                                mt * 128);
                }
            }
        } else if (warp == kWarpB) {
            // query chunks: once per distinct chunk of the range, double-buffered
            uint32_t h = b0;
            for (int c = u0 / MT; c <= (u1 - 1) / MT; ++c, ++h) {
                const int buf = h & 1;
                if (h >= 2 && !mbar_wait_bounded(&g.bempty[buf], ((h >> 1) - 1) & 1, cx, 2)) break;
                const int kc = chunk_kb(c) * 64;
                char* dstb = g.b_buf + buf * kBChunkBytes;
                const int per_row = kc / 8;                      // 16-byte pieces per row
                for (int e = lane; e < kGemmN * per_row; e += 32) {
                    const int r = e / per_row, pc = e - r * per_row;
                    const int kb = pc >> 3, j = pc & 7;
                    const char* src = x.row(r < n ? r : 0) + (size_t)(c * L.KC + 8 * pc) * 2;
                    cp_async16_zfill(dstb + kb * kBTileBytes + r * 128 + ((j ^ (r & 7)) << 4), src,
                                     r < n ? 16u : 0u);
                }
                cp_async_commit();
                cp_async_wait<0>();
                fence_proxy_async_smem();
                mbar_arrive(&g.bfull[buf]);
            }
        } else if (warp == kWarpMma && lane == 0) {
            const uint32_t idesc = idesc_bf16_f32(128, kGemmN);
            uint32_t gi = ring0, h = b0, a = a0;
            int cur_c = -1;
            for (int u = u0; u < u1; ++u, ++a) {
                const int c = u / MT;
                const int nkb = chunk_kb(c);
                if (c != cur_c) {
                    if (cur_c >= 0) { tc_commit(&g.bempty[h & 1]); ++h; }
                    cur_c = c;
                    if (!mbar_wait_bounded(&g.bfull[h & 1], (h >> 1) & 1, cx, 3)) goto done;
                }
                const int acc = a & 1;
                if (a >= a0 + 2 || a >= 2) {
                    if (a >= 2 && !mbar_wait_bounded(&g.tfree[acc], ((a >> 1) - 1) & 1, cx, 4)) goto done;
                }
                tc_fence_after();
                const uint32_t d_tmem = tmem + acc * kGemmN;
                const uint32_t b_base = smem_u32(g.b_buf + (h & 1) * kBChunkBytes);
                for (int kb = 0; kb < nkb; ++kb, ++gi) {
                    const int s = gi % kGemmStages;
                    if (!mbar_wait_bounded(&g.full[s], (gi / kGemmStages) & 1, cx, 5)) goto done;
                    tc_fence_after();
                    const uint32_t a_addr = smem_u32(g.a_ring + s * kATileBytes);
                    const uint32_t b_addr = b_base + kb * kBTileBytes;
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        tc_mma_f16(d_tmem, sw128_desc(a_addr + 32 * k), sw128_desc(b_addr + 32 * k),
                                   idesc, (kb > 0 || k > 0) ? 1u : 0u);
                    tc_commit(&g.empty[s]);
                }
                tc_commit(&g.tfull[acc]);
            }
            if (cur_c >= 0) tc_commit(&g.bempty[h & 1]);
        } else if (warp >= kWarpEpi0) {
            // accumulator rows 32 (warp % 4) .. +31, all 32 query columns
            const int sub = warp & 3;
            for (int u = u0, a = (int)a0; u < u1; ++u, ++a) {
                const int c = u / MT, mt = u - c * MT;
                const int acc = a & 1;
                if (!mbar_wait_bounded(&g.tfull[acc], (a >> 1) & 1, cx, 6)) break;
                tc_fence_after();
                uint32_t r0[16], r1[16];
                const uint32_t ta = tmem + ((uint32_t)(32 * sub) << 16) + acc * kGemmN;
                tmem_ld16(ta, r0);
                tmem_ld16(ta + 16, r1);
                tmem_ld_wait();
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&g.tfree[acc]);
                const int m = mt * 128 + 32 * sub + lane;
                if (m < L.N) {
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const int q = j;
                        if (q < n) {
                            const float v = __uint_as_float(j < 16 ? r0[j] : r1[j - 16]);
                            if (L.C == 1) store_out(direct, q, m, apply_act(v, L.act));
                            else __stcg(Pbuf + ((size_t)c * n + q) * L.Npad + m, v);
                        }
                    }
                }
            }
        }
    }
done:
    __syncthreads();
    if (threadIdx.x == 0 && u0 < u1) {
        uint32_t tiles = 0;
        for (int u = u0; u < u1; ++u) tiles += chunk_kb(u / MT);
        *g.ring_it = ring0 + tiles;
        *g.b_it = b0 + (uint32_t)((u1 - 1) / MT - u0 / MT + 1);
        *g.acc_it = a0 + (uint32_t)(u1 - u0);
    }
    __syncthreads();
    return !has_error(cx.ctl);
}

// out[q][m] = act(sum over chunks, in chunk order) for m < N.
static __device__ void gemm_reduce(const StageCtx& cx, const LayerParams& L, int n, const float* Pbuf,
                                   const LayerOut& o) {
    const int total = n * L.N;
    const size_t cstride = (size_t)n * L.Npad;
    for (int e = cx.rank * kThreads + threadIdx.x; e < total; e += cx.nctas * kThreads) {
        const int q = e / L.N, m = e - q * L.N;
        const float* p = Pbuf + (size_t)q * L.Npad + m;
        float s = 0.f;
        int c = 0;
        for (; c + 8 <= L.C; c += 8) {
            float v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = __ldcg(p + (size_t)(c + u) * cstride);
#pragma unroll
            for (int u = 0; u < 8; ++u) s += v[u];
        }
        for (; c < L.C; ++c) s += __ldcg(p + (size_t)c * cstride);
        store_out(o, q, m, apply_act(s, L.act));
    }
}

// The whole GEMM_BF16 stage.
static __device__ bool gemm_body(const StageCtx& cx, const StageParams& P, RowRef in, int n,
                                 RowRef out, const FinalOut& fo) {
    RowRef x = in;
    for (int l = 0; l < P.n_layers; ++l) {
        const LayerParams& L = P.layer[l];
        const bool last = (l == P.n_layers - 1);
        LayerOut o;
        if (last && P.top_k == 0) {
            o = LayerOut{out, 0};
        } else if (last) {
            o = LayerOut{RowRef{cx.scratch + L.h_off, 0, ~0ull, (size_t)L.N * sizeof(float)}, 1};
        } else {
            o = LayerOut{RowRef{cx.scratch + L.h_off, 0, ~0ull, (size_t)L.N * 2}, 0};
        }
        float* Pbuf = reinterpret_cast<float*>(cx.scratch + L.p_off);
        if (!gemm_layer_tasks(cx, L, x, n, Pbuf, o)) return false;
        if (!group_barrier(cx.gs, cx.nctas, cx.ctl, cx.limit_ns, cx.where)) return false;
        if (L.C > 1) {
            gemm_reduce(cx, L, n, Pbuf, o);
            if (!group_barrier(cx.gs, cx.nctas, cx.ctl, cx.limit_ns, cx.where)) return false;
        }
        x = o.rows;
        if (last && P.top_k > 0) topk_rows(cx, x, n, L.N, P.top_k, fo);
    }
    return true;
}

}  // namespace camelot
