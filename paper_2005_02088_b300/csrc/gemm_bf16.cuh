// GEMM_BF16 stage body: dense layers on the 5th-generation tensor cores.
//
// Each layer computes y[q][m] = act(sum_k W[m][k] x[q][k]) for a batch of at
// most 32 queries.  The batch is small, so the operands are swapped: the
// weights are the M = 128 operand (one 128-row tile per task, streamed by TMA
// through a 6-stage shared-memory ring with the 128-byte swizzle) and the
// queries are the N = 32 operand (the task's K-chunk of all queries, staged
// once per task with cp.async in the same swizzled layout).  One thread issues
// tcgen05.mma (M=128, N=32, K=16 per instruction) accumulating in TMEM; the
// epilogue reads the accumulator with tcgen05.ld.  A task is (128-row tile,
// K-chunk); chunk partials are added in chunk order, so the result is the
// same whatever the number of CTAs.
#pragma once
#include <cuda_bf16.h>

#include "device_sync.cuh"
#include "stage_params.h"
#include "stages.cuh"
#include "tc_ptx.cuh"

namespace camelot {

constexpr int kGemmStages = 6;                   // weight-tile ring depth
constexpr int kGemmN = 32;                       // queries per MMA (N)
constexpr int kGemmMaxKC = 1024;                 // largest K-chunk (elements)
constexpr uint32_t kATileBytes = 128 * 64 * 2;   // one 128 x 64 bf16 weight tile
constexpr uint32_t kBTileBytes = kGemmN * 64 * 2;
constexpr uint32_t kTmemCols = 32;

struct GemmSmem {
    char* a_ring;          // kGemmStages x 16 KB
    char* b_tile;          // (kGemmMaxKC / 64) x 4 KB
    uint64_t* full;        // [kGemmStages] weight tile landed
    uint64_t* empty;       // [kGemmStages] MMAs reading the stage are done
    uint64_t* accb;        // accumulator complete
    uint32_t* tmem_slot;   // TMEM base address written by tcgen05.alloc
    uint32_t* ring_it;     // weight tiles issued so far (phase tracking)
    uint32_t* acc_it;      // tasks finished so far
};

__device__ __forceinline__ GemmSmem gemm_smem(float* smem) {
    char* base = reinterpret_cast<char*>(
        (reinterpret_cast<uintptr_t>(smem) + 1023) & ~static_cast<uintptr_t>(1023));
    GemmSmem g;
    g.a_ring = base;
    g.b_tile = base + kGemmStages * kATileBytes;
    char* tail = g.b_tile + (kGemmMaxKC / 64) * kBTileBytes;
    g.full = reinterpret_cast<uint64_t*>(tail);
    g.empty = g.full + kGemmStages;
    g.accb = g.empty + kGemmStages;
    g.tmem_slot = reinterpret_cast<uint32_t*>(g.accb + 1);
    g.ring_it = g.tmem_slot + 1;
    g.acc_it = g.ring_it + 1;
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
        mbar_init(g.accb, 1);
        *g.ring_it = 0;
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
            record_error(cx.ctl, DEV_ERR_GROUP_BARRIER, 400 + cx.where);
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

// One layer's (tile, chunk) tasks.  Returns false on a failed wait.
static __device__ bool gemm_layer_tasks(const StageCtx& cx, const LayerParams& L, RowRef x, int n,
                                        float* Pbuf, const LayerOut& direct) {
    const GemmSmem g = gemm_smem(cx.smem);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int MT = L.Npad / 128;
    const int ntask = MT * L.C;
    const uint32_t idesc = idesc_bf16_f32(128, kGemmN);
    const uint32_t tmem = *g.tmem_slot;
    __shared__ int s_ok;
    for (int t = cx.rank; t < ntask; t += cx.nctas) {
        const int mt = t / L.C, c = t - mt * L.C;
        const int k0 = c * L.KC;
        const int kc = min(L.KC, L.K - k0);
        const int nkb = kc / 64;
        // the queries' K-chunk, swizzled: 16-byte piece j of row r of k-block kb
        // lands at kb * 4096 + r * 128 + ((j ^ (r & 7)) * 16)
        const int pieces = kGemmN * (kc / 8);
        for (int e = threadIdx.x; e < pieces; e += kThreads) {
            const int r = e / (kc / 8), p = e - r * (kc / 8);
            const int kb = p >> 3, j = p & 7;
            const char* src = x.row(r < n ? r : 0) + (size_t)(k0 + 8 * p) * 2;
            char* dst = g.b_tile + kb * kBTileBytes + r * 128 + ((j ^ (r & 7)) << 4);
            cp_async16_zfill(dst, src, r < n ? 16u : 0u);
        }
        cp_async_commit();
        cp_async_wait<0>();
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // visible to the tensor cores
        __syncthreads();
        if (threadIdx.x == 0) {
            int ok = 1;
            const uint32_t base_it = *g.ring_it;
            int issued = 0;
            for (int kb = 0; kb < nkb && ok; ++kb) {
                while (ok && issued < nkb && issued < kb + kGemmStages) {
                    const uint32_t gi = base_it + issued;
                    const int s = gi % kGemmStages;
                    if (gi >= (uint32_t)kGemmStages &&
                        !mbar_wait_bounded(&g.empty[s], ((gi / kGemmStages) - 1) & 1, cx, 1))
                        ok = 0;
                    if (!ok) break;
                    mbar_arrive_expect_tx(&g.full[s], kATileBytes);
                    tma_load_2d(g.a_ring + s * kATileBytes, &L.tmap, &g.full[s], k0 + issued * 64,
                                mt * 128);
                    ++issued;
                }
                if (!ok) break;
                const uint32_t gi = base_it + kb;
                const int s = gi % kGemmStages;
                if (!mbar_wait_bounded(&g.full[s], (gi / kGemmStages) & 1, cx, 2)) { ok = 0; break; }
                tc_fence_after();
                const uint32_t a_addr = smem_u32(g.a_ring + s * kATileBytes);
                const uint32_t b_addr = smem_u32(g.b_tile + kb * kBTileBytes);
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    tc_mma_f16(tmem, sw128_desc(a_addr + 32 * k), sw128_desc(b_addr + 32 * k), idesc,
                               (kb > 0 || k > 0) ? 1u : 0u);
                tc_commit(&g.empty[s]);
            }
            if (ok) tc_commit(g.accb);
            *g.ring_it = base_it + issued;
            s_ok = ok;
        }
        __syncthreads();
        if (!s_ok) return false;
        const uint32_t ai = *g.acc_it;
        if (!mbar_wait_bounded(g.accb, ai & 1, cx, 3)) return false;
        tc_fence_after();
        // epilogue: warp w reads TMEM lanes 32 (w % 4) .. +31 (its 32 output rows)
        // and columns 16 (w / 4) .. +15 (16 of the queries)
        const int sub = warp & 3, half = warp >> 2;
        uint32_t r[16];
        tmem_ld16(tmem + ((uint32_t)(32 * sub) << 16) + 16 * half, r);
        tmem_ld_wait();
        const int m = mt * 128 + 32 * sub + lane;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const int q = 16 * half + j;
            if (q < n && m < L.N) {
                const float v = __uint_as_float(r[j]);
                if (L.C == 1) store_out(direct, q, m, apply_act(v, L.act));
                else __stcg(Pbuf + ((size_t)c * n + q) * L.Npad + m, v);
            }
        }
        tc_fence_before();
        __syncthreads();
        if (threadIdx.x == 0) *g.acc_it = ai + 1;
        __syncthreads();
    }
    return true;
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
