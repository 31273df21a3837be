// GEMM_BF16 / GEMM_FP8 stage body: dense layers on the 5th-generation tensor
// cores, bf16 (kind::f16) or e4m3 (kind::f8f6f4) operands, f32 accumulation.
//
// Each layer computes y[q][m] = act(vscale * sum_k W[m][k] x[q][k]) for a batch
// of at most 32 queries (or of up to 8192 token rows).  The batch is small, so
// the operands are swapped: the weights are the M = 128 operand (128-row x
// 128-byte tiles, stored pre-tiled and pre-swizzled as contiguous 16 KB
// blocks) and the input rows are the N operand (N = 32 for query batches, 128
// for token-level stages; NT-row x 128-byte tiles in the same swizzled form,
// written so by the producer or re-tiled once per layer).  One warp streams
// both operands with 1-D bulk copies through a shared-memory ring; one thread
// in each of two warps issues tcgen05.mma (M=128, N=NT) into its own pair of
// TMEM accumulators; four warps drain finished accumulators.  A unit is
// (row tile, K-chunk, 128-row weight tile); chunk partials are added in chunk
// order, so the result is the same whatever the number of CTAs.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "device_sync.cuh"
#include "stage_params.h"
#include "stages.cuh"
#include "tc_ptx.cuh"

namespace camelot {

constexpr int kKbPerStage = 2;                   // k-blocks per stage: one 32 KB weight copy
constexpr uint32_t kATileBytes = 128 * 128;      // one weight tile: 128 rows x 128 bytes
constexpr uint32_t kRingBytes = 200 * 1024;      // shared memory of the stage ring
constexpr int kMaxGemmStages = kMaxRingSlots;
constexpr int kIssuers = 2;                      // MMA-issuing warps
constexpr uint32_t kTmemCols = 512;              // two accumulators per issuer, up to 128 columns each

// Ring geometry for NT rows per MMA (N = 32 for batches of queries, 128 for
// token-level stages): query tiles of NT rows x 128 bytes; stages of two weight
// and two query tiles (40 KB / 64 KB), as many as fit the ring (5 / 3).
template <int NT>
struct RingGeom {
    static constexpr uint32_t kBTile = NT * 128;
    static constexpr uint32_t kStage = kKbPerStage * (kATileBytes + kBTile);
    static constexpr int kStages = (int)(kRingBytes / kStage) < kMaxGemmStages ? (int)(kRingBytes / kStage)
                                                                                 : kMaxGemmStages;
};

// Warp roles inside a CTA running tensor-core layers.
constexpr int kWarpTma = 0;     // weight and query tiles, bulk copies
constexpr int kWarpEpi0 = 4;    // warps 4..7 read the accumulators
// warps 1 and 3 issue tcgen05.mma (one thread each): issuer 0 takes the
// CTA's even units, issuer 1 the odd ones
__device__ __forceinline__ int issuer_of_warp(int warp) { return warp == 1 ? 0 : (warp == 3 ? 1 : -1); }

struct GemmSmem {
    char* ring;            // stages of 2 weight tiles then 2 query tiles (RingGeom)
    uint64_t* full;        // [stages][kIssuers] both operands landed (1 arrival + tx bytes), one
                           // barrier per slot and issuer: see gemm_layer_tasks
    uint64_t* empty;       // [stages] MMAs reading the stage are done
    uint64_t* tfull;       // [2 * kIssuers] accumulator complete
    uint64_t* tfree;       // [2 * kIssuers] accumulator read out (4 arrivals: epilogue warps)
    uint32_t* tmem_slot;   // TMEM base address written by tcgen05.alloc
    uint32_t* fills;       // [kMaxGemmStages] times each ring slot has been filled (all calls of this CTA)
    uint32_t* acc_it;      // [kIssuers] units finished so far by each issuer
    uint32_t* ipar;        // [kIssuers] bit s: phase parity of the issuer's next wait on slot s (all calls)
    char* stage_out;       // [4 epilogue warps][kEpiStageBytes] staging of tiled output blocks
};
constexpr uint32_t kEpiStageBytes = 32 * 32 * 2;   // one 32-row x 32-column block of bf16
// the barriers and counters of GemmSmem fit the 1024 bytes between the ring and stage_out
static_assert(8 * (kMaxGemmStages * kIssuers + kMaxGemmStages + 4 * kIssuers) +
                  4 * (1 + kMaxGemmStages + 2 * kIssuers) <= 1024,
              "GEMM barrier block");

__device__ __forceinline__ GemmSmem gemm_smem(float* smem) {
    char* base = reinterpret_cast<char*>(
        (reinterpret_cast<uintptr_t>(smem) + 1023) & ~static_cast<uintptr_t>(1023));
    GemmSmem g;
    g.ring = base;
    uint64_t* bars = reinterpret_cast<uint64_t*>(base + kRingBytes);
    g.full = bars;
    g.empty = g.full + kMaxGemmStages * kIssuers;
    g.tfull = g.empty + kMaxGemmStages;
    g.tfree = g.tfull + 2 * kIssuers;
    g.tmem_slot = reinterpret_cast<uint32_t*>(g.tfree + 2 * kIssuers);
    g.fills = g.tmem_slot + 1;
    g.acc_it = g.fills + kMaxGemmStages;
    g.ipar = g.acc_it + kIssuers;
    g.stage_out = base + kRingBytes + 1024;
    return g;
}

// Once per launch by every CTA that runs GEMM_BF16 work: barriers and TMEM.
__device__ __forceinline__ void gemm_setup(float* smem) {
    GemmSmem g = gemm_smem(smem);
    if (threadIdx.x == 0) {
        for (int s = 0; s < kMaxGemmStages; ++s) {
            for (int w = 0; w < kIssuers; ++w) mbar_init(&g.full[s * kIssuers + w], 1);
            mbar_init(&g.empty[s], 1);
        }
        for (int b = 0; b < 2 * kIssuers; ++b) {
            mbar_init(&g.tfull[b], 1);
            mbar_init(&g.tfree[b], 4);
        }
        for (int s = 0; s < kMaxGemmStages; ++s) g.fills[s] = 0;
        for (int w = 0; w < kIssuers; ++w) g.acc_it[w] = 0;
        for (int w = 0; w < kIssuers; ++w) g.ipar[w] = 0;
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

// Output of one layer: bf16 rows, f32 rows (logits) or e4m3 rows.
enum OutFmt : int { OUT_BF16 = 0, OUT_F32 = 1, OUT_E4M3 = 2 };
struct LayerOut {
    RowRef rows;
    int fmt;
    int act;
    float vscale;   // accumulator scale
    float qscale;   // e4m3: the stored code is e4m3(value / qscale)
    int tiled;      // bf16 / e4m3 rows in the tiled layout (the next layer's operand), from rows.base
    size_t rowb;    // bytes per row (tiled)
    int th;         // rows per tile (tiled)
};

__device__ __forceinline__ void store_out(const LayerOut& o, int q, int m, float acc) {
    const float v = apply_act(acc * o.vscale, o.act);
    if (o.fmt == OUT_F32) {
        reinterpret_cast<float*>(o.rows.row(q))[m] = v;
    } else if (o.fmt == OUT_BF16) {
        const __nv_bfloat16 b = __float2bfloat16_rn(v);
        if (o.tiled) *reinterpret_cast<__nv_bfloat16*>(o.rows.base + tiled_offset(q, (size_t)m * 2, o.rowb, o.th)) = b;
        else reinterpret_cast<__nv_bfloat16*>(o.rows.row(q))[m] = b;
    } else {
        const __nv_fp8_storage_t c = __nv_cvt_float_to_fp8(v / o.qscale, __NV_SATFINITE, __NV_E4M3);
        if (o.tiled) *reinterpret_cast<__nv_fp8_storage_t*>(o.rows.base + tiled_offset(q, (size_t)m, o.rowb, o.th)) = c;
        else reinterpret_cast<__nv_fp8_storage_t*>(o.rows.row(q))[m] = c;
    }
}

// Epilogue stores of one 32-row block of an accumulator: this lane holds
// output column m of rows row0 .. row0 + 31 (r0: the first 16, r1: the rest),
// of which the first jn are real.  The branches on the output kind sit
// outside the unrolled row loops, so each path is straight-line code.
__device__ __forceinline__ float epi_val(const uint32_t (&r0)[16], const uint32_t (&r1)[16], int j) {
    return __uint_as_float(j < 16 ? r0[j] : r1[j - 16]);
}

// Chunk partials (f32, row stride ld floats), reduced afterwards.
__device__ __forceinline__ void epi_partials(float* dst, size_t ld, const uint32_t (&r0)[16],
                                             const uint32_t (&r1)[16], int jn) {
#pragma unroll
    for (int j = 0; j < 32; ++j)
        if (j < jn) __stcg(dst + (size_t)j * ld, epi_val(r0, r1, j));
}

// Final values: act(acc * vscale), stored as o describes; called by all 32
// lanes of an epilogue warp (lane l holds column m = m0 + l; columns >= N
// are not stored).  Tiled bf16 outputs (the next layer's operand) pass
// through the warp's staging block in shared memory, so that the global
// stores are whole 16-byte pieces of rows (N is a multiple of 8).
__device__ __forceinline__ void epi_direct(const LayerOut& o, int row0, int m, int N, const uint32_t (&r0)[16],
                                           const uint32_t (&r1)[16], int jn, char* stg) {
    float v[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) v[j] = epi_val(r0, r1, j) * o.vscale;
    if (o.act == ACT_GELU) {
#pragma unroll
        for (int j = 0; j < 32; ++j) v[j] = apply_act(v[j], ACT_GELU);
    } else if (o.act == ACT_RELU) {
#pragma unroll
        for (int j = 0; j < 32; ++j) v[j] = apply_act(v[j], ACT_RELU);
    }
    if (o.fmt == OUT_F32) {
#pragma unroll
        for (int j = 0; j < 32; ++j)
            if (j < jn && m < N) reinterpret_cast<float*>(o.rows.row(row0 + j))[m] = v[j];
    } else if (o.fmt == OUT_BF16) {
        if (o.tiled) {
            const int lane = threadIdx.x & 31, m0 = m - lane;
            __nv_bfloat16* sb = reinterpret_cast<__nv_bfloat16*>(stg);
#pragma unroll
            for (int j = 0; j < 32; ++j) sb[j * 32 + lane] = __float2bfloat16_rn(v[j]);
            __syncwarp();
            // 32 rows x 4 pieces of 16 bytes; lane l takes pieces l, l + 32, ...
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int pc = 32 * i + lane, j = pc >> 2, c = pc & 3;
                if (j < jn && m0 + 8 * c < N)
                    __stcg(reinterpret_cast<uint4*>(o.rows.base + tiled_offset(row0 + j, (size_t)(m0 + 8 * c) * 2,
                                                                               o.rowb, o.th)),
                           *reinterpret_cast<const uint4*>(stg + j * 64 + c * 16));
            }
            __syncwarp();
        } else {
#pragma unroll
            for (int j = 0; j < 32; ++j)
                if (j < jn && m < N) reinterpret_cast<__nv_bfloat16*>(o.rows.row(row0 + j))[m] = __float2bfloat16_rn(v[j]);
        }
    } else {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            if (j < jn && m < N) {
                const __nv_fp8_storage_t c = __nv_cvt_float_to_fp8(v[j] / o.qscale, __NV_SATFINITE, __NV_E4M3);
                if (o.tiled) *reinterpret_cast<__nv_fp8_storage_t*>(o.rows.base + tiled_offset(row0 + j, (size_t)m, o.rowb, o.th)) = c;
                else reinterpret_cast<__nv_fp8_storage_t*>(o.rows.row(row0 + j))[m] = c;
            }
        }
    }
}

// What a stage needs to know about its unit, worked out once per unit.
struct UnitInfo {
    int c, mt, row0;   // K-chunk, weight tile, first input row
    int nkb, ns;       // 128-byte k-blocks in the chunk, ring stages of the unit
};

// The order in which a CTA's ring stages carry its units: units are taken in
// pairs (r, r + 1) relative to the CTA's first unit, and the stages of a pair
// alternate between its two units, so both issuers always have stages in the
// ring.  f(info, r, j, gi) is called for stage j of unit u0 + r at ring
// position gi, in ring order; it returns false to stop.
template <class Info, class F>
__device__ __forceinline__ bool for_each_stage(int u0, int u1, uint32_t ring0, Info info, F&& f) {
    uint32_t gi = ring0;
    for (int r = 0; u0 + r < u1; r += 2) {
        const int ua = u0 + r;
        const bool pair = ua + 1 < u1;
        const UnitInfo a = info(ua);
        const UnitInfo b = pair ? info(ua + 1) : UnitInfo{0, 0, 0, 0, 0};
        const int nmax = a.ns > b.ns ? a.ns : b.ns;
        for (int j = 0; j < nmax; ++j) {
            if (j < a.ns && !f(a, r, j, gi++)) return false;
            if (j < b.ns && !f(b, r + 1, j, gi++)) return false;
        }
    }
    return true;
}

// A layer of exactly two K-chunks whose units pair up inside every CTA: each
// CTA's units start at an even unit and come in an even number, and units are
// then ordered chunk-minor, so that the pair (2i, 2i + 1) is chunks 0 and 1 of
// one weight tile, run by the CTA's two issuers into two accumulators.  The
// epilogue adds the pair itself, (0 + p0) + p1 in f32 as the reduce pass would,
// so the layer writes no partials and needs no reduce pass: the result is the
// same bits as the unpaired path's.
__device__ __forceinline__ bool gemm_pairs_fused(const LayerParams& L, int rows, int nctas, int nt) {
    if (L.C != 2) return false;
    const int U = (L.Npad / 128) * 2 * ((rows + nt - 1) / nt);
    return (U / 2) % nctas == 0;
}

// One layer over `rows` input rows (queries, or tokens of a token-level
// stage), taken 32 at a time.  Work units u = (row tile rt, chunk c, 128-row
// weight tile mt) in that order (u = (rt * C + c) * MT + mt; in a layer whose
// chunk pairs are fused, u = (rt * MT + mt) * 2 + c); CTA r takes the
// contiguous units [r U / p, (r+1) U / p).
// Every unit accumulates the same K range in the same MMA order, issued by
// one thread into one accumulator, whichever CTA or issuer runs it.  Each ring
// stage carries two consecutive weight tiles (one 32 KB bulk copy: the copy
// engine's cost is per operation, so larger copies stream faster; kept in L2
// with the evict-last policy) and the matching two query tiles of xt (one
// 8 KB bulk copy).
// ESZ = bytes per operand element (2: bf16 / kind::f16, 1: e4m3 / kind::f8f6f4),
// a template parameter so that each instantiation's MMA loop holds one kind.
template <int ESZ, int NT>
static __device__ bool gemm_layer_tasks(const StageCtx& cx, const LayerParams& L, const char* xt, int rows,
                                        float* Pbuf, const LayerOut& direct) {
    using G = RingGeom<NT>;
    // ring slots of this layer: all that fit (G::kStages), or fewer when the stage asks for fewer;
    // the full ring (the usual case) keeps a constant divisor
    const uint32_t nslot = (L.ring > 0 && L.ring < G::kStages) ? (uint32_t)L.ring : (uint32_t)G::kStages;
    const bool full_ring = nslot == (uint32_t)G::kStages;
    auto slot_of = [=](uint32_t gi) { return (int)(full_ring ? gi % (uint32_t)G::kStages : gi % nslot); };
    auto round_of = [=](uint32_t gi) { return full_ring ? gi / (uint32_t)G::kStages : gi / nslot; };
    constexpr uint32_t kBTileBytes = G::kBTile;
    constexpr uint32_t kStageBytes = G::kStage;
    constexpr int kGemmN = NT;
    const GemmSmem g = gemm_smem(cx.smem);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int MT = L.Npad / 128;
    const int CM = MT * L.C;                        // units per row tile
    const int U = CM * ((rows + kGemmN - 1) / kGemmN);
    const int u0 = (int)((long long)cx.rank * U / cx.nctas);
    const int u1 = (int)((long long)(cx.rank + 1) * U / cx.nctas);
    // ring positions count from 0 in every call: position gi uses slot gi mod
    // nslot, the fills[slot] + gi / nslot -th fill of that slot, so the barrier
    // phases stay right whatever the tile height (and so the stage size) or the
    // slot count of the calls before
    const uint32_t ring0 = 0;
    uint32_t accb[kIssuers];
#pragma unroll
    for (int w = 0; w < kIssuers; ++w) accb[w] = g.acc_it[w];
    const uint32_t tmem = *g.tmem_slot;
    // k-blocks are 128 bytes wide: 64 bf16 or 128 e4m3 columns
    // layer constants in registers: the lambdas below capture by value, so the
    // asm statements' memory clobbers do not force reloads
    const int K = L.K, KC = L.KC, N = L.N, Npad = L.Npad, C = L.C;
    constexpr int esz = ESZ;
    auto chunk_kb = [=](int c) { return min(KC, K - c * KC) * esz / 128; };
    const size_t kc_bytes = (size_t)KC * esz;
    const bool fused = gemm_pairs_fused(L, rows, cx.nctas, NT);
    auto info = [=](int u) {
        UnitInfo ui;
        const int rt = u / CM, v = u - rt * CM;
        ui.c = fused ? (v & 1) : v / MT;
        ui.mt = fused ? (v >> 1) : v - ui.c * MT;
        ui.row0 = rt * kGemmN;
        ui.nkb = chunk_kb(ui.c);
        ui.ns = (ui.nkb + kKbPerStage - 1) / kKbPerStage;
        return ui;
    };
    // accumulator of the unit that is issuer w's k-th (counting all its
    // earlier units): two per issuer, alternating
    auto acc_of = [](int w, uint32_t k) { return 2 * w + (int)(k & 1u); };
    const int iw = issuer_of_warp(warp);

    if (u0 < u1) {
        if (warp == kWarpTma && lane == 0) {
            // the operands were written by generic stores (other CTAs, other
            // stages) and are read here by the async proxy
            fence_proxy_async_global();
            // tiles (mt, kb) and (mt, kb+1) are adjacent in memory: one bulk copy
            const uint64_t pol = l2_policy_evict_last();
            const char* wt = reinterpret_cast<const char*>(L.w);
            const int KB = K * esz / 128;                // weight tiles per 128-row block
            for_each_stage(u0, u1, ring0, info, [=](UnitInfo ui, int r, int j, uint32_t gi) {
                const int kb = j * kKbPerStage;
                const int nk = min(kKbPerStage, ui.nkb - kb);
                const int s = slot_of(gi);
                const uint32_t use = g.fills[s] + round_of(gi);
                if (use >= 1 && !mbar_wait_bounded(&g.empty[s], (use - 1) & 1, cx, 1))
                    return false;
                const size_t kbg = ui.c * (kc_bytes / 128) + kb;   // first k-block of the stage
                uint64_t* fb = &g.full[s * kIssuers + (r & 1)];      // the issuer that reads it
                mbar_arrive_expect_tx(fb, nk * (kATileBytes + kBTileBytes));
                bulk_load_hint(g.ring + s * kStageBytes, wt + ((size_t)ui.mt * KB + kbg) * kATileBytes,
                               nk * kATileBytes, fb, pol);
                bulk_load_hint(g.ring + s * kStageBytes + kKbPerStage * kATileBytes,
                               xt + ((size_t)(ui.row0 / kGemmN) * KB + kbg) * kBTileBytes, nk * kBTileBytes,
                               fb, pol);
                return true;
            });
        } else if (iw >= 0 && lane == 0) {
            constexpr bool f8 = ESZ == 1;
            constexpr uint32_t idesc = f8 ? idesc_e4m3_f32(128, NT) : idesc_bf16_f32(128, NT);
            uint32_t k = accb[iw];
            // A slot's successive fills can go to different issuers (the
            // stages of a unit pair alternate), and the fill before this one
            // may still be landing when this issuer arrives: on a barrier
            // shared by both issuers the parity wait would then pass one
            // phase early.  Each (slot, issuer) barrier is waited on by one
            // thread only, in fill order, so its phase is never more than one
            // behind the wait, and the wait needs only its parity: bit s of
            // par, flipped at every wait on slot s and kept in shared memory
            // for the next call (a register here, no per-slot array).
            uint32_t par = g.ipar[iw];
            for_each_stage(u0, u1, ring0, info, [=](UnitInfo ui, int r, int j, uint32_t gi) mutable {
                if ((r & 1) != iw) return true;
                const int acc = acc_of(iw, k);
                const int ns = ui.ns;
                if (j == 0 && k >= 2 && !mbar_wait_bounded(&g.tfree[acc], ((k >> 1) - 1) & 1, cx, 4))
                    return false;
                const int kb = j * kKbPerStage;
                const int nk = min(kKbPerStage, ui.nkb - kb);
                const int s = slot_of(gi);
                if (!mbar_wait_bounded(&g.full[s * kIssuers + iw], (par >> s) & 1u, cx, 5)) return false;
                par ^= 1u << s;
                g.ipar[iw] = par;
                tc_fence_after();
                // descriptors of the stage's first A and B slices; a slice 32
                // bytes further along is the start field + 2 (the field is
                // address >> 4 and shared memory stays below 256 KB, so the
                // additions never carry out of it)
                const uint32_t d_tmem = tmem + acc * kGemmN;
                const uint32_t sbase = smem_u32(g.ring + s * kStageBytes);
                const uint64_t da = sw128_desc(sbase);
                const uint64_t db = sw128_desc(sbase + kKbPerStage * kATileBytes);
                auto mma = [&](int t, int kk) {
                    const uint64_t a = da + (t * kATileBytes + 32 * kk) / 16;
                    const uint64_t b = db + (t * kBTileBytes + 32 * kk) / 16;
                    const uint32_t accum = (kb + t > 0 || kk > 0) ? 1u : 0u;
                    if constexpr (f8) tc_mma_f8(d_tmem, a, b, idesc, accum);
                    else tc_mma_f16(d_tmem, a, b, idesc, accum);
                };
                if (nk == kKbPerStage) {
#pragma unroll
                    for (int t = 0; t < kKbPerStage; ++t)
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk) mma(t, kk);
                } else {
                    for (int t = 0; t < nk; ++t)
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk) mma(t, kk);
                }
                tc_commit(&g.empty[s]);
                if (j == ns - 1) {
                    tc_commit(&g.tfull[acc]);
                    ++k;
                }
                return true;
            });
        } else if (warp >= kWarpEpi0) {
            // accumulator rows 32 (warp % 4) .. +31, the NT query columns 32 at
            // a time; units in order, each from its issuer's accumulator
            const int sub = warp & 3;
            uint32_t kw[kIssuers];
#pragma unroll
            for (int w = 0; w < kIssuers; ++w) kw[w] = accb[w];
            // a fused pair: issuer 0's accumulator holds chunk 0, issuer 1's chunk 1
            for (int u = u0; u < u1; u += fused ? 2 : 1) {
                const int w = (u - u0) & 1;
                const uint32_t k = kw[w]++;
                const uint32_t k1 = fused ? kw[1]++ : 0u;
                const UnitInfo ui = info(u);
                const int c = ui.c, mt = ui.mt, row0 = ui.row0;
                const int acc = acc_of(w, k), acc1 = acc_of(1, k1);
                if (!mbar_wait_bounded(&g.tfull[acc], (k >> 1) & 1, cx, 6)) break;
                if (fused && !mbar_wait_bounded(&g.tfull[acc1], (k1 >> 1) & 1, cx, 6)) break;
                tc_fence_after();
                const int m = mt * 128 + 32 * sub + lane;
#pragma unroll 1
                for (int q0 = 0; q0 < NT; q0 += 32) {
                    uint32_t r0[16], r1[16];
                    const uint32_t ta = tmem + ((uint32_t)(32 * sub) << 16) + acc * NT + q0;
                    if (fused) {
                        // (0 + p0) + p1, each addition rounded once, as the reduce pass adds
                        const uint32_t tb = tmem + ((uint32_t)(32 * sub) << 16) + acc1 * NT + q0;
                        uint32_t t[16];
                        tmem_ld16(ta, r0);
                        tmem_ld16(tb, t);
                        tmem_ld_wait();
#pragma unroll
                        for (int i = 0; i < 16; ++i)
                            r0[i] = __float_as_uint(__fadd_rn(__fadd_rn(0.f, __uint_as_float(r0[i])), __uint_as_float(t[i])));
                        tmem_ld16(ta + 16, r1);
                        tmem_ld16(tb + 16, t);
                        tmem_ld_wait();
#pragma unroll
                        for (int i = 0; i < 16; ++i)
                            r1[i] = __float_as_uint(__fadd_rn(__fadd_rn(0.f, __uint_as_float(r1[i])), __uint_as_float(t[i])));
                    } else {
                        tmem_ld16(ta, r0);
                        tmem_ld16(ta + 16, r1);
                        tmem_ld_wait();
                    }
                    if (q0 + 32 >= NT) {           // the accumulator(s) have been read out
                        tc_fence_before();
                        __syncwarp();
                        if (lane == 0) {
                            mbar_arrive(&g.tfree[acc]);
                            if (fused) mbar_arrive(&g.tfree[acc1]);
                        }
                    }
                    const int jn = min(32, rows - (row0 + q0));   // real rows of this block
                    if (jn > 0) {   // (warp-uniform)
                        if (C > 1 && !fused) {
                            if (m < N) epi_partials(Pbuf + ((size_t)c * rows + row0 + q0) * Npad + m, Npad, r0, r1, jn);
                        } else {
                            epi_direct(direct, row0 + q0, m, N, r0, r1, jn, g.stage_out + sub * kEpiStageBytes);
                        }
                    }
                }
            }
        }
    }
    // direct (C == 1 or fused) outputs may be the next layer's bulk-copied operand
    fence_proxy_async_global();
    __syncthreads();
    if (threadIdx.x == 0 && u0 < u1) {
        uint32_t stages = 0;
        for (int u = u0; u < u1; ++u) stages += info(u).ns;
        for (uint32_t sl = 0; sl < nslot; ++sl)
            g.fills[sl] += (stages + (nslot - 1 - sl)) / nslot;
        const uint32_t cnt = (uint32_t)(u1 - u0);
        g.acc_it[0] = accb[0] + (cnt + 1) / 2;
        g.acc_it[1] = accb[1] + cnt / 2;
    }
    __syncthreads();
    return !has_error(cx.ctl);
}

// out[q][m] = act(sum over chunks, in chunk order) for m < N.  Each thread
// owns two groups of four consecutive outputs and keeps 2 x 8 float4 loads in
// flight; the four lanes of a float4 are summed independently, each in chunk
// order, so the result equals the scalar chunk-order sum.
static __device__ void gemm_reduce(const StageCtx& cx, const LayerParams& L, int n, const float* Pbuf,
                                   const LayerOut& o) {
    const int m4n = L.Npad / 4;                   // float4 groups per query row
    const int total = n * m4n;
    const size_t cstride4 = (size_t)n * m4n;      // float4 stride between chunks
    const float4* P4 = reinterpret_cast<const float4*>(Pbuf);
    const int nthreads = cx.nctas * kThreads;
    for (int base = cx.rank * kThreads + threadIdx.x; base < total; base += 2 * nthreads) {
        const int e0 = base, e1 = base + nthreads;
        const bool has1 = e1 < total;
        float4 s0 = make_float4(0.f, 0.f, 0.f, 0.f), s1 = s0;
        for (int c = 0; c < L.C; c += 8) {
            float4 v0[8], v1[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                if (c + u < L.C) {
                    v0[u] = __ldcg(P4 + (size_t)(c + u) * cstride4 + e0);
                    if (has1) v1[u] = __ldcg(P4 + (size_t)(c + u) * cstride4 + e1);
                }
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                if (c + u < L.C) {
                    s0.x += v0[u].x; s0.y += v0[u].y; s0.z += v0[u].z; s0.w += v0[u].w;
                    if (has1) { s1.x += v1[u].x; s1.y += v1[u].y; s1.z += v1[u].z; s1.w += v1[u].w; }
                }
            }
        }
        for (int h = 0; h < 2; ++h) {
            if (h == 1 && !has1) break;
            const int e = h ? e1 : e0;
            const float4 v = h ? s1 : s0;
            const int q = e / m4n, m = (e - q * m4n) * 4;
            const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
                if (m + i < L.N) store_out(o, q, m + i, vv[i]);
        }
    }
    fence_proxy_async_global();   // the outputs may be the next layer's bulk-copied operand
}

// The whole GEMM_BF16 / GEMM_FP8 stage.  Hidden rows and the rows handed to
// the next stage are bf16 (GEMM_BF16) or e4m3 codes (GEMM_FP8); a final stage
// keeps its logits in f32.
// Rewrite `rows` input rows of `rowb` bytes (x) as NT-row x 128-byte tiles:
// tile (rt, kb) at (rt * rowb / 128 + kb) * NT * 128, row r's 16-byte piece j
// at (r % NT) * 128 + (j ^ (r % 8)) * 16, the layout the MMA reads; rows past
// `rows` in the last tile are zero.  All CTAs of the instance share the work;
// the writes are fenced for the bulk copies that read them after the next
// barrier.
template <int NT>
static __device__ void retile_rows(const StageCtx& cx, RowRef x, int rows, size_t rowb, char* xt) {
    // one warp per (row, run of 256 16-byte pieces): 8 coalesced loads in
    // flight per lane, then stores of whole 128-byte tile rows
    const int pieces = (int)(rowb / 16);
    const int KB = (int)(rowb / 128);
    const int runs = (pieces + 255) / 256;
    const int total = (rows + NT - 1) / NT * NT * runs;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int w = cx.rank * kWarps + warp; w < total; w += cx.nctas * kWarps) {
        const int r = w / runs, p0 = (w - r * runs) * 256;
        uint4 v[8];
        const uint4* src = r < rows ? reinterpret_cast<const uint4*>(x.row(r)) : nullptr;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int p = p0 + 32 * i + lane;
            v[i] = (src != nullptr && p < pieces) ? __ldcs(src + p) : make_uint4(0u, 0u, 0u, 0u);
        }
        const int rt = r / NT, rr = r % NT;
        char* trow = xt + (size_t)rt * KB * (NT * 128) + rr * 128;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int p = p0 + 32 * i + lane;
            if (p < pieces)
                *reinterpret_cast<uint4*>(trow + (size_t)(p >> 3) * (NT * 128) + (((p & 7) ^ (rr & 7)) << 4)) = v[i];
        }
    }
    fence_proxy_async_global();
}

// Rows of a token-level stage: the T rows of query q follow each other in its
// query row, so row r of a contiguous batch is at base + r * (stride / T).
__device__ __forceinline__ RowRef token_rows(const RowRef& q, int T) {
    return RowRef{q.base + q.first * q.stride, 0, ~0ull, q.stride / (size_t)T};
}

// Top-k of a final query stage (32-row tiles) whose last layer leaves each of
// its 128-logit weight tiles complete in one CTA (one K-chunk, or fused chunk
// pairs): each CTA reduces its own tiles to k candidates per query right after
// its epilogue (no group barrier between the layer and the top-k), and the
// candidates are merged afterwards: by the pipeline's leader once the other
// CTAs have reported, or after one group barrier in a direct launch.  The
// order is total (value descending, index ascending), so the result is the
// row-wise top-k's.
__device__ __forceinline__ bool gemm_topk_cands(const StageParams& P, int rows, int nctas) {
    const LayerParams& L = P.layer[P.n_layers - 1];
    return P.top_k > 0 && P.rows <= 1 && P.tile_h == 32 && (L.C == 1 || gemm_pairs_fused(L, rows, nctas, 32));
}

// Candidate (value bits, index) of query q, tile mt, rank r.
__device__ __forceinline__ int2* gemm_cand(const StageCtx& cx, const StageParams& P, int q, int mt, int r) {
    const int MT = P.layer[P.n_layers - 1].Npad / 128;
    return reinterpret_cast<int2*>(cx.scratch + P.cand_off) + ((size_t)q * MT + mt) * kMaxTopK + r;
}

// Warp-wide best of four independent (value, index) pairs at once (value
// descending, index ascending on ties): the four shuffle chains interleave.
__device__ __forceinline__ void warp_best4(float (&v)[4], int (&i)[4]) {
#pragma unroll
    for (int off = 16; off; off >>= 1) {
        float ov[4];
        int oi[4];
#pragma unroll
        for (int g = 0; g < 4; ++g) {
            ov[g] = __shfl_xor_sync(0xffffffffu, v[g], off);
            oi[g] = __shfl_xor_sync(0xffffffffu, i[g], off);
        }
#pragma unroll
        for (int g = 0; g < 4; ++g)
            if (ov[g] > v[g] || (ov[g] == v[g] && oi[g] < i[g])) { v[g] = ov[g]; i[g] = oi[g]; }
    }
}

// This CTA's tiles (the tiles of its units, in the unit order of
// gemm_layer_tasks): warp w takes queries w, w + 8, w + 16, w + 24 of a 32-row
// tile together (four logits per lane and query, all loads in flight at once),
// then k rounds of warp-wide best.  The logits rows are copied to the sink on
// the way.
static __device__ void gemm_tile_cands(const StageCtx& cx, const StageParams& P, RowRef z, int n,
                                       const FinalOut& fo) {
    const LayerParams& L = P.layer[P.n_layers - 1];
    const int MT = L.Npad / 128, k = P.top_k;
    const int per = L.C == 1 ? 1 : 2;                     // units per tile
    const int U = MT * per * ((n + 31) / 32);
    const int u0 = (int)((long long)cx.rank * U / cx.nctas);
    const int u1 = (int)((long long)(cx.rank + 1) * U / cx.nctas);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    static_assert(kWarps * 4 == 32, "four queries per warp cover a 32-row tile");
    for (int t = u0 / per; t < u1 / per; ++t) {
        const int rt = t / MT, mt = t - rt * MT;
        float v[4][4];
        int ix[4][4];
#pragma unroll
        for (int g = 0; g < 4; ++g) {
            const int q = rt * 32 + warp + kWarps * g;
            const float* zr = q < n ? reinterpret_cast<const float*>(z.row(q)) : nullptr;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int m = mt * 128 + 32 * j + lane;
                const bool ok = zr != nullptr && m < L.N;
                v[g][j] = ok ? __ldcg(zr + m) : -INFINITY;
                ix[g][j] = ok ? m : 0x7fffffff;
            }
        }
        if (fo.logits.base != nullptr) {
#pragma unroll
            for (int g = 0; g < 4; ++g) {
                const int q = rt * 32 + warp + kWarps * g;
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (q < n && ix[g][j] != 0x7fffffff) reinterpret_cast<float*>(fo.logits.row(q))[ix[g][j]] = v[g][j];
            }
        }
        for (int r = 0; r < k; ++r) {
            float bv[4];
            int bi[4];
#pragma unroll
            for (int g = 0; g < 4; ++g) {
                bv[g] = v[g][0];
                bi[g] = ix[g][0];
#pragma unroll
                for (int j = 1; j < 4; ++j)
                    if (v[g][j] > bv[g] || (v[g][j] == bv[g] && ix[g][j] < bi[g])) { bv[g] = v[g][j]; bi[g] = ix[g][j]; }
            }
            warp_best4(bv, bi);
#pragma unroll
            for (int g = 0; g < 4; ++g) {
                const int q = rt * 32 + warp + kWarps * g;
                if (lane == 0 && q < n) *gemm_cand(cx, P, q, mt, r) = make_int2(__float_as_int(bv[g]), bi[g]);
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (ix[g][j] == bi[g]) { v[g][j] = -INFINITY; ix[g][j] = 0x7fffffff; }
            }
        }
    }
}

// Merge of the candidates into the final top-k of queries first_q + w,
// first_q + w + q_stride, ... (w the warp; `first_q` counts the calling CTA's
// warps), four queries per warp at once.  A lane takes candidates lane and
// lane + 32 of each (at most 64: MT k <= 64) or scans lane, lane + 32, ... (a
// query at a time) for wider layers, in (tile, rank) order, which for equal
// values is index order, into its sorted top kMaxTopK.
__device__ __forceinline__ void cand_insert(float (&bv)[kMaxTopK], int (&bi)[kMaxTopK], float cv, int ci) {
    if (cv > bv[kMaxTopK - 1] || bi[kMaxTopK - 1] == 0x7fffffff) {
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
__device__ __forceinline__ void cand_pop(float (&bv)[kMaxTopK], int (&bi)[kMaxTopK]) {
#pragma unroll
    for (int t = 0; t + 1 < kMaxTopK; ++t) { bv[t] = bv[t + 1]; bi[t] = bi[t + 1]; }
    bv[kMaxTopK - 1] = -INFINITY;
    bi[kMaxTopK - 1] = 0x7fffffff;
}

static __device__ void gemm_cand_merge(const StageCtx& cx, const StageParams& P, int n, const FinalOut& fo,
                                       int first_q, int q_stride) {
    const int MT = P.layer[P.n_layers - 1].Npad / 128, k = P.top_k, NC = MT * k;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (NC <= 64) {
        for (int q0 = first_q + warp; q0 < n; q0 += 4 * q_stride) {
            int2 e[4][2];
#pragma unroll
            for (int g = 0; g < 4; ++g) {
                const int q = q0 + g * q_stride;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int c = lane + 32 * h, mt = c / k;
                    e[g][h] = (q < n && c < NC) ? __ldcg(gemm_cand(cx, P, q, mt, c - mt * k))
                                                : make_int2(__float_as_int(-INFINITY), 0x7fffffff);
                }
            }
            float bv[4][kMaxTopK];
            int bi[4][kMaxTopK];
#pragma unroll
            for (int g = 0; g < 4; ++g) {
#pragma unroll
                for (int r = 0; r < kMaxTopK; ++r) { bv[g][r] = -INFINITY; bi[g][r] = 0x7fffffff; }
#pragma unroll
                for (int h = 0; h < 2; ++h) cand_insert(bv[g], bi[g], __int_as_float(e[g][h].x), e[g][h].y);
            }
            for (int r = 0; r < k; ++r) {
                float v[4];
                int i[4];
#pragma unroll
                for (int g = 0; g < 4; ++g) { v[g] = bv[g][0]; i[g] = bi[g][0]; }
                warp_best4(v, i);
#pragma unroll
                for (int g = 0; g < 4; ++g) {
                    const int q = q0 + g * q_stride;
                    if (lane == 0 && q < n) {
                        fo.idx[(size_t)q * k + r] = i[g];
                        fo.val[(size_t)q * k + r] = v[g];
                    }
                    if (bi[g][0] == i[g]) cand_pop(bv[g], bi[g]);
                }
            }
        }
        return;
    }
    for (int q = first_q + warp; q < n; q += q_stride) {
        float bv[kMaxTopK];
        int bi[kMaxTopK];
#pragma unroll
        for (int r = 0; r < kMaxTopK; ++r) { bv[r] = -INFINITY; bi[r] = 0x7fffffff; }
        for (int c = lane; c < NC; c += 32) {
            const int mt = c / k;
            const int2 e = __ldcg(gemm_cand(cx, P, q, mt, c - mt * k));
            cand_insert(bv, bi, __int_as_float(e.x), e.y);
        }
        for (int r = 0; r < k; ++r) {
            float v = bv[0];
            int i = bi[0];
            warp_best(v, i);
            if (lane == 0) {
                fo.idx[(size_t)q * k + r] = i;
                fo.val[(size_t)q * k + r] = v;
            }
            if (bi[0] == i) cand_pop(bv, bi);
        }
    }
}

template <int NT>
static __device__ bool gemm_body_nt(const StageCtx& cx, const StageParams& P, RowRef in, int n,
                                    RowRef out, const FinalOut& fo) {
    const int T = P.rows;
    const int rows = n * T;
    RowRef x = T > 1 ? token_rows(in, T) : in;
    if (T > 1 && out.base != nullptr && !P.out_tiled) out = token_rows(out, T);
    const int hfmt = P.kind == KIND_GEMM_FP8 ? OUT_E4M3 : OUT_BF16;
    const size_t hsz = P.kind == KIND_GEMM_FP8 ? 1 : 2;
    // the first layer's operand: the input slot itself when the producer wrote
    // it tiled, else a tiled copy
    const char* xt = P.in_tiled ? in.base + in.first * in.stride : nullptr;
    for (int l = 0; l < P.n_layers; ++l) {
        const LayerParams& L = P.layer[l];
        const bool last = (l == P.n_layers - 1);
        LayerOut o;
        if (last && P.top_k == 0) {
            o = LayerOut{out, hfmt, L.act, L.vscale, L.qscale, P.out_tiled, (size_t)L.N * hsz, P.out_tile_h};
        } else if (last) {
            o = LayerOut{RowRef{cx.scratch + L.h_off, 0, ~0ull, (size_t)L.N * sizeof(float)}, OUT_F32, L.act,
                         L.vscale, 0.f, 0, 0, NT};
        } else {   // hidden rows, tiled for the next layer
            o = LayerOut{RowRef{cx.scratch + L.h_off, 0, ~0ull, (size_t)L.N * hsz}, hfmt, L.act, L.vscale,
                         L.qscale, 1, (size_t)L.N * hsz, NT};
        }
        float* Pbuf = reinterpret_cast<float*>(cx.scratch + L.p_off);
        if (xt == nullptr) {
            char* buf = cx.scratch + P.tile_off;
            retile_rows<NT>(cx, x, rows, (size_t)L.K * L.esz, buf);
            if (!group_barrier(cx.gs, cx.nctas, cx.ctl, cx.limit_ns, cx.where)) return false;
            xt = buf;
        }
        const bool ok = L.esz == 1 ? gemm_layer_tasks<1, NT>(cx, L, xt, rows, Pbuf, o)
                                   : gemm_layer_tasks<2, NT>(cx, L, xt, rows, Pbuf, o);
        if (!ok) return false;
        if (last && NT == 32 && gemm_topk_cands(P, rows, cx.nctas)) {
            gemm_tile_cands(cx, P, o.rows, n, fo);
            if (cx.defer_topk) return true;            // the pipeline's leader merges
            if (!group_barrier(cx.gs, cx.nctas, cx.ctl, cx.limit_ns, cx.where)) return false;
            gemm_cand_merge(cx, P, n, fo, cx.rank * kWarps, cx.nctas * kWarps);
            return true;
        }
        if (!group_barrier(cx.gs, cx.nctas, cx.ctl, cx.limit_ns, cx.where)) return false;
        if (L.C > 1 && !gemm_pairs_fused(L, rows, cx.nctas, NT)) {
            gemm_reduce(cx, L, rows, Pbuf, o);
            if (!group_barrier(cx.gs, cx.nctas, cx.ctl, cx.limit_ns, cx.where)) return false;
        }
        if (!last) xt = cx.scratch + L.h_off;   // written (and fenced) before the barriers above
        x = o.rows;
        if (last && P.top_k > 0) {
            if (T > 1) token_argmax(cx, x, n, T, L.N, P.res_k, fo);
            else topk_rows(cx, x, n, L.N, P.top_k, fo);
        }
    }
    return true;
}

// Query-batch stages stream 32-row operand tiles, token-level stages 128-row
// tiles (four times the work per MMA at about the same issue cost).
static __device__ bool gemm_body(const StageCtx& cx, const StageParams& P, RowRef in, int n,
                                 RowRef out, const FinalOut& fo) {
    return P.tile_h == 128 ? gemm_body_nt<128>(cx, P, in, n, out, fo) : gemm_body_nt<32>(cx, P, in, n, out, fo);
}

}  // namespace camelot
