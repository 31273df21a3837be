// Host runtime of libcamelot: stage preparation, pipeline rings and lifecycle,
// submission, completion polling, trace replay and the host-staged relay.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <time.h>
#include <immintrin.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <chrono>
#include <thread>
#include <vector>

#include "../../include/camelot.h"
#include "pipeline_params.h"

namespace camelot {
cudaError_t launch_pipeline_kernel(const PipeParams* dparams, int grid, cudaStream_t stream, uint32_t kinds);
cudaError_t launch_stage_direct(const StageParams* dsp, int kind, RowRef in, int n, RowRef out, int32_t* idx,
                                float* val, RowRef logits, char* scratch, GroupSync* gs, Ctl* ctl,
                                long long limit_ns, int grid, cudaStream_t stream);
cudaError_t configure_kernels();
cudaError_t max_coresident_ctas(int* per_sm);
}  // namespace camelot

using namespace camelot;

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
static thread_local std::string g_err;

static camelot_status fail(camelot_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

#define CUDA_TRY(expr)                                                                      \
    do {                                                                                    \
        cudaError_t e_ = (expr);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return fail(e_ == cudaErrorMemoryAllocation ? CAMELOT_ENOMEM : CAMELOT_ECUDA,   \
                        "%s failed: %s", #expr, cudaGetErrorString(e_));                   \
    } while (0)

extern "C" const char* camelot_last_error(void) { return g_err.c_str(); }
void camelot_internal_set_error(const char* msg) { g_err = msg; }
extern "C" int camelot_version(void) { return 200; }

static int64_t host_now_ns() {
    timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return (int64_t)ts.tv_sec * 1000000000ll + ts.tv_nsec;
}

static size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

static int sm_count() {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n;
}

static camelot_status ensure_configured() {
    static std::once_flag once;
    static cudaError_t err = cudaSuccess;
    std::call_once(once, [] { err = configure_kernels(); });
    if (err != cudaSuccess) return fail(CAMELOT_ECUDA, "kernel configuration failed: %s",
                                        cudaGetErrorString(err));
    return CAMELOT_OK;
}

// ---------------------------------------------------------------------------
// stages
// ---------------------------------------------------------------------------
struct camelot_stage {
    camelot_stage_desc desc;
    float wscale[kMaxLayers] = {1.f, 1.f, 1.f, 1.f};   // tensor-core layers: weight scale s_w
    StageParams sp;            // host copy (device pointers inside)
    StageParams* d_sp = nullptr;
    std::vector<void*> allocs; // device buffers owned by the stage
    int device = 0;
};

camelot_status camelot_internal_quantize_e4m3(const float* w, int N, int K, int Npad, void** out, float* scale);

static void stage_free(camelot_stage* st) {
    for (void* p : st->allocs) cudaFree(p);
    if (st->d_sp) cudaFree(st->d_sp);
    delete st;
}

// K-chunk of a tensor-core layer with MT 128-row weight tiles.  With 8 or more
// row tiles and K >= 512, two chunks: 2 MT units per row tile of queries,
// which pair up inside each CTA when the instance's CTA count divides MT times
// the row tiles (chunks 0 and 1 of a weight tile on the CTA's two issuers,
// added in its epilogue), so the layer writes no partials and runs no reduce
// pass (37632 -> 1024 at batch 32 on 8 SMs: saves
// the ~10 us reduce pass of a ~144 us batch); one chunk would leave one issuer
// of each CTA idle and run a single accumulator chain (1024 -> 1024 and
// 1024 -> 1000 at batch 32 on 8 SMs: ~2 us less per layer of ~8-10 us).  Fewer row tiles: the whole
// K up to 1024 columns (one chunk: no partial sums and no reduce pass), above
// that as few equal chunks as give about 64 units, at most one per 1024 columns.
// Chunks are rounded up to 128 columns (whole 128-byte k-blocks for bf16 and
// e4m3 alike).
static int choose_kc_gemm(int K, int MT) {
    if (MT >= 8 && K >= 512) return ((K + 1) / 2 + 127) / 128 * 128;
    if (K <= 1024) return K;
    const int C = std::max(1, std::min((K + 1023) / 1024, (64 + MT - 1) / MT));
    return ((K + C - 1) / C + 127) / 128 * 128;
}

// K-chunk of a task layer: about 128 chunks over K, a multiple of 4 in [32, kMaxKC].
static int choose_kc(int K) {
    int kc = (K + 127) / 128;
    kc = (kc + 3) / 4 * 4;
    kc = std::max(32, std::min(kMaxKC, kc));
    return std::min(kc, K);
}

// Scratch layout of one instance for batches of up to B rows.
static size_t layout_scratch(StageParams& sp, int B) {
    size_t p_bytes = 0, h_bytes = 0, t_bytes = 0;
    for (int l = 0; l < sp.n_layers; ++l) {
        LayerParams& L = sp.layer[l];
        if (is_tensor_kind(sp.kind)) {
            const size_t rows = (size_t)B * std::max(1, sp.rows);
            const size_t th = (size_t)sp.tile_h;
            const size_t rows_pad = (rows + th - 1) / th * th;   // hidden rows are kept tiled
            if (L.C > 1) p_bytes = std::max(p_bytes, (size_t)L.C * rows * L.Npad * sizeof(float));
            h_bytes = std::max(h_bytes, rows_pad * L.Npad * sizeof(float));
            t_bytes = std::max(t_bytes, rows_pad * (size_t)L.K * L.esz);
            continue;
        }
        const size_t G = (L.C + kWarps - 1) / kWarps;    // chunk groups
        if (!L.head) p_bytes = std::max(p_bytes, G * B * L.Npad * sizeof(float));
        h_bytes = std::max(h_bytes, (size_t)B * L.N * sizeof(float));
    }
    size_t off = 0;
    const size_t p_off = off;
    off = align_up(off + p_bytes, 256);
    const size_t h0 = off;
    off = align_up(off + h_bytes, 256);
    const size_t h1 = off;
    off = align_up(off + h_bytes, 256);
    for (int l = 0; l < sp.n_layers; ++l) {
        sp.layer[l].p_off = p_off;
        sp.layer[l].h_off = (l % 2 == 0) ? h0 : h1;
    }
    sp.res_off = off;
    off = align_up(off + (size_t)B * kMaxTopK * 8, 256);
    sp.tile_off = off;
    off = align_up(off + t_bytes, 256);
    sp.cand_off = off;
    if (is_tensor_kind(sp.kind) && sp.top_k > 0 && sp.n_layers > 0)
        off = align_up(off + (size_t)B * (sp.layer[sp.n_layers - 1].Npad / 128) * kMaxTopK * 8, 256);
    return off;
}

extern "C" camelot_status camelot_stage_prepare(const camelot_stage_desc* d, camelot_stage** out) {
    if (!d || !out) return fail(CAMELOT_EINVAL, "null argument");
    *out = nullptr;
    if (d->max_batch < 1 || d->max_batch > 256)
        return fail(CAMELOT_EINVAL, "max_batch %d outside 1..256", d->max_batch);
    if (d->top_k < 0 || d->top_k > kMaxTopK)
        return fail(CAMELOT_EINVAL, "top_k %d outside 0..%d", d->top_k, kMaxTopK);
    const bool tc_kind = d->kind == CAMELOT_STAGE_GEMM_BF16 || d->kind == CAMELOT_STAGE_GEMM_FP8;
    if (d->ring_slots != 0 && (!tc_kind || d->ring_slots < 2 || d->ring_slots > kMaxRingSlots))
        return fail(CAMELOT_EINVAL, "ring_slots %d: 0, or 2..%d for tensor-core kinds", d->ring_slots,
                    kMaxRingSlots);
    camelot_status cs = ensure_configured();
    if (cs != CAMELOT_OK) return cs;
    StageParams sp{};
    sp.kind = d->kind;
    sp.top_k = d->top_k;
    sp.max_batch = d->max_batch;
    sp.rows = 1;
    sp.tile_h = 32;
    sp.out_tile_h = 32;
    sp.res_k = d->top_k;
    auto* st = new camelot_stage();
    st->desc = *d;
    cudaGetDevice(&st->device);
    auto bail = [&](camelot_status s) { stage_free(st); return s; };

    switch (d->kind) {
        case CAMELOT_STAGE_NORMALIZE_U8:
        case CAMELOT_STAGE_NORMALIZE_U8_E4M3:
        case CAMELOT_STAGE_NORM_POOL2_BF16: {
            const int H = d->dims[0], W = d->dims[1], C = d->dims[2];
            if (H <= 0 || W <= 0 || C <= 0) return bail(fail(CAMELOT_EINVAL, "image dims must be > 0"));
            if (d->top_k != 0) return bail(fail(CAMELOT_EINVAL, "image stages cannot be final"));
            sp.H = H; sp.W = W; sp.C = C;
            sp.in_row_bytes = (size_t)H * W * C;
            if (d->kind == CAMELOT_STAGE_NORMALIZE_U8 || d->kind == CAMELOT_STAGE_NORMALIZE_U8_E4M3) {
                if (sp.in_row_bytes % 16)
                    return bail(fail(CAMELOT_EINVAL, "H*W*C must be a multiple of 16"));
                sp.out_row_bytes = sp.in_row_bytes * (d->kind == CAMELOT_STAGE_NORMALIZE_U8 ? 4 : 1);
            } else {
                if (H % 2 || W % 2) return bail(fail(CAMELOT_EINVAL, "H and W must be even"));
                if ((2 * W * C) % 16 || 2 * W * C > 8192)
                    return bail(fail(CAMELOT_EINVAL, "2*W*C must be a multiple of 16 and <= 8192"));
                sp.out_row_bytes = (size_t)(H / 2) * (W / 2) * C * 2;
            }
            sp.scratch_bytes = 0;
            break;
        }
        case CAMELOT_STAGE_MLP_FP32: {
            const int L = d->n_layers;
            if (L < 1 || L > kMaxLayers) return bail(fail(CAMELOT_EINVAL, "n_layers %d outside 1..4", L));
            for (int l = 0; l <= L; ++l)
                if (d->dims[l] <= 0) return bail(fail(CAMELOT_EINVAL, "dims[%d] must be > 0", l));
            for (int l = 0; l < L; ++l) {
                if (d->dims[l] % 4) return bail(fail(CAMELOT_EINVAL, "layer input width dims[%d]=%d must be a multiple of 4", l, d->dims[l]));
                if (!d->weights[l]) return bail(fail(CAMELOT_EINVAL, "weights[%d] is null", l));
                if (d->act[l] < 0 || d->act[l] > 2) return bail(fail(CAMELOT_EINVAL, "act[%d] invalid", l));
            }
            if (d->top_k > d->dims[L]) return bail(fail(CAMELOT_EINVAL, "top_k exceeds the final width"));
            sp.n_layers = L;
            sp.in_row_bytes = (size_t)d->dims[0] * 4;
            sp.out_row_bytes = d->top_k ? 0 : (size_t)d->dims[L] * 4;
            if (!d->top_k && d->dims[L] % 4)
                return bail(fail(CAMELOT_EINVAL, "an intermediate stage's output width must be a multiple of 4"));
            sp.out_width = d->dims[L];
            for (int l = 0; l < L; ++l) {
                LayerParams& Lp = sp.layer[l];
                const int K = d->dims[l], N = d->dims[l + 1];
                Lp.K = K; Lp.N = N; Lp.act = d->act[l];
                Lp.head = (l == L - 1 && d->top_k > 0 && N <= 32) ? 1 : 0;
                std::vector<float> w((size_t)N * K);
                if (cudaMemcpy(w.data(), d->weights[l], w.size() * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
                    return bail(fail(CAMELOT_EINVAL, "weights[%d] is not readable device memory", l));
                std::vector<float> packed;
                if (Lp.head) {
                    Lp.Npad = N; Lp.KC = K; Lp.C = 1;
                    packed = std::move(w);
                } else {
                    Lp.Npad = (N + kNBlock - 1) / kNBlock * kNBlock;
                    Lp.KC = choose_kc(K);
                    Lp.C = (K + Lp.KC - 1) / Lp.KC;
                    // block-major [Npad/64][K/4][64][4]: a task's chunk of a
                    // 64-neuron block is one contiguous run (one bulk copy)
                    const size_t KQ = (size_t)K / 4;
                    packed.assign(KQ * Lp.Npad * 4, 0.f);
                    for (int n = 0; n < N; ++n)
                        for (size_t kq = 0; kq < KQ; ++kq)
                            for (int j = 0; j < 4; ++j)
                                packed[(((size_t)(n / 64) * KQ + kq) * 64 + n % 64) * 4 + j] =
                                    w[(size_t)n * K + 4 * kq + j];
                }
                void* dp = nullptr;
                if (cudaMalloc(&dp, packed.size() * 4) != cudaSuccess)
                    return bail(fail(CAMELOT_ENOMEM, "weight copy allocation failed"));
                st->allocs.push_back(dp);
                if (cudaMemcpy(dp, packed.data(), packed.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess)
                    return bail(fail(CAMELOT_ECUDA, "weight upload failed"));
                Lp.w = (const float*)dp;
            }
            sp.scratch_bytes = layout_scratch(sp, d->max_batch);
            break;
        }
        case CAMELOT_STAGE_GEMM_BF16:
        case CAMELOT_STAGE_GEMM_FP8: {
            const bool f8 = d->kind == CAMELOT_STAGE_GEMM_FP8;
            const int esz = f8 ? 1 : 2;
            const int L = d->n_layers;
            const int T = std::max(1, d->rows_per_query);
            if (T > 1 && d->top_k > 1)
                return bail(fail(CAMELOT_EINVAL, "a token-level final stage emits argmax tags: top_k must be 1"));
            if ((size_t)T * d->max_batch > 8192)
                return bail(fail(CAMELOT_EINVAL, "rows_per_query x max_batch exceeds 8192 rows"));
            sp.rows = T;
            sp.tile_h = T > 1 ? 128 : 32;
            sp.res_k = T > 1 && d->top_k ? std::min(T, kMaxTopK) : d->top_k;
            if (L < 1 || L > kMaxLayers) return bail(fail(CAMELOT_EINVAL, "n_layers %d outside 1..4", L));
            if (d->max_batch > 32) return bail(fail(CAMELOT_EINVAL, "tensor-core stages take batches of at most 32"));
            for (int l = 0; l <= L; ++l)
                if (d->dims[l] <= 0) return bail(fail(CAMELOT_EINVAL, "dims[%d] must be > 0", l));
            if (f8)
                for (int l = 0; l <= (d->top_k ? L - 1 : L); ++l)
                    if (!(d->scales[l] > 0.f) || !std::isfinite(d->scales[l]))
                        return bail(fail(CAMELOT_EINVAL, "scales[%d] must be finite and > 0", l));
            for (int l = 0; l < L; ++l) {
                if ((d->dims[l] * esz) % 128)
                    return bail(fail(CAMELOT_EINVAL, "layer input width dims[%d]=%d must be a multiple of %d", l,
                                     d->dims[l], 128 / esz));
                if (!d->weights[l]) return bail(fail(CAMELOT_EINVAL, "weights[%d] is null", l));
                if (d->act[l] < 0 || d->act[l] > 2) return bail(fail(CAMELOT_EINVAL, "act[%d] invalid", l));
            }
            if (d->top_k > d->dims[L]) return bail(fail(CAMELOT_EINVAL, "top_k exceeds the final width"));
            if (!d->top_k && d->dims[L] % 8)
                return bail(fail(CAMELOT_EINVAL, "an intermediate stage's output width must be a multiple of 8"));
            sp.n_layers = L;
            sp.in_row_bytes = (size_t)T * d->dims[0] * esz;
            sp.out_row_bytes = d->top_k ? 0 : (size_t)T * d->dims[L] * esz;
            sp.out_width = T > 1 ? T : d->dims[L];   // token-level: the sink row holds T tags
            for (int l = 0; l < L; ++l) {
                LayerParams& Lp = sp.layer[l];
                const int K = d->dims[l], N = d->dims[l + 1];
                Lp.K = K; Lp.N = N; Lp.act = d->act[l]; Lp.head = 0;
                Lp.Npad = (N + 127) / 128 * 128;
                // token-level stages have row tiles enough to fill the SMs: no split-K
                Lp.KC = T > 1 ? K : choose_kc_gemm(K, Lp.Npad / 128);
                Lp.C = (K + Lp.KC - 1) / Lp.KC;
                Lp.esz = esz;
                Lp.ring = d->ring_slots;
                Lp.vscale = 1.f;
                Lp.qscale = 0.f;
                if (f8) {
                    void* q = nullptr;
                    float sw = 0.f;
                    const camelot_status qs = camelot_internal_quantize_e4m3((const float*)d->weights[l], N, K,
                                                                             Lp.Npad, &q, &sw);
                    if (qs != CAMELOT_OK) return bail(qs);
                    st->allocs.push_back(q);
                    st->wscale[l] = sw;
                    Lp.w = (const float*)q;
                    Lp.vscale = sw * d->scales[l];
                    const bool out_codes = l < L - 1 || d->top_k == 0;
                    Lp.qscale = out_codes ? d->scales[l + 1] : 0.f;
                    continue;
                }
                std::vector<uint16_t> w((size_t)N * K);
                if (cudaMemcpy(w.data(), d->weights[l], w.size() * 2, cudaMemcpyDeviceToHost) != cudaSuccess)
                    return bail(fail(CAMELOT_EINVAL, "weights[%d] is not readable device memory", l));
                // tile (mt, kb): 128 rows x 64 columns, 16-byte piece j of row r at
                // r * 128 + ((j ^ (r & 7)) * 16) -- the 128-byte-swizzle layout
                const int KB = K / 64;
                std::vector<uint16_t> t((size_t)Lp.Npad * K, 0);
                for (int mt = 0; mt < Lp.Npad / 128; ++mt)
                    for (int kb = 0; kb < KB; ++kb) {
                        uint16_t* tile = t.data() + ((size_t)mt * KB + kb) * (128 * 64);
                        for (int r = 0; r < 128; ++r) {
                            const int row = mt * 128 + r;
                            if (row >= N) continue;
                            for (int j = 0; j < 8; ++j)
                                memcpy(tile + r * 64 + ((j ^ (r & 7)) * 8),
                                       w.data() + (size_t)row * K + kb * 64 + 8 * j, 16);
                        }
                    }
                void* dp = nullptr;
                if (cudaMalloc(&dp, t.size() * 2) != cudaSuccess)
                    return bail(fail(CAMELOT_ENOMEM, "weight copy allocation failed"));
                st->allocs.push_back(dp);
                if (cudaMemcpy(dp, t.data(), t.size() * 2, cudaMemcpyHostToDevice) != cudaSuccess)
                    return bail(fail(CAMELOT_ECUDA, "weight upload failed"));
                Lp.w = (const float*)dp;
            }
            sp.scratch_bytes = layout_scratch(sp, d->max_batch);
            break;
        }
        case CAMELOT_STAGE_COMPUTE_SYNTH:
        case CAMELOT_STAGE_STREAM_SYNTH: {
            const bool stream = d->kind == CAMELOT_STAGE_STREAM_SYNTH;
            const int W = d->dims[0];
            if (W <= 0 || W % 4) return bail(fail(CAMELOT_EINVAL, "dims[0] (row width W) must be a positive multiple of 4"));
            if (d->top_k > W) return bail(fail(CAMELOT_EINVAL, "top_k exceeds the row width"));
            sp.W = W;
            sp.in_row_bytes = (size_t)W * 4;
            sp.out_row_bytes = d->top_k ? 0 : (size_t)W * 4;
            sp.out_width = W;
            if (!stream) {
                if (d->dims[1] < 0) return bail(fail(CAMELOT_EINVAL, "dims[1] (FMA steps) must be >= 0"));
                sp.H = d->dims[1];
            } else {
                const int R = d->dims[1], L = d->dims[2];
                if (R <= 0 || L <= 0 || R % W || L % W || R > L)
                    return bail(fail(CAMELOT_EINVAL, "STREAM_SYNTH dims {W, R, L}: R, L positive multiples of W, R <= L"));
                if (!d->weights[0] || (reinterpret_cast<uintptr_t>(d->weights[0]) & 15))
                    return bail(fail(CAMELOT_EINVAL, "weights[0] (the table) must be a 16-byte aligned pointer"));
                cudaPointerAttributes a{};
                if (cudaPointerGetAttributes(&a, d->weights[0]) != cudaSuccess) {
                    cudaGetLastError();
                    return bail(fail(CAMELOT_EINVAL, "weights[0] is not device or mapped pinned host memory"));
                }
                const void* dp = nullptr;
                if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) dp = d->weights[0];
                else if (a.type == cudaMemoryTypeHost && a.devicePointer) dp = a.devicePointer;
                if (!dp) return bail(fail(CAMELOT_EINVAL, "weights[0] is not device or mapped pinned host memory"));
                sp.H = R / W;
                sp.C = L / W - R / W + 1;
                sp.layer[0].w = (const float*)dp;
                sp.layer[0].act = a.type == cudaMemoryTypeHost ? 1 : 0;   // table in pinned host memory
            }
            // scratch: a final stage's output rows, then the result arrays
            size_t off = 0;
            sp.layer[0].h_off = 0;
            if (d->top_k) off = align_up((size_t)d->max_batch * W * 4, 256);
            sp.res_off = off;
            off = align_up(off + (size_t)d->max_batch * kMaxTopK * 8, 256);
            sp.tile_off = off;
            sp.scratch_bytes = off;
            break;
        }
        case CAMELOT_STAGE_EMBED_GATHER: {
            const int V = d->dims[0], D = d->dims[1], T = d->dims[2];
            if (V <= 0 || D <= 0 || T <= 0 || D % 8)
                return bail(fail(CAMELOT_EINVAL, "EMBED_GATHER dims {V, D, T}: positive, D a multiple of 8"));
            if (d->top_k != 0) return bail(fail(CAMELOT_EINVAL, "an embedding stage cannot be final"));
            if (!d->weights[0]) return bail(fail(CAMELOT_EINVAL, "weights[0] (the table) is null"));
            sp.H = V; sp.W = D; sp.rows = T;
            sp.in_row_bytes = (size_t)T * 4;
            sp.out_row_bytes = (size_t)T * D * 2;
            void* tab = nullptr;
            if (cudaMalloc(&tab, (size_t)V * D * 2) != cudaSuccess)
                return bail(fail(CAMELOT_ENOMEM, "table copy allocation failed"));
            st->allocs.push_back(tab);
            if (cudaMemcpy(tab, d->weights[0], (size_t)V * D * 2, cudaMemcpyDeviceToDevice) != cudaSuccess)
                return bail(fail(CAMELOT_EINVAL, "weights[0] is not readable device memory"));
            sp.layer[0].w = (const float*)tab;
            sp.scratch_bytes = 0;
            break;
        }
        default:
            return bail(fail(CAMELOT_EINVAL, "unknown stage kind %d", d->kind));
    }
    st->sp = sp;
    if (cudaMalloc(&st->d_sp, sizeof(StageParams)) != cudaSuccess)
        return bail(fail(CAMELOT_ENOMEM, "allocation failed"));
    if (cudaMemcpy(st->d_sp, &st->sp, sizeof(StageParams), cudaMemcpyHostToDevice) != cudaSuccess)
        return bail(fail(CAMELOT_ECUDA, "upload failed"));
    *out = st;
    return CAMELOT_OK;
}

extern "C" camelot_status camelot_stage_release(camelot_stage* st) {
    if (!st) return fail(CAMELOT_EINVAL, "null stage");
    stage_free(st);
    return CAMELOT_OK;
}

static const size_t kDirectHeader = align_up(sizeof(Ctl), 256) + align_up(sizeof(GroupSync), 256);

// Internal helpers shared with noalloc.cu (not part of the C ABI).
const StageParams* camelot_internal_stage_params(const camelot_stage* st) { return &st->sp; }
size_t camelot_internal_layout_scratch(StageParams& sp, int B) {
    return (sp.kind == KIND_MLP_FP32 || is_tensor_kind(sp.kind)) ? layout_scratch(sp, B) : sp.scratch_bytes;
}
int camelot_internal_sm_count() { return sm_count(); }
camelot_status camelot_internal_fail(camelot_status st, const char* msg) { return fail(st, "%s", msg); }
size_t camelot_internal_query_bytes(const camelot_pipeline* p);

extern "C" camelot_status camelot_stage_info(const camelot_stage* st, size_t* in_row,
                                             size_t* out_row, uint32_t n, size_t* scratch) {
    if (!st) return fail(CAMELOT_EINVAL, "null stage");
    if (in_row) *in_row = st->sp.in_row_bytes;
    if (out_row) *out_row = st->sp.out_row_bytes;
    if (scratch) *scratch = kDirectHeader + st->sp.scratch_bytes;   // laid out for max_batch
    (void)n;
    return CAMELOT_OK;
}


extern "C" camelot_status camelot_stage_export_weights(const camelot_stage* st, int layer, void* out,
                                                       size_t bytes, float* weight_scale) {
    if (!st || !out) return fail(CAMELOT_EINVAL, "null argument");
    if (!is_tensor_kind(st->sp.kind)) return fail(CAMELOT_EINVAL, "not a tensor-core stage");
    if (layer < 0 || layer >= st->sp.n_layers) return fail(CAMELOT_EINVAL, "layer %d outside 0..%d", layer,
                                                           st->sp.n_layers - 1);
    const LayerParams& L = st->sp.layer[layer];
    const size_t rowb = (size_t)L.K * L.esz;
    if (bytes != (size_t)L.N * rowb)
        return fail(CAMELOT_EINVAL, "%zu bytes given, %zu needed", bytes, (size_t)L.N * rowb);
    std::vector<unsigned char> t((size_t)L.Npad * rowb);
    if (cudaMemcpy(t.data(), L.w, t.size(), cudaMemcpyDeviceToHost) != cudaSuccess)
        return fail(CAMELOT_ECUDA, "weight read-back failed");
    // undo the tiling: tile (mt, kb) holds rows 128 mt.. and bytes 128 kb.. of
    // each row, row r's 16-byte piece j at r * 128 + (j ^ (r % 8)) * 16
    const size_t KB = rowb / 128;
    unsigned char* o = (unsigned char*)out;
    for (int row = 0; row < L.N; ++row) {
        const int mt = row / 128, r = row % 128;
        for (size_t kb = 0; kb < KB; ++kb) {
            const unsigned char* tile = t.data() + ((size_t)mt * KB + kb) * 16384;
            for (int j = 0; j < 8; ++j)
                memcpy(o + (size_t)row * rowb + kb * 128 + 16 * j, tile + r * 128 + ((j ^ (r & 7)) * 16), 16);
        }
    }
    if (weight_scale) *weight_scale = st->wscale[layer];
    return CAMELOT_OK;
}

extern "C" camelot_status camelot_stage_launch(const camelot_stage* st, int n_ctas, const void* in,
                                               uint32_t n, void* out, int32_t* out_idx,
                                               float* out_val, float* out_logits, void* scratch,
                                               size_t scratch_bytes, void* stream) {
    if (!st) return fail(CAMELOT_EINVAL, "null stage");
    const StageParams& sp = st->sp;
    if (n == 0 || (int)n > sp.max_batch)
        return fail(CAMELOT_EINVAL, "n=%u outside 1..max_batch=%d", n, sp.max_batch);
    if (n_ctas < 1 || n_ctas > sm_count())
        return fail(CAMELOT_EINVAL, "n_ctas=%d outside 1..%d", n_ctas, sm_count());
    if (!in) return fail(CAMELOT_EINVAL, "null input");
    if (sp.top_k == 0 && !out) return fail(CAMELOT_EINVAL, "intermediate stage needs `out`");
    if (sp.top_k > 0 && (!out_idx || !out_val)) return fail(CAMELOT_EINVAL, "final stage needs out_idx and out_val");
    size_t need = 0;
    camelot_stage_info(st, nullptr, nullptr, n, &need);
    if (!scratch || scratch_bytes < need)
        return fail(CAMELOT_EINVAL, "scratch of %zu bytes needed, %zu given", need, scratch_bytes);
    if (((uintptr_t)scratch) % 256) return fail(CAMELOT_EINVAL, "scratch must be 256-byte aligned");
    cudaStream_t s = (cudaStream_t)stream;
    char* base = (char*)scratch;
    Ctl* ctl = (Ctl*)base;
    GroupSync* gs = (GroupSync*)(base + align_up(sizeof(Ctl), 256));
    CUDA_TRY(cudaMemsetAsync(base, 0, kDirectHeader, s));
    RowRef rin{(char*)in, 0, ~0ull, sp.in_row_bytes};
    RowRef rout{(char*)out, 0, ~0ull, sp.out_row_bytes};
    RowRef rlog{(char*)out_logits, 0, ~0ull, sp.out_width * sizeof(float)};
    CUDA_TRY(launch_stage_direct(st->d_sp, sp.kind, rin, (int)n, rout, out_idx, out_val, rlog,
                                 base + kDirectHeader, gs, ctl, 2000000000ll, n_ctas, s));
    return CAMELOT_OK;
}

// ---------------------------------------------------------------------------
// pipelines
// ---------------------------------------------------------------------------
extern "C" void camelot_options_default(camelot_options* o) {
    if (!o) return;
    o->query_slots = 65536;
    o->batch_slots = 8;
    o->max_wait_ns = 200000;
    o->idle_exit_ns = 500000000;
    o->wait_limit_ns = 2000000000;
    o->logits_sink = nullptr;
    o->exit_after_trace = 0;
    o->data_slots = 0;
    o->device_data = 0;
    o->qos_ns = 0;
    o->qos_margin_ns = 0;
    for (int b = 0; b < 32; ++b) o->batch_latency_ns[b] = 0;
}

struct HostRing {   // one batch ring's allocations
    unsigned long long* seq = nullptr;
    BatchHdr* hdr = nullptr;
    char* data = nullptr;
    unsigned long long* cursors = nullptr;   // [head line, tail line]
    unsigned int slots = 0;
    size_t slot_bytes = 0;
    // host-staged
    unsigned long long* note_pub = nullptr;
    unsigned int* note_n = nullptr;
    unsigned long long* note_free = nullptr;
};

struct camelot_pipeline {
    int device = 0;
    int n_stages = 0;
    camelot_stage* stages[kMaxStages] = {};
    camelot_alloc alloc{};
    camelot_handoff mode = CAMELOT_HANDOFF_GLOBAL;
    camelot_options opt{};
    int grid = 0;
    uint32_t kinds = 0;                // bit k: some stage is of kind k
    bool tiled[kMaxStages] = {};       // boundary s carries tiled rows
    PipeParams hp{};
    PipeParams* dp = nullptr;
    Ctl* ctl = nullptr;
    HostFlags* hflags = nullptr;       // pinned
    unsigned long long* hstatus = nullptr;  // pinned (inside hflags' page)
    GroupSync* groups = nullptr;
    char* scratch = nullptr;
    HostRing out_rings[kMaxStages], in_rings[kMaxStages];
    unsigned ring_slots[kMaxStages] = {};
    QDesc* qring = nullptr;            // pinned
    char* qdata = nullptr;             // pinned (device_data = 0) or device memory
    cudaStream_t h2d = nullptr;        // device_data: submit's copies
    CompSlot* comp = nullptr;          // pinned
    QMeta* meta = nullptr;             // device
    TraceDev* trace = nullptr;         // device
    cudaStream_t kstream = nullptr, side = nullptr;
    cudaEvent_t kdone = nullptr, kstart = nullptr;
    bool launched = false;
    bool timed = false;          // the last launch's duration has been added
    double last_launch_ms = 0.0, total_launch_ms = 0.0;
    std::mutex launch_mu;
    std::atomic<uint64_t> next_ticket{0};
    std::atomic<uint64_t> next_poll{0};
    uint64_t launches = 0;
    bool trace_active = false;
    uint64_t trace_end = 0;
    uint64_t data_floor = 0;      // first ticket whose data row is tracked by its descriptor
    std::atomic<bool> failed{false};
    std::string fail_msg;
    // relay (host-staged)
    std::thread relay;
    std::atomic<bool> relay_stop{false};
    std::atomic<bool> relay_hold{false};   // fault injection: the relay moves nothing
    std::atomic<uint64_t> relayed_bytes{0};
    cudaStream_t r_d2h[kMaxStages] = {}, r_h2d[kMaxStages] = {};
    std::vector<cudaEvent_t> r_ev[kMaxStages];
    char* r_stage[kMaxStages] = {};          // pinned staging [slots][slot_bytes]
    BatchHdr* r_hdr[kMaxStages] = {};        // pinned
    unsigned long long* r_valA[kMaxStages] = {};
    unsigned long long* r_valB[kMaxStages] = {};
    std::atomic<int> relay_err{0};
};

static void free_ring(HostRing& r) {
    if (r.seq) cudaFree(r.seq);
    if (r.hdr) cudaFree(r.hdr);
    if (r.data) cudaFree(r.data);
    if (r.cursors) cudaFree(r.cursors);
    if (r.note_pub) cudaFreeHost(r.note_pub);
    if (r.note_n) cudaFreeHost(r.note_n);
    if (r.note_free) cudaFreeHost(r.note_free);
    r = HostRing{};
}

static camelot_status alloc_ring(HostRing& r, unsigned slots, size_t slot_bytes, bool notes) {
    r.slots = slots;
    r.slot_bytes = slot_bytes;
    CUDA_TRY(cudaMalloc(&r.seq, slots * sizeof(unsigned long long)));
    CUDA_TRY(cudaMalloc(&r.hdr, slots * sizeof(BatchHdr)));
    CUDA_TRY(cudaMalloc(&r.data, slots * slot_bytes));
    CUDA_TRY(cudaMalloc(&r.cursors, 2 * sizeof(Line64)));
    CUDA_TRY(cudaMemset(r.cursors, 0, 2 * sizeof(Line64)));
    CUDA_TRY(cudaMemset(r.hdr, 0, slots * sizeof(BatchHdr)));
    std::vector<unsigned long long> iota(slots);
    for (unsigned i = 0; i < slots; ++i) iota[i] = i;
    CUDA_TRY(cudaMemcpy(r.seq, iota.data(), slots * 8, cudaMemcpyHostToDevice));
    if (notes) {
        CUDA_TRY(cudaHostAlloc((void**)&r.note_pub, slots * 8, cudaHostAllocMapped | cudaHostAllocPortable));
        CUDA_TRY(cudaHostAlloc((void**)&r.note_n, slots * 4, cudaHostAllocMapped | cudaHostAllocPortable));
        CUDA_TRY(cudaHostAlloc((void**)&r.note_free, slots * 8, cudaHostAllocMapped | cudaHostAllocPortable));
        for (unsigned i = 0; i < slots; ++i) {
            r.note_pub[i] = 0;
            r.note_n[i] = 0;
            r.note_free[i] = i;
        }
    }
    return CAMELOT_OK;
}

static RingDev ring_view(const HostRing& r) {
    RingDev v{};
    v.seq = r.seq;
    v.hdr = r.hdr;
    v.data = r.data;
    v.head = r.cursors;
    v.tail = (unsigned long long*)((char*)r.cursors + sizeof(Line64));
    v.slots = r.slots;
    v.slot_bytes = r.slot_bytes;
    v.note_pub = r.note_pub;
    v.note_n = r.note_n;
    v.note_free = r.note_free;
    return v;
}

static void pipeline_free(camelot_pipeline* p) {
    if (p->relay.joinable()) {
        p->relay_stop = true;
        p->relay.join();
    }
    if (p->kstream) cudaStreamSynchronize(p->kstream);
    for (int s = 0; s < kMaxStages; ++s) {
        free_ring(p->out_rings[s]);
        free_ring(p->in_rings[s]);
        if (p->r_d2h[s]) cudaStreamDestroy(p->r_d2h[s]);
        if (p->r_h2d[s]) cudaStreamDestroy(p->r_h2d[s]);
        for (auto e : p->r_ev[s]) cudaEventDestroy(e);
        if (p->r_stage[s]) cudaFreeHost(p->r_stage[s]);
        if (p->r_hdr[s]) cudaFreeHost(p->r_hdr[s]);
        if (p->r_valA[s]) cudaFreeHost(p->r_valA[s]);
        if (p->r_valB[s]) cudaFreeHost(p->r_valB[s]);
    }
    if (p->dp) cudaFree(p->dp);
    if (p->ctl) cudaFree(p->ctl);
    if (p->groups) cudaFree(p->groups);
    if (p->scratch) cudaFree(p->scratch);
    if (p->trace) cudaFree(p->trace);
    if (p->hflags) cudaFreeHost(p->hflags);
    if (p->qring) cudaFreeHost(p->qring);
    if (p->qdata) {
        if (p->opt.device_data) cudaFree(p->qdata);
        else cudaFreeHost(p->qdata);
    }
    if (p->h2d) cudaStreamDestroy(p->h2d);
    if (p->comp) cudaFreeHost(p->comp);
    if (p->meta) cudaFree(p->meta);
    if (p->kdone) cudaEventDestroy(p->kdone);
    if (p->kstart) cudaEventDestroy(p->kstart);
    if (p->kstream) cudaStreamDestroy(p->kstream);
    if (p->side) cudaStreamDestroy(p->side);
    delete p;
}

static camelot_status set_failed(camelot_pipeline* p, const char* why) {
    p->failed = true;
    p->fail_msg = why;
    return fail(CAMELOT_ESTATE, "pipeline failed: %s", why);
}

// Checks the device error word and the state of the last launch; relaunches
// the persistent kernel if it has ended (idle exit) and `want_running`.
static camelot_status check_and_run(camelot_pipeline* p, bool want_running) {
    std::lock_guard<std::mutex> g(p->launch_mu);
    if (p->failed) return fail(CAMELOT_ESTATE, "pipeline failed: %s", p->fail_msg.c_str());
    const unsigned long long st = *(volatile unsigned long long*)p->hstatus;
    if (st != 0ull) {
        char buf[128];
        snprintf(buf, sizeof buf, "device error %u at %u", (unsigned)(st & 0xffffffffu),
                 (unsigned)(st >> 32));
        return set_failed(p, buf);
    }
    if (p->relay_err.load()) return set_failed(p, "host-staged relay copy failed");
    bool running = false;
    if (p->launched) {
        cudaError_t e = cudaEventQuery(p->kdone);
        if (e == cudaErrorNotReady) running = true;
        else if (e != cudaSuccess) {
            char buf[160];
            snprintf(buf, sizeof buf, "persistent kernel failed: %s", cudaGetErrorString(e));
            return set_failed(p, buf);
        }
    }
    if (p->launched && !running && !p->timed) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, p->kstart, p->kdone) == cudaSuccess) {
            p->last_launch_ms = ms;
            p->total_launch_ms += ms;
        }
        p->timed = true;
    }
    if (running || !want_running) return CAMELOT_OK;
    // (re)launch: clear the per-launch exit counters and the group barriers
    cudaError_t e = cudaMemsetAsync(&p->ctl->exited[0], 0, sizeof(p->ctl->exited), p->kstream);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->groups, 0, sizeof(GroupSync) *
                                              (size_t)p->hp.inst_begin[p->n_stages - 1] +
                                              sizeof(GroupSync) * p->hp.inst[p->n_stages - 1],
                                              p->kstream);
    if (e == cudaSuccess) e = cudaEventRecord(p->kstart, p->kstream);
    if (e == cudaSuccess) e = launch_pipeline_kernel(p->dp, p->grid, p->kstream, p->kinds);
    if (e == cudaSuccess) e = cudaEventRecord(p->kdone, p->kstream);
    if (e != cudaSuccess) {
        char buf[160];
        snprintf(buf, sizeof buf, "launch failed: %s", cudaGetErrorString(e));
        return set_failed(p, buf);
    }
    p->launched = true;
    p->timed = false;
    p->launches++;
    return CAMELOT_OK;
}

// Host-staged handoff (Sec. 4.2 / 6.1): every published batch is copied from
// the producer's device slot to pinned host memory and from there into the
// consumer's device slot; the copies run on one D2H and one H2D stream per
// stage boundary, so consecutive batches overlap.
// Copy the first `rows` rows of a batch slot: a plain copy of rows x rowb bytes,
// or, for a slot tiled in th-row tiles (th > 0), the whole row tiles plus, for
// a partial last tile, the first rows x 128 bytes of each of its th x 128-byte
// tiles (one 2-D copy).  Returns the bytes moved.
static size_t copy_batch_rows(char* dst, const char* src, size_t rows, size_t rowb, int th,
                              cudaMemcpyKind kind, cudaStream_t st, cudaError_t* e) {
    if (th == 0) {
        *e = cudaMemcpyAsync(dst, src, rows * rowb, kind, st);
        return rows * rowb;
    }
    const size_t full = rows / th, part = rows % th, tile_set = (size_t)th * rowb;   // bytes of one row tile
    size_t moved = 0;
    *e = cudaSuccess;
    if (full) {
        *e = cudaMemcpyAsync(dst, src, full * tile_set, kind, st);
        moved += full * tile_set;
    }
    if (part && *e == cudaSuccess) {
        const size_t off = full * tile_set, pitch = (size_t)th * 128;
        *e = cudaMemcpy2DAsync(dst + off, pitch, src + off, pitch, part * 128, rowb / 128, kind, st);
        moved += part * 128 * (rowb / 128);
    }
    return moved;
}

static void relay_main(camelot_pipeline* p) {
    cudaSetDevice(p->device);
    std::vector<uint64_t> cur(p->n_stages, 0);
    int idle = 0;
    while (!p->relay_stop.load(std::memory_order_relaxed)) {
        if (p->relay_hold.load(std::memory_order_relaxed)) {
            std::this_thread::sleep_for(std::chrono::microseconds(50));
            continue;
        }
        bool progress = false;
        for (int s = 0; s + 1 < p->n_stages; ++s) {
            HostRing& A = p->out_rings[s];
            HostRing& Bq = p->in_rings[s + 1];
            const uint64_t t = cur[s];
            const unsigned a = (unsigned)(t % A.slots), b = (unsigned)(t % Bq.slots);
            if (((volatile unsigned long long*)A.note_pub)[a] != t + 1) continue;
            if (((volatile unsigned long long*)Bq.note_free)[b] != t) continue;
            std::atomic_thread_fence(std::memory_order_acquire);
            const unsigned n = ((volatile unsigned int*)A.note_n)[a];
            const size_t T = (size_t)std::max(1, p->stages[s]->sp.rows);
            const size_t rowb = p->stages[s]->sp.out_row_bytes / T;
            char* stg = p->r_stage[s] + (size_t)b * A.slot_bytes;
            cudaError_t e = cudaMemcpyAsync(&p->r_hdr[s][b], &A.hdr[a], sizeof(BatchHdr),
                                            cudaMemcpyDeviceToHost, p->r_d2h[s]);
            size_t bytes = 0;
            const int th = p->tiled[s] ? p->stages[s + 1]->sp.tile_h : 0;
            if (!e) bytes = copy_batch_rows(stg, A.data + (size_t)a * A.slot_bytes, (size_t)n * T, rowb, th,
                                            cudaMemcpyDeviceToHost, p->r_d2h[s], &e);
            p->r_valA[s][a] = t + A.slots;
            if (!e) e = cudaMemcpyAsync(&A.seq[a], &p->r_valA[s][a], 8, cudaMemcpyHostToDevice,
                                        p->r_d2h[s]);
            if (!e) e = cudaEventRecord(p->r_ev[s][b], p->r_d2h[s]);
            if (!e) e = cudaStreamWaitEvent(p->r_h2d[s], p->r_ev[s][b], 0);
            if (!e) e = cudaMemcpyAsync(&Bq.hdr[b], &p->r_hdr[s][b], sizeof(BatchHdr),
                                        cudaMemcpyHostToDevice, p->r_h2d[s]);
            if (!e) copy_batch_rows(Bq.data + (size_t)b * Bq.slot_bytes, stg, (size_t)n * T, rowb, th,
                                    cudaMemcpyHostToDevice, p->r_h2d[s], &e);
            p->r_valB[s][b] = t + 1;
            if (!e) e = cudaMemcpyAsync(&Bq.seq[b], &p->r_valB[s][b], 8, cudaMemcpyHostToDevice,
                                        p->r_h2d[s]);
            if (e) { p->relay_err = 1; return; }
            p->relayed_bytes += 2 * bytes;
            cur[s] = t + 1;
            progress = true;
        }
        if (progress) { idle = 0; continue; }
        if (++idle < 2000) _mm_pause();
        else std::this_thread::yield();
    }
}

extern "C" camelot_status camelot_pipeline_create(camelot_stage* const* stages, int n_stages,
                                                  const camelot_alloc* alloc, camelot_handoff mode,
                                                  const camelot_options* opts,
                                                  camelot_pipeline** out) {
    if (!stages || !alloc || !out) return fail(CAMELOT_EINVAL, "null argument");
    *out = nullptr;
    if (n_stages < 1 || n_stages > kMaxStages)
        return fail(CAMELOT_EINVAL, "n_stages %d outside 1..%d", n_stages, kMaxStages);
    if (alloc->n_stages != n_stages) return fail(CAMELOT_EINVAL, "alloc.n_stages != n_stages");
    if (mode != CAMELOT_HANDOFF_GLOBAL && mode != CAMELOT_HANDOFF_HOST_STAGED)
        return fail(CAMELOT_EINVAL, "unknown handoff mode");
    camelot_options o;
    camelot_options_default(&o);
    if (opts) o = *opts;
    if (o.query_slots < 64 || (o.query_slots & (o.query_slots - 1)))
        return fail(CAMELOT_EINVAL, "query_slots must be a power of two >= 64");
    if (o.batch_slots < 2 || o.batch_slots > 4096) return fail(CAMELOT_EINVAL, "batch_slots outside 2..4096");
    if (o.data_slots == 0) o.data_slots = o.query_slots;
    if (o.data_slots < 64 || (o.data_slots & (o.data_slots - 1)) || o.data_slots > o.query_slots)
        return fail(CAMELOT_EINVAL, "data_slots must be a power of two in 64..query_slots");
    if (o.max_wait_ns < 0 || o.idle_exit_ns < 1000000 || o.wait_limit_ns < 1000000)
        return fail(CAMELOT_EINVAL, "max_wait_ns >= 0, idle_exit_ns and wait_limit_ns >= 1 ms required");
    if (o.qos_ns < 0 || o.qos_margin_ns < 0) return fail(CAMELOT_EINVAL, "qos_ns and qos_margin_ns must be >= 0");
    for (int b = 0; b < 32; ++b)
        if (o.batch_latency_ns[b] < 0) return fail(CAMELOT_EINVAL, "batch_latency_ns[%d] < 0", b);
    const int B = alloc->batch;
    if (B < 1 || B > 32) return fail(CAMELOT_EINVAL, "batch %d outside 1..32", B);
    int total = 0;
    for (int s = 0; s < n_stages; ++s) {
        const camelot_stage* st = stages[s];
        if (!st) return fail(CAMELOT_EINVAL, "stage %d is null", s);
        if (alloc->instances[s] < 1 || alloc->sm_quota[s] < 1)
            return fail(CAMELOT_EINVAL, "stage %d: instances and sm_quota must be >= 1", s);
        if (st->sp.max_batch < B) return fail(CAMELOT_EINVAL, "stage %d: max_batch < batch", s);
        const bool last = (s == n_stages - 1);
        if (last != (st->sp.top_k > 0))
            return fail(CAMELOT_EINVAL, "stage %d: only the last stage may (and must) have top_k > 0", s);
        if (!last && st->sp.out_row_bytes != stages[s + 1]->sp.in_row_bytes)
            return fail(CAMELOT_EINVAL, "stage %d output row (%zu B) != stage %d input row (%zu B)", s,
                        st->sp.out_row_bytes, s + 1, stages[s + 1]->sp.in_row_bytes);
        total += alloc->instances[s] * alloc->sm_quota[s];
    }
    camelot_status cs = ensure_configured();
    if (cs != CAMELOT_OK) return cs;
    int per_sm = 0;
    CUDA_TRY(max_coresident_ctas(&per_sm));
    const int sms = sm_count();
    if (per_sm < 1 || total > per_sm * sms)
        return fail(CAMELOT_EINVAL, "allocation needs %d SMs, the device offers %d", total, sms * per_sm);
    if (is_tensor_kind(stages[0]->sp.kind) && stages[0]->sp.rows > 1)
        return fail(CAMELOT_EINVAL, "a token-level tensor-core stage cannot be the first stage");
    {
        const int fk = stages[n_stages - 1]->sp.kind;
        if (o.logits_sink && fk != KIND_MLP_FP32 && !is_tensor_kind(fk) && fk != KIND_COMPUTE_SYNTH &&
            fk != KIND_STREAM_SYNTH)
            return fail(CAMELOT_EINVAL, "logits_sink needs a dense or artifact final stage");
    }

    auto* p = new camelot_pipeline();
    auto bail = [&](camelot_status s) { pipeline_free(p); return s; };
#define P_TRY(expr)                                                                         \
    do {                                                                                    \
        cudaError_t e_ = (expr);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return bail(fail(e_ == cudaErrorMemoryAllocation ? CAMELOT_ENOMEM : CAMELOT_ECUDA, \
                             "%s failed: %s", #expr, cudaGetErrorString(e_)));              \
    } while (0)
    cudaGetDevice(&p->device);
    p->n_stages = n_stages;
    for (int s = 0; s < n_stages; ++s) p->stages[s] = stages[s];
    p->alloc = *alloc;
    p->mode = mode;
    p->opt = o;
    p->grid = total;
    for (int s = 0; s < n_stages; ++s) p->kinds |= 1u << stages[s]->sp.kind;
    P_TRY(cudaStreamCreateWithFlags(&p->kstream, cudaStreamNonBlocking));
    P_TRY(cudaStreamCreateWithFlags(&p->side, cudaStreamNonBlocking));
    P_TRY(cudaEventCreate(&p->kdone));
    P_TRY(cudaEventCreate(&p->kstart));

    PipeParams& hp = p->hp;
    hp.n_stages = n_stages;
    hp.B = B;
    hp.handoff = mode;
    hp.total_ctas = total;
    int cta = 0, inst = 0;
    size_t scr = 0;
    for (int s = 0; s < n_stages; ++s) {
        hp.cta_begin[s] = cta;
        hp.inst[s] = alloc->instances[s];
        hp.quota[s] = alloc->sm_quota[s];
        hp.inst_begin[s] = inst;
        hp.st[s] = stages[s]->sp;
        StageParams tmp = stages[s]->sp;
        const bool dense = tmp.kind == KIND_MLP_FP32 || is_tensor_kind(tmp.kind);
        const size_t per = dense ? align_up(layout_scratch(tmp, B), 256) : align_up(tmp.scratch_bytes, 256);
        hp.st[s] = tmp;   // scratch offsets laid out for batch B
        hp.inst_scratch[s] = per;
        hp.scratch_off[s] = scr;
        scr += per * alloc->instances[s];
        cta += alloc->instances[s] * alloc->sm_quota[s];
        inst += alloc->instances[s];
    }
    hp.cta_begin[n_stages] = cta;
    // boundaries into a tensor-core stage carry the rows in its tiled operand
    // layout when the producer can write it (no re-tiling pass per batch)
    for (int s = 0; s + 1 < n_stages; ++s) {
        const int pk = stages[s]->sp.kind, ck = stages[s + 1]->sp.kind;
        const bool producer_can = pk == KIND_NORM_POOL2_BF16 || pk == KIND_NORMALIZE_U8_E4M3 ||
                                  pk == KIND_EMBED_GATHER || is_tensor_kind(pk);
        p->tiled[s] = is_tensor_kind(ck) && producer_can;
        hp.st[s].out_tiled = p->tiled[s] ? 1 : 0;
        hp.st[s].out_tile_h = stages[s + 1]->sp.tile_h;
        hp.st[s + 1].in_tiled = p->tiled[s] ? 1 : 0;
    }
    P_TRY(cudaMalloc(&p->ctl, sizeof(Ctl)));
    P_TRY(cudaMemset(p->ctl, 0, sizeof(Ctl)));
    P_TRY(cudaMalloc(&p->groups, sizeof(GroupSync) * inst));
    P_TRY(cudaMemset(p->groups, 0, sizeof(GroupSync) * inst));
    if (scr) P_TRY(cudaMalloc(&p->scratch, scr));
    P_TRY(cudaHostAlloc((void**)&p->hflags, 2 * sizeof(HostFlags), cudaHostAllocMapped | cudaHostAllocPortable));
    memset((void*)p->hflags, 0, 2 * sizeof(HostFlags));
    p->hstatus = (unsigned long long*)&p->hflags[1].stop;
    hp.ctl = p->ctl;
    hp.host_stop = &p->hflags[0].stop;
    hp.host_status = (volatile unsigned long long*)p->hstatus;
    hp.groups = p->groups;
    hp.scratch = p->scratch;
    // batch rings
    for (int s = 0; s + 1 < n_stages; ++s) {
        const size_t T = (size_t)std::max(1, stages[s]->sp.rows);
        const size_t slot_bytes = align_up(
            p->tiled[s] ? tiled_bytes((size_t)B * T, stages[s]->sp.out_row_bytes / T, stages[s + 1]->sp.tile_h)
                        : (size_t)B * stages[s]->sp.out_row_bytes, 256);
        const bool staged = (mode == CAMELOT_HANDOFF_HOST_STAGED);
        // every producer and consumer instance of the boundary can hold a slot,
        // with as many again in flight
        const unsigned need = 2u * (unsigned)(alloc->instances[s] + alloc->instances[s + 1]);
        const unsigned slots = std::max(o.batch_slots, need);
        p->ring_slots[s] = slots;
        cs = alloc_ring(p->out_rings[s], slots, slot_bytes, staged);
        if (cs != CAMELOT_OK) return bail(cs);
        hp.out_ring[s] = ring_view(p->out_rings[s]);
        if (staged) {
            cs = alloc_ring(p->in_rings[s + 1], slots, slot_bytes, true);
            if (cs != CAMELOT_OK) return bail(cs);
            // the producer side publishes notes, the consumer side frees them
            hp.out_ring[s].note_free = nullptr;
            hp.in_ring[s + 1] = ring_view(p->in_rings[s + 1]);
            hp.in_ring[s + 1].note_pub = nullptr;
            hp.in_ring[s + 1].note_n = nullptr;
            P_TRY(cudaStreamCreateWithFlags(&p->r_d2h[s], cudaStreamNonBlocking));
            P_TRY(cudaStreamCreateWithFlags(&p->r_h2d[s], cudaStreamNonBlocking));
            p->r_ev[s].resize(slots);
            for (auto& e : p->r_ev[s]) P_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
            P_TRY(cudaHostAlloc((void**)&p->r_stage[s], (size_t)slots * slot_bytes, cudaHostAllocPortable));
            P_TRY(cudaHostAlloc((void**)&p->r_hdr[s], slots * sizeof(BatchHdr), cudaHostAllocPortable));
            P_TRY(cudaHostAlloc((void**)&p->r_valA[s], slots * 8, cudaHostAllocPortable));
            P_TRY(cudaHostAlloc((void**)&p->r_valB[s], slots * 8, cudaHostAllocPortable));
        } else {
            hp.out_ring[s].note_pub = nullptr;
            hp.out_ring[s].note_n = nullptr;
            hp.out_ring[s].note_free = nullptr;
            hp.in_ring[s + 1] = hp.out_ring[s];
        }
    }
    // query ring and completion ring (pinned, mapped)
    const size_t R = o.query_slots;
    const size_t q_row = stages[0]->sp.in_row_bytes;
    P_TRY(cudaHostAlloc((void**)&p->qring, R * sizeof(QDesc), cudaHostAllocMapped | cudaHostAllocPortable));
    const size_t D = o.data_slots;
    if (o.device_data) {
        P_TRY(cudaMalloc(&p->qdata, D * q_row));
        P_TRY(cudaStreamCreateWithFlags(&p->h2d, cudaStreamNonBlocking));
    } else {
        P_TRY(cudaHostAlloc((void**)&p->qdata, D * q_row, cudaHostAllocMapped | cudaHostAllocPortable));
    }
    P_TRY(cudaHostAlloc((void**)&p->comp, R * sizeof(CompSlot), cudaHostAllocMapped | cudaHostAllocPortable));
    memset((void*)p->qring, 0, R * sizeof(QDesc));
    memset((void*)p->comp, 0, R * sizeof(CompSlot));
    P_TRY(cudaMalloc(&p->meta, R * sizeof(QMeta)));
    for (size_t i = 0; i < R; ++i) p->qring[i].seq = i;
    hp.qring = p->qring;
    hp.qdata = p->qdata;
    hp.qmask = R - 1;
    hp.dmask = D - 1;
    hp.q_row = q_row;
    hp.comp = p->comp;
    hp.meta = p->meta;
    hp.cmask = R - 1;
    hp.sink = o.logits_sink;
    hp.sink_ld = stages[n_stages - 1]->sp.out_width;
    P_TRY(cudaMalloc(&p->trace, sizeof(TraceDev)));
    P_TRY(cudaMemset(p->trace, 0, sizeof(TraceDev)));
    hp.trace = p->trace;
    hp.max_wait_ns = o.max_wait_ns;
    for (int b = 0; b < 32; ++b) {
        long long w = o.max_wait_ns;
        if (o.qos_ns > 0) w = std::min(w, std::max(0ll, (long long)(o.qos_ns - o.qos_margin_ns - o.batch_latency_ns[b])));
        hp.trig_wait_ns[b] = w;
    }
    hp.idle_ns = o.idle_exit_ns;
    hp.limit_ns = o.wait_limit_ns;
    hp.exit_after_trace = o.exit_after_trace ? 1 : 0;
    P_TRY(cudaMalloc(&p->dp, sizeof(PipeParams)));
    P_TRY(cudaMemcpy(p->dp, &hp, sizeof(PipeParams), cudaMemcpyHostToDevice));
    if (mode == CAMELOT_HANDOFF_HOST_STAGED) p->relay = std::thread(relay_main, p);
#undef P_TRY
    *out = p;
    return CAMELOT_OK;
}

extern "C" camelot_status camelot_submit(camelot_pipeline* p, uint32_t stream_id, const void* queries,
                                         uint32_t n, const int64_t* arrival_ns,
                                         uint64_t* first_query_id) {
    if (!p) return fail(CAMELOT_EINVAL, "null pipeline");
    if (n == 0) { if (first_query_id) *first_query_id = p->next_ticket; return CAMELOT_OK; }
    if (!queries) return fail(CAMELOT_EINVAL, "null queries");
    if (p->failed) return fail(CAMELOT_ESTATE, "pipeline failed: %s", p->fail_msg.c_str());
    const uint64_t polled = p->next_poll.load(std::memory_order_acquire);
    if (p->trace_active) {
        if (polled < p->trace_end) return fail(CAMELOT_ESTATE, "a trace is running");
        p->trace_active = false;
    }
    const uint64_t R = p->opt.query_slots, mask = R - 1;
    const uint64_t t0 = p->next_ticket.load(std::memory_order_relaxed);
    if (t0 + n - polled > R) return fail(CAMELOT_EAGAIN, "completion ring full (poll first)");
    const uint64_t D = p->opt.data_slots, dmask = D - 1;
    if (n > D) return fail(CAMELOT_EINVAL, "n=%u exceeds data_slots=%llu", n, (unsigned long long)D);
    for (uint32_t i = 0; i < n; ++i) {
        const uint64_t t = t0 + i;
        if (p->qring[t & mask].seq != t) return fail(CAMELOT_EAGAIN, "query ring full");
        // the data row of ticket t last held ticket u = t - D (u < t0 since n <= D):
        // stage 0 must have released u's descriptor (seq = u + R)
        if (D < R && t >= D) {
            const uint64_t u = t - D;
            // tickets before the last trace's end were all done when it was armed
            if (u >= p->data_floor && p->qring[u & mask].seq != u + R)
                return fail(CAMELOT_EAGAIN, "query data ring full");
        }
    }
    const size_t row = p->hp.q_row;
    const int64_t now = host_now_ns();
    if (p->opt.device_data) {
        // rows t0 .. t0+n-1 occupy one or two contiguous runs of the ring
        const uint64_t first = t0 & dmask;
        const uint64_t run1 = std::min<uint64_t>(n, D - first);
        if (cudaMemcpyAsync(p->qdata + first * row, queries, run1 * row, cudaMemcpyHostToDevice, p->h2d) !=
                cudaSuccess ||
            (run1 < n && cudaMemcpyAsync(p->qdata, (const char*)queries + run1 * row, (n - run1) * row,
                                         cudaMemcpyHostToDevice, p->h2d) != cudaSuccess) ||
            cudaStreamSynchronize(p->h2d) != cudaSuccess)
            return fail(CAMELOT_ECUDA, "query copy to the device data ring failed");
    }
    for (uint32_t i = 0; i < n; ++i) {
        const uint64_t t = t0 + i;
        if (!p->opt.device_data)
            memcpy(p->qdata + (t & dmask) * row, (const char*)queries + (size_t)i * row, row);
        QDesc& d = p->qring[t & mask];
        d.t_arrival = arrival_ns ? arrival_ns[i] : now;
        d.stream_id = stream_id;
    }
    std::atomic_thread_fence(std::memory_order_release);
    for (uint32_t i = 0; i < n; ++i) p->qring[(t0 + i) & mask].seq = t0 + i + 1;
    p->next_ticket.store(t0 + n, std::memory_order_release);
    if (first_query_id) *first_query_id = t0;
    return check_and_run(p, true);
}

extern "C" camelot_status camelot_submit_trace(camelot_pipeline* p, uint32_t stream_id,
                                               const void* queries, uint32_t n,
                                               const int64_t* arrival_off_ns,
                                               uint64_t* first_query_id) {
    if (!p) return fail(CAMELOT_EINVAL, "null pipeline");
    if (!queries || !arrival_off_ns || n == 0) return fail(CAMELOT_EINVAL, "empty trace");
    if (p->failed) return fail(CAMELOT_ESTATE, "pipeline failed: %s", p->fail_msg.c_str());
    const uint64_t base = p->next_ticket.load();
    if (p->next_poll.load() != base) return fail(CAMELOT_ESTATE, "queries are outstanding");
    const uint64_t R = p->opt.query_slots;
    if (n > R) return fail(CAMELOT_EINVAL, "trace longer than query_slots");
    cudaSetDevice(p->device);
    TraceDev td{};
    td.data = (const char*)queries;
    td.off = (const long long*)arrival_off_ns;
    td.base = base;
    td.n = n;
    td.stream_id = stream_id;
    td.armed = 0;
    static const unsigned long long zero = 0;
    static const unsigned int one = 1;
    // disarm, reset the trace clock, write the fields, then arm
    CUDA_TRY(cudaMemcpyAsync(&p->trace->armed, &td.armed, sizeof(unsigned), cudaMemcpyHostToDevice, p->side));
    CUDA_TRY(cudaMemcpyAsync(&p->ctl->trace_t0.v, &zero, 8, cudaMemcpyHostToDevice, p->side));
    CUDA_TRY(cudaMemcpyAsync(p->trace, &td, sizeof(TraceDev), cudaMemcpyHostToDevice, p->side));
    CUDA_TRY(cudaMemcpyAsync(&p->trace->armed, &one, sizeof(unsigned), cudaMemcpyHostToDevice, p->side));
    CUDA_TRY(cudaStreamSynchronize(p->side));
    // tickets after the trace: each host ring slot now expects the first
    // ticket >= base + n that maps to it
    const uint64_t next = base + n, mask = R - 1;
    for (uint64_t s = 0; s < R; ++s) {
        uint64_t t = next + ((s - next) & mask);
        p->qring[s].seq = t;
    }
    p->trace_active = true;
    p->trace_end = next;
    p->data_floor = next;
    p->next_ticket.store(next, std::memory_order_release);
    if (first_query_id) *first_query_id = base;
    return check_and_run(p, true);
}

// The completion of ticket t, once every word of its slot carries the flag
// t + 1 (each 8-byte word is written atomically by the device: 32 data bits,
// 32 flag bits).  Returns false while any word is still missing.
static bool read_completion(const CompSlot& cs, uint64_t t, camelot_completion* c) {
    const volatile unsigned long long* w = cs.w;
    const uint32_t flag = (uint32_t)(t + 1);
    uint32_t d[kCompWords];
    for (int i = 0; i < CW_USED; ++i) {
        const unsigned long long x = w[i];
        if ((uint32_t)(x >> 32) != flag) return false;
        d[i] = (uint32_t)x;
    }
    std::atomic_thread_fence(std::memory_order_acquire);
    auto u64 = [&](int lo) { return (int64_t)((uint64_t)d[lo] | ((uint64_t)d[lo + 1] << 32)); };
    memset(c, 0, sizeof(*c));
    c->query_id = t;
    c->stream_id = d[CW_STREAM];
    c->status = (int32_t)d[CW_STATUS];
    c->batch_size = (int32_t)d[CW_BATCH];
    c->t_arrival_ns = u64(CW_T_ARR);
    c->t_batch_ns = u64(CW_T_BATCH);
    c->t_done_ns = u64(CW_T_DONE);
    for (int r = 0; r < kMaxTopK; ++r) {
        c->idx[r] = (int32_t)d[CW_IDX + r];
        uint32_t v = d[CW_VAL + r];
        memcpy(&c->val[r], &v, 4);
    }
    return true;
}

extern "C" camelot_status camelot_poll(camelot_pipeline* p, camelot_completion* out, uint32_t max,
                                       uint32_t* n_out, int64_t timeout_us) {
    if (!p || !n_out || (max && !out)) return fail(CAMELOT_EINVAL, "null argument");
    *n_out = 0;
    const uint64_t mask = p->opt.query_slots - 1;
    const int64_t t_start = host_now_ns();
    uint32_t got = 0;
    int spins = 0;
    for (;;) {
        uint64_t t = p->next_poll.load(std::memory_order_relaxed);
        while (got < max) {
            if (!read_completion(p->comp[t & mask], t, &out[got])) break;
            out[got].t_poll_ns = host_now_ns();
            ++got;
            ++t;
        }
        if (got) {
            p->next_poll.store(t, std::memory_order_release);
            *n_out = got;
            return CAMELOT_OK;
        }
        if ((spins & 1023) == 0) {
            const bool outstanding = t < p->next_ticket.load(std::memory_order_acquire);
            camelot_status cs = check_and_run(p, outstanding);
            if (cs != CAMELOT_OK) return cs;
        }
        if (max == 0 || timeout_us == 0) return CAMELOT_OK;
        if (timeout_us > 0 && host_now_ns() - t_start > timeout_us * 1000)
            return fail(CAMELOT_ETIMEDOUT, "no completion within %lld us", (long long)timeout_us);
        if (++spins < 4000) _mm_pause();
        else std::this_thread::yield();
    }
}

extern "C" camelot_status camelot_pipeline_stall_relay(camelot_pipeline* p, int stall) {
    if (!p) return fail(CAMELOT_EINVAL, "null pipeline");
    if (p->mode != CAMELOT_HANDOFF_HOST_STAGED) return fail(CAMELOT_EINVAL, "not a host-staged pipeline");
    p->relay_hold.store(stall != 0);
    return CAMELOT_OK;
}

extern "C" camelot_status camelot_pipeline_stats(camelot_pipeline* p, camelot_stats* out) {
    if (!p || !out) return fail(CAMELOT_EINVAL, "null argument");
    memset(out, 0, sizeof *out);
    out->submitted = p->next_ticket.load();
    out->completed = p->next_poll.load();
    Line64 b[kMaxStages];
    CUDA_TRY(cudaMemcpyAsync(b, &p->ctl->batches[0], sizeof b, cudaMemcpyDeviceToHost, p->side));
    CUDA_TRY(cudaStreamSynchronize(p->side));
    for (int s = 0; s < kMaxStages; ++s) out->batches[s] = b[s].v;
    CUDA_TRY(cudaMemcpyAsync(b, &p->ctl->busy_ns[0], sizeof b, cudaMemcpyDeviceToHost, p->side));
    CUDA_TRY(cudaStreamSynchronize(p->side));
    for (int s = 0; s < kMaxStages; ++s) out->busy_ns[s] = b[s].v;
    CUDA_TRY(cudaMemcpyAsync(b, &p->ctl->body_ns[0], sizeof b, cudaMemcpyDeviceToHost, p->side));
    CUDA_TRY(cudaStreamSynchronize(p->side));
    for (int s = 0; s < kMaxStages; ++s) out->body_ns[s] = b[s].v;
    CUDA_TRY(cudaMemcpyAsync(b, &p->ctl->acq_ns[0], sizeof b, cudaMemcpyDeviceToHost, p->side));
    CUDA_TRY(cudaStreamSynchronize(p->side));
    for (int s = 0; s < kMaxStages; ++s) out->acquire_ns[s] = b[s].v;
    out->kernel_launches = p->launches;
    out->relayed_bytes = p->relayed_bytes.load();
    size_t slot = 0, ring = 0;
    for (int s = 0; s < kMaxStages; ++s) {
        for (HostRing* r : {&p->out_rings[s], &p->in_rings[s]}) {
            if (!r->data) continue;
            slot = std::max(slot, r->slot_bytes);
            ring += (size_t)r->slots * r->slot_bytes;
        }
    }
    out->device_bytes_per_batch_slot = slot;
    out->device_ring_bytes = ring;
    const unsigned long long st = *(volatile unsigned long long*)p->hstatus;
    out->device_status = (int32_t)(st & 0xffffffffu);
    out->device_where = (int32_t)(st >> 32);
    check_and_run(p, false);   // folds in the duration of a launch that has ended
    out->last_launch_ms = p->last_launch_ms;
    out->total_launch_ms = p->total_launch_ms;
    return CAMELOT_OK;
}

extern "C" camelot_status camelot_pipeline_destroy(camelot_pipeline* p) {
    if (!p) return fail(CAMELOT_EINVAL, "null pipeline");
    cudaSetDevice(p->device);
    p->hflags[0].stop = 1;
    std::atomic_thread_fence(std::memory_order_seq_cst);
    if (p->relay.joinable()) {
        p->relay_stop = true;
        p->relay.join();
    }
    cudaError_t e = cudaStreamSynchronize(p->kstream);
    for (int s = 0; s < kMaxStages; ++s) {
        if (p->r_d2h[s]) cudaStreamSynchronize(p->r_d2h[s]);
        if (p->r_h2d[s]) cudaStreamSynchronize(p->r_h2d[s]);
    }
    pipeline_free(p);
    if (e != cudaSuccess) return fail(CAMELOT_ECUDA, "persistent kernel ended with: %s", cudaGetErrorString(e));
    return CAMELOT_OK;
}

size_t camelot_internal_query_bytes(const camelot_pipeline* p) { return p->hp.q_row; }
