// Camelot CPU oracle -- TEST INFRASTRUCTURE ONLY.
//
// A plain, slow, FP64 restatement of what the Camelot query pipeline computes,
// written from the paper (Zhang et al., "Towards QoS-Aware and Resource-Efficient
// GPU Microservices Based on Spatial Multitasking GPUs In Datacenters").  Only the
// tests, the package's smoke check and the benchmark's CPU-baseline leg may load
// it; the product library never does, and this file shares no code, header or
// constant table with the CUDA path.
//
// Parts (each function below cites the passage it follows):
//   1. stage math of the synthetic microservices (stand-ins for the Sec. 3
//      suite): u8 normalisation, 2x2 pooling, dense layers with ReLU / erf-GELU,
//      argmax / top-k, the number formats the reduced-precision arms use, and
//      the FP8 arm's per-tensor quantisation and scaled dense layers, and the
//      artifact compute / memory / host-link stages (binary32 by definition);
//   2. whole-pipeline references (the plain 2-stage and the 3-stage BF16 pipelines);
//   3. an event-driven simulator of the wait queue, batch trigger and
//      multi-instance stage pipeline (Sec. 5.2 steps 1-2, Sec. 4.1);
//   4. the two allocation policies (Eq. 1, Eq. 3) by exhaustive enumeration,
//      and the simulated-annealing solver the paper adopts (end of Sec. 7.3);
//   5. the latency-predictor MLP forward / backward / Adam (Sec. 7.1, with an
//      MLP in place of the paper's decision tree).
//
// Parity status: every function here is pinned by a `-m "not gpu"` test
// (closed forms, brute force, library routines, finite differences); none is
// "parity unpinned".
//
// Build: g++ -O2 -std=c++17 -fopenmp -shared -fPIC camelot_oracle.cpp
#include <cmath>
#include <cstdint>
#include <cstring>
#include <algorithm>
#include <deque>
#include <functional>
#include <queue>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

extern "C" {

// ---------------------------------------------------------------------------
// 1. Stage math
// ---------------------------------------------------------------------------

// Activation codes shared by every dense-layer routine of the oracle.
enum { ORC_ACT_NONE = 0, ORC_ACT_RELU = 1, ORC_ACT_GELU = 2 };

// Normalisation stage of the image pipelines (stand-in for the Sec. 3
// preprocessing microservice): y = (x - 127.5) / 64, element by element, the
// flattened order being the input's HWC order.
void orc_normalize_u8(const uint8_t* x, int64_t n, double* y) {
    for (int64_t i = 0; i < n; ++i) y[i] = ((double)x[i] - 127.5) / 64.0;
}

// 2x2 average pooling followed by the same normalisation (3-stage image
// pipeline): y[q, h, w, c] = ((x00 + x01 + x10 + x11) / 4 - 127.5) / 64 where
// x_ab = x[q, 2h+a, 2w+b, c]; input [nq, H, W, C] u8, output [nq, H/2, W/2, C].
void orc_norm_pool2(const uint8_t* x, int64_t nq, int H, int W, int C, double* y) {
    const int Ho = H / 2, Wo = W / 2;
    for (int64_t q = 0; q < nq; ++q) {
        const uint8_t* xq = x + q * (int64_t)H * W * C;
        double* yq = y + q * (int64_t)Ho * Wo * C;
        for (int h = 0; h < Ho; ++h)
            for (int w = 0; w < Wo; ++w)
                for (int c = 0; c < C; ++c) {
                    double s = 0.0;
                    for (int a = 0; a < 2; ++a)
                        for (int b = 0; b < 2; ++b)
                            s += (double)xq[((int64_t)(2 * h + a) * W + (2 * w + b)) * C + c];
                    yq[((int64_t)h * Wo + w) * C + c] = (s / 4.0 - 127.5) / 64.0;
                }
    }
}

// erf-form GELU: 0.5 * v * (1 + erf(v / sqrt(2))).
double orc_gelu(double v) { return 0.5 * v * (1.0 + std::erf(v / std::sqrt(2.0))); }

static double apply_act(double v, int act) {
    if (act == ORC_ACT_RELU) return v > 0.0 ? v : 0.0;
    if (act == ORC_ACT_GELU) return orc_gelu(v);
    return v;
}

// Dense layer of a stage: y[q, j] = act(sum_k w[j, k] * x[q, k]), w row-major
// [N, K], no bias.  If `absdot` is non-null it receives sum_k |w[j, k] x[q, k]|,
// the scale the FP32 tolerance is stated against.
void orc_linear(const double* x, int64_t nq, int K, const double* w, int N, int act,
                double* y, double* absdot) {
    for (int64_t q = 0; q < nq; ++q)
        for (int j = 0; j < N; ++j) {
            double s = 0.0, a = 0.0;
            const double* wr = w + (int64_t)j * K;
            const double* xr = x + q * (int64_t)K;
            for (int k = 0; k < K; ++k) {
                s += wr[k] * xr[k];
                a += std::fabs(wr[k] * xr[k]);
            }
            y[q * N + j] = apply_act(s, act);
            if (absdot) absdot[q * N + j] = a;
        }
}

// Index of the largest of z[q, 0..N-1]; among equal maxima the lowest index.
void orc_argmax(const double* z, int64_t nq, int N, int32_t* idx) {
    for (int64_t q = 0; q < nq; ++q) {
        int best = 0;
        for (int j = 1; j < N; ++j)
            if (z[q * N + j] > z[q * N + best]) best = j;
        idx[q] = best;
    }
}

// The k largest of z[q, :], ordered by value descending then index ascending.
void orc_topk(const double* z, int64_t nq, int N, int k, int32_t* idx, double* val) {
    std::vector<int> order(N);
    for (int64_t q = 0; q < nq; ++q) {
        const double* zq = z + q * N;
        for (int j = 0; j < N; ++j) order[j] = j;
        std::stable_sort(order.begin(), order.end(), [zq](int a, int b) {
            if (zq[a] != zq[b]) return zq[a] > zq[b];
            return a < b;
        });
        for (int r = 0; r < k; ++r) {
            idx[q * k + r] = order[r];
            if (val) val[q * k + r] = zq[order[r]];
        }
    }
}

// ---- number formats ------------------------------------------------------
// Round to binary32 (round-to-nearest-even of the C conversion).
void orc_round_f32(const double* in, int64_t n, double* out) {
    for (int64_t i = 0; i < n; ++i) out[i] = (double)(float)in[i];
}

// Round to bfloat16: first to binary32, then keep the top 16 bits of the
// binary32 pattern with round-to-nearest-even on the dropped 16 bits (the
// bfloat16 format is the upper half of binary32).  NaN stays NaN.
static float f32_to_bf16_value(float f) {
    uint32_t u;
    std::memcpy(&u, &f, 4);
    if ((u & 0x7F800000u) == 0x7F800000u && (u & 0x007FFFFFu)) {
        u |= 0x00400000u;  // quiet NaN
    } else {
        const uint32_t lsb = (u >> 16) & 1u;
        u += 0x7FFFu + lsb;
    }
    u &= 0xFFFF0000u;
    float r;
    std::memcpy(&r, &u, 4);
    return r;
}
void orc_round_bf16(const double* in, int64_t n, double* out) {
    for (int64_t i = 0; i < n; ++i) out[i] = (double)f32_to_bf16_value((float)in[i]);
}
// Bit pattern of the bfloat16 value (for golden fixtures).
void orc_bf16_bits(const double* in, int64_t n, uint16_t* out) {
    for (int64_t i = 0; i < n; ++i) {
        float r = f32_to_bf16_value((float)in[i]);
        uint32_t u;
        std::memcpy(&u, &r, 4);
        out[i] = (uint16_t)(u >> 16);
    }
}

// Round to OCP FP8 E4M3 (1 sign, 4 exponent bits with bias 7, 3 mantissa bits,
// no infinities, largest finite 448, smallest normal 2^-6, subnormal spacing
// 2^-9), round-to-nearest-even on the binary32 value, saturating to +-448.
void orc_round_e4m3(const double* in, int64_t n, double* out) {
    for (int64_t i = 0; i < n; ++i) {
        double v = (double)(float)in[i];
        if (std::isnan(v)) { out[i] = v; continue; }
        double a = std::fabs(v);
        double r;
        if (a == 0.0) {
            r = 0.0;
        } else {
            int e = (int)std::floor(std::log2(a));
            if (e < -6) e = -6;               // subnormal range shares the 2^-9 quantum
            double quantum = std::ldexp(1.0, e - 3);
            double m = a / quantum;           // exact: quantum is a power of two
            double fl = std::floor(m);
            double fr = m - fl;
            double k = fl;
            if (fr > 0.5 || (fr == 0.5 && std::fmod(fl, 2.0) != 0.0)) k = fl + 1.0;
            r = k * quantum;
            if (r > 448.0) r = 448.0;
        }
        out[i] = std::copysign(r, v);
    }
}

// Value of each OCP FP8 E4M3 code: bit 7 sign, bits 6-3 exponent (bias 7),
// bits 2-0 mantissa; exponent field 0 encodes subnormals m * 2^-9; S.1111.111
// is NaN (the format has no infinities).
void orc_e4m3_decode(const uint8_t* codes, int64_t n, double* out) {
    for (int64_t i = 0; i < n; ++i) {
        const int c = codes[i];
        const int e = (c >> 3) & 15, m = c & 7;
        double v;
        if (e == 15 && m == 7) v = std::nan("");
        else if (e == 0) v = std::ldexp((double)m, -9);
        else v = std::ldexp(1.0 + m / 8.0, e - 7);
        out[i] = (c & 0x80) ? -v : v;
    }
}

// Per-tensor quantisation of the FP8 arm (the scaling the configuration fixes:
// s = max|w| / 448 computed in binary32, codes e4m3(w / s) with the quotient
// rounded to binary32 first, as the kernel computes it).  Writes the code
// values to q and returns s.
double orc_quantize_e4m3(const double* w, int64_t n, double* q) {
    double amax = 0.0;
    for (int64_t i = 0; i < n; ++i) amax = std::max(amax, std::fabs((double)(float)w[i]));
    const double s = (double)(float)(amax / 448.0);
    for (int64_t i = 0; i < n; ++i) {
        const double t = (double)(float)((double)(float)w[i] / s);
        orc_round_e4m3(&t, 1, q + i);
    }
    return s;
}

// Dense layer of the FP8 arm on code values: y[q, j] = act(vscale * sum_k
// wq[j, k] xq[q, k]) with the sum in FP64 (vscale = the binary32 product of the
// weight and input scales).  If yq is given, the output codes e4m3(y / s_out)
// (quotient rounded to binary32).  absdot (nullable): sum_k |wq xq| * vscale.
void orc_linear_fp8(const double* xq, int64_t nq, int K, const double* wq, int N, double vscale,
                    int act, double s_out, double* y, double* yq, double* absdot) {
    for (int64_t q = 0; q < nq; ++q)
        for (int j = 0; j < N; ++j) {
            double acc = 0.0, a = 0.0;
            for (int k = 0; k < K; ++k) {
                acc += wq[(int64_t)j * K + k] * xq[q * K + k];
                a += std::fabs(wq[(int64_t)j * K + k] * xq[q * K + k]);
            }
            const double v = apply_act(acc * vscale, act);
            y[q * N + j] = v;
            if (absdot) absdot[q * N + j] = a * vscale;
            if (yq) {
                const double t = (double)(float)(v / s_out);
                orc_round_e4m3(&t, 1, yq + q * N + j);
            }
        }
}

// Embedding gather of the text-tagging microservice: row t of query q is
// E[tok[q, t]] for 0 <= tok < V, and a zero row for padding (any other ID).
void orc_embed_gather(const int32_t* tok, int64_t n_rows, const double* E, int V, int D, double* out) {
    for (int64_t r = 0; r < n_rows; ++r) {
        const int32_t t = tok[r];
        for (int d = 0; d < D; ++d) out[r * D + d] = (t >= 0 && t < V) ? E[(int64_t)t * D + d] : 0.0;
    }
}

// Artifact compute-intensive stage (the c_i of Sec. 2.3 and Sec. 8.5, whose
// arithmetic intensity is a parameter): every value x runs `steps` iterations
// of y <- fma(y, 127/128, x / 128) from y = 0.  The stage is defined in
// binary32 with one rounding per fused step, so this reference computes in
// binary32 too (std::fma on floats rounds once); the exact real result is
// x (1 - (127/128)^steps).
void orc_compute_synth(const float* x, int64_t n, int steps, float* y) {
    for (int64_t i = 0; i < n; ++i) {
        const float b = x[i] * 0.0078125f;
        float a = 0.0f;
        for (int k = 0; k < steps; ++k) a = std::fma(a, 0.9921875f, b);
        y[i] = a;
    }
}

// Artifact memory- / host-link-intensive stage (the m_i and p_i of Sec. 8.5):
// row q of width W gets y_j = x_j + T[b + j] + T[b + W + j] + ... (R / W table
// windows, added left to right in binary32), b = W * (h mod (L / W - R / W + 1)),
// h = the high 32 bits of the 64-bit product bits(x_0) * 0x9E3779B97F4A7C15.
void orc_stream_synth(const float* x, int64_t nq, int W, const float* T, int64_t L, int R, float* y) {
    const uint64_t starts = (uint64_t)(L / W - R / W + 1);
    for (int64_t q = 0; q < nq; ++q) {
        const float* xr = x + q * W;
        uint32_t bits;
        std::memcpy(&bits, xr, 4);
        const uint32_t h = (uint32_t)(((uint64_t)bits * 0x9E3779B97F4A7C15ull) >> 32);
        const int64_t b = (int64_t)(h % (uint32_t)starts) * W;
        for (int j = 0; j < W; ++j) {
            float a = xr[j];
            for (int r = 0; r < R / W; ++r) a = a + T[b + (int64_t)r * W + j];
            y[q * W + j] = a;
        }
    }
}

// ---------------------------------------------------------------------------
// 2. Whole-pipeline references
// ---------------------------------------------------------------------------

// Plain 2-stage image pipeline: stage 1 normalises [64, 64, 3] u8 to 12288
// values; stage 2 is relu(W1 y) -> relu(W2 .) -> W3 . (no bias, no activation on
// the logits) followed by argmax.  FP64 throughout.  `dims` = {K0, N1, N2, N3};
// weights row-major; outputs logits [nq, N3] and idx [nq].  Queries are
// independent, so they are spread over `nthreads` OpenMP threads (0 = all).
void orc_pipeline_mlp(const uint8_t* x, int64_t nq, const int* dims, const double* w1,
                      const double* w2, const double* w3, double* logits, int32_t* idx,
                      int nthreads) {
    const int K0 = dims[0], N1 = dims[1], N2 = dims[2], N3 = dims[3];
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for num_threads(nthreads) schedule(dynamic, 1)
#endif
    for (int64_t q = 0; q < nq; ++q) {
        std::vector<double> y(K0), h1(N1), h2(N2), z(N3);
        orc_normalize_u8(x + q * (int64_t)K0, K0, y.data());
        orc_linear(y.data(), 1, K0, w1, N1, ORC_ACT_RELU, h1.data(), nullptr);
        orc_linear(h1.data(), 1, N1, w2, N2, ORC_ACT_RELU, h2.data(), nullptr);
        orc_linear(h2.data(), 1, N2, w3, N3, ORC_ACT_NONE, z.data(), nullptr);
        for (int j = 0; j < N3; ++j) logits[q * N3 + j] = z[j];
        orc_argmax(z.data(), 1, N3, idx + q);
    }
    (void)nthreads;
}

// 3-stage image pipeline: stage 1 = 2x2 pool + normalise ([H, W, 3] u8 ->
// H/2 * W/2 * 3 values); stage 2 = gelu(Wb gelu(Wa y)); stage 3 = logits Wc h
// and the top-k indices.  `emulate_bf16` != 0 rounds where the BF16 arm
// rounds: the stage-1 output, every weight, and each GELU output to bfloat16;
// the logits stay unrounded (FP32 on the device).  0 = pure FP64 on the given
// weights.  dims = {K0, N1, N2, N3}.
void orc_pipeline_gemm3(const uint8_t* x, int64_t nq, int H, int W, const int* dims,
                        const double* wa, const double* wb, const double* wc, int top_k,
                        int emulate_bf16, double* logits, int32_t* idx, int nthreads) {
    const int K0 = dims[0], N1 = dims[1], N2 = dims[2], N3 = dims[3];
    std::vector<double> wa_r(wa, wa + (int64_t)N1 * K0), wb_r(wb, wb + (int64_t)N2 * N1),
        wc_r(wc, wc + (int64_t)N3 * N2);
    if (emulate_bf16) {
        orc_round_bf16(wa_r.data(), (int64_t)wa_r.size(), wa_r.data());
        orc_round_bf16(wb_r.data(), (int64_t)wb_r.size(), wb_r.data());
        orc_round_bf16(wc_r.data(), (int64_t)wc_r.size(), wc_r.data());
    }
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for num_threads(nthreads) schedule(dynamic, 1)
#endif
    for (int64_t q = 0; q < nq; ++q) {
        std::vector<double> y(K0), h1(N1), h2(N2), z(N3);
        orc_norm_pool2(x + q * (int64_t)H * W * 3, 1, H, W, 3, y.data());
        if (emulate_bf16) orc_round_bf16(y.data(), K0, y.data());
        orc_linear(y.data(), 1, K0, wa_r.data(), N1, ORC_ACT_GELU, h1.data(), nullptr);
        if (emulate_bf16) orc_round_bf16(h1.data(), N1, h1.data());
        orc_linear(h1.data(), 1, N1, wb_r.data(), N2, ORC_ACT_GELU, h2.data(), nullptr);
        if (emulate_bf16) orc_round_bf16(h2.data(), N2, h2.data());
        orc_linear(h2.data(), 1, N2, wc_r.data(), N3, ORC_ACT_NONE, z.data(), nullptr);
        for (int j = 0; j < N3; ++j) logits[q * N3 + j] = z[j];
        orc_topk(z.data(), 1, N3, top_k, idx + q * top_k, nullptr);
    }
    (void)nthreads;
}

// ---------------------------------------------------------------------------
// 3. Event-driven pipeline simulator (Sec. 5.2 steps 1-2; Sec. 4.1)
// ---------------------------------------------------------------------------
//
// Queries arrive at times `arr` (seconds, ascending) into the wait queue.  The
// batch trigger (Sec. 5.2 step 2) issues a batch when `B` queries wait, or when
// the oldest waiting query has waited `t_wait` (the "about to violate QoS"
// rule, with its threshold given as a wait bound).  Stage s has `inst[s]`
// identical instances; a batch of b queries occupies one instance of stage s
// for `tau[s * B + (b - 1)]` seconds, times the next value of the stage's
// multiplier stream `mult[s][...]` when `mult_len` > 0 (used for random service
// times).  Between stage s and s+1 there are `cap[s]` batch slots: a stage-s
// batch claims a slot when it starts and the slot is freed when the stage-(s+1)
// batch that reads it finishes.  Stage 0 is the batcher's consumer.  Any free
// instance takes the oldest ready batch (FIFO per stage).  Output: completion
// time of every query (`done`, seconds) and the size of every issued batch in
// order (`batch_sizes`, may be null; capacity nq).  Returns the number of
// batches issued.
//
// QoS form of the trigger (Sec. 5.2 step 2, "the first query tends to suffer
// from QoS violation"): with `lat` non-null, a batch of k = min(waiting, B)
// queries also leaves once the oldest has waited qos_budget - lat[k - 1], where
// lat[k - 1] is the predicted latency of a k-query batch and qos_budget the QoS
// bound less its margin: waiting longer would make the oldest query's wait plus
// its batch's latency exceed the budget.  The wait bound is the smaller of that
// and t_wait (at once when it is <= 0).  `issue` (nullable, capacity nq)
// receives the time each batch was issued.
int64_t orc_simulate_qos(const double* arr, int64_t nq, int B, double t_wait, double qos_budget,
                         const double* lat, int n_stages, const int* inst, const double* tau,
                         const int* cap, const double* mult, int64_t mult_len, double* done,
                         int32_t* batch_sizes, double* issue) {
    struct Batch { int64_t first; int n; };
    struct Ev {
        double t; int stage; int64_t seq; int64_t batch;
        bool operator>(const Ev& o) const {
            if (t != o.t) return t > o.t;
            if (stage != o.stage) return stage < o.stage;   // later stages first
            return seq > o.seq;
        }
    };
    std::vector<Batch> batches;
    std::priority_queue<Ev, std::vector<Ev>, std::greater<Ev>> evq;
    std::vector<int> idle(inst, inst + n_stages);
    std::vector<std::deque<int64_t>> ready(n_stages);      // batches waiting for stage s
    std::vector<int> slots_used(n_stages > 0 ? n_stages : 1, 0);  // slots s -> s+1 in use
    std::vector<int64_t> mult_pos(n_stages, 0);
    int64_t next_arr = 0, next_issue = 0, seq = 0, completed = 0;
    double t = 0.0;

    auto service = [&](int s, int b) {
        double v = tau[(int64_t)s * B + (b - 1)];
        if (mult_len > 0) {
            v *= mult[(int64_t)s * mult_len + (mult_pos[s] % mult_len)];
            mult_pos[s]++;
        }
        return v;
    };
    auto out_slot_free = [&](int s) { return s == n_stages - 1 || slots_used[s] < cap[s]; };
    // how long the oldest of `waiting` queries may wait before its batch leaves
    auto wait_bound = [&](int64_t waiting) {
        if (!lat) return t_wait;
        const int k = (int)std::min<int64_t>(waiting, B);
        return std::min(t_wait, std::max(0.0, qos_budget - lat[k - 1]));
    };

    while (completed < nq) {
        // Dispatch everything that can start at time t, later stages first.
        bool progress = true;
        while (progress) {
            progress = false;
            for (int s = n_stages - 1; s >= 1; --s) {
                while (idle[s] > 0 && !ready[s].empty() && out_slot_free(s)) {
                    int64_t bi = ready[s].front();
                    ready[s].pop_front();
                    idle[s]--;
                    if (s < n_stages - 1) slots_used[s]++;
                    evq.push({t + service(s, batches[bi].n), s, seq++, bi});
                    progress = true;
                }
            }
            // Stage 0 pulls straight from the wait queue through the batch trigger.
            while (idle[0] > 0 && out_slot_free(0) && next_issue < next_arr) {
                int64_t waiting = next_arr - next_issue;
                bool full = waiting >= B;
                bool late = t >= arr[next_issue] + wait_bound(waiting);  // same sum as the event time
                if (!full && !late) break;
                int b = (int)std::min<int64_t>(waiting, B);
                batches.push_back({next_issue, b});
                if (batch_sizes) batch_sizes[batches.size() - 1] = b;
                if (issue) issue[batches.size() - 1] = t;
                next_issue += b;
                idle[0]--;
                if (n_stages > 1) slots_used[0]++;
                evq.push({t + service(0, b), 0, seq++, (int64_t)batches.size() - 1});
                progress = true;
            }
        }
        // Next event: a finish, an arrival, or the oldest waiting query's deadline.
        double t_next = INFINITY;
        if (!evq.empty()) t_next = evq.top().t;
        if (next_arr < nq) t_next = std::min(t_next, arr[next_arr]);
        if (next_issue < next_arr && idle[0] > 0 && out_slot_free(0))
            t_next = std::min(t_next, arr[next_issue] + wait_bound(next_arr - next_issue));
        if (!(t_next < INFINITY)) break;  // nothing can happen: stuck (should not occur)
        t = std::max(t, t_next);
        while (next_arr < nq && arr[next_arr] <= t) next_arr++;
        while (!evq.empty() && evq.top().t <= t) {
            Ev e = evq.top();
            evq.pop();
            int s = e.stage;
            idle[s]++;
            if (s > 0) slots_used[s - 1]--;           // its input slot is released
            if (s == n_stages - 1) {
                const Batch& b = batches[e.batch];
                for (int i = 0; i < b.n; ++i) done[b.first + i] = e.t;
                completed += b.n;
            } else {
                ready[s + 1].push_back(e.batch);
            }
        }
    }
    return (int64_t)batches.size();
}

int64_t orc_simulate(const double* arr, int64_t nq, int B, double t_wait, int n_stages,
                     const int* inst, const double* tau, const int* cap, const double* mult,
                     int64_t mult_len, double* done, int32_t* batch_sizes) {
    return orc_simulate_qos(arr, nq, B, t_wait, 0.0, nullptr, n_stages, inst, tau, cap, mult, mult_len, done,
                            batch_sizes, nullptr);
}

// ---------------------------------------------------------------------------
// 4. Allocation policies (Eq. 1 and Eq. 3, Table 2) and the annealing solver
// ---------------------------------------------------------------------------
//
// Problem data, for n stages, L quota levels (quota of level l = (l+1) * unit
// SMs) and nb candidate batch sizes (index bi):
//   f[(bi*n + i)*L + l]  predicted throughput of ONE instance of stage i (qps),
//   bw[(bi*n + i)*L + l] its global-memory bandwidth demand (GB/s),
//   d[(bi*n + i)*L + l]  its duration for one batch (s),
//   mem[bi*n + i]        its global-memory footprint (bytes) at that batch size.
// Constraints (Eq. 1 with one GPU, C = 1): sum N_i p_i <= S (Constraint-1);
// sum N_i <= I and N_i >= 1 (Constraint-2; a stage with no instance serves
// nothing); sum N_i bw_i(p_i) <= BW (Constraint-3); sum N_i mem_i <= F
// (Constraint-4); sum_i d_i(p_i) <= QoS (Constraint-5, read as the sum of stage
// durations).  Policy 0 (Eq. 1) maximises min_i N_i f_i(p_i).  Policy 1 (Eq. 3)
// minimises sum N_i p_i subject to the same constraints plus
// min_i N_i f_i(p_i) >= load (the throughput requirement the low-load policy
// needs to be meaningful) and sum N_i p_i <= S.  Ties: policy 0 prefers the
// larger objective, then fewer SMs; policy 1 the fewer SMs, then larger
// throughput; then the lexicographically smallest (bi, N_1..N_n, l_1..l_n).
// Host link (optional): stages that read pinned host memory share the host
// link the way all stages share HBM; with hb[(bi*n + i)*L + l] an instance's
// host-link demand (GB/s) the same form as Constraint-3 applies to it:
// sum N_i hb_i(p_i) <= HB (Sec. 6.1 names the link's contention; Eq. 1 itself
// has no term for it).
struct OrcProblem {
    int n, L, nb, unit, S, I;
    const double *f, *bw, *d, *mem;
    double BW, F, qos, load;
    int policy;
    const double* hb = nullptr;
    double HB = 0.0;
};

static bool orc_eval(const OrcProblem& P, int bi, const int* N, const int* l, double* thr,
                     int* sms) {
    int64_t sm = 0, ninst = 0;
    double bws = 0.0, mems = 0.0, dsum = 0.0, tmin = INFINITY, hbs = 0.0;
    for (int i = 0; i < P.n; ++i) {
        if (N[i] < 1 || l[i] < 0 || l[i] >= P.L) return false;
        int64_t k = ((int64_t)bi * P.n + i) * P.L + l[i];
        sm += (int64_t)N[i] * (l[i] + 1) * P.unit;
        ninst += N[i];
        bws += N[i] * P.bw[k];
        mems += N[i] * P.mem[(int64_t)bi * P.n + i];
        dsum += P.d[k];
        if (P.hb) hbs += N[i] * P.hb[k];
        tmin = std::min(tmin, N[i] * P.f[k]);
    }
    if (sm > P.S || ninst > P.I || bws > P.BW || mems > P.F || dsum > P.qos) return false;
    if (P.hb && hbs > P.HB) return false;
    if (P.policy == 1 && tmin < P.load) return false;
    *thr = tmin;
    *sms = (int)sm;
    return true;
}

// true if candidate (thr, sms) beats the incumbent under the policy's order
// (the lexicographic tie-break comes from the enumeration order).
static bool orc_better(int policy, double thr, int sms, double bthr, int bsms) {
    if (policy == 0) {
        if (thr != bthr) return thr > bthr;
        return sms < bsms;
    }
    if (sms != bsms) return sms < bsms;
    return thr > bthr;
}

// Exhaustive enumeration.  Writes the best (bi, N[], l[]) and returns 1, or 0
// if no allocation is feasible.
static int orc_exhaustive(const OrcProblem& P, int* best_bi, int* best_N, int* best_l, double* best_thr,
                          int* best_sms);
int orc_allocate_exhaustive(int n, int L, int nb, int unit, int S, int I, const double* f,
                            const double* bw, const double* d, const double* mem, double BW,
                            double F, double qos, double load, int policy, int* best_bi,
                            int* best_N, int* best_l, double* best_thr, int* best_sms) {
    OrcProblem P{n, L, nb, unit, S, I, f, bw, d, mem, BW, F, qos, load, policy};
    return orc_exhaustive(P, best_bi, best_N, best_l, best_thr, best_sms);
}
// The same with the host-link constraint (hb as f, HB the link's budget).
int orc_allocate_exhaustive_hl(int n, int L, int nb, int unit, int S, int I, const double* f,
                               const double* bw, const double* d, const double* mem, double BW,
                               double F, double qos, double load, int policy, const double* hb,
                               double HB, int* best_bi, int* best_N, int* best_l, double* best_thr,
                               int* best_sms) {
    OrcProblem P{n, L, nb, unit, S, I, f, bw, d, mem, BW, F, qos, load, policy, hb, HB};
    return orc_exhaustive(P, best_bi, best_N, best_l, best_thr, best_sms);
}
static int orc_exhaustive(const OrcProblem& P, int* best_bi, int* best_N, int* best_l, double* best_thr,
                          int* best_sms) {
    const int n = P.n, L = P.L, nb = P.nb, unit = P.unit, S = P.S, I = P.I, policy = P.policy;
    std::vector<int> N(n, 1), l(n, 0);
    bool found = false;
    double bthr = 0.0;
    int bsms = 0;
    const int maxN = std::max(1, std::min(I, S / unit));
    for (int bi = 0; bi < nb; ++bi) {
        // Odometer over N_1..N_n (1..maxN) then l_1..l_n (0..L-1), lexicographic.
        std::fill(N.begin(), N.end(), 1);
        while (true) {
            std::fill(l.begin(), l.end(), 0);
            while (true) {
                double thr;
                int sms;
                if (orc_eval(P, bi, N.data(), l.data(), &thr, &sms) &&
                    (!found || orc_better(policy, thr, sms, bthr, bsms))) {
                    found = true;
                    bthr = thr;
                    bsms = sms;
                    *best_bi = bi;
                    std::copy(N.begin(), N.end(), best_N);
                    std::copy(l.begin(), l.end(), best_l);
                }
                int j = n - 1;
                while (j >= 0 && ++l[j] == L) { l[j] = 0; --j; }
                if (j < 0) break;
            }
            int j = n - 1;
            while (j >= 0 && ++N[j] > maxN) { N[j] = 1; --j; }
            if (j < 0) break;
        }
    }
    if (found) { *best_thr = bthr; *best_sms = bsms; }
    return found ? 1 : 0;
}

// SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): the annealer's random source.
static uint64_t splitmix64_next(uint64_t* s) {
    uint64_t z = (*s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
static double splitmix64_unit(uint64_t* s) { return (splitmix64_next(s) >> 11) * 0x1.0p-53; }

// Lexicographic order on (bi, N_1..N_n, l_1..l_n): the tie-break of both solvers.
static bool orc_key_less(int n, int bi, const int* N, const int* l, int bbi, const int* bN,
                         const int* bl) {
    if (bi != bbi) return bi < bbi;
    for (int i = 0; i < n; ++i) if (N[i] != bN[i]) return N[i] < bN[i];
    for (int i = 0; i < n; ++i) if (l[i] != bl[i]) return l[i] < bl[i];
    return false;
}

// Simulated annealing over V = [N_1..N_n, p_1..p_n] (end of Sec. 7.3): each
// iteration moves one coordinate of V by one step (an instance, or one quota
// level of `unit` SMs) to get V'; V' is dropped if it violates a constraint;
// otherwise it is accepted if it is better, or with a probability exp(gain/T)
// that shrinks as T cools geometrically by `alpha` per iteration.  The best
// state seen is kept apart from the current one.  Candidate batch sizes are
// scanned in an outer loop.  Gain scale: policy 0 divides the throughput change
// by the start state's throughput, policy 1 the SM change by S.  Start state:
// N_i = 1 at the lowest quota level, or, if that is infeasible, the first
// feasible state among up to 20000 uniformly drawn ones.
// Returns 1 if a feasible state was found.
int orc_allocate_anneal(int n, int L, int nb, int unit, int S, int I, const double* f,
                        const double* bw, const double* d, const double* mem, double BW,
                        double F, double qos, double load, int policy, int iters, double T0,
                        double alpha, uint64_t seed, int* best_bi, int* best_N, int* best_l,
                        double* best_thr, int* best_sms) {
    OrcProblem P{n, L, nb, unit, S, I, f, bw, d, mem, BW, F, qos, load, policy};
    uint64_t rs = seed;
    bool found = false;
    double bthr = 0.0;
    int bsms = 0;
    const int maxN = std::max(1, std::min(I, S / unit));
    std::vector<int> N(n), l(n), Nc(n), lc(n);
    for (int bi = 0; bi < nb; ++bi) {
        std::fill(N.begin(), N.end(), 1);
        std::fill(l.begin(), l.end(), 0);
        double thr = 0.0;
        int sms = 0;
        bool have = orc_eval(P, bi, N.data(), l.data(), &thr, &sms);
        for (int tries = 0; tries < 20000 && !have; ++tries) {
            for (int i = 0; i < n; ++i) {
                N[i] = 1 + (int)(splitmix64_next(&rs) % (uint64_t)maxN);
                l[i] = (int)(splitmix64_next(&rs) % (uint64_t)L);
            }
            have = orc_eval(P, bi, N.data(), l.data(), &thr, &sms);
        }
        if (!have) continue;
        const double scale = (policy == 0) ? std::max(thr, 1e-300) : (double)S;
        auto offer = [&](const std::vector<int>& Nv, const std::vector<int>& lv, double t_,
                         int s_) {
            bool take = !found || orc_better(policy, t_, s_, bthr, bsms) ||
                        (t_ == bthr && s_ == bsms &&
                         orc_key_less(n, bi, Nv.data(), lv.data(), *best_bi, best_N, best_l));
            if (take) {
                found = true; bthr = t_; bsms = s_; *best_bi = bi;
                std::copy(Nv.begin(), Nv.end(), best_N);
                std::copy(lv.begin(), lv.end(), best_l);
            }
        };
        offer(N, l, thr, sms);
        double T = T0;
        for (int it = 0; it < iters; ++it, T *= alpha) {
            Nc = N; lc = l;
            const int coord = (int)(splitmix64_next(&rs) % (uint64_t)(2 * n));
            const int dir = (splitmix64_next(&rs) & 1) ? 1 : -1;
            const double u = splitmix64_unit(&rs);
            if (coord < n) Nc[coord] += dir; else lc[coord - n] += dir;
            double thr2;
            int sms2;
            if (!orc_eval(P, bi, Nc.data(), lc.data(), &thr2, &sms2)) continue;
            const double gain = (policy == 0) ? (thr2 - thr) / scale : (double)(sms - sms2) / scale;
            if (gain > 0.0 || (T > 0.0 && u < std::exp(gain / T))) {
                N = Nc; l = lc; thr = thr2; sms = sms2;
                offer(N, l, thr, sms);
            }
        }
    }
    if (found) { *best_thr = bthr; *best_sms = bsms; }
    return found ? 1 : 0;
}

// Minimum number of GPUs (Eq. 2): y = max(sum_i C(i,s) / G, sum_i M(i,s) / F),
// rounded up to a whole GPU.
double orc_min_gpus(const double* C, const double* M, int n, double G, double F) {
    double c = 0.0, m = 0.0;
    for (int i = 0; i < n; ++i) { c += C[i]; m += M[i]; }
    return std::ceil(std::max(c / G, m / F));
}

// ---------------------------------------------------------------------------
// 5. Latency predictor (Sec. 7.1; an MLP stands in for the decision tree)
// ---------------------------------------------------------------------------
//
// Network 12 -> 64 -> 64 -> 1: h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2),
// y = W3 h2 + b3.  Flat parameter vector, in order: W1 [64x12 row-major], b1
// [64], W2 [64x64], b2 [64], W3 [1x64], b3 [1] (5057 values).  relu'(0) = 0.
enum { PR_IN = 12, PR_H = 64 };
static const int64_t PR_NPARAM = PR_H * PR_IN + PR_H + PR_H * PR_H + PR_H + PR_H + 1;

int64_t orc_pred_nparams(void) { return PR_NPARAM; }

void orc_pred_forward(const double* th, const double* X, int64_t n, double* y) {
    const double *W1 = th, *b1 = W1 + PR_H * PR_IN, *W2 = b1 + PR_H, *b2 = W2 + PR_H * PR_H,
                 *W3 = b2 + PR_H, *b3 = W3 + PR_H;
    double h1[PR_H], h2[PR_H];
    for (int64_t q = 0; q < n; ++q) {
        const double* x = X + q * PR_IN;
        for (int j = 0; j < PR_H; ++j) {
            double s = b1[j];
            for (int k = 0; k < PR_IN; ++k) s += W1[j * PR_IN + k] * x[k];
            h1[j] = s > 0 ? s : 0;
        }
        for (int j = 0; j < PR_H; ++j) {
            double s = b2[j];
            for (int k = 0; k < PR_H; ++k) s += W2[j * PR_H + k] * h1[k];
            h2[j] = s > 0 ? s : 0;
        }
        double s = b3[0];
        for (int k = 0; k < PR_H; ++k) s += W3[k] * h2[k];
        y[q] = s;
    }
}

// Mean-squared-error loss L = (1/n) sum_q (y_q - t_q)^2 and its gradient with
// respect to every parameter (backpropagation through the three layers).
double orc_pred_grad(const double* th, const double* X, const double* t, int64_t n,
                     double* g) {
    const double *W1 = th, *b1 = W1 + PR_H * PR_IN, *W2 = b1 + PR_H, *b2 = W2 + PR_H * PR_H,
                 *W3 = b2 + PR_H, *b3 = W3 + PR_H;
    double *gW1 = g, *gb1 = gW1 + PR_H * PR_IN, *gW2 = gb1 + PR_H, *gb2 = gW2 + PR_H * PR_H,
           *gW3 = gb2 + PR_H, *gb3 = gW3 + PR_H;
    std::fill(g, g + PR_NPARAM, 0.0);
    double loss = 0.0;
    double a1[PR_H], h1[PR_H], a2[PR_H], h2[PR_H], dh2[PR_H], da2[PR_H], dh1[PR_H], da1[PR_H];
    for (int64_t q = 0; q < n; ++q) {
        const double* x = X + q * PR_IN;
        for (int j = 0; j < PR_H; ++j) {
            double s = b1[j];
            for (int k = 0; k < PR_IN; ++k) s += W1[j * PR_IN + k] * x[k];
            a1[j] = s; h1[j] = s > 0 ? s : 0;
        }
        for (int j = 0; j < PR_H; ++j) {
            double s = b2[j];
            for (int k = 0; k < PR_H; ++k) s += W2[j * PR_H + k] * h1[k];
            a2[j] = s; h2[j] = s > 0 ? s : 0;
        }
        double y = b3[0];
        for (int k = 0; k < PR_H; ++k) y += W3[k] * h2[k];
        double r = y - t[q];
        loss += r * r;
        double dy = 2.0 * r / (double)n;
        gb3[0] += dy;
        for (int k = 0; k < PR_H; ++k) { gW3[k] += dy * h2[k]; dh2[k] = dy * W3[k]; }
        for (int j = 0; j < PR_H; ++j) da2[j] = a2[j] > 0 ? dh2[j] : 0.0;
        for (int k = 0; k < PR_H; ++k) dh1[k] = 0.0;
        for (int j = 0; j < PR_H; ++j) {
            gb2[j] += da2[j];
            for (int k = 0; k < PR_H; ++k) {
                gW2[j * PR_H + k] += da2[j] * h1[k];
                dh1[k] += W2[j * PR_H + k] * da2[j];
            }
        }
        for (int j = 0; j < PR_H; ++j) da1[j] = a1[j] > 0 ? dh1[j] : 0.0;
        for (int j = 0; j < PR_H; ++j) {
            gb1[j] += da1[j];
            for (int k = 0; k < PR_IN; ++k) gW1[j * PR_IN + k] += da1[j] * x[k];
        }
    }
    return loss / (double)n;
}

// One Adam step (Kingma & Ba 2015) on every parameter, step number t >= 1:
// m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2; th -= lr * (m / (1-b1^t)) /
// (sqrt(v / (1-b2^t)) + eps).
void orc_adam_step(double* th, const double* g, double* m, double* v, int64_t np, int t,
                   double lr, double b1, double b2, double eps) {
    const double c1 = 1.0 - std::pow(b1, t), c2 = 1.0 - std::pow(b2, t);
    for (int64_t i = 0; i < np; ++i) {
        m[i] = b1 * m[i] + (1.0 - b1) * g[i];
        v[i] = b2 * v[i] + (1.0 - b2) * g[i] * g[i];
        th[i] -= lr * (m[i] / c1) / (std::sqrt(v[i] / c2) + eps);
    }
}

}  // extern "C"
