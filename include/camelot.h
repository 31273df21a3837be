/*
 * camelot.h -- C ABI of libcamelot.so, a B300-native (sm_103a) runtime for
 * multi-stage GPU microservice query pipelines in the manner of Camelot
 * (Zhang et al., "Towards QoS-Aware and Resource-Efficient GPU Microservices
 * Based on Spatial Multitasking GPUs In Datacenters").
 *
 * What the library does, in the paper's terms:
 *   - Each microservice stage runs as instances that own a fixed number of SMs
 *     (the SM quota p_i of Table 2; instances N_i), all inside ONE persistent
 *     cooperative kernel whose CTAs are partitioned into stage instances, one
 *     CTA per SM.  This replaces the MPS quotas of Sec. 5.2 step 5.
 *   - Stage i hands a batch to stage i+1 through device global memory: a ring
 *     slot plus an acquire/release sequence flag; the consumer reads the slot
 *     in place (the global-memory-based communication of Sec. 6.2).  The
 *     comparison arm copies every handoff device -> pinned host -> device (the
 *     default main-memory mechanism of Sec. 4.2 and Sec. 6.1).
 *   - Queries wait in a queue and are batched when B of them wait or when the
 *     oldest would otherwise pass the QoS bound, given the predicted latency
 *     of the batch, or has waited a fixed bound (Sec. 5.2 steps 1-2).
 *   - camelot_allocate solves the peak-load policy (Eq. 1) and the low-load
 *     resource policy (Eq. 3) over instance counts and SM quotas.
 *
 * Conventions (all entry points):
 *   - Every call returns a camelot_status; nothing throws across the ABI.  On
 *     error no partial effect is left behind unless stated, and
 *     camelot_last_error() returns a thread-local message.
 *   - Pointers documented as "device" must be device (or managed) memory of the
 *     current CUDA device; "host" pointers are ordinary host memory.  The
 *     library never takes ownership of caller memory.
 *   - A pipeline is driven by one submitting thread and one polling thread at
 *     most (they may be the same thread).
 *   - The library prints nothing; it allocates device memory only inside
 *     camelot_stage_prepare, camelot_pipeline_create, camelot_predictor_create,
 *     camelot_corunner_start, camelot_xring_create / open, camelot_server_create
 *     and camelot_fp8_scale (a 4-byte result word).
 */
#ifndef CAMELOT_H_
#define CAMELOT_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */
typedef enum {
    CAMELOT_OK = 0,
    CAMELOT_EINVAL = 1,      /* bad argument (message says which)                        */
    CAMELOT_ENOMEM = 2,      /* device or pinned host allocation failed                  */
    CAMELOT_EAGAIN = 3,      /* back-pressure: the query ring is full; nothing was queued */
    CAMELOT_ETIMEDOUT = 4,   /* a bounded wait (device or host) gave up                  */
    CAMELOT_ECUDA = 5,       /* a CUDA runtime/driver call failed                         */
    CAMELOT_ESTATE = 6,      /* the pipeline is in an error state or the call is out of order */
    CAMELOT_EINFEASIBLE = 7  /* camelot_allocate: no allocation satisfies the constraints */
} camelot_status;

/* Thread-local description of the last failure on this thread ("" if none). */
const char* camelot_last_error(void);

/* Library version as an integer (major * 10000 + minor * 100 + patch). */
int camelot_version(void);

/* ------------------------------------------------------------- stages */
/* Stage kinds.  The synthetic microservices stand in for the suite of
 * Sec. 3 (Table 1); their definitions are the workload configurations:
 *   NORMALIZE_U8   : u8 image [H][W][C] (HWC) -> f32 [H*W*C], y = (x - 127.5) / 64.
 *   NORM_POOL2_BF16: u8 image [H][W][C] -> bf16 [H/2][W/2][C], y = rne_bf16(
 *                    (mean of the 2x2 block - 127.5) / 64).  H, W even.
 *   MLP_FP32       : f32 rows -> chain of FP32 dense layers y = act(W x) (no
 *                    bias), then, if top_k > 0, the top-k indices/values of the
 *                    last layer (top_k = 1 is argmax; ties -> lowest index).
 *                    FP32 FFMA arithmetic, no TF32.
 *   GEMM_BF16      : bf16 rows -> chain of dense layers on the tensor cores
 *                    (bf16 operands, f32 accumulation in TMEM), each layer's
 *                    output rounded to bf16 after its activation, except the
 *                    last layer of a final (top_k > 0) stage, whose f32 output
 *                    feeds the top-k.  Widths dims[0..L-1] multiples of 64.
 *   GEMM_FP8       : e4m3 rows -> the same chain with OCP FP8 E4M3 operands and
 *                    per-tensor scales, f32 accumulation.  Layer l's input code c
 *                    stands for c * scales[l]; its weights are quantised at
 *                    prepare time to e4m3(w / s_w), s_w = max|W_l| / 448 (f32),
 *                    rounding to nearest even, saturating; its output value is
 *                    act(acc * f32(s_w * scales[l])), stored as the code
 *                    e4m3(value / scales[l+1]) for hidden layers (and for the
 *                    last layer of an intermediate stage, with scales[L]), f32
 *                    for the last layer of a final stage.  Widths dims[0..L-1]
 *                    multiples of 128; batches of at most 32.
 *   NORMALIZE_U8_E4M3: u8 image -> e4m3 codes of 128 y (y as NORMALIZE_U8), i.e.
 *                    e4m3(2 x - 255): the next stage reads them with scale 1/128.
 *   EMBED_GATHER   : int32 token IDs [T] -> bf16 rows [T][D], row t = E[tok[t]] for
 *                    0 <= tok < V and zero for any other ID (padding).  dims =
 *                    {V, D, T}, D a multiple of 8; weights[0] = E, bf16 [V][D].
 *   COMPUTE_SYNTH  : artifact compute-intensive stage (the c_i of Sec. 2.3 and
 *                    Sec. 8.5): f32 rows of W -> f32 rows of W, y_j = the n-th
 *                    iterate of y <- fma(y, 127/128, x_j / 128) from y = 0 (n FMA
 *                    steps per value, each rounded once in f32; the exact value
 *                    is x_j (1 - (127/128)^n)).  dims = {W, n}, W a multiple of 4.
 *   STREAM_SYNTH   : artifact memory- or host-link-intensive stage (m_i, p_i):
 *                    f32 rows of W -> f32 rows of W, y_j = x_j + T[b + j] +
 *                    T[b + W + j] + ... (R / W terms, added left to right in f32)
 *                    over the table T of L f32 values in weights[0]: device
 *                    memory for m_i, pinned host memory mapped into the device
 *                    (cudaHostAllocMapped) for p_i.  The window start b = W (h mod
 *                    (L / W - R / W + 1)), h = the high 32 bits of the 64-bit
 *                    product bits(x_0) * 0x9E3779B97F4A7C15.  dims = {W, R, L}, W
 *                    a multiple of 4, R and L multiples of W, R <= L.  The table
 *                    is NOT copied: it must stay valid while the stage exists.
 * COMPUTE_SYNTH and STREAM_SYNTH may be final (top_k > 0: top-k of the row).
 * Token-level tensor-core stages: a GEMM_BF16 / GEMM_FP8 stage with
 * rows_per_query T > 1 treats each query as T rows (its input row is T x
 * dims[0] elements) and runs the dense chain on every row; a final such stage
 * must have top_k = 1 and emits the argmax of every row (a tag per token):
 * result arrays hold the tags and maxima of the first min(T, 5) rows, and the
 * logits output / logits_sink row of a query holds its T tags as int32. */
typedef enum {
    CAMELOT_STAGE_NORMALIZE_U8 = 1,
    CAMELOT_STAGE_NORM_POOL2_BF16 = 2,
    CAMELOT_STAGE_MLP_FP32 = 3,
    CAMELOT_STAGE_GEMM_BF16 = 4,
    CAMELOT_STAGE_GEMM_FP8 = 5,
    CAMELOT_STAGE_NORMALIZE_U8_E4M3 = 6,
    CAMELOT_STAGE_EMBED_GATHER = 7,
    CAMELOT_STAGE_COMPUTE_SYNTH = 8,
    CAMELOT_STAGE_STREAM_SYNTH = 9
} camelot_stage_kind;

typedef enum { CAMELOT_ACT_NONE = 0, CAMELOT_ACT_RELU = 1, CAMELOT_ACT_GELU = 2 } camelot_act;

#define CAMELOT_MAX_LAYERS 4
#define CAMELOT_MAX_STAGES 8
#define CAMELOT_MAX_TOPK 5

typedef struct {
    int32_t kind;                       /* camelot_stage_kind                              */
    int32_t n_layers;                   /* dense kinds: 1..CAMELOT_MAX_LAYERS; else 0       */
    int32_t dims[CAMELOT_MAX_LAYERS + 1]; /* dense: dims[0] = input width, dims[l+1] = width
                                           after layer l.  Image kinds: {H, W, C, 0, 0}.   */
    int32_t act[CAMELOT_MAX_LAYERS];    /* dense: camelot_act per layer                     */
    int32_t top_k;                      /* 0: the stage's output rows go to the next stage;
                                           1..CAMELOT_MAX_TOPK: final stage, emits top-k   */
    int32_t max_batch;                  /* largest batch the stage must accept (1..256)    */
    const void* weights[CAMELOT_MAX_LAYERS]; /* dense: device pointers, row-major
                                           [dims[l+1]][dims[l]], f32 for MLP_FP32 and GEMM_FP8,
                                           bf16 for GEMM_BF16.  Read once by
                                           camelot_stage_prepare. */
    float scales[CAMELOT_MAX_LAYERS + 1]; /* GEMM_FP8 only (> 0): scales[l] is the scale of
                                           layer l's input codes; scales[n_layers] that of
                                           an intermediate stage's output codes (static
                                           scales, calibrated by the caller) */
    int32_t rows_per_query;             /* tensor-core kinds: rows per query (0 or 1 = one;
                                           T > 1 = token-level, see above); else 0 */
    int32_t ring_slots;                 /* tensor-core kinds: slots of the bulk-copy ring that
                                           streams weight and operand tiles (0 = as many as
                                           fit in shared memory, at most 5; 2..5 = at most
                                           that many).  Results do not depend on it.  Other
                                           kinds: 0.  EINVAL outside these values. */
} camelot_stage_desc;

/* A prepared stage: validated descriptor plus the library's own copy of its
 * weights in the layout its kernels read (one copy per stage, shared by every
 * instance of the stage, as in Sec. 7.4's weight sharing). */
typedef struct camelot_stage camelot_stage;

/* Validate `desc` and copy its weights into kernel layout (device memory owned
 * by the returned object).  The caller's weight buffers may be freed after the
 * call returns.  Errors: EINVAL (shape/kind), ENOMEM, ECUDA. */
camelot_status camelot_stage_prepare(const camelot_stage_desc* desc, camelot_stage** out);
camelot_status camelot_stage_release(camelot_stage* st);

/* The weights of tensor-core layer l as the stage's kernels use them, row-major
 * [dims[l+1]][dims[l]] element codes (bf16 bit patterns for GEMM_BF16, e4m3
 * codes for GEMM_FP8) written to host memory `out` of `bytes` bytes (exactly
 * rows x columns x element size), and (nullable) the weight scale s_w (1 for
 * bf16).  Errors: EINVAL (not a tensor-core stage, bad layer or size), ECUDA. */
camelot_status camelot_stage_export_weights(const camelot_stage* st, int layer, void* out, size_t bytes,
                                            float* weight_scale);

/* Static activation scale of an FP8 layer input (the calibration of the FP8
 * arm): *scale = f32(max |x| / 448) over the n f32 values at x (device),
 * computed by a reduction kernel on `stream` (NULL = legacy default stream);
 * the call waits for it.  448 is the largest finite E4M3 magnitude, so the
 * calibration values map onto the code range.  Errors: EINVAL (null pointer,
 * n = 0, a maximum that is zero or infinite), ENOMEM, ECUDA. */
camelot_status camelot_fp8_scale(const float* x, size_t n, void* stream, float* scale);

/* Row sizes in bytes of one query's input and output for the stage (output
 * bytes are 0 for a final stage), and the device scratch bytes a direct launch
 * of `n` rows needs. */
camelot_status camelot_stage_info(const camelot_stage* st, size_t* in_row_bytes,
                                  size_t* out_row_bytes, uint32_t n, size_t* scratch_bytes);

/* Direct, non-persistent launch of one stage on `n_ctas` CTAs (one per SM; the
 * SM quota) over a batch of n rows -- the same device code the pipeline runs
 * per batch.  Asynchronous on `stream` (a cudaStream_t; NULL = legacy default
 * stream).
 *   in      device, n * in_row_bytes, rows contiguous.
 *   out     device, n * out_row_bytes (intermediate stages), else may be NULL.
 *   out_idx device int32 [n][k] (final stages), else NULL; k = top_k, or
 *           min(T, 5) for a token-level stage.
 *   out_val device f32   [n][k] (final stages), else NULL.
 *   out_logits device f32 [n][dims[n_layers]] or NULL: the final layer's
 *           output before top-k (dense kinds only); int32 [n][T] tags for a
 *           token-level stage.
 *   scratch device, >= camelot_stage_info(...) bytes, 256-byte aligned; the
 *           call clears what must start at zero.
 * Errors: EINVAL (n = 0 or > max_batch, n_ctas outside 1..SM count, missing
 * buffer), ECUDA (launch failure). */
camelot_status camelot_stage_launch(const camelot_stage* st, int n_ctas, const void* in,
                                    uint32_t n, void* out, int32_t* out_idx, float* out_val,
                                    float* out_logits, void* scratch, size_t scratch_bytes,
                                    void* stream);

/* Allocation-free form of camelot_stage_launch (the paper has no counterpart;
 * it serves callers of this library that cannot allocate device memory at the
 * point where they run a stage: an application whose memory manager owns the
 * whole device pool, a serving loop that cannot afford the latency or the
 * device-wide synchronisation of cudaMalloc/cudaFree mid-request, or a
 * plug-in that is only handed its input and output buffers).  Same arguments
 * and results as camelot_stage_launch, minus the scratch, for every stage kind
 * except the tensor-core ones (GEMM_BF16, GEMM_FP8: refused with EINVAL; use
 * camelot_stage_launch).  The stage's scratch lives in a static 16 MiB device
 * array that every GPU loading the library holds until the process exits.
 * Nothing is allocated by this call.
 *   - The first call on a device (with that device current) looks up the
 *     array's device address and sets the kernel's shared-memory limit; make
 *     that first call before any stream capture.  The address is kept for the
 *     life of the process: do not use this call after a cudaDeviceReset.
 *   - Every call on a device shares the one array and leaves its contents
 *     behind; the call clears the part that must start at zero.  Calls whose
 *     kernels overlap on the GPU (other streams, other host threads) race on
 *     the array and give wrong results: order them on one stream.
 *   - If a wait inside the kernel gives up (2 s), the call's outputs are
 *     overwritten with a failure pattern once every CTA is done: final
 *     stages get -1 in every out_idx entry and NaN in out_val and out_logits;
 *     intermediate stages get 0xFF in every output byte (NaN in f32, bf16 and
 *     e4m3).  After synchronising the stream, a negative index or a NaN says
 *     the call failed.
 *   - Errors: EINVAL when the batch needs more than the 16 MiB (the FP32 stage
 *     of the plain 2-stage pipeline needs about 37 KB per query and fits at
 *     every batch it accepts; very wide layers may not) or the stage is a
 *     tensor-core stage, plus those of camelot_stage_launch. */
camelot_status camelot_stage_launch_noalloc(const camelot_stage* st, int n_ctas, const void* in,
                                            uint32_t n, void* out, int32_t* out_idx,
                                            float* out_val, float* out_logits, void* stream);

/* Profiling of one stage (Sec. 7.1: the allocator's inputs are measured by
 * running each microservice alone under a given SM percentage and batch):
 * issue `runs` back-to-back camelot_stage_launch calls with the same arguments
 * on `stream`, with a CUDA event between consecutive launches, wait for them,
 * and write each launch's event-to-event duration in milliseconds to ms_out
 * (host, [runs]).  runs in 1..65536.  Errors: those of camelot_stage_launch,
 * ECUDA. */
camelot_status camelot_stage_time(const camelot_stage* st, int n_ctas, const void* in, uint32_t n,
                                  void* out, int32_t* out_idx, float* out_val, float* out_logits,
                                  void* scratch, size_t scratch_bytes, void* stream, uint32_t runs,
                                  float* ms_out);

/* Bandwidth-hog co-runner for profiling under memory contention (the
 * co-location interference of Sec. 4.2 and the bandwidth term of Eq. 1):
 * a kernel of n_ctas CTAs, one per SM (each reserves 120 KB of shared memory,
 * so no stage CTA can share its SM), that streams `bytes` (rounded down to a
 * multiple of 16) from src to dst (device, 16-byte aligned, not overlapping)
 * pass after pass until camelot_corunner_stop, or until max_ns nanoseconds
 * have passed (its own deadline, so it always ends).  Returns once every CTA is
 * resident (ETIMEDOUT, with the kernel stopped, if that takes over 5 s), so a
 * stage launched afterwards gets the other SMs.  n_ctas in 1..SM count, at most
 * 256.  The caller keeps src and dst alive until stop returns. */
typedef struct camelot_corunner camelot_corunner;
camelot_status camelot_corunner_start(const void* src, void* dst, size_t bytes, int n_ctas,
                                      int64_t max_ns, camelot_corunner** out);
/* Stop the co-runner, wait for it, free it, and report (nullable) the bytes it
 * moved (read + written, full passes) per second of its run, in GB/s.  Returns
 * ETIMEDOUT if it had already stopped at its own deadline (c is freed either
 * way). */
camelot_status camelot_corunner_stop(camelot_corunner* c, double* gbytes_per_s);

/* ------------------------------------------------------- latency predictor */
/* A learned stand-in for the per-microservice performance models of Sec. 7.1
 * (which are decision trees there): an MLP 12 -> 64 -> 64 -> 1 in FP32 with
 * ReLU hidden layers and a linear output, h1 = relu(W1 x + b1), h2 = relu(W2 h1
 * + b2), y = W3 h2 + b3, where x is the feature vector z-scored with the stored
 * mean and inverse standard deviation.  Parameters are one flat FP32 vector of
 * CAMELOT_PRED_PARAMS values in the order W1 [64x12 row-major], b1 [64], W2
 * [64x64], b2 [64], W3 [64], b3 [1].  Training minimises the mean squared error
 * (1/n) sum_q (y_q - t_q)^2 with Adam (beta1 0.9, beta2 0.999, eps 1e-8).  All
 * computation runs in the library's kernels; forward, grad and train_step are
 * asynchronous on `stream`, and calls on one predictor must be ordered on one
 * stream (they share its device scratch). */
#define CAMELOT_PRED_FEATURES 12
#define CAMELOT_PRED_PARAMS 5057
typedef struct camelot_predictor camelot_predictor;

/* Allocate a predictor on the current device with parameters init_params
 * (host, CAMELOT_PRED_PARAMS floats), zero Adam moments, identity feature
 * scaling (mean 0, inv_std 1).  Holds ~71 MB of device scratch for minibatches
 * of up to 65536 samples.  Errors: EINVAL, ENOMEM, ECUDA. */
camelot_status camelot_predictor_create(const float* init_params, camelot_predictor** out);
/* Replace the parameters (host) and reset the Adam moments and step count.
 * Synchronous. */
camelot_status camelot_predictor_set_params(camelot_predictor* p, const float* params);
/* Copy the parameters to host memory (CAMELOT_PRED_PARAMS floats).  The caller
 * first synchronises the stream its training ran on. */
camelot_status camelot_predictor_get_params(camelot_predictor* p, float* out);
/* Feature scaling applied by later launches: x_k = (raw_k - mean[k]) *
 * inv_std[k] (host arrays of CAMELOT_PRED_FEATURES floats). */
camelot_status camelot_predictor_set_norm(camelot_predictor* p, const float* mean, const float* inv_std);
/* y[q] = network(X[q]) for q < n.  X: device [n][12] row-major raw features;
 * y: device [n].  Errors: EINVAL (null pointer, n = 0), ECUDA. */
camelot_status camelot_predictor_forward(camelot_predictor* p, const float* X, uint32_t n, float* y,
                                         void* stream);
/* Gradient of the mean squared error over a minibatch of n samples (1..65536)
 * with respect to every parameter: sample q is row idx[q] of X and t (device
 * uint32 [n]; NULL = rows 0..n-1).  X: device [rows][12]; t: device [rows]
 * targets; grad: device [CAMELOT_PRED_PARAMS]; loss (device float, nullable)
 * receives the minibatch loss.  Each gradient is summed over the samples in
 * minibatch order, so the result is deterministic.  Errors: EINVAL, ECUDA. */
camelot_status camelot_predictor_grad(camelot_predictor* p, const float* X, const float* t,
                                      const uint32_t* idx, uint32_t n, float* grad, float* loss,
                                      void* stream);
/* One Adam step (step count + 1, bias corrections 1 - beta^step) on the
 * gradient camelot_predictor_grad would give for the same arguments, with
 * learning rate lr > 0.  loss (device, nullable) receives the minibatch loss
 * before the step. */
camelot_status camelot_predictor_train_step(camelot_predictor* p, const float* X, const float* t,
                                            const uint32_t* idx, uint32_t n, float lr, float* loss,
                                            void* stream);
camelot_status camelot_predictor_destroy(camelot_predictor* p);

/* Algorithmic work of one stage, the inputs of the predictor's features and
 * of the allocator's bandwidth and memory terms (Table 2: C(i,s) FLOPs, M the
 * memory footprint). */
typedef struct {
    int32_t stage_id;        /* the stage's identity as the predictor's first feature */
    int32_t pad_;
    double flop_per_query;   /* FLOPs of one query                                   */
    double bytes_per_batch;  /* bytes read once per batch (the weights)              */
    double bytes_per_query;  /* bytes read and written per query (input + output row) */
    double mem_bytes;        /* device memory of one instance (Constraint-4's M)      */
} camelot_stage_cost;

/* Raw predictor features of n configurations (host, float [n][12], the order
 * the predictor is trained on): for stage costs[s], s = stage[r] (an index
 * into costs), batch b = batch[r], quota p = sms[r] SMs, a co-runner on c =
 * co_sms[r] SMs (0 = none) streaming g = co_gbs[r] GB/s when alone:
 *   [id, b, p, F, Y, F / Y, c, c > 0 ? g : 0, c > 0, p + c, log2 b, 1 / p]
 * with id = costs[s].stage_id,
 * F = b flop_per_query and Y = bytes_per_batch + b bytes_per_query.  The
 * paper's features are the batch size and the SM share from solo runs (Sec.
 * 7.1); the work and co-runner terms let the model see contention (Sec. 4.2).
 * Host-only.  Errors: EINVAL (null pointer, stage index, b < 1, p < 1). */
camelot_status camelot_predictor_features(const camelot_stage_cost* costs, int n_stages, uint32_t n,
                                          const int32_t* stage, const int32_t* batch, const int32_t* sms,
                                          const int32_t* co_sms, const double* co_gbs, float* X);

/* The allocator's table (Table 2 quantities) from batch latencies: for
 * lat_s[b][i][l] (host, [n_batches][n_stages][n_levels], seconds, > 0) the
 * duration d = lat_s, the throughput of one instance f = B_b / d, its
 * bandwidth demand (bytes_per_batch + B_b bytes_per_query) / d / 1e9 GB/s, and
 * mem[b][i] = costs[i].mem_bytes; outputs are host arrays of the same shapes,
 * laid out as camelot_profile expects.  Host-only.  Errors: EINVAL. */
camelot_status camelot_profile_from_latency(const camelot_stage_cost* costs, int n_stages,
                                            const int32_t* batch_sizes, int n_batches, int n_levels,
                                            const double* lat_s, double* thr, double* bw, double* dur,
                                            double* mem);

/* The performance model inside the allocator (Sec. 7.1-7.2): fills the
 * camelot_profile arrays thr, bw, dur ([n_batches][n_stages][n_levels]) and
 * mem ([n_batches][n_stages]) from the predictor's latency estimate for every
 * batch size, stage and quota level (level l = (l + 1) unit SMs), beside a
 * co-runner on co_sms SMs streaming co_gbs GB/s alone (0 = none).  The network
 * predicts log of the latency in microseconds.  Builds the features as
 * camelot_predictor_features does, runs the forward kernel on the rows in one
 * launch (in the predictor's own scratch, at most 65536 rows) and converts as
 * camelot_profile_from_latency does.  Synchronous (legacy default stream);
 * must not overlap other calls on the same predictor.  Errors: EINVAL, ECUDA. */
camelot_status camelot_profile_predict(camelot_predictor* p, const camelot_stage_cost* costs, int n_stages,
                                       const int32_t* batch_sizes, int n_batches, int unit, int n_levels,
                                       int32_t co_sms, double co_gbs, double* thr, double* bw, double* dur,
                                       double* mem);

/* ----------------------------------------------------------- pipelines */
typedef enum {
    CAMELOT_HANDOFF_GLOBAL = 0,      /* pointer + flag in device memory, no copy (Sec. 6.2) */
    CAMELOT_HANDOFF_HOST_STAGED = 1  /* D2H to pinned host, then H2D (Sec. 4.2 / 6.1)      */
} camelot_handoff;

/* Instances and SM quotas per stage: the allocation vector V of Sec. 7.3
 * ([N_1..N_n, p_1..p_n]) plus the batch size s. */
typedef struct {
    int32_t n_stages;
    int32_t instances[CAMELOT_MAX_STAGES]; /* N_i >= 1                                     */
    int32_t sm_quota[CAMELOT_MAX_STAGES];  /* p_i: SMs (= CTAs) per instance, >= 1          */
    int32_t batch;                         /* B: largest batch the trigger forms            */
} camelot_alloc;

typedef struct {
    uint32_t query_slots;   /* capacity of the query ring and of the completion ring
                               (power of two, default 65536)                          */
    uint32_t batch_slots;   /* least capacity of each inter-stage batch ring (default 8;
                               raised to 2 x the instances on both sides)              */
    int64_t max_wait_ns;    /* batch trigger: a partial batch leaves once its oldest query
                               has waited this long (default 200000)                   */
    int64_t idle_exit_ns;   /* the persistent kernel ends after this long without work;
                               the next submit or poll relaunches it (default 500 ms)  */
    int64_t wait_limit_ns;  /* every other device wait gives up after this and puts the
                               pipeline in the error state (default 2 s)               */
    float* logits_sink;     /* optional device f32 [query_slots][final width]: the final
                               layer's output of query q lands in row q % query_slots  */
    int32_t exit_after_trace; /* 1: the persistent kernel ends as soon as a trace has been
                               fully taken and drained (one launch per trace, which makes
                               the launch's CUDA-event time the trace's device time)  */
    uint32_t data_slots;    /* rows of the buffer that holds submitted query bytes
                               (power of two in 64..query_slots; 0 = query_slots).  The
                               buffer takes data_slots x the stage-0 row bytes, pinned or
                               on the device, allocated at pipeline_create: 0 with 65536
                               query slots and 150 KB rows is ~10 GB and seconds of
                               allocation; a pipeline fed only by camelot_submit_trace
                               needs the minimum, 64; one call of camelot_submit takes at
                               most data_slots queries                                    */
    int32_t device_data;    /* 0: that buffer is pinned, mapped host memory which stage 0
                               reads over the host link; 1: it is device memory which
                               camelot_submit fills with DMA copies (cudaMemcpyAsync,
                               at most two per call) and waits for before publishing   */
    /* QoS-aware batch trigger (Sec. 5.2 step 2: a partial batch leaves once its
     * first query "tends to suffer" a QoS violation).  With qos_ns > 0, a batch of
     * b < B ready queries leaves once its oldest query has waited
     *     min(max_wait_ns, qos_ns - qos_margin_ns - batch_latency_ns[b - 1])
     * (at once if that is <= 0): its wait plus the predicted latency of a b-query
     * batch through all stages would otherwise pass QoS - margin.  qos_ns = 0
     * keeps the plain max_wait_ns rule.  batch_latency_ns[b - 1] is the predicted
     * end-to-end service latency of a batch of b (b = 1..32), e.g. filled by
     * camelot_trigger_latency from the allocation's profile. */
    int64_t qos_ns;
    int64_t qos_margin_ns;
    int64_t batch_latency_ns[32];
} camelot_options;

/* Fill `o` with the defaults above (qos_ns = qos_margin_ns = 0 and a zero
 * latency table: the plain max_wait_ns trigger). */
void camelot_options_default(camelot_options* o);

typedef struct camelot_pipeline camelot_pipeline;

/* Build a pipeline of n_stages prepared stages (stage i's output row must be
 * stage i+1's input row; the last stage must have top_k > 0) with allocation
 * `alloc` (sum_i N_i * p_i must not exceed the SM count; each stage's
 * max_batch >= alloc->batch), the given handoff mode and options (NULL =
 * defaults).  Allocates the rings (device memory; the query and completion
 * rings in pinned, mapped host memory).  The persistent kernel is launched by
 * the first submit (and relaunched by any later submit or poll that finds it
 * ended).
 * The stages must outlive the pipeline.  Errors: EINVAL, ENOMEM, ECUDA. */
camelot_status camelot_pipeline_create(camelot_stage* const* stages, int n_stages,
                                       const camelot_alloc* alloc, camelot_handoff mode,
                                       const camelot_options* opts, camelot_pipeline** out);

/* Queue n queries from host memory (n * stage-0 input row bytes, rows
 * contiguous; pinned memory makes the device_data copies run at the DMA
 * engine's rate); the bytes are copied before return.  Query IDs are assigned
 * consecutively from *first_query_id (a per-pipeline counter starting at 0).
 * arrival_ns (host, nullable) gives each query's arrival stamp on the host
 * CLOCK_MONOTONIC scale; NULL stamps them with the time of the call.  All or
 * nothing: EAGAIN if fewer than n slots are free (poll to free them), ESTATE
 * if the pipeline is in the error state or a trace is running.  n = 0 queues
 * nothing, returns OK and stores the next query ID (queries may be NULL). */
camelot_status camelot_submit(camelot_pipeline* p, uint32_t stream_id, const void* queries,
                              uint32_t n, const int64_t* arrival_ns, uint64_t* first_query_id);

/* Replay an arrival trace whose queries already reside in device memory:
 * query i (bytes at queries + i * row bytes, device) arrives arrival_off_ns[i]
 * nanoseconds (device int64 array, non-decreasing) after the device starts the
 * trace; the batch trigger waits for each arrival on the device clock, so the
 * host is out of the loop.  Requires no outstanding queries and n <=
 * query_slots.  Completion stamps of trace queries are on the device clock.
 * The device buffers must stay valid until the trace's completions are polled.
 * Errors: EINVAL (null buffer, n = 0, n > query_slots), ESTATE (outstanding
 * queries / error state). */
camelot_status camelot_submit_trace(camelot_pipeline* p, uint32_t stream_id, const void* queries,
                                    uint32_t n, const int64_t* arrival_off_ns,
                                    uint64_t* first_query_id);

typedef struct {
    uint64_t query_id;
    uint32_t stream_id;
    int32_t status;                 /* 0 = ok                                            */
    int32_t idx[CAMELOT_MAX_TOPK];  /* top-k indices of the final stage (k = its top_k)   */
    float val[CAMELOT_MAX_TOPK];    /* and their values                                   */
    int32_t batch_size;             /* size of the batch the query travelled in           */
    int32_t pad_;
    int64_t t_arrival_ns;           /* submit: host clock; trace: device clock            */
    int64_t t_batch_ns;             /* device clock: batch formed by the trigger           */
    int64_t t_done_ns;              /* device clock: final stage finished                  */
    int64_t t_poll_ns;              /* host clock: when camelot_poll returned it           */
} camelot_completion;

/* Copy up to max completions, strictly in query-ID order, into out; *n_out
 * receives the count.  Waits up to timeout_us (0 = do not wait, < 0 = wait
 * without a bound) for the first completion.  Returns ETIMEDOUT only if
 * timeout_us > 0 elapsed with nothing to return; ESTATE (with the completions
 * delivered so far) if the device reported an error. */
camelot_status camelot_poll(camelot_pipeline* p, camelot_completion* out, uint32_t max,
                            uint32_t* n_out, int64_t timeout_us);

typedef struct {
    uint64_t submitted, completed;          /* query counters                            */
    uint64_t batches[CAMELOT_MAX_STAGES];   /* batches finished per stage                */
    uint64_t kernel_launches;               /* persistent-kernel launches so far          */
    uint64_t relayed_bytes;                 /* host-staged mode: bytes copied D2H + H2D   */
    uint64_t device_bytes_per_batch_slot;   /* device bytes of one inter-stage slot       */
    uint64_t device_ring_bytes;             /* device bytes held by all inter-stage rings */
    int32_t device_status, device_where;    /* first device error (0 = none)              */
    double last_launch_ms;                  /* CUDA-event duration of the last finished launch */
    double total_launch_ms;                 /* sum over finished launches                  */
    uint64_t busy_ns[CAMELOT_MAX_STAGES];   /* per stage, summed over its batches (device clock):
                                               from the instance holding a batch's work (input
                                               and output slots) to the batch published, so
                                               busy_ns / batches is the in-pipeline service time
                                               of one batch, hand-over included              */
    uint64_t body_ns[CAMELOT_MAX_STAGES];   /* per stage, summed over its batches: the time the
                                               instance's first CTA spent in the stage's own
                                               computation (busy_ns - body_ns is the batch
                                               protocol and the wait for the other CTAs)    */
    uint64_t acquire_ns[CAMELOT_MAX_STAGES];/* per stage, summed over its batches: the time its
                                               instances' leaders spent finding a batch's work
                                               (for stage 0 the batch trigger, which includes
                                               waiting for arrivals; for later stages waiting
                                               for a published input batch)                  */
} camelot_stats;

camelot_status camelot_pipeline_stats(camelot_pipeline* p, camelot_stats* out);

/* Fault injection on the host, for tests of the device-side timeouts: while
 * `stall` is non-zero the relay thread of a host-staged pipeline copies no
 * batch, as if the host link had stopped.  Producers then find no free slot
 * downstream; their bounded waits give up after wait_limit_ns and the
 * pipeline enters the error state (later calls return ESTATE; destroy stays
 * clean).  Nothing is faulted on the GPU.  Errors: EINVAL (null pipeline, not
 * host-staged). */
camelot_status camelot_pipeline_stall_relay(camelot_pipeline* p, int stall);

/* Stop the persistent kernel (it exits at its next check), wait for it and
 * free every resource.  Completions not yet polled are dropped. */
camelot_status camelot_pipeline_destroy(camelot_pipeline* p);

/* -------------------------------------------------------- serving loop */
/* A serving loop over several pipelines sharing the GPU, with admission by
 * device memory (Sec. 5.1: a query is started only once the memory it needs is
 * free; services are co-located, Sec. 4.2).  camelot_server_submit queues
 * queries per pipeline in pinned host memory and returns at once; one server
 * thread admits them in FIFO order per pipeline, round robin over pipelines, at
 * most max_admit at a time, while the query bytes in flight on the device (all
 * pipelines) stay within device_bytes_budget and the pipeline has ring room,
 * by camelot_submit (so each pipeline should use device_data = 1: the admitted
 * bytes then live in its device data ring); it polls every pipeline and keeps
 * the completions for camelot_server_poll.  Batching happens on the device, per
 * pipeline, over whatever has been admitted.  The server is the only thread
 * that may submit to or poll its pipelines while it exists; the pipelines
 * (caller-owned) must outlive it. */
#define CAMELOT_MAX_SERVER_PIPELINES 16
typedef struct camelot_server camelot_server;
typedef struct {
    uint64_t device_bytes_budget;  /* query bytes in flight on the device, all pipelines
                                      (0 = no limit beyond the rings)               */
    uint32_t host_queue_queries;   /* host queue capacity per pipeline (default 4096)  */
    uint32_t max_admit;            /* queries admitted per pipeline per round (64)     */
} camelot_server_options;
typedef struct {
    uint64_t submitted, admitted, completed;  /* queries                               */
    uint64_t waiting;                         /* in the host queue, not yet admitted   */
    uint64_t deferred;                        /* admission rounds that found no room   */
    uint64_t inflight_bytes;                  /* this pipeline's query bytes on device */
    uint64_t peak_inflight_bytes;
    uint64_t total_inflight_bytes;            /* all pipelines                         */
    int32_t status;                           /* camelot_status of the pipeline        */
    int32_t pad_;
} camelot_lane_stats;

void camelot_server_options_default(camelot_server_options* o);
/* Errors: EINVAL (n outside 1..16, null pipeline, budget below one query),
 * ENOMEM. */
camelot_status camelot_server_create(camelot_pipeline* const* pipelines, int n,
                                     const camelot_server_options* opts, camelot_server** out);
/* Copy n queries (host, rows contiguous, the pipeline's stage-0 row bytes each)
 * into pipeline `pipeline`'s host queue with their arrival stamps (host
 * CLOCK_MONOTONIC ns; NULL = now).  All or nothing: EAGAIN if the host queue
 * lacks room; ESTATE if the pipeline failed. */
camelot_status camelot_server_submit(camelot_server* s, int pipeline, uint32_t stream_id,
                                     const void* queries, uint32_t n, const int64_t* arrival_ns);
/* Up to max completions of `pipeline`, in query-ID order; waits up to
 * timeout_us for the first (0 = no wait, < 0 = no bound).  ETIMEDOUT if
 * timeout_us > 0 passed with nothing; ESTATE if the pipeline failed. */
camelot_status camelot_server_poll(camelot_server* s, int pipeline, camelot_completion* out,
                                   uint32_t max, uint32_t* n_out, int64_t timeout_us);
camelot_status camelot_server_stats(camelot_server* s, int pipeline, camelot_lane_stats* out);
/* Stop the server thread and free the queues (queued, unadmitted queries are
 * dropped; admitted ones stay in their pipelines). */
camelot_status camelot_server_destroy(camelot_server* s);

/* ------------------------------------------------------- cross-process ring */
/* Handoff between stages that run in different processes (the paper's
 * deployment, Sec. 6.2: each microservice is a process and the next stage maps
 * the previous one's global-memory output through a CUDA IPC handle).  A ring
 * of `slots` device buffers of `slot_bytes` each, created by the producer
 * process, mapped by the consumer process through cudaIpcOpenMemHandle, and
 * two inter-process CUDA events per slot: ready[k] (the producer's writes to
 * slot k are done) and free[k] (the consumer's reads of slot k are done).
 * Ordering on the GPU is by stream waits on those events; no kernel ever waits
 * for another process.  The host side of each process tells the other which
 * slot it has recorded (over any host channel, e.g. a pipe): a begin call may
 * only be made after the matching end call of the other side has returned,
 * because a stream wait sees an event's most recent record.
 *   producer: produce_begin(k) -> write slot k on the stream -> produce_end(k)
 *   consumer: consume_begin(k) -> read slot k on the stream  -> consume_end(k)
 * Both sides must use the same device. */
typedef struct camelot_xring camelot_xring;
#define CAMELOT_XRING_MAX_SLOTS 64
typedef struct {
    uint64_t slot_bytes;
    uint32_t slots;
    int32_t device;
    unsigned char mem[64];                                /* cudaIpcMemHandle_t      */
    unsigned char ready[CAMELOT_XRING_MAX_SLOTS][64];     /* cudaIpcEventHandle_t    */
    unsigned char free_[CAMELOT_XRING_MAX_SLOTS][64];
} camelot_xring_handle;

/* Producer side: allocate the slots (one device allocation, 256-byte aligned
 * slots) and the events, and fill the handle to send to the consumer.  Errors:
 * EINVAL (slots outside 1..64, slot_bytes 0), ENOMEM, ECUDA. */
camelot_status camelot_xring_create(uint64_t slot_bytes, uint32_t slots, camelot_xring** out,
                                    camelot_xring_handle* handle);
/* Consumer side (another process): map the slots and open the events.
 * Errors: EINVAL (malformed handle, other device), ECUDA (the handle does not
 * open in this process, e.g. the creating process itself). */
camelot_status camelot_xring_open(const camelot_xring_handle* handle, camelot_xring** out);
/* Device address of slot k (NULL for k out of range). */
void* camelot_xring_slot(const camelot_xring* x, uint32_t k);
/* Stream-ordered begin / end of one side's use of slot k (`stream` is a
 * cudaStream_t; NULL = legacy default stream).  produce_begin waits for
 * free[k], produce_end records ready[k]; consume_begin waits for ready[k],
 * consume_end records free[k].  Errors: EINVAL (k, wrong side), ECUDA. */
camelot_status camelot_xring_produce_begin(camelot_xring* x, uint32_t k, void* stream);
camelot_status camelot_xring_produce_end(camelot_xring* x, uint32_t k, void* stream);
camelot_status camelot_xring_consume_begin(camelot_xring* x, uint32_t k, void* stream);
camelot_status camelot_xring_consume_end(camelot_xring* x, uint32_t k, void* stream);
/* Unmap (consumer) or free (producer, after the consumer has closed) the ring
 * and its events. */
camelot_status camelot_xring_destroy(camelot_xring* x);

/* ------------------------------------------------------------ allocator */
typedef enum {
    CAMELOT_POLICY_MAX_PEAK = 0,  /* Eq. 1: maximise min_i N_i f_i(p_i)                   */
    CAMELOT_POLICY_MIN_SM = 1     /* Eq. 3: minimise sum_i N_i p_i at the given load      */
} camelot_policy;

typedef enum {
    CAMELOT_SOLVER_EXHAUSTIVE = 0, /* enumerate every (batch, N, p): exact                */
    CAMELOT_SOLVER_ANNEAL = 1      /* simulated annealing over V (end of Sec. 7.3)        */
} camelot_solver;

/* Per-instance performance table (the predicted f, g/bandwidth, duration and
 * memory of Table 2), for n_stages stages, n_levels SM-quota levels (level l
 * means (l + 1) * unit SMs) and n_batches candidate batch sizes.  Arrays are
 * row-major [n_batches][n_stages][n_levels] (mem: [n_batches][n_stages]). */
typedef struct {
    int32_t n_stages, n_levels, n_batches, unit;
    const int32_t* batch_sizes;  /* [n_batches]                                          */
    const double* thr_qps;       /* f_i(p): queries/s of ONE instance                    */
    const double* bw_gbs;        /* its global-memory bandwidth demand, GB/s            */
    const double* dur_s;         /* its duration for one batch, s                        */
    const double* mem_bytes;     /* its global-memory footprint, bytes                   */
    const double* host_gbs;      /* its host-link bandwidth demand, GB/s (stages reading
                                    pinned host memory); NULL = none for every stage      */
} camelot_profile;

typedef struct {
    int32_t total_sms;      /* S (C * R with C = 1 GPU)                                   */
    int32_t max_instances;  /* I: most instances in total                                 */
    double bw_gbs;          /* BW: bandwidth budget (Constraint-3)                        */
    double mem_bytes;       /* F: memory budget (Constraint-4)                            */
    double qos_s;           /* QoS bound on the sum of stage durations (Constraint-5)     */
    double load_qps;        /* MIN_SM only: throughput the allocation must sustain        */
    int32_t solver;         /* camelot_solver                                              */
    int32_t anneal_iters;   /* annealing: iterations per batch size (default 5000 if 0)   */
    double anneal_t0;       /* initial temperature (relative; default 1.0 if 0)           */
    double anneal_alpha;    /* geometric cooling factor (default 0.995 if 0)              */
    uint64_t seed;          /* annealing random stream (SplitMix64)                        */
    double host_gbs;        /* host-link budget, Constraint-3's form applied to the link
                               that host-memory stages share (0 = no budget)              */
} camelot_constraints;

/* Solve the chosen policy.  On success fills out (n_stages, instances,
 * sm_quota, batch = batch_sizes[chosen]) and *objective (the min-throughput for
 * MAX_PEAK, the SM count for MIN_SM).  Constraints: sum N_i p_i <= S, sum N_i <=
 * I, N_i >= 1, sum N_i bw_i <= BW, sum N_i mem_i <= F, sum_i dur_i <= QoS, when
 * both prof->host_gbs and c->host_gbs are given sum N_i host_i <= c->host_gbs,
 * and for MIN_SM min_i N_i f_i >= load.  Ties: better objective, then fewer SMs (MAX_PEAK)
 * or higher throughput (MIN_SM), then the lexicographically smallest
 * (batch index, N, level).  Errors: EINVAL, EINFEASIBLE.  Host-only; no GPU use. */
camelot_status camelot_allocate(const camelot_profile* prof, camelot_policy policy,
                                const camelot_constraints* c, camelot_alloc* out,
                                double* objective);

/* Predicted end-to-end service latency of a batch of b queries (b = 1..32)
 * through the stages of `alloc` at their allocated quotas, for the QoS-aware
 * batch trigger (Sec. 5.2 step 2 uses the predicted latency to decide when the
 * first query is at risk): out_ns[b - 1] = sum_i dur_i(b, level_i) with level_i
 * = sm_quota[i] / unit - 1 (quotas must be multiples of the profile's unit
 * within its levels).  dur is interpolated linearly between the profile's batch
 * sizes; below the smallest one it is the smallest one's duration, above the
 * largest it grows in proportion to b.  Host-only.  Errors: EINVAL. */
camelot_status camelot_trigger_latency(const camelot_profile* prof, const camelot_alloc* alloc,
                                       int64_t* out_ns);

/* The per-batch hand-over cost of a pipeline in the allocator's table: a
 * stage inside a pipeline spends a different time per batch than when it is
 * timed alone by separate launches: the batch's work is acquired from a ring,
 * posted to the instance's CTAs, counted back and published, co-located
 * stages share the memory system, and no launch overhead is paid.  With
 * handover_s[i] the measured difference for stage i (its service time per
 * batch in a saturated pipeline -- camelot_stats.busy_ns / batches plus the
 * per-batch acquisition cost -- minus the solo duration at the same quota; it
 * may be negative), every entry becomes d' = d + handover_s[i], f' = B / d',
 * bandwidth' = bandwidth d / d' (the same bytes in the new time).  Outputs are
 * arrays shaped like the profile's (they may be the profile's own).
 * Host-only.  Errors: EINVAL (also when a corrected duration is not > 0). */
camelot_status camelot_profile_add_handover(const camelot_profile* prof, const double* handover_s,
                                            double* thr, double* bw, double* dur);

/* Event-driven simulation of the pipeline on its profile (the allocator's
 * model of Sec. 5.2 and Eq. 1): n_queries Poisson arrivals at rate_qps (a
 * SplitMix64 stream from seed), the batch trigger (B = alloc->batch, or the
 * oldest waited max_wait_s), alloc->instances[i] instances of stage i, each
 * batch of b queries served in the profiled duration at the stage's quota
 * (interpolated as camelot_trigger_latency does) plus handover_s[i] (NULL =
 * 0; the sum must stay > 0); unbounded buffers between stages.  Reports the p50 and p99 latency
 * (arrival to last stage done) over the queries after the first 10 %, and the
 * throughput: completions per second after the first 10 % of them.
 * Host-only.  Errors: EINVAL. */
camelot_status camelot_simulate_profile(const camelot_profile* prof, const camelot_alloc* alloc,
                                        const double* handover_s, double max_wait_s, double rate_qps,
                                        uint32_t n_queries, uint64_t seed, double* p50_s, double* p99_s,
                                        double* thr_qps);

#ifdef __cplusplus
}
#endif
#endif /* CAMELOT_H_ */
