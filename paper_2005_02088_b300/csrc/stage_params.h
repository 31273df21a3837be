// Plain-data description of a prepared stage, shared by the host runtime and
// the device code (passed by value in kernel parameters).
#pragma once
#include <cstddef>
#include <cstdint>

namespace camelot {

constexpr int kMaxLayers = 4;
constexpr int kMaxStages = 8;
constexpr int kMaxTopK = 5;
constexpr int kThreads = 256;          // threads per CTA (one CTA per SM)
constexpr int kWarps = kThreads / 32;
constexpr int kQGroup = 16;            // queries per register tile of the FP32 layers
constexpr int kNBlock = 128;           // neurons per warp task (4 per lane)
constexpr int kMaxKC = 128;            // largest K-chunk of a warp task
constexpr int kMRing = 3;              // FP32 layers: bulk-copy ring slots per warp
constexpr int kMQuads = 3;             // FP32 layers: weight k-quads per ring slot
constexpr int kMaxRingSlots = 5;       // tensor-core layers: most bulk-copy ring slots
constexpr size_t kSmemBytes = 216 * 1024;  // dynamic shared memory per CTA: > half an SM,
                                           // so exactly one CTA fits on an SM

enum StageKind : int32_t { KIND_NORMALIZE_U8 = 1, KIND_NORM_POOL2_BF16 = 2, KIND_MLP_FP32 = 3,
                           KIND_GEMM_BF16 = 4, KIND_GEMM_FP8 = 5, KIND_NORMALIZE_U8_E4M3 = 6,
                           KIND_EMBED_GATHER = 7, KIND_COMPUTE_SYNTH = 8, KIND_STREAM_SYNTH = 9 };
__host__ __device__ inline bool is_tensor_kind(int32_t k) { return k == KIND_GEMM_BF16 || k == KIND_GEMM_FP8; }
enum Act : int32_t { ACT_NONE = 0, ACT_RELU = 1, ACT_GELU = 2 };

// One dense layer in kernel layout.
//  - "task" layers (N > 32 or not the last layer of a final stage): weights
//    packed as quads of k, [K/4][Npad][4] f32, Npad = N rounded up to 128, rows
//    >= N zero; computed as (query-group, 128-neuron block, K-chunk) warp tasks
//    whose partial sums are reduced over chunks in chunk order.
//  - "head" layer (last layer of a final stage with N <= 32): weights row-major
//    [N][K]; one warp computes a whole query.
//  - tensor-core layers (GEMM_BF16, GEMM_FP8): weights bf16 or e4m3 in tiles of
//    128 rows x 128 bytes (64 bf16 or 128 e4m3 columns); tile (mt, kb) is a
//    contiguous 16 KB block at ((mt * KB) + kb) * 16 KB, KB = K * esz / 128,
//    holding rows 128 mt.. and the kb-th 128-byte column block in the
//    128-byte-swizzle layout (row r's 16-byte piece j at r * 128 + (j ^ (r % 8))
//    * 16); rows >= N are zero and Npad = N rounded up to 128.  K is cut into
//    chunks of KC (128 / esz columns at least) whose fp32 partials are reduced
//    in chunk order.  An output value is act(acc * vscale); FP8 hidden outputs
//    are stored as e4m3(value / qscale).
struct LayerParams {
    const float* w;     // device, kernel layout (see above)
    int32_t K, N, Npad;
    int32_t KC, C;      // K-chunk and number of chunks
    int32_t act;
    int32_t head;       // 1 = head layer
    int32_t esz;        // tensor-core layers: bytes per element (2 bf16, 1 e4m3)
    float vscale;       // tensor-core layers: accumulator scale (1 for bf16)
    float qscale;       // FP8 layers: scale of the output codes (0 = f32 / bf16 output)
    int32_t ring;       // tensor-core layers: ring slots to use (0 = all that fit)
    size_t p_off;       // scratch offset of this layer's partial sums (task layers)
    size_t h_off;       // scratch offset of its output rows (hidden layers / logits)
};

struct StageParams {
    int32_t kind;
    int32_t n_layers;
    int32_t top_k;          // 0 = intermediate stage
    int32_t max_batch;
    int32_t H, W, C;        // image kinds; EMBED_GATHER: H = vocabulary, W = row width D;
                            // COMPUTE_SYNTH: W = row width, H = FMA steps; STREAM_SYNTH: W = row
                            // width, H = table windows per query (R / W), C = window starts
                            // (L / W - R / W + 1), layer[0].w = the table
    int32_t rows;           // rows per query: tokens (EMBED_GATHER, token-level tensor-core stages), else 1
    int32_t res_k;          // results per query in the final-stage result arrays (top_k, or tags of
                            // the first tokens for a token-level stage)
    int32_t in_tiled;       // set per pipeline: the input rows arrive in the tiled layout below
    int32_t out_tiled;      // set per pipeline: write the output rows in the tiled layout
    int32_t tile_h;         // tensor-core kinds: rows per operand tile (32; 128 for token-level stages)
    int32_t out_tile_h;     // set per pipeline: tile height of the consumer's tiled layout
    int32_t pad_;
    size_t in_row_bytes;
    size_t out_row_bytes;   // 0 for final stages
    size_t out_width;       // final stages: width of the last layer (logits per query)
    size_t scratch_bytes;   // per instance (for max_batch)
    size_t res_off;         // scratch offset of final results: idx [B][5] int32, val [B][5] f32
    size_t tile_off;        // tensor-core kinds: scratch offset of a layer's input in tiled form
    size_t cand_off;        // final tensor-core kinds: scratch offset of the top-k candidates,
                            // (value bits, index) int32 pairs [rows][last layer's 128-row tiles][kMaxTopK]
    LayerParams layer[kMaxLayers];
};

// Tiled row layout read by the tensor-core stages (their MMA operand format):
// rows of rowb bytes (a multiple of 128) in h-row x 128-byte tiles (h = 32 or
// 128, nothing else); tile (rt, kb) = rows h rt.. and bytes 128 kb.. of each row, h x 128
// bytes at (rt * rowb / 128 + kb) * h * 128; row r's 16-byte piece j at
// (r % h) * 128 + (j ^ (r % 8)) * 16 inside it.  Byte `b` of row r:
__host__ __device__ inline size_t tiled_offset(int r, size_t b, size_t rowb, int h) {
    const int lg = h == 128 ? 7 : 5;               // h is 32 or 128
    const size_t p = b >> 4, kb = p >> 3, j = p & 7;
    const int rt = r >> lg, rr = r & (h - 1);
    return ((((size_t)rt * (rowb >> 7)) + kb) << (lg + 7)) + (size_t)rr * 128 + ((j ^ (size_t)(rr & 7)) << 4) +
           (b & 15);
}
// Bytes a tiled batch of `rows` rows occupies (whole row tiles of h rows).
__host__ __device__ inline size_t tiled_bytes(size_t rows, size_t rowb, int h) {
    return (rows + h - 1) / h * h * rowb;
}

// Row addressing: row q is at base + ((first + q) & mask) * stride.  Ring
// slots wrap with mask = slots - 1; contiguous buffers use mask = ~0.
struct RowRef {
    char* base;
    uint64_t first;
    uint64_t mask;
    size_t stride;
    __host__ __device__ char* row(uint64_t q) const {
        return base + ((first + q) & mask) * stride;
    }
};

}  // namespace camelot
