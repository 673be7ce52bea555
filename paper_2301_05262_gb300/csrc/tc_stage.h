// Job tables of the tensor-core level kernels (net_bf16.cu): one launch per
// stage serves up to kMaxViews views of any size.
#pragma once

#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

#include "nsm_common.cuh"

namespace nsm {

constexpr int kMaxViews = 32;
constexpr int kTcStages = 5;  // enc0 (+ gather), enc1, bottleneck, dec1, dec0 (+ head)

// TMA: as PLAIN, the rows staged by tensor-memory-access copies (one thread)
enum TcPro { TPRO_GATHER = 0, TPRO_PLAIN = 1, TPRO_UP_SKIP = 2, TPRO_UP = 3, TPRO_TMA = 4 };
// STORE_PAIR: like STORE, as BF16 hi + lo pairs [H][W][2][COUT];
// HEAD_PAR: the level-0 decoder on the coarse grid (four output parities per
// coarse pixel, 1x1 per parity, head, sigmoid; fine visibility [2H][2W])
enum TcEpi { TEPI_POOL = 0, TEPI_SKIP_POOL = 1, TEPI_STORE = 2, TEPI_HEAD = 3, TEPI_HEAD4 = 4, TEPI_STORE_PAIR = 5,
             TEPI_HEAD_PAR = 6 };

// One view's work in one stage.
struct TcJob {
    GatherParams g;             // GATHER prologue: the view's G-buffer, map, emitter, camera
    int H, W;                   // the stage's resolution for this view
    int tiles_x, tiles_y;       // tiles per row / column (filled at launch); tiles run column-major
    // activations read by the tensor cores straight from memory (PLAIN inputs)
    // are BF16 hi + lo pairs, [pixel][part][C] (part 0 = hi, 1 = lo); those
    // the up-sampling producers read are FP32 [pixel][C] (same 4 bytes per channel)
    const uint16_t* in;         // PLAIN: [H][W][2][CIN]
    const float* in_f;          // UP*: [H/2][W/2][CIN]
    const float* skip;          // UP_SKIP: [H][W][CIN]
    uint16_t* out;              // POOL / SKIP_POOL: pooled [H/2][W/2][2][COUT]; STORE_PAIR: [H][W][2][COUT]
    float* out_f;               // STORE: [H][W][COUT]
    float* out_skip;            // SKIP_POOL: [H][W][COUT]
    // FP8 form: every activation E4M3 [pixel][C], 1 byte per channel
    const uint8_t* in8;         // PLAIN: [H][W][CIN]; UP*: [H/2][W/2][CIN]
    const uint8_t* skip8;       // UP_SKIP: [H][W][CIN]
    uint8_t* out8;              // POOL / SKIP_POOL: pooled [H/2][W/2][COUT]; STORE: [H][W][COUT]
    uint8_t* out_skip8;         // SKIP_POOL: [H][W][COUT]
    float* vis;                 // HEAD: [H][W]; HEAD_PAR: [2H][2W]; HEAD4 writes out_f [H][W][4]
    // TMA prologue: tensor map of `in` as [H][W][2 CIN / 8 chunks][8 BF16],
    // box = one 16-byte chunk plane of kSW pixels of one row (zero fill outside)
    CUtensorMap tmap;           // (the type carries the 64-byte alignment TMA needs)
};

// Kernel parameter of a stage launch (passed by value, __grid_constant__).
struct TcBatch {
    int nviews;
    int tile_start[kMaxViews + 1];  // prefix sums of the views' tile counts
    TcJob job[kMaxViews];
    const uint4* b3img;         // packed 3x3 weights (shared-memory image, hi then lo)
    const uint4* b1img;         // packed 1x1 weights
    const float* bias3;
    const float* bias1;
    const float* head;          // HEAD: weights [16] then bias; HEAD4: weights [4][16] then biases [4]
    const float* w3;            // HEAD_PAR: FP32 3x3 weights [COUT][CIN][3][3] (exact border ring)
    const float* w1;            // HEAD_PAR: FP32 1x1 weights [COUT][COUT]
    const float* scale3;        // FP8 form: per-output-channel weight scales of the 3x3
    const float* scale1;        // and of the 1x1
    int* err;                   // device error word
    // Per-view completion times (batched serving), or null: [0] the batch's
    // start (%globaltimer, ns, written by the first stage), [1 + v] the time
    // view v's last output pixel was written (level-0 decoder), [1 + kMaxViews
    // + v] the completion counter of view v
    unsigned long long* timing;
};
constexpr int kTimingWords = 1 + 2 * kMaxViews;

struct Activations;

int tc_stage_variants(int stage);
int tc_stage_rows(int stage, int variant);
int tc_stage_warps(int stage, int variant, int* producer_warps);  // epilogue warps
// MMA schedule: 0 = a tile's 1x1 right after its 3x3; 1 = the next tile's 3x3
// first, then the previous tile's 1x1 (overlaps the epilogue's 3x3 read-out)
int tc_stage_order(int stage, int variant);
int tc_default_variant(int stage);
const void* tc_stage_kernel(int stage, int variant);
int tc_stage_occupancy(int stage, int variant);
void tc_make_batches(const GatherParams* g, const Activations* act, float* const* vis, int n, const float* params,
                     const uint16_t* img, int* err, TcBatch* out);
cudaError_t tc_launch_stage(int stage, int variant, TcBatch& b, int ctas_per_sm, cudaStream_t stream);
void tc_fill_tiles(TcBatch& b, int rows);  // tile counts of every view for tile height rows
// Tile table (and, for TMA variants, the views' tensor maps) of a stage's batch
cudaError_t tc_prepare_stage(int stage, int variant, TcBatch& b);
// Tensor map of a PLAIN stage input ([H][W][2][cin] BF16) for the TMA prologue
cudaError_t tc_encode_input_map(CUtensorMap* map, const uint16_t* in, int H, int W, int cin);

}  // namespace nsm
