// kaze_batch.h -- layouts shared by the batched persistent kernel
// (k_batch.cu) and its host runtime (kaze_batch_api.cu).
#pragma once

#include <stdint.h>

#include "kaze_internal.h"

namespace kz {
namespace batch {

constexpr int kBatchThreads = 256;  // threads per persistent CTA
constexpr int kExtremaRows = 4;     // rows per extrema item
constexpr int kTilesPerItem = 4;    // 32x32 stencil tiles per item (one tile row)

// Chunk lengths for which the batch kernel carries compiled (register)
// solvers; must match KZ_BATCH_ROW_M / KZ_BATCH_COL_M in k_batch.cu.
constexpr int kRowCompiledM[] = {11, 21, 31};
constexpr int kColCompiledM[] = {9, 13, 17, 19};

enum ItemKind : uint8_t {
    IT_PRESMOOTH = 0,  // kTilesPerItem 32x32 tiles of L_0 = G_sigma0 * I
    IT_GMAX,           // ... of the gradient maximum
    IT_GHIST,          // ... of the gradient histogram
    IT_PCT,            // percentile pick -> k (one per image)
    IT_COND,           // ... of the conductance of level `level`
    IT_ROWS,           // 4 rows of the row solves of level `level`
    IT_COLS,           // strip of columns: column solves + average -> L_level
    IT_DOH,            // 64x64 tile of the response of level `level`
    IT_EXTREMA,        // kExtremaRows rows of extrema of level `level`
};

struct Item {
    uint8_t kind;
    uint8_t level;
    uint16_t image;
    uint32_t index;  // tile / row group / strip / band
};

// One image of the batch, in device memory.
struct ImageDesc {
    const float* img;  // input (updated per call)
    int img_pitch;
    int w, h, pitch;
    long long plane;   // floats per plane
    float* levels;     // N planes
    float* doh;        // N planes
    float* g;          // conductance scratch
    float* ux;         // row-solution scratch
    float* k;          // contrast factor
    unsigned* hmax;    // bit pattern of the gradient maximum
    unsigned* hist;    // nbins counts
    kaze_keypoint* kp; // keypoint buffer of kp_cap entries
    unsigned* kp_count;
    int kp_cap;
    int mrow;          // row chunk length (64 chunks)
    int mcol;          // column chunk length (64 chunks, 4-column strips)
    int mcol32;        // column chunk length (32 chunks, 8-column strips)
    int tiles32_x, tiles64_x;
    int groups32_x;    // items per tile row of the 32x32 stencils
};

struct BatchParams {
    const ImageDesc* imgs;
    const Item* items;
    int n_items;
    unsigned* next;          // work-queue head
    unsigned* done;          // [image][slot] completed items
    const unsigned* need;    // [image][slot] items per stage
    int slots;               // slots per image
    int* status;             // bit 0: a bounded wait ran out
    long long spin_limit;    // cycles a wait may take
    GaussTaps taps0, tapsd;
    LevelTable tab;
    float tau[kMaxLevels];        // t_i - t_{i-1}
    float doh_scale[kMaxLevels];  // norm_i / (1024 s_i^2)^2
    double pct;
    int nbins, diffusivity;
    float thr, edge_r, k_override;
    int cols;                // columns per strip (4 or 8)
    int N;                   // levels
};

// Stage slots of one image.
__host__ __device__ inline int slot_presmooth() { return 0; }
__host__ __device__ inline int slot_gmax() { return 1; }
__host__ __device__ inline int slot_ghist() { return 2; }
__host__ __device__ inline int slot_pct() { return 3; }
__host__ __device__ inline int slot_cond(int l) { return 4 + 3 * (l - 1); }
__host__ __device__ inline int slot_rows(int l) { return 5 + 3 * (l - 1); }
__host__ __device__ inline int slot_cols(int l) { return 6 + 3 * (l - 1); }
// response and extrema slots follow the 3 (N - 1) evolution slots; the
// kernel reaches them through these with kMaxLevels-sized spacing
__host__ __device__ inline int slot_doh(int l) { return 4 + 3 * (kMaxLevels - 1) + l; }
__host__ __device__ inline int slot_extrema(int l) { return 4 + 3 * (kMaxLevels - 1) + kMaxLevels + l; }
__host__ __device__ inline int slots_per_image() { return 4 + 3 * (kMaxLevels - 1) + 2 * kMaxLevels; }
constexpr int kSlotWords = (4 + 3 * (kMaxLevels - 1) + 2 * kMaxLevels + 31) / 32;  // bit words per image

cudaError_t configure_batch_kernel(int smem);
cudaError_t batch_occupancy(int smem, int* blocks_per_sm);
cudaError_t launch_batch(const BatchParams& p, int grid, int smem, cudaStream_t st);

}  // namespace batch
}  // namespace kz
