// Internal types of the batched forward (ss_batch_submit / plans).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "ss_device.cuh"

namespace ss {

// One instance as the batched kernel sees it (copied to shared memory per warp;
// a multiple of 4 bytes so lanes can copy it word by word).
struct __align__(16) BatchItemDesc {
    Tile T;
    LevelTab L;
    Outputs O;
    const float* stats;     // (global max, global min) of the instance's heights
    int64_t n_rays;         // nx * ny (grid mode)
    int32_t levels;
    int32_t poly;           // the rise series is valid for every ray
    int32_t tile_w;         // ray-rectangle width of chunks (0 = row-major runs)
    int32_t pad;
};

struct BatchArgs {
    const BatchItemDesc* items;
    const int64_t* chunk_prefix;    // [n_items + 1]: first chunk of each instance
    unsigned long long* counter;    // work-queue head (zeroed before the launch)
    int64_t total_chunks;
    int32_t n_items;
    int32_t chunk_rays;
    int32_t kleaf;
    int32_t refill_min;
    int32_t light_only;             // SS_FLAG_LIGHT_ONLY
    int32_t strip;                  // rays per seeded strip (1 = no seeding)
    int32_t colseed;                // rectangular chunks: single rays, column seeds
    int32_t seed_w;                 // half-width of a seed window
    int32_t lane_leaves;            // SS_FLAG_LANE_LEAVES: leaves in the walking lane
};

constexpr int32_t kBatchSeedW = 64;    // widest chunk with a column-seed table

constexpr size_t kBatchHeader = 256;   // queue counter, padded
inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

size_t batch_workspace_bytes(int32_t n_items);
void batch_layout(void* ws, int32_t n_items, unsigned long long** counter, BatchItemDesc** items,
                  int64_t** prefix);
cudaError_t launch_batch_forward(const BatchArgs& a, int block, bool count, cudaStream_t s);

}  // namespace ss
