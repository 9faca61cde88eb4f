// Internal host-side interface between the C ABI (api.cu) and the kernel
// translation units.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "ss_device.cuh"

namespace ss {

// Layout of the maximum-mipmap buffer (levels 1..L-1, then two stats floats).
struct MipLayout {
    int32_t levels;                 // including level 0
    int32_t w[kMaxLevels], h[kMaxLevels];
    int64_t pitch[kMaxLevels];      // level 0: not used (heights keep their own pitch)
    int64_t offset[kMaxLevels];     // elements from the buffer start (level >= 1)
    int64_t stats_offset;           // (global max, global min)
    int64_t total_elems;
};

bool mip_layout(int32_t nx, int32_t ny, MipLayout* L);

struct FwdArgs {
    Tile T;
    Pyramid P;
    Rays R;
    Outputs O;
    const float* stats;   // device: (global max, global min) of the heights
    int32_t kleaf;
    uint32_t flags;
    int64_t rays_per_block;   // rays owned by one block
    int32_t refill_min;       // waiting lanes that trigger a warp service
    int32_t poly;             // 1: the rise series is valid for every ray
    int32_t tile_w;           // grid mode: ray-rectangle width (0 = row-major runs)
    int32_t strip;            // descent: rays per strip (1 = no seeding)
    int32_t colseed;          // descent, grid rays in rectangles: column seeds
    int32_t seed_w;           // descent: half-width of a seed window
};

constexpr int32_t kColSeedMaxW = 512;    // widest rectangle with a column-seed table
constexpr int32_t kListSeedCols = 512;   // listed rays: columns of consecutive ids

struct BwdArgs {
    Tile T;
    Rays R;
    const int32_t* argmin;
    const float* cost;          // optional forward cost (saturation pre-test)
    const float* grad_light;
    float* grad_h;
    int64_t grad_pitch;
    double* grad_sun;
    double ds_de[3], ds_da[3];
    uint32_t* status;           // device status word (non-finite dL/dlight), or null
};

cudaError_t launch_build_maxmip(const float* h, int32_t nx, int32_t ny, int64_t pitch,
                                float* mip, const MipLayout& L, cudaStream_t s);
cudaError_t launch_dp_forward(const FwdArgs& a, int block, cudaStream_t s);
cudaError_t launch_uniform_forward(const FwdArgs& a, int block, cudaStream_t s);
cudaError_t launch_backward(const BwdArgs& a, int block, cudaStream_t s);
size_t backward_det_workspace_bytes(int32_t nx, int32_t ny);
cudaError_t launch_backward_det(const BwdArgs& a, int block, void* workspace, cudaStream_t s);

// camera of the view-ray caster (mirrors ss_camera)
struct ViewCamera {
    double pos[3], forward[3], right[3], up[3];
    double tan_x, tan_y;
    int32_t width, height;
};

int64_t view_blocks(int32_t width, int32_t height);
size_t view_workspace_bytes(int32_t width, int32_t height);
cudaError_t launch_view_rays(const Tile& T, const Pyramid& P, const ViewCamera& cam, double step,
                             int64_t K, const float* stats, float* uv, int32_t* pixel,
                             int64_t* count, void* workspace, cudaStream_t s);

constexpr int kGreedyMaxRuns = 8;
cudaError_t launch_greedy(const Tile& T, const Pyramid& P, const Rays& R, const int32_t* levels,
                          int32_t n_runs, float* light, float* cost, float* t_star,
                          cudaStream_t s, const float* stats, bool f32);

constexpr int kShadeMaxLights = 8;
struct ShadeLight {       // mirrors ss_light
    double elevation_rad, azimuth_rad, intensity;
    const float* lit;
};
cudaError_t launch_shade(const Tile& T, const Rays& R, const ShadeLight* lights, int32_t n_lights,
                         float* E, cudaStream_t s);

int device_sm_count();

}  // namespace ss
