// C ABI (include/softshadow.h): argument validation on the host, then kernel
// launches on the caller's stream.  Nothing here allocates device memory.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <mutex>
#include <vector>

#include "../../include/softshadow.h"
#include "ss_batch.h"
#include "ss_launch.h"
#include "ss_walk.cuh"

namespace {

thread_local char g_last_error[256] = "";

ss_status cuda_fail(cudaError_t e, const char* where) {
    snprintf(g_last_error, sizeof(g_last_error), "%s: %s", where, cudaGetErrorString(e));
    return SS_ERR_CUDA;
}

bool finite_pos(double x) { return isfinite(x) && x > 0.0; }

ss_status check_tile(const ss_heightfield* hf, int32_t min_dim) {
    if (!hf || !hf->h) return SS_ERR_INVALID_ARG;
    if (hf->nx < min_dim || hf->ny < min_dim || hf->nx > SS_MAX_DIM || hf->ny > SS_MAX_DIM)
        return SS_ERR_BAD_SIZE;
    if (hf->pitch < hf->nx) return SS_ERR_BAD_SIZE;
    if ((double)hf->pitch * (double)hf->ny > 4294967295.0) return SS_ERR_BAD_SIZE;
    if (!finite_pos(hf->texel_m) || !finite_pos(hf->radius_m)) return SS_ERR_INVALID_ARG;
    if (hf->projection != SS_PROJ_GNOMONIC && hf->projection != SS_PROJ_POLAR_STEREO)
        return SS_ERR_INVALID_ARG;
    return SS_OK;
}

ss_status check_sun(const ss_sun* sun) {
    if (!sun) return SS_ERR_INVALID_ARG;
    if (!isfinite(sun->elevation_rad) || !isfinite(sun->azimuth_rad)) return SS_ERR_INVALID_ARG;
    if (!(fabs(sun->elevation_rad) < M_PI / 2)) return SS_ERR_INVALID_ARG;
    if (!finite_pos(sun->angular_radius_rad) || !(sun->angular_radius_rad < M_PI / 2))
        return SS_ERR_INVALID_ARG;
    return SS_OK;
}

constexpr uint32_t kFwdFlags =
    SS_FLAG_COUNT_SAMPLES | SS_FLAG_NO_EARLY_EXIT | SS_FLAG_LIGHT_ONLY | SS_FLAG_LANE_LEAVES;

static_assert(SS_DEV_NONFINITE_HEIGHT == ss::kDevNonfiniteHeight &&
                  SS_DEV_NONFINITE_RAY == ss::kDevNonfiniteRay &&
                  SS_DEV_NONFINITE_GRAD == ss::kDevNonfiniteGrad,
              "status bits");

ss_status check_params(const ss_params* p, double g, int32_t* J, double* delta,
                       uint32_t allowed_flags = kFwdFlags) {
    if (!p) return SS_ERR_INVALID_ARG;
    if (!finite_pos(p->max_len_m)) return SS_ERR_INVALID_ARG;
    if (!isfinite(p->step_texels) || p->step_texels < 0.0) return SS_ERR_INVALID_ARG;
    if (p->flags & ~allowed_flags) return SS_ERR_INVALID_ARG;
    if (p->block_threads != 0 &&
        (p->block_threads < 32 || p->block_threads > 256 || p->block_threads % 32 != 0))
        return SS_ERR_INVALID_ARG;
    if (p->leaf_level < -1 || p->leaf_level > 16) return SS_ERR_INVALID_ARG;
    if (p->rays_per_thread < 0 || p->rays_per_thread > 4096) return SS_ERR_INVALID_ARG;
    if (p->refill_min < 0 || p->refill_min > 32) return SS_ERR_INVALID_ARG;
    if (p->ray_tile_w < 0 || p->ray_tile_w > SS_MAX_DIM) return SS_ERR_INVALID_ARG;
    if (p->strip_len < 0 || p->strip_len > 256) return SS_ERR_INVALID_ARG;
    if (p->seed_width < 0 || p->seed_width > 16) return SS_ERR_INVALID_ARG;
    double st = p->step_texels == 0.0 ? 0.5 : p->step_texels;
    double d = st * g;
    if (!finite_pos(d)) return SS_ERR_INVALID_ARG;
    double jj = floor(p->max_len_m / d);
    if (!(jj <= (double)SS_MAX_SAMPLES)) return SS_ERR_BAD_SIZE;
    *J = (int32_t)jj;
    *delta = d;
    return SS_OK;
}

ss_status check_rays(const ss_rays* r, const ss_heightfield* hf, int64_t* n) {
    if (!r) return SS_ERR_INVALID_ARG;
    if (r->mode == SS_RAYS_GRID) {
        *n = (int64_t)hf->nx * hf->ny;
    } else if (r->mode == SS_RAYS_LIST) {
        if (r->n < 0) return SS_ERR_BAD_SIZE;
        if (r->n > 0 && !r->uv) return SS_ERR_INVALID_ARG;
        *n = r->n;
    } else {
        return SS_ERR_INVALID_ARG;
    }
    return SS_OK;
}

void sun_vector(const ss_sun* s, double v[3]) {
    double ce = cos(s->elevation_rad);
    v[0] = ce * sin(s->azimuth_rad);
    v[1] = ce * cos(s->azimuth_rad);
    v[2] = sin(s->elevation_rad);
}

ss::Tile make_tile(const ss_heightfield* hf, const ss_sun* sun, int32_t J, double delta) {
    ss::Tile T{};
    T.h = hf->h;
    T.pitch = hf->pitch;
    T.nx = hf->nx;
    T.ny = hf->ny;
    T.proj = hf->projection;
    T.J = J;
    T.g = hf->texel_m;
    T.R = hf->radius_m;
    T.cx = 0.5 * (hf->nx - 1);
    T.cy = 0.5 * (hf->ny - 1);
    double s[3];
    sun_vector(sun, s);
    T.sx = s[0];
    T.sy = s[1];
    T.sz = s[2];
    T.delta = delta;
    T.inv_gR = 1.0 / (hf->texel_m * hf->radius_m);
    T.inv_R = 1.0 / hf->radius_m;
    T.inv_g = 1.0 / hf->texel_m;
    T.alpha = sun->angular_radius_rad;
    T.delta_f = (float)delta;
    T.inv_delta_f = (float)(1.0 / delta);
    T.sz_f = (float)s[2];
    T.sx_f = (float)s[0];
    T.sy_f = (float)s[1];
    T.R_f = (float)hf->radius_m;
    T.g_f = (float)hf->texel_m;
    T.cx_f = (float)T.cx;
    T.cy_f = (float)T.cy;
    T.alpha_f = (float)sun->angular_radius_rad;
    auto split = [](double x, float& hi, float& lo) {
        hi = (float)x;
        lo = (float)(x - (double)hi);
    };
    const double g = hf->texel_m, R = hf->radius_m;
    split(g, T.g_hi, T.g_lo);
    float r_hi;
    split(R, r_hi, T.R_lo);
    split(R * R, T.RR_hi, T.RR_lo);
    split(delta, T.delta_hi, T.delta_lo);
    split(T.inv_gR, T.igR_hi, T.igR_lo);
    split(R * s[0], T.Rsx_hi, T.Rsx_lo);
    split(R * s[1], T.Rsy_hi, T.Rsy_lo);
    float sz_hi, sx_hi, sy_hi;
    split(s[2], sz_hi, T.sz_lo);
    split(s[0], sx_hi, T.sx_lo);
    split(s[1], sy_hi, T.sy_lo);
    split(2.0 * R / g, T.k2_hi, T.k2_lo);
    T.szR_f = (float)(s[2] / R);
    return T;
}

ss::Pyramid make_pyramid(const ss_heightfield* hf, const float* mip, const ss::MipLayout& L) {
    ss::Pyramid P{};
    P.levels = L.levels;
    P.ptr[0] = hf->h;
    P.pitch[0] = hf->pitch;
    for (int l = 1; l < L.levels; ++l) {
        P.ptr[l] = mip + L.offset[l];
        P.pitch[l] = L.pitch[l];
    }
    return P;
}

// The float32 ray rise uses a 5-term series in x = t (2 rho sin e + t) / rho^2
// when |x| <= 1/32 holds for every ray of the launch.  Bound: |sin e| <=
// |s_z| + sin(theta) |s_xy| with theta the angle from the tile centre to its
// corner (x3 for listed origins, which may lie off the tile), and rho >= R/2
// (heights above -R/2); then |x| <= t (4 |sin e| / R + 4 t / R^2).
bool rise_series_ok(const ss_heightfield* hf, const ss_sun* sun, double tmax, int32_t mode) {
    const double hx = 0.5 * (hf->nx - 1) * hf->texel_m, hy = 0.5 * (hf->ny - 1) * hf->texel_m;
    double st = sqrt(hx * hx + hy * hy) / hf->radius_m;
    if (mode != SS_RAYS_GRID) st *= 3.0;
    st = fmin(st, 1.0);
    const double sz = fabs(sin(sun->elevation_rad)), sxy = fabs(cos(sun->elevation_rad));
    const double se = fmin(1.0, sz + st * sxy);
    const double R = hf->radius_m;
    return tmax * (4.0 * se / R + 4.0 * tmax / (R * R)) <= 0.03125;
}

enum class FwdKind { Descent, Uniform };

// rays per descent strip when strips are used by default (each ray seeded from
// the previous one's argmin)
constexpr int32_t kDefaultStrip = 10;
// default ray-rectangle width of the descent on grid rays
constexpr int32_t kDefaultTileW = 256;

ss_status shadow_common(FwdKind kind, const ss_heightfield* hf, const float* mip,
                        const ss_rays* rays, const ss_sun* sun, const ss_params* params,
                        const ss_outputs* out, ss_stream_t stream) {
    ss_status st = check_tile(hf, 2);
    if (st != SS_OK) return st;
    if ((st = check_sun(sun)) != SS_OK) return st;
    int32_t J;
    double delta;
    if ((st = check_params(params, hf->texel_m, &J, &delta)) != SS_OK) return st;
    int64_t n;
    if ((st = check_rays(rays, hf, &n)) != SS_OK) return st;
    if (!mip || !out) return SS_ERR_INVALID_ARG;
    if (n == 0) return SS_OK;
    if (!out->light || !out->argmin) return SS_ERR_INVALID_ARG;
    if ((params->flags & SS_FLAG_COUNT_SAMPLES) && !out->counters) return SS_ERR_INVALID_ARG;
    ss::MipLayout L;
    if (!ss::mip_layout(hf->nx, hf->ny, &L)) return SS_ERR_BAD_SIZE;
    ss::FwdArgs a{};
    a.T = make_tile(hf, sun, J, delta);
    a.P = make_pyramid(hf, mip, L);
    a.R.mode = rays->mode;
    a.R.n = n;
    a.R.uv = rays->uv;
    a.R.lift = rays->mode == SS_RAYS_LIST ? rays->lift_m : nullptr;
    a.R.status = out->status;
    a.O.light = out->light;
    a.O.argmin = out->argmin;
    a.O.cost = out->cost;
    a.O.status = out->status;
    a.O.counters = (params->flags & SS_FLAG_COUNT_SAMPLES) ? out->counters : nullptr;
    a.stats = mip + L.stats_offset;
    a.kleaf = params->leaf_level >= 0 ? params->leaf_level : (rays->mode == SS_RAYS_GRID ? 1 : 2);
    a.flags = params->flags;
    const bool light_only = (params->flags & SS_FLAG_LIGHT_ONLY) != 0;
    const bool descent = kind == FwdKind::Descent;
    // Defaults (measured on GB300: 4096^2 mid workload, polar view).  The
    // descent (exact and light-only) draws grid rays row by row across 256 x 24
    // ray rectangles, each seeded from the last finished ray of its column
    // (column seeds, window +-1, leaf level 1); listed rays are read as 512
    // columns of consecutive ids and drawn the same way (window +-2: adjacent
    // view rays can be several texels apart; leaf level 2).  Uniform stepping
    // draws single rays from row-major runs.
    int block = params->block_threads ? params->block_threads : 256;
    const int32_t rpt = params->rays_per_thread > 0 ? params->rays_per_thread
                        : !descent                     ? 16
                        : rays->mode == SS_RAYS_GRID   ? 24
                                                       : 12;
    a.rays_per_block = (int64_t)block * rpt;
    a.poly = rise_series_ok(hf, sun, J * delta, rays->mode) ? 1 : 0;
    a.tile_w = params->ray_tile_w;
    if (a.tile_w == 0 && descent && rays->mode == SS_RAYS_GRID &&
        a.rays_per_block % kDefaultTileW == 0)
        a.tile_w = kDefaultTileW;
    if (a.tile_w > 0 && a.rays_per_block % a.tile_w != 0) return SS_ERR_INVALID_ARG;
    a.colseed = (descent && params->strip_len == 0 &&
                 (rays->mode != SS_RAYS_GRID || a.tile_w <= ss::kColSeedMaxW))
                    ? 1 : 0;
    // strips: explicit strip_len, else (no column seeds) strips of kDefaultStrip,
    // none in light-only mode
    a.strip = !descent ? 1
              : params->strip_len > 0 ? params->strip_len
              : light_only ? 1 : kDefaultStrip;
    a.seed_w = params->seed_width > 0 ? params->seed_width : (rays->mode == SS_RAYS_GRID ? 1 : 2);
    // warp services: the task descent (exact walks with column seeds, see
    // ss_forward.cuh) waits for 14 idle lanes on gnomonic tiles and 22 on
    // stereographic ones, the single-lane walk for 10 (sweeps over sun
    // directions and chunk shapes on the 4096^2 tile, and over 6-22 on the
    // polar view at 8192^2 and 16384^2)
    const bool grid_gn = rays->mode == SS_RAYS_GRID && hf->projection == SS_PROJ_GNOMONIC;
    const bool tasks = descent && !light_only && a.colseed &&
                       !(params->flags & SS_FLAG_LANE_LEAVES) && a.kleaf <= (grid_gn ? 1 : 2) &&
                       (rays->mode != SS_RAYS_GRID || a.tile_w > 0);
    const bool stereo = hf->projection != SS_PROJ_GNOMONIC;
    a.refill_min = params->refill_min > 0 ? params->refill_min
                   : tasks                ? (stereo ? 22 : 14)
                   : descent              ? 10
                                          : 6;
    cudaError_t e = kind == FwdKind::Descent
                        ? ss::launch_dp_forward(a, block, (cudaStream_t)stream)
                        : ss::launch_uniform_forward(a, block, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, kind == FwdKind::Descent ? "ss_shadow_forward" : "ss_shadow_uniform");
    return SS_OK;
}

// ------------------------------------------------------------------ batch
struct BatchPrep {
    std::vector<unsigned char> image;   // workspace contents after the header
    ss::BatchArgs args{};
    std::vector<ss::MipLayout> layouts;
    int block = 256;
    bool count = false;
};

ss_status batch_prepare(const ss_batch_item* items, int32_t n, const ss_params* params, void* ws,
                        size_t ws_bytes, BatchPrep& B) {
    if (!items || !params || !ws) return SS_ERR_INVALID_ARG;
    if (n < 1 || n > (1 << 20)) return SS_ERR_BAD_SIZE;
    if (ws_bytes < ss::batch_workspace_bytes(n)) return SS_ERR_OUT_OF_MEMORY;
    if (params->block_threads != 0 &&
        (params->block_threads < 32 || params->block_threads > 256 || params->block_threads % 32))
        return SS_ERR_INVALID_ARG;
    B.block = params->block_threads ? params->block_threads : 256;
    B.count = (params->flags & SS_FLAG_COUNT_SAMPLES) != 0;
    // Defaults (64-instance batch on GB300): exact walks take 64 x 64-texel
    // chunks (128 rays per lane) with column seeds and services at 14 idle
    // lanes; light-only walks runs of 512 texels (16 rays per lane) with
    // services at 6.
    const bool batch_light = (params->flags & SS_FLAG_LIGHT_ONLY) != 0;
    const int32_t rpt = params->rays_per_thread > 0 ? params->rays_per_thread
                        : batch_light              ? 16
                                                   : 128;
    const int32_t chunk = 32 * rpt;
    const int32_t tile_w = params->ray_tile_w > 0 || params->rays_per_thread > 0 || batch_light
                               ? params->ray_tile_w
                               : ss::kBatchSeedW;
    if (tile_w > 0 && chunk % tile_w != 0) return SS_ERR_INVALID_ARG;
    const size_t desc_bytes = ss::align256((size_t)n * sizeof(ss::BatchItemDesc));
    B.image.assign(desc_bytes + (size_t)(n + 1) * sizeof(int64_t), 0);
    auto* descs = reinterpret_cast<ss::BatchItemDesc*>(B.image.data());
    auto* prefix = reinterpret_cast<int64_t*>(B.image.data() + desc_bytes);
    B.layouts.resize(n);
    prefix[0] = 0;
    for (int32_t i = 0; i < n; ++i) {
        const ss_batch_item& it = items[i];
        ss_status st = check_tile(&it.hf, 2);
        if (st != SS_OK) return st;
        if (it.hf.projection != SS_PROJ_GNOMONIC) return SS_ERR_UNSUPPORTED;
        if ((st = check_sun(&it.sun)) != SS_OK) return st;
        int32_t J;
        double delta;
        if ((st = check_params(params, it.hf.texel_m, &J, &delta)) != SS_OK) return st;
        if (!it.mip || !it.out.light || !it.out.argmin) return SS_ERR_INVALID_ARG;
        if (B.count && !it.out.counters) return SS_ERR_INVALID_ARG;
        if (!ss::mip_layout(it.hf.nx, it.hf.ny, &B.layouts[i])) return SS_ERR_BAD_SIZE;
        ss::BatchItemDesc& d = descs[i];
        d.T = make_tile(&it.hf, &it.sun, J, delta);
        const ss::Pyramid P = make_pyramid(&it.hf, it.mip, B.layouts[i]);
        for (int l = 0; l < ss::kMaxLevels; ++l) {
            d.L.ptr[l] = l < P.levels ? P.ptr[l] : nullptr;
            d.L.pitch[l] = l < P.levels ? (uint32_t)P.pitch[l] : 0u;
        }
        d.levels = P.levels;
        d.O.light = it.out.light;
        d.O.argmin = it.out.argmin;
        d.O.cost = it.out.cost;
        d.O.counters = B.count ? it.out.counters : nullptr;
        d.O.status = it.out.status;
        d.stats = it.mip + B.layouts[i].stats_offset;
        d.n_rays = (int64_t)it.hf.nx * it.hf.ny;
        d.poly = rise_series_ok(&it.hf, &it.sun, J * delta, SS_RAYS_GRID) ? 1 : 0;
        d.tile_w = tile_w;
        prefix[i + 1] = prefix[i] + ss::chunk_count(d.n_rays, it.hf.nx, it.hf.ny, chunk, tile_w);
    }
    unsigned long long* counter;
    ss::BatchItemDesc* ditems;
    int64_t* dprefix;
    ss::batch_layout(ws, n, &counter, &ditems, &dprefix);
    B.args.items = ditems;
    B.args.chunk_prefix = dprefix;
    B.args.counter = counter;
    B.args.total_chunks = prefix[n];
    B.args.n_items = n;
    B.args.chunk_rays = chunk;
    B.args.kleaf = params->leaf_level < 0 ? 1 : params->leaf_level;   // grid rays
    B.args.refill_min = params->refill_min > 0 ? params->refill_min : (batch_light ? 6 : 14);
    B.args.light_only = (params->flags & SS_FLAG_LIGHT_ONLY) ? 1 : 0;
    B.args.strip = params->strip_len > 0 ? params->strip_len
                                         : (B.args.light_only ? 1 : kDefaultStrip);
    B.args.colseed = (params->strip_len == 0 && !B.args.light_only && tile_w > 0) ? 1 : 0;
    B.args.seed_w = params->seed_width > 0 ? params->seed_width : 1;   // grid rays
    B.args.lane_leaves = (params->flags & SS_FLAG_LANE_LEAVES) ? 1 : 0;
    return SS_OK;
}

// queue reset + mipmap builds + persistent kernel, all on stream s
cudaError_t batch_enqueue(const BatchPrep& B, const ss_batch_item* items, int32_t n,
                          cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(B.args.counter, 0, sizeof(unsigned long long), s);
    for (int32_t i = 0; e == cudaSuccess && i < n; ++i)
        e = ss::launch_build_maxmip(items[i].hf.h, items[i].hf.nx, items[i].hf.ny,
                                    items[i].hf.pitch, items[i].mip, B.layouts[i], s);
    if (e == cudaSuccess) e = ss::launch_batch_forward(B.args, B.block, B.count, s);
    return e;
}

// ss_shadow_backward / ss_shadow_backward_ws
ss_status backward_common(const ss_heightfield* hf, const ss_rays* rays, const ss_sun* sun,
                          const ss_params* params, const int32_t* argmin, const float* cost,
                          const float* grad_light, float* grad_h, double* grad_sun,
                          void* workspace, size_t workspace_bytes, uint32_t* status,
                          bool with_ws, ss_stream_t stream) {
    ss_status st = check_tile(hf, 2);
    if (st != SS_OK) return st;
    if ((st = check_sun(sun)) != SS_OK) return st;
    int32_t J;
    double delta;
    const uint32_t allowed = with_ws ? (kFwdFlags | SS_FLAG_DETERMINISTIC_BWD) : kFwdFlags;
    if ((st = check_params(params, hf->texel_m, &J, &delta, allowed)) != SS_OK) return st;
    int64_t n;
    if ((st = check_rays(rays, hf, &n)) != SS_OK) return st;
    const bool det = (params->flags & SS_FLAG_DETERMINISTIC_BWD) != 0;
    if (det) {
        if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255) != 0)
            return SS_ERR_INVALID_ARG;
        if (workspace_bytes < ss::backward_det_workspace_bytes(hf->nx, hf->ny))
            return SS_ERR_OUT_OF_MEMORY;
    }
    if (n == 0) return SS_OK;
    if (!argmin || !grad_light || !grad_h || !grad_sun) return SS_ERR_INVALID_ARG;
    ss::BwdArgs a{};
    a.T = make_tile(hf, sun, J, delta);
    a.R.mode = rays->mode;
    a.R.n = n;
    a.R.uv = rays->uv;
    a.R.lift = rays->mode == SS_RAYS_LIST ? rays->lift_m : nullptr;
    a.argmin = argmin;
    a.cost = cost;
    a.grad_light = grad_light;
    a.grad_h = grad_h;
    a.grad_pitch = hf->pitch;
    a.grad_sun = grad_sun;
    a.status = status;
    double e = sun->elevation_rad, az = sun->azimuth_rad;
    a.ds_de[0] = -sin(e) * sin(az);
    a.ds_de[1] = -sin(e) * cos(az);
    a.ds_de[2] = cos(e);
    a.ds_da[0] = cos(e) * cos(az);
    a.ds_da[1] = -cos(e) * sin(az);
    a.ds_da[2] = 0.0;
    int block = params->block_threads ? params->block_threads : 256;
    cudaError_t ce = det ? ss::launch_backward_det(a, block, workspace, (cudaStream_t)stream)
                         : ss::launch_backward(a, block, (cudaStream_t)stream);
    if (ce != cudaSuccess)
        return cuda_fail(ce, with_ws ? "ss_shadow_backward_ws" : "ss_shadow_backward");
    return SS_OK;
}

}  // namespace

struct ss_batch_plan {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

extern "C" {

const char* ss_status_string(ss_status s) {
    switch (s) {
        case SS_OK: return "SS_OK";
        case SS_ERR_INVALID_ARG: return "SS_ERR_INVALID_ARG: invalid argument";
        case SS_ERR_BAD_SIZE: return "SS_ERR_BAD_SIZE: size out of range";
        case SS_ERR_OUT_OF_MEMORY: return "SS_ERR_OUT_OF_MEMORY: workspace too small";
        case SS_ERR_CUDA: return "SS_ERR_CUDA: CUDA error";
        case SS_ERR_TIMEOUT: return "SS_ERR_TIMEOUT: bounded device wait expired";
        case SS_ERR_INTERNAL: return "SS_ERR_INTERNAL: internal consistency check failed";
        case SS_ERR_UNSUPPORTED: return "SS_ERR_UNSUPPORTED: not supported by this build";
    }
    return "unknown ss_status";
}

const char* ss_last_error_string(void) { return g_last_error; }

const char* ss_version(void) { return "softshadow-gb300 0.1 (sm_103a)"; }

int32_t ss_maxmip_levels(int32_t nx, int32_t ny) {
    ss::MipLayout L;
    return ss::mip_layout(nx, ny, &L) ? L.levels : 0;
}

size_t ss_maxmip_bytes(int32_t nx, int32_t ny) {
    ss::MipLayout L;
    return ss::mip_layout(nx, ny, &L) ? (size_t)L.total_elems * sizeof(float) : 0;
}

ss_status ss_maxmip_level_info(int32_t nx, int32_t ny, int32_t level, int32_t* width,
                               int32_t* height, int64_t* pitch, int64_t* offset_elems) {
    ss::MipLayout L;
    if (!ss::mip_layout(nx, ny, &L)) return SS_ERR_BAD_SIZE;
    if (level < 0 || level > L.levels) return SS_ERR_INVALID_ARG;
    if (level == L.levels) {   // the stats block: max, min, non-finite count
        if (width) *width = 3;
        if (height) *height = 1;
        if (pitch) *pitch = 3;
        if (offset_elems) *offset_elems = L.stats_offset;
        return SS_OK;
    }
    if (width) *width = L.w[level];
    if (height) *height = L.h[level];
    if (pitch) *pitch = level == 0 ? (int64_t)nx : L.pitch[level];
    if (offset_elems) *offset_elems = level == 0 ? -1 : L.offset[level];
    return SS_OK;
}

ss_status ss_build_maxmip(const ss_heightfield* hf, float* mip, ss_stream_t stream) {
    ss_status st = check_tile(hf, 1);
    if (st != SS_OK) return st;
    if (!mip) return SS_ERR_INVALID_ARG;
    ss::MipLayout L;
    if (!ss::mip_layout(hf->nx, hf->ny, &L)) return SS_ERR_BAD_SIZE;
    cudaError_t e = ss::launch_build_maxmip(hf->h, hf->nx, hf->ny, hf->pitch, mip, L,
                                            (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "ss_build_maxmip");
    return SS_OK;
}

ss_status ss_shadow_forward(const ss_heightfield* hf, const float* mip, const ss_rays* rays,
                            const ss_sun* sun, const ss_params* params, const ss_outputs* out,
                            ss_stream_t stream) {
    return shadow_common(FwdKind::Descent, hf, mip, rays, sun, params, out, stream);
}

ss_status ss_shadow_uniform(const ss_heightfield* hf, const float* mip, const ss_rays* rays,
                            const ss_sun* sun, const ss_params* params, const ss_outputs* out,
                            ss_stream_t stream) {
    return shadow_common(FwdKind::Uniform, hf, mip, rays, sun, params, out, stream);
}

ss_status ss_shadow_backward(const ss_heightfield* hf, const ss_rays* rays, const ss_sun* sun,
                             const ss_params* params, const int32_t* argmin, const float* cost,
                             const float* grad_light, float* grad_h, double* grad_sun,
                             ss_stream_t stream) {
    return backward_common(hf, rays, sun, params, argmin, cost, grad_light, grad_h, grad_sun,
                           nullptr, 0, nullptr, false, stream);
}

size_t ss_backward_workspace_bytes(int32_t nx, int32_t ny, uint32_t flags) {
    if (nx < 2 || ny < 2 || nx > SS_MAX_DIM || ny > SS_MAX_DIM) return 0;
    if (!(flags & SS_FLAG_DETERMINISTIC_BWD)) return 0;
    return ss::backward_det_workspace_bytes(nx, ny);
}

ss_status ss_shadow_backward_ws(const ss_heightfield* hf, const ss_rays* rays, const ss_sun* sun,
                                const ss_params* params, const int32_t* argmin,
                                const float* cost, const float* grad_light, float* grad_h,
                                double* grad_sun, void* workspace, size_t workspace_bytes,
                                uint32_t* status, ss_stream_t stream) {
    return backward_common(hf, rays, sun, params, argmin, cost, grad_light, grad_h, grad_sun,
                           workspace, workspace_bytes, status, true, stream);
}

size_t ss_batch_workspace_bytes(int32_t n_items) {
    if (n_items < 1 || n_items > (1 << 20)) return 0;
    return ss::batch_workspace_bytes(n_items);
}

ss_status ss_batch_submit(const ss_batch_item* items, int32_t n_items, const ss_params* params,
                          void* workspace, size_t workspace_bytes, ss_stream_t stream) {
    BatchPrep B;
    ss_status st = batch_prepare(items, n_items, params, workspace, workspace_bytes, B);
    if (st != SS_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    // pageable source: the call returns once the image has been staged
    cudaError_t e = cudaMemcpyAsync(static_cast<unsigned char*>(workspace) + ss::kBatchHeader,
                                    B.image.data(), B.image.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = batch_enqueue(B, items, n_items, s);
    if (e != cudaSuccess) return cuda_fail(e, "ss_batch_submit");
    return SS_OK;
}

ss_status ss_batch_plan_create(const ss_batch_item* items, int32_t n_items,
                               const ss_params* params, void* workspace, size_t workspace_bytes,
                               ss_batch_plan** plan) {
    if (!plan) return SS_ERR_INVALID_ARG;
    *plan = nullptr;
    BatchPrep B;
    ss_status st = batch_prepare(items, n_items, params, workspace, workspace_bytes, B);
    if (st != SS_OK) return st;
    cudaError_t e = cudaMemcpy(static_cast<unsigned char*>(workspace) + ss::kBatchHeader,
                               B.image.data(), B.image.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "ss_batch_plan_create (upload)");
    cudaStream_t cs;
    if ((e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking)) != cudaSuccess)
        return cuda_fail(e, "ss_batch_plan_create (stream)");
    ss_batch_plan* p = new ss_batch_plan();
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaError_t e1 = batch_enqueue(B, items, n_items, cs);
        cudaError_t e2 = cudaStreamEndCapture(cs, &p->graph);
        e = e1 != cudaSuccess ? e1 : e2;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&p->exec, p->graph, 0);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) {
        if (p->graph) cudaGraphDestroy(p->graph);
        delete p;
        return cuda_fail(e, "ss_batch_plan_create (capture)");
    }
    *plan = p;
    return SS_OK;
}

ss_status ss_batch_plan_launch(ss_batch_plan* plan, ss_stream_t stream) {
    if (!plan || !plan->exec) return SS_ERR_INVALID_ARG;
    cudaError_t e = cudaGraphLaunch(plan->exec, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "ss_batch_plan_launch");
    return SS_OK;
}

ss_status ss_batch_plan_destroy(ss_batch_plan* plan) {
    if (!plan) return SS_ERR_INVALID_ARG;
    if (plan->exec) cudaGraphExecDestroy(plan->exec);
    if (plan->graph) cudaGraphDestroy(plan->graph);
    delete plan;
    return SS_OK;
}

}  // extern "C"

// ----------------------------------------------- batch without any allocation
// Some callers cannot allocate device memory for the batch workspace: a
// renderer's per-frame loop, where cudaMalloc may synchronise the whole device
// and stall the frame; host programs whose device memory belongs to another
// allocator (an engine or framework pool) that third-party libraries must not
// bypass; code that may not call allocation routines at all.  For them,
// ss_batch_submit_static keeps its workspace in a fixed array in the library's
// device image instead of a caller buffer.
namespace {

constexpr int32_t kStaticMaxItems = SS_BATCH_STATIC_MAX_ITEMS;
constexpr size_t kStaticBytes =
    ss::kBatchHeader +
    (((size_t)kStaticMaxItems * sizeof(ss::BatchItemDesc) + 255) & ~(size_t)255) +
    (((size_t)(kStaticMaxItems + 1) * sizeof(int64_t) + 255) & ~(size_t)255);

// Every GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_batch_static_scratch[kStaticBytes];

constexpr int kMaxDevices = 256;
std::mutex g_static_mu;
void* g_static_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once
// per device (a host-side name of a __device__ array is not a device address).
ss_status static_scratch(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "ss_batch_submit_static (device)");
    if (dev < 0 || dev >= kMaxDevices) return SS_ERR_INTERNAL;
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_batch_static_scratch);
        if (e != cudaSuccess || !p) return cuda_fail(e, "ss_batch_submit_static (symbol)");
        g_static_ptr[dev] = p;
    }
    *out = g_static_ptr[dev];
    return SS_OK;
}

}  // namespace

extern "C" {

size_t ss_batch_static_scratch_bytes(void) { return kStaticBytes; }

ss_status ss_batch_submit_static(const ss_batch_item* items, int32_t n_items,
                                 const ss_params* params, ss_stream_t stream) {
    if (n_items > kStaticMaxItems) {
        snprintf(g_last_error, sizeof(g_last_error),
                 "ss_batch_submit_static: %d items exceed the static scratch limit of %d",
                 (int)n_items, (int)kStaticMaxItems);
        return SS_ERR_BAD_SIZE;
    }
    if (!items || !params) return SS_ERR_INVALID_ARG;
    if (n_items < 1) return SS_ERR_BAD_SIZE;
    void* ws = nullptr;
    ss_status st = static_scratch(&ws);
    if (st != SS_OK) return st;
    BatchPrep B;
    st = batch_prepare(items, n_items, params, ws, kStaticBytes, B);
    if (st != SS_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    // descriptors from the previous call are overwritten; the queue counter is
    // reset by batch_enqueue before the kernel runs
    cudaError_t e = cudaMemcpyAsync(static_cast<unsigned char*>(ws) + ss::kBatchHeader,
                                    B.image.data(), B.image.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = batch_enqueue(B, items, n_items, s);
    if (e != cudaSuccess) return cuda_fail(e, "ss_batch_submit_static");
    return SS_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ view rays
extern "C" {

size_t ss_view_workspace_bytes(int32_t width, int32_t height) {
    if (width < 1 || height < 1 || (int64_t)width * height >= ((int64_t)1 << 31)) return 0;
    return ss::view_workspace_bytes(width, height);
}

ss_status ss_view_rays(const ss_heightfield* hf, const float* mip, const ss_camera* cam,
                       double step_m, double max_dist_m, float* uv, int32_t* pixel,
                       int64_t* count, void* workspace, size_t workspace_bytes,
                       ss_stream_t stream) {
    ss_status st = check_tile(hf, 2);
    if (st != SS_OK) return st;
    if (!cam || !mip || !uv || !count || !workspace) return SS_ERR_INVALID_ARG;
    if (cam->width < 1 || cam->height < 1 ||
        (int64_t)cam->width * cam->height >= ((int64_t)1 << 31))
        return SS_ERR_BAD_SIZE;
    for (int k = 0; k < 3; ++k)
        if (!isfinite(cam->pos[k]) || !isfinite(cam->forward[k]) || !isfinite(cam->right[k]) ||
            !isfinite(cam->up[k]))
            return SS_ERR_INVALID_ARG;
    if (!isfinite(cam->tan_half_x) || !isfinite(cam->tan_half_y)) return SS_ERR_INVALID_ARG;
    if (!finite_pos(step_m) || !finite_pos(max_dist_m)) return SS_ERR_INVALID_ARG;
    const double K = floor(max_dist_m / step_m);
    if (!(K >= 1.0) || K >= 2147483648.0) return SS_ERR_BAD_SIZE;
    if (workspace_bytes < ss_view_workspace_bytes(cam->width, cam->height)) return SS_ERR_BAD_SIZE;
    ss::MipLayout L;
    if (!ss::mip_layout(hf->nx, hf->ny, &L)) return SS_ERR_BAD_SIZE;
    const ss_sun unused = { 0.1, 0.0, 1e-3 };   // the view kernels read only the tile geometry
    const ss::Tile T = make_tile(hf, &unused, 0, 1.0);
    const ss::Pyramid P = make_pyramid(hf, mip, L);
    ss::ViewCamera vc{};
    for (int k = 0; k < 3; ++k) {
        vc.pos[k] = cam->pos[k];
        vc.forward[k] = cam->forward[k];
        vc.right[k] = cam->right[k];
        vc.up[k] = cam->up[k];
    }
    vc.tan_x = cam->tan_half_x;
    vc.tan_y = cam->tan_half_y;
    vc.width = cam->width;
    vc.height = cam->height;
    cudaError_t e = ss::launch_view_rays(T, P, vc, step_m, (int64_t)K, mip + L.stats_offset, uv,
                                         pixel, count, workspace, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "ss_view_rays");
    return SS_OK;
}

}  // extern "C"

// ------------------------------------------------------------ greedy descent
extern "C" {

static ss_status greedy_common(const ss_heightfield* hf, const float* mip, const ss_rays* rays,
                               const ss_sun* sun, const int32_t* levels, int32_t n_runs,
                               float* light, float* cost, float* t_star, ss_stream_t stream,
                               bool f32) {
    ss_status st = check_tile(hf, 2);
    if (f32 && hf->projection != SS_PROJ_GNOMONIC) return SS_ERR_UNSUPPORTED;
    if (st != SS_OK) return st;
    if ((st = check_sun(sun)) != SS_OK) return st;
    int64_t n;
    if ((st = check_rays(rays, hf, &n)) != SS_OK) return st;
    if (!mip || !levels || n_runs < 1 || n_runs > SS_GREEDY_MAX_RUNS) return SS_ERR_INVALID_ARG;
    const int32_t L = ss_maxmip_levels(hf->nx, hf->ny);
    for (int i = 0; i < n_runs; ++i)
        if (levels[i] < 1 || levels[i] > L) return SS_ERR_INVALID_ARG;
    if (n == 0) return SS_OK;
    if (!light) return SS_ERR_INVALID_ARG;
    ss::MipLayout ML;
    if (!ss::mip_layout(hf->nx, hf->ny, &ML)) return SS_ERR_BAD_SIZE;
    const ss::Tile T = make_tile(hf, sun, 0, hf->texel_m);
    const ss::Pyramid P = make_pyramid(hf, mip, ML);
    ss::Rays R{};
    R.mode = rays->mode;
    R.n = n;
    R.uv = rays->uv;
    R.lift = rays->mode == SS_RAYS_LIST ? rays->lift_m : nullptr;
    cudaError_t e = ss::launch_greedy(T, P, R, levels, n_runs, light, cost, t_star,
                                      (cudaStream_t)stream, mip + ML.stats_offset, f32);
    if (e != cudaSuccess) return cuda_fail(e, f32 ? "ss_shadow_greedy_f32" : "ss_shadow_greedy");
    return SS_OK;
}

ss_status ss_shadow_greedy(const ss_heightfield* hf, const float* mip, const ss_rays* rays,
                           const ss_sun* sun, const int32_t* levels, int32_t n_runs,
                           float* light, float* cost, float* t_star, ss_stream_t stream) {
    return greedy_common(hf, mip, rays, sun, levels, n_runs, light, cost, t_star, stream, false);
}

ss_status ss_shadow_greedy_f32(const ss_heightfield* hf, const float* mip, const ss_rays* rays,
                               const ss_sun* sun, const int32_t* levels, int32_t n_runs,
                               float* light, float* cost, float* t_star, ss_stream_t stream) {
    return greedy_common(hf, mip, rays, sun, levels, n_runs, light, cost, t_star, stream, true);
}

}  // extern "C"

// ---------------------------------------------------------- shading epilogue
extern "C" {

ss_status ss_shade(const ss_heightfield* hf, const ss_rays* rays, const ss_light* lights,
                   int32_t n_lights, float* irradiance, ss_stream_t stream) {
    ss_status st = check_tile(hf, 2);
    if (st != SS_OK) return st;
    int64_t n;
    if ((st = check_rays(rays, hf, &n)) != SS_OK) return st;
    if (!lights || n_lights < 1 || n_lights > SS_SHADE_MAX_LIGHTS) return SS_ERR_INVALID_ARG;
    ss::ShadeLight L[ss::kShadeMaxLights];
    for (int l = 0; l < n_lights; ++l) {
        const ss_light& x = lights[l];
        if (!isfinite(x.elevation_rad) || !isfinite(x.azimuth_rad) || !isfinite(x.intensity) ||
            !(fabs(x.elevation_rad) <= M_PI / 2) || !x.lit)
            return SS_ERR_INVALID_ARG;
        L[l].elevation_rad = x.elevation_rad;
        L[l].azimuth_rad = x.azimuth_rad;
        L[l].intensity = x.intensity;
        L[l].lit = x.lit;
    }
    if (n == 0) return SS_OK;
    if (!irradiance) return SS_ERR_INVALID_ARG;
    const ss_sun unused = { 0.1, 0.0, 1e-3 };   // only the tile geometry is read
    const ss::Tile T = make_tile(hf, &unused, 0, 1.0);
    ss::Rays R{};
    R.mode = rays->mode;
    R.n = n;
    R.uv = rays->uv;
    cudaError_t e = ss::launch_shade(T, R, L, n_lights, irradiance, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "ss_shade");
    return SS_OK;
}

}  // extern "C"
