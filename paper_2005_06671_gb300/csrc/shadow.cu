// Forward (exact max-mip descent and uniform stepping) and backward kernels.
//
// Work decomposition: one thread walks one shadow ray at a time; each block
// owns a contiguous range of ray ids (grid mode: row-major texels, so a warp's
// rays are neighbours whose samples touch neighbouring texels) and its lanes
// draw rays from that range as they finish (see refill()).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "ss_launch.h"
#include "ss_walk.cuh"

namespace ss {

// Minimum resident 256-thread blocks per SM for the forward kernels (caps
// registers at 65536 / (256 * SS_FWD_MIN_BLOCKS)).
#ifndef SS_FWD_MIN_BLOCKS
#define SS_FWD_MIN_BLOCKS 4
#endif

// Scheduling shared by both forward kernels.  Block b owns rays
// [b*rays_per_block, ...) (the grid oversubscribes the SMs so the hardware
// block scheduler balances them).  Each lane walks one ray.  A lane whose ray
// is finished keeps its result in registers and waits; once at least
// refill_min lanes of the warp are waiting (or all are), the warp services
// them together: finished rays are written, and the waiting lanes draw the
// next rays of the block pool (one shared-memory atomic per warp).
__device__ __forceinline__ ChunkRange block_pool(const FwdArgs& a, int32_t* s_next) {
    if (threadIdx.x == 0) *s_next = 0;
    return chunk_range(blockIdx.x, ray_count(a.T, a.R), a.T.nx, a.T.ny, (int32_t)a.rays_per_block,
                       a.R.mode == 0 ? a.tile_w : 0);
}

// Draw rays for this warp's lanes with r < 0; returns the new local index or -1.
__device__ __forceinline__ int32_t draw(const ChunkRange& P, int32_t* s_next, int32_t r,
                                        bool& open) {
    const unsigned idle = __ballot_sync(kFull, r < 0);
    const int nidle = __popc(idle);
    int base = 0;
    if ((threadIdx.x & 31) == 0 && nidle > 0) base = atomicAdd(s_next, nidle);
    base = __shfl_sync(kFull, base, 0);
    if (base + nidle >= P.cnt) open = false;
    if (r >= 0) return r;
    const int my = base + __popc(idle & lanemask_lt());
    return my < P.cnt ? my : -1;
}

// ---------------------------------------------------------------- descent
// Each loop iteration is one probe of the exact descent (walk_step) per
// walking lane.
template <bool kCount, bool kGrid, bool kPoly, bool kLight>
__global__ void __launch_bounds__(256, SS_FWD_MIN_BLOCKS) dp_forward_kernel(const FwdArgs a) {
    __shared__ LevelTab s_lev;
    __shared__ int32_t s_next;
    if (threadIdx.x < kMaxLevels) {
        s_lev.ptr[threadIdx.x] = a.P.ptr[threadIdx.x];
        s_lev.pitch[threadIdx.x] = (uint32_t)a.P.pitch[threadIdx.x];
    }
    const ChunkRange P = block_pool(a, &s_next);
    __syncthreads();
    const float span = a.stats[0] - a.stats[1];
    const int32_t kleaf = a.kleaf, levels = a.P.levels;

    int32_t r = -1;
    bool done = false, open = true;
    RayF rf;
    Walk w;
    w.best = INFINITY;
    w.bestj = -1;
    while (true) {
        unsigned act = __ballot_sync(kFull, r >= 0 && !done);
        if (act == 0 || (open && __popc(~act) >= a.refill_min)) {
            if (done) {
                finish_ray(a.T, a.R, a.O, chunk_ray(P, a.T.nx, r), w.best, w.bestj, w.nb, w.nl);
                r = -1;
                done = false;
            }
            if (open) {
                const int32_t nr = draw(P, &s_next, r, open);
                if (nr >= 0 && r < 0) {
                    r = nr;
                    setup_ray<kGrid, kLight>(a.T, a.R, chunk_ray(P, a.T.nx, r), span, rf);
                    walk_begin<kLight>(w, rf, kleaf);
                    if (rf.j_hi < rf.j_lo) {   // no usable sample: written at once
                        finish_ray(a.T, a.R, a.O, chunk_ray(P, a.T.nx, r), w.best, w.bestj, 0, 0);
                        r = -1;
                    }
                }
            }
            act = __ballot_sync(kFull, r >= 0 && !done);
            if (act == 0) {
                if (!open) break;
                continue;
            }
        }
        if (r < 0 || done) continue;
        done = walk_step<kCount, kGrid, kPoly, kLight>(a.T, s_lev, levels, kleaf, rf, w);
    }
}

// ---------------------------------------------------------------- uniform
// Every usable sample in order, same scheduling as the descent.  Early exit
// (exact): with H(t) = h_p + rise(t) convex and H(0) = h_p <= max h,
// g(t) = (H(t) - max h - G)/t is non-decreasing and bounds every later
// sample's cost from below; once g(t_j) >= best no later sample can win.
// G = 3 guards covers the float32 rounding of both sides.
template <bool kCount, bool kGrid, bool kPoly, bool kLight>
__global__ void __launch_bounds__(256, SS_FWD_MIN_BLOCKS) uniform_forward_kernel(const FwdArgs a) {
    __shared__ int32_t s_next;
    const ChunkRange P = block_pool(a, &s_next);
    __syncthreads();
    const float hmax = a.stats[0];
    const float span = a.stats[0] - a.stats[1];
    const bool allow_exit = !(a.flags & 0x2u);

    int32_t r = -1;
    bool done = false, open = true;
    RayF rf;
    float best = INFINITY, hmax_rel = 0.0f, G = 0.0f;
    int32_t bestj = -1, nl = 0, j = 0;
    bool exit_ok = false;
    while (true) {
        unsigned act = __ballot_sync(kFull, r >= 0 && !done);
        if (act == 0 || (open && __popc(~act) >= a.refill_min)) {
            if (done) {
                finish_ray(a.T, a.R, a.O, chunk_ray(P, a.T.nx, r), best, bestj, 0, nl);
                r = -1;
                done = false;
            }
            if (open) {
                const int32_t nr = draw(P, &s_next, r, open);
                if (nr >= 0 && r < 0) {
                    r = nr;
                    setup_ray<kGrid, kLight>(a.T, a.R, chunk_ray(P, a.T.nx, r), span, rf);
                    best = kLight ? rf.c_sat : INFINITY;
                    bestj = -1;
                    nl = 0;
                    j = rf.j_lo;
                    hmax_rel = hmax - rf.href;
                    exit_ok = allow_exit && (rf.X <= hmax_rel);
                    const float tJ = (float)rf.j_hi * a.T.delta_f;
                    const float rb = fmaxf(rise_bound(rf, tJ),
                                           0.5f * rf.B * rf.B * rf.inv_2rho);
                    G = 3.0f * kGuardRel * (rf.guard0 + fabsf(hmax_rel) + rb);
                    if (rf.j_hi < rf.j_lo) {   // no usable sample: written at once
                        finish_ray(a.T, a.R, a.O, chunk_ray(P, a.T.nx, r), best, bestj, 0, 0);
                        r = -1;
                    }
                }
            }
            act = __ballot_sync(kFull, r >= 0 && !done);
            if (act == 0) {
                if (!open) break;
                continue;
            }
        }
        if (r < 0 || done) continue;
        float rise;
        const float c = leaf_cost<kGrid, kPoly>(a.T, rf, j, rise);
        if (kCount) ++nl;
        const bool improve = c < best;
        best = improve ? c : best;
        bestj = improve ? j : bestj;
        bool stop = (j >= rf.j_hi);
        if (exit_ok && (j & 3) == 0) {
            const float t = __fmul_rn((float)j, a.T.delta_f);
            const float h = kGrid ? rise : rf.X + rise;
            stop = stop || ((h - hmax_rel) - G) / t >= best;
        }
        ++j;
        done = kLight ? (stop || best <= -rf.c_sat) : stop;
    }
}

// ---------------------------------------------------------------- backward
// d light / d (heights, sun) at the forward argmin, FP64 per ray (only rays in
// the penumbra have a non-zero gradient).  Heights: atomicAdd (float32);
// sun: block reduction in FP64, then one atomicAdd per block and component.
__global__ void __launch_bounds__(256) backward_kernel(const BwdArgs a) {
    const int64_t n = ray_count(a.T, a.R);
    double gs[5] = { 0.0, 0.0, 0.0, 0.0, 0.0 };
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += stride) {
        int32_t j = a.argmin[r];
        float gl = a.grad_light[r];
        if (j < 1 || gl == 0.0f) continue;
        // the forward's float32 cost rules out rays whose light is certainly
        // saturated (the same test the forward uses before its FP64 re-evaluation)
        if (a.cost && fabsf(a.cost[r]) * cos_elev_f32(a.T, a.R, r) >= 1.001f * a.T.alpha_f)
            continue;
        double up, vp, hp, href, ow[4];
        int32_t oi0, oj0;
        ray_origin(a.T, a.R, r, up, vp, hp, href, oi0, oj0, ow);
        Geom64 G;
        geom64(a.T, up, vp, hp, G);
        double U, V;
        double c = leaf_cost64(a.T, G, j, &U, &V);
        const double cos_e = cos_elev(G);
        double d = c * cos_e / a.T.alpha;
        if (!(d > -1.0 && d < 1.0)) continue;
        double gd = (double)gl * (2.0 / M_PI) * sqrt(1.0 - d * d);   // dL/dd
        double gc = gd * cos_e / a.T.alpha;                         // dL/dc
        double t = (double)j * a.T.delta;
        // sample texels and the bilinear gradient at (U, V)
        int32_t i0 = (int32_t)floor(U), j0 = (int32_t)floor(V);
        i0 = min(max(i0, 0), a.T.nx - 2);
        j0 = min(max(j0, 0), a.T.ny - 2);
        double fu = U - i0, fv = V - j0;
        const float* hr = a.T.h + (int64_t)j0 * a.T.pitch + i0;
        double h00 = hr[0], h10 = hr[1], h01 = hr[a.T.pitch], h11 = hr[a.T.pitch + 1];
        double du = (1.0 - fv) * (h10 - h00) + fv * (h11 - h01);
        double dv = (1.0 - fu) * (h01 - h00) + fu * (h11 - h10);
        double w[4] = { (1.0 - fu) * (1.0 - fv), fu * (1.0 - fv), (1.0 - fu) * fv, fu * fv };
        float* gp = a.grad_h + (int64_t)j0 * a.grad_pitch + i0;
        atomicAdd(gp, (float)(-gc * w[0] / t));
        atomicAdd(gp + 1, (float)(-gc * w[1] / t));
        atomicAdd(gp + a.grad_pitch, (float)(-gc * w[2] / t));
        atomicAdd(gp + a.grad_pitch + 1, (float)(-gc * w[3] / t));
        // origin height: moves the ray up along n_p and shifts its texel image
        double B = 2.0 * G.rho * G.sin_e;
        double qn = sqrt(G.rho * G.rho + t * (B + t));
        double dHdhp = (G.rho + t * G.sin_e) / qn;
        double jd = (double)j, den = 1.0 + G.b * jd;
        double dUdhp = -G.Au * jd / (G.rho * den * den);
        double dVdhp = -G.Av * jd / (G.rho * den * den);
        double dcdhp = (dHdhp - (du * dUdhp + dv * dVdhp)) / t;
        float* go = a.grad_h + (int64_t)oj0 * a.grad_pitch + oi0;
        double go_s = gc * dcdhp;
        if (ow[0] != 0.0) atomicAdd(go, (float)(go_s * ow[0]));
        if (ow[1] != 0.0) atomicAdd(go + 1, (float)(go_s * ow[1]));
        if (ow[2] != 0.0) atomicAdd(go + a.grad_pitch, (float)(go_s * ow[2]));
        if (ow[3] != 0.0) atomicAdd(go + a.grad_pitch + 1, (float)(go_s * ow[3]));
        // sun direction: q = p + t s; dc/ds = q/|q| - grad_q h(texel image of q)
        double q[3] = { G.rho * G.nhat[0] + t * a.T.sx, G.rho * G.nhat[1] + t * a.T.sy,
                        G.rho * G.nhat[2] + t * a.T.sz };
        double kq = a.T.R / a.T.g;
        double JU[3] = { kq / q[2], 0.0, -kq * q[0] / (q[2] * q[2]) };
        double JV[3] = { 0.0, kq / q[2], -kq * q[1] / (q[2] * q[2]) };
        double ce_term = cos_e > 0.0 ? (-G.sin_e / cos_e) : 0.0;
        double gsv[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            double dcds = q[i] / qn - (du * JU[i] + dv * JV[i]);
            gsv[i] = gc * dcds + gd * (c / a.T.alpha) * ce_term * G.nhat[i];
        }
        gs[0] += gsv[0] * a.ds_de[0] + gsv[1] * a.ds_de[1] + gsv[2] * a.ds_de[2];
        gs[1] += gsv[0] * a.ds_da[0] + gsv[1] * a.ds_da[1] + gsv[2] * a.ds_da[2];
        gs[2] += gsv[0];
        gs[3] += gsv[1];
        gs[4] += gsv[2];
    }
    // block reduction of the sun gradient
    __shared__ double red[5][8];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        double v = gs[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) red[k][threadIdx.x >> 5] = v;
    }
    __syncthreads();
    if (threadIdx.x < 5) {
        double v = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[threadIdx.x][w];
        if (v != 0.0) atomicAdd(a.grad_sun + threadIdx.x, v);
    }
}

// ---------------------------------------------------------------- launchers
static int g_sm_count = 0;

int device_sm_count() {
    if (g_sm_count == 0) {
        int dev = 0, n = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess)
            g_sm_count = n;
        else
            g_sm_count = 1;
    }
    return g_sm_count;
}

// Grid-stride kernels: one wave of resident blocks (occupancy x SMs), fewer
// when there is not enough work.
template <typename K>
static int resident_grid(K kernel, int block, int64_t n_threads) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, 0) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    int64_t cap = (int64_t)device_sm_count() * per_sm;
    int64_t want = (n_threads + block - 1) / block;
    if (want < 1) want = 1;
    return (int)(want < cap ? want : cap);
}

static int pool_grid(const FwdArgs& a) {
    const int64_t n = a.R.mode == 0 ? (int64_t)a.T.nx * a.T.ny : a.R.n;
    return (int)chunk_count(n, a.T.nx, a.T.ny, (int32_t)a.rays_per_block,
                            a.R.mode == 0 ? a.tile_w : 0);
}

#define SS_FWD_CASE(C, G, P, L) \
    case ((C) << 3) | ((G) << 2) | ((P) << 1) | (L): return Launch<C, G, P, L>::go(a, grid, block, s);

// runtime flags -> the kernel instance (counters, grid mode, rise series, light-only)
template <template <bool, bool, bool, bool> class Launch>
static cudaError_t dispatch(const FwdArgs& a, int block, cudaStream_t s) {
    const int idx = ((a.O.counters != nullptr) << 3) | ((a.R.mode == 0) << 2) | ((a.poly != 0) << 1) |
                    ((a.flags & 0x4u) ? 1 : 0);
    const int grid = pool_grid(a);
    switch (idx) {
        SS_FWD_CASE(0, 0, 0, 0) SS_FWD_CASE(0, 0, 0, 1) SS_FWD_CASE(0, 0, 1, 0) SS_FWD_CASE(0, 0, 1, 1)
        SS_FWD_CASE(0, 1, 0, 0) SS_FWD_CASE(0, 1, 0, 1) SS_FWD_CASE(0, 1, 1, 0) SS_FWD_CASE(0, 1, 1, 1)
        SS_FWD_CASE(1, 0, 0, 0) SS_FWD_CASE(1, 0, 0, 1) SS_FWD_CASE(1, 0, 1, 0) SS_FWD_CASE(1, 0, 1, 1)
        SS_FWD_CASE(1, 1, 0, 0) SS_FWD_CASE(1, 1, 0, 1) SS_FWD_CASE(1, 1, 1, 0) SS_FWD_CASE(1, 1, 1, 1)
    }
    return cudaErrorInvalidValue;
}
#undef SS_FWD_CASE

template <bool C, bool G, bool P, bool L>
struct DpLaunch {
    static cudaError_t go(const FwdArgs& a, int grid, int block, cudaStream_t s) {
        dp_forward_kernel<C, G, P, L><<<grid, block, 0, s>>>(a);
        return cudaGetLastError();
    }
};

template <bool C, bool G, bool P, bool L>
struct UniLaunch {
    static cudaError_t go(const FwdArgs& a, int grid, int block, cudaStream_t s) {
        uniform_forward_kernel<C, G, P, L><<<grid, block, 0, s>>>(a);
        return cudaGetLastError();
    }
};

cudaError_t launch_dp_forward(const FwdArgs& a, int block, cudaStream_t s) {
    return dispatch<DpLaunch>(a, block, s);
}

cudaError_t launch_uniform_forward(const FwdArgs& a, int block, cudaStream_t s) {
    return dispatch<UniLaunch>(a, block, s);
}

cudaError_t launch_backward(const BwdArgs& a, int block, cudaStream_t s) {
    int64_t n = a.R.mode == 0 ? (int64_t)a.T.nx * a.T.ny : a.R.n;
    backward_kernel<<<resident_grid(backward_kernel, block, n), block, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace ss
