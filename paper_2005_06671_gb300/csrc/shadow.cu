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

namespace ss {

__device__ __forceinline__ int64_t ray_count(const Tile& T, const Rays& R) {
    return R.mode == 0 ? (int64_t)T.nx * T.ny : R.n;
}

// cos(eps_p) of ray r's origin in float32 (relative error ~1e-7), enough to
// decide whether its light is saturated.
__device__ __forceinline__ float cos_elev_f32(const FwdArgs& a, int64_t r) {
    float u, v;
    if (a.R.mode == 0) {
        const int64_t vv = r / a.T.nx;
        u = (float)(r - vv * a.T.nx);
        v = (float)vv;
    } else {
        u = a.R.uv[2 * r];
        v = a.R.uv[2 * r + 1];
    }
    const float g = (float)a.T.g, R = (float)a.T.R;
    const float X = (u - (float)a.T.cx) * g, Y = (v - (float)a.T.cy) * g;
    const float se = (X * (float)a.T.sx + Y * (float)a.T.sy + R * (float)a.T.sz) *
                     rsqrtf(X * X + Y * Y + R * R);
    return sqrtf(fmaxf(0.0f, 1.0f - se * se));
}

// Final value of one ray: re-evaluate the argmin sample in FP64 unless the
// light is certainly saturated (|c*| cos(eps) >= 1.001 alpha), then the
// disc-occlusion formula (Eq. discfrac).
__device__ __forceinline__ void finish_ray(const FwdArgs& a, int64_t r, float best,
                                           int32_t bestj, int32_t nb, int32_t nl) {
    float light, cost;
    if (bestj < 0) {
        light = 1.0f;
        cost = INFINITY;
    } else if (fabsf(best) * cos_elev_f32(a, r) >= 1.001f * a.T.alpha_f) {
        light = best > 0.0f ? 1.0f : 0.0f;
        cost = best;
    } else {
        double up, vp, hp, href, ow[4];
        int32_t oi0, oj0;
        ray_origin(a.T, a.R, r, up, vp, hp, href, oi0, oj0, ow);
        Geom64 G;
        geom64(a.T, up, vp, hp, G);
        double c = leaf_cost64(a.T, G, bestj);
        light = (float)disc_light64(c * G.cos_e / a.T.alpha);
        cost = (float)c;
    }
    a.O.light[r] = light;
    a.O.argmin[r] = bestj;
    if (a.O.cost) a.O.cost[r] = cost;
    if (a.O.counters) {
        a.O.counters[2 * r] = nb;
        a.O.counters[2 * r + 1] = nl;
    }
}

template <bool kGrid>
__device__ __forceinline__ void setup_ray(const FwdArgs& a, int64_t r, float span, RayF& rf) {
    double up, vp, hp, href;
    if (kGrid) {
        const int64_t v = r / a.T.nx, u = r - v * a.T.nx;
        up = (double)u;
        vp = (double)v;
        hp = href = (double)a.T.h[v * a.T.pitch + u];
    } else {
        double ow[4];
        int32_t oi0, oj0;
        ray_origin(a.T, a.R, r, up, vp, hp, href, oi0, oj0, ow);
    }
    Geom64 G;
    geom64(a.T, up, vp, hp, G);
    make_rayf(a.T, G, href, span, rf);
    if (kGrid) rf.X = 0.0f;
}

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

constexpr unsigned kFull = 0xffffffffu;

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
struct BlockPool {
    int64_t lo;
    int32_t cnt;
};

__device__ __forceinline__ BlockPool block_pool(const FwdArgs& a, int32_t* s_next) {
    if (threadIdx.x == 0) *s_next = 0;
    BlockPool P;
    const int64_t n = ray_count(a.T, a.R);
    P.lo = (int64_t)blockIdx.x * a.rays_per_block;
    const int64_t c = n - P.lo;
    P.cnt = (int32_t)(c < a.rays_per_block ? c : a.rays_per_block);
    return P;
}

// Draw rays for this warp's lanes with r < 0; returns the new local index or -1.
__device__ __forceinline__ int32_t draw(const BlockPool& P, int32_t* s_next, int32_t r,
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
// Stackless depth-first walk over aligned sample blocks [s0+1, s0+2^k]:
// a block's bound (probe) is compared with the running minimum; blocks that
// cannot win are skipped, the others split; blocks of <= 2^kleaf samples are
// evaluated sample by sample.  After a block, the walk continues at
// s0 += 2^k with k = ctz(s0), the next block in near-to-far order, so samples
// are evaluated in increasing j and a strict '<' keeps the smallest j among
// equal costs.  Each loop iteration is exactly one probe per walking lane.
// Blocks are aligned to their size, so for k = ctz(s0) the block may end past
// j_hi; it is clipped.  The leaf level bounds the smallest block that gets a
// bound probe: runs of 2^(kleaf+1) samples are evaluated directly.
template <bool kCount, bool kGrid, bool kPoly>
__global__ void __launch_bounds__(256, SS_FWD_MIN_BLOCKS) dp_forward_kernel(const FwdArgs a) {
    __shared__ LevelTab s_lev;
    __shared__ int32_t s_next;
    if (threadIdx.x < kMaxLevels) {
        s_lev.ptr[threadIdx.x] = a.P.ptr[threadIdx.x];
        s_lev.pitch[threadIdx.x] = (uint32_t)a.P.pitch[threadIdx.x];
    }
    const BlockPool P = block_pool(a, &s_next);
    __syncthreads();
    const float span = a.stats[0] - a.stats[1];
    const int32_t kleaf = a.kleaf, levels = a.P.levels;

    int32_t r = -1;
    bool done = false, open = true;
    RayF rf;
    float best = INFINITY;
    int32_t bestj = -1, nb = 0, nl = 0, s0 = 0, k = 0;
    while (true) {
        unsigned act = __ballot_sync(kFull, r >= 0 && !done);
        if (act == 0 || (open && __popc(~act) >= a.refill_min)) {
            if (done) {
                finish_ray(a, P.lo + r, best, bestj, nb, nl);
                r = -1;
                done = false;
            }
            if (open) {
                const int32_t nr = draw(P, &s_next, r, open);
                if (nr >= 0 && r < 0) {
                    r = nr;
                    setup_ray<kGrid>(a, P.lo + r, span, rf);
                    best = INFINITY;
                    bestj = -1;
                    nb = nl = s0 = 0;
                    // While best is +inf every block on the left spine is split
                    // without a bound being able to prune it, so the walk starts
                    // directly with the first run of leaves (same order, same result).
                    k = 0;
                    if (rf.j_hi < rf.j_lo) {   // no usable sample: written at once
                        finish_ray(a, P.lo + r, best, bestj, 0, 0);
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
        const bool leaf = (k == 0);
        const int32_t s1 = s0 + 1;
        int32_t ja = leaf ? s1 : max(s1, rf.j_lo);
        int32_t jb = leaf ? s1 : min(s0 + (1 << k), rf.j_hi);
        const bool valid = leaf ? (s1 >= rf.j_lo) : (ja <= jb);
        ja = valid ? ja : rf.j_lo;
        jb = valid ? jb : rf.j_lo;
        const float v = probe<kGrid, kPoly>(a.T, s_lev, levels, rf, ja, jb, leaf);
        const bool improve = valid && leaf && (v < best);
        best = improve ? v : best;
        bestj = improve ? ja : bestj;
        const bool descend = valid && !leaf && !(v > best);
        if (kCount) {
            nl += (valid && leaf) ? 1 : 0;
            nb += (valid && !leaf) ? 1 : 0;
        }
        const int32_t s_adv = s0 + (1 << k);
        const int32_t k_adv = __ffs(s_adv) - 1;
        s0 = descend ? s0 : s_adv;
        k = descend ? ((k - 1 > kleaf) ? k - 1 : 0) : ((k_adv <= kleaf) ? 0 : k_adv);
        done = !descend && (s_adv >= rf.j_hi);
    }
}

// ---------------------------------------------------------------- uniform
// Every usable sample in order, same scheduling as the descent.  Early exit
// (exact): with H(t) = h_p + rise(t) convex and H(0) = h_p <= max h,
// g(t) = (H(t) - max h - G)/t is non-decreasing and bounds every later
// sample's cost from below; once g(t_j) >= best no later sample can win.
// G = 3 guards covers the float32 rounding of both sides.
template <bool kCount, bool kGrid, bool kPoly>
__global__ void __launch_bounds__(256, SS_FWD_MIN_BLOCKS) uniform_forward_kernel(const FwdArgs a) {
    __shared__ int32_t s_next;
    const BlockPool P = block_pool(a, &s_next);
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
                finish_ray(a, P.lo + r, best, bestj, 0, nl);
                r = -1;
                done = false;
            }
            if (open) {
                const int32_t nr = draw(P, &s_next, r, open);
                if (nr >= 0 && r < 0) {
                    r = nr;
                    setup_ray<kGrid>(a, P.lo + r, span, rf);
                    best = INFINITY;
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
                        finish_ray(a, P.lo + r, best, bestj, 0, 0);
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
        done = stop;
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
        double up, vp, hp, href, ow[4];
        int32_t oi0, oj0;
        ray_origin(a.T, a.R, r, up, vp, hp, href, oi0, oj0, ow);
        Geom64 G;
        geom64(a.T, up, vp, hp, G);
        double U, V;
        double c = leaf_cost64(a.T, G, j, &U, &V);
        double d = c * G.cos_e / a.T.alpha;
        if (!(d > -1.0 && d < 1.0)) continue;
        double gd = (double)gl * (2.0 / M_PI) * sqrt(1.0 - d * d);   // dL/dd
        double gc = gd * G.cos_e / a.T.alpha;                         // dL/dc
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
        double ce_term = G.cos_e > 0.0 ? (-G.sin_e / G.cos_e) : 0.0;
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
    int64_t n = a.R.mode == 0 ? (int64_t)a.T.nx * a.T.ny : a.R.n;
    return (int)((n + a.rays_per_block - 1) / a.rays_per_block);
}

template <template <bool, bool, bool> class Launch>
static cudaError_t dispatch(const FwdArgs& a, int block, cudaStream_t s) {
    const bool cnt = a.O.counters != nullptr, grid = a.R.mode == 0, poly = a.poly != 0;
    const int g = pool_grid(a);
    if (cnt) {
        if (grid) return poly ? Launch<true, true, true>::go(a, g, block, s) : Launch<true, true, false>::go(a, g, block, s);
        return poly ? Launch<true, false, true>::go(a, g, block, s) : Launch<true, false, false>::go(a, g, block, s);
    }
    if (grid) return poly ? Launch<false, true, true>::go(a, g, block, s) : Launch<false, true, false>::go(a, g, block, s);
    return poly ? Launch<false, false, true>::go(a, g, block, s) : Launch<false, false, false>::go(a, g, block, s);
}

template <bool C, bool G, bool P>
struct DpLaunch {
    static cudaError_t go(const FwdArgs& a, int grid, int block, cudaStream_t s) {
        dp_forward_kernel<C, G, P><<<grid, block, 0, s>>>(a);
        return cudaGetLastError();
    }
};

template <bool C, bool G, bool P>
struct UniLaunch {
    static cudaError_t go(const FwdArgs& a, int grid, int block, cudaStream_t s) {
        uniform_forward_kernel<C, G, P><<<grid, block, 0, s>>>(a);
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
