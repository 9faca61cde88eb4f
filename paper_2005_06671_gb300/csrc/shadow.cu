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

// Final value of one ray: re-evaluate the argmin sample in FP64 when the light
// is not saturated, then apply the disc-occlusion formula (Eq. discfrac).
__device__ __forceinline__ void finish_ray(const FwdArgs& a, int64_t r, const RayF& rf,
                                           float best, int32_t bestj, int32_t nb, int32_t nl) {
    float light, cost;
    if (bestj < 0) {
        light = 1.0f;
        cost = INFINITY;
    } else {
        float d = best * rf.cos_e / a.T.alpha_f;
        if (fabsf(d) < 1.001f) {
            double up, vp, hp, href, ow[4];
            int32_t oi0, oj0;
            ray_origin(a.T, a.R, r, up, vp, hp, href, oi0, oj0, ow);
            Geom64 G;
            geom64(a.T, up, vp, hp, G);
            double c = leaf_cost64(a.T, G, bestj);
            double dd = c * G.cos_e / a.T.alpha;
            light = (float)disc_light64(dd);
            cost = (float)c;
        } else {
            light = d > 0.0f ? 1.0f : 0.0f;
            cost = best;
        }
    }
    a.O.light[r] = light;
    a.O.argmin[r] = bestj;
    if (a.O.cost) a.O.cost[r] = cost;
    if (a.O.counters) {
        a.O.counters[2 * r] = nb;
        a.O.counters[2 * r + 1] = nl;
    }
}

__device__ __forceinline__ void setup_ray(const FwdArgs& a, int64_t r, float span, RayF& rf) {
    double up, vp, hp, href, ow[4];
    int32_t oi0, oj0;
    ray_origin(a.T, a.R, r, up, vp, hp, href, oi0, oj0, ow);
    Geom64 G;
    geom64(a.T, up, vp, hp, G);
    make_rayf(a.T, G, href, span, rf);
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
// [b*rays_per_block, ...) (grid oversubscribes the SMs so the hardware block
// scheduler balances them).  Each lane walks one ray; when at least
// refill_min lanes of a warp are idle, those lanes take the next rays of the
// block pool at once (ballot + one shared-memory atomic per warp), so lanes
// whose rays finish early do not idle until the slowest lane is done.
struct BlockPool {
    int64_t lo;
    int32_t cnt;
};

__device__ __forceinline__ BlockPool block_pool(const FwdArgs& a, int32_t* s_next) {
    if (threadIdx.x == 0) *s_next = 0;
    BlockPool P;
    const int64_t n = ray_count(a.T, a.R);
    P.lo = (int64_t)blockIdx.x * a.rays_per_block;
    int64_t c = n - P.lo;
    P.cnt = (int32_t)(c < a.rays_per_block ? c : a.rays_per_block);
    return P;
}

// Returns the ray index this lane should start (or -1); updates `open`.
__device__ __forceinline__ int64_t refill(const FwdArgs& a, const BlockPool& P, int32_t* s_next,
                                          bool idle_lane, bool& open) {
    const unsigned idle = __ballot_sync(kFull, idle_lane);
    if (!open || idle == 0 || (idle != kFull && __popc(idle) < a.refill_min)) return -1;
    const int nidle = __popc(idle);
    int base = 0;
    if ((threadIdx.x & 31) == 0) base = atomicAdd(s_next, nidle);
    base = __shfl_sync(kFull, base, 0);
    if (base + nidle >= P.cnt) open = false;
    if (!idle_lane) return -1;
    const int my = base + __popc(idle & lanemask_lt());
    return my < P.cnt ? P.lo + my : -1;
}

// ---------------------------------------------------------------- descent
// Stackless depth-first walk over aligned sample blocks [s0+1, s0+2^k]:
// a block's bound (probe) is compared with the running minimum; blocks that
// cannot win are skipped, the others split; blocks of <= 2^kleaf samples are
// evaluated sample by sample.  After a block, the walk continues at
// s0 += 2^k with k = ctz(s0), the next block in near-to-far order, so samples
// are evaluated in increasing j and a strict '<' keeps the smallest j among
// equal costs.  Each loop iteration is exactly one probe per active lane.
template <bool kCount>
__global__ void __launch_bounds__(256, SS_FWD_MIN_BLOCKS) dp_forward_kernel(const FwdArgs a) {
    __shared__ const float* s_ptr[kMaxLevels];
    __shared__ int64_t s_pitch[kMaxLevels];
    __shared__ int32_t s_next;
    if (threadIdx.x < kMaxLevels) {
        s_ptr[threadIdx.x] = a.P.ptr[threadIdx.x];
        s_pitch[threadIdx.x] = a.P.pitch[threadIdx.x];
    }
    const BlockPool P = block_pool(a, &s_next);
    __syncthreads();
    const float span = a.stats[0] - a.stats[1];
    const int32_t kleaf = a.kleaf, levels = a.P.levels;

    int64_t r = -1;
    RayF rf;
    float best = INFINITY;
    int32_t bestj = -1, nb = 0, nl = 0, s0 = 0, k = 0;
    bool open = true;
    while (true) {
        const int64_t nr = refill(a, P, &s_next, r < 0, open);
        if (nr >= 0) {
            r = nr;
            setup_ray(a, r, span, rf);
            best = INFINITY;
            bestj = -1;
            nb = nl = s0 = 0;
            const int32_t K = rf.j_hi <= 1 ? 0 : 32 - __clz(rf.j_hi - 1);   // 2^K >= j_hi
            k = K > kleaf ? K : 0;
            if (rf.j_hi < rf.j_lo) {   // no usable sample
                finish_ray(a, r, rf, best, bestj, 0, 0);
                r = -1;
            }
        }
        if (__ballot_sync(kFull, r >= 0) == 0) {
            if (!open) break;
            continue;
        }
        if (r < 0) continue;
        const bool leaf = (k == 0);
        int32_t ja = leaf ? s0 + 1 : max(s0 + 1, rf.j_lo);
        int32_t jb = leaf ? s0 + 1 : min(s0 + (1 << k), rf.j_hi);
        const bool valid = leaf ? (ja >= rf.j_lo) : (ja <= jb);
        if (!valid) ja = jb = rf.j_lo;   // keep the probe in range; result unused
        const float v = probe(a.T, s_ptr, s_pitch, levels, rf, ja, jb, leaf);
        bool advance = true;
        if (valid) {
            if (leaf) {
                if (kCount) ++nl;
                if (v < best) {
                    best = v;
                    bestj = ja;
                }
            } else {
                if (kCount) ++nb;
                if (!(v > best)) {
                    k = (k - 1 > kleaf) ? k - 1 : 0;
                    advance = false;
                }
            }
        }
        if (advance) {
            s0 += 1 << k;
            if (s0 >= rf.j_hi) {
                finish_ray(a, r, rf, best, bestj, nb, nl);
                r = -1;
            } else {
                k = __ffs(s0) - 1;
                if (k <= kleaf) k = 0;
            }
        }
    }
}

// ---------------------------------------------------------------- uniform
// Every usable sample in order, same scheduling as the descent.  Early exit
// (exact): with H(t) = h_p + rise(t) convex and H(0) = h_p <= max h,
// g(t) = (H(t) - max h - G)/t is non-decreasing and bounds every later
// sample's cost from below; once g(t_j) >= best no later sample can win.
// G = 3 guards covers the float32 rounding of both sides.
template <bool kCount>
__global__ void __launch_bounds__(256, SS_FWD_MIN_BLOCKS) uniform_forward_kernel(const FwdArgs a) {
    __shared__ int32_t s_next;
    const BlockPool P = block_pool(a, &s_next);
    __syncthreads();
    const float hmax = a.stats[0];
    const float span = a.stats[0] - a.stats[1];
    const bool allow_exit = !(a.flags & 0x2u);

    int64_t r = -1;
    RayF rf;
    float best = INFINITY, hmax_rel = 0.0f, G = 0.0f;
    int32_t bestj = -1, nl = 0, j = 0;
    bool exit_ok = false, open = true;
    while (true) {
        const int64_t nr = refill(a, P, &s_next, r < 0, open);
        if (nr >= 0) {
            r = nr;
            setup_ray(a, r, span, rf);
            best = INFINITY;
            bestj = -1;
            nl = 0;
            j = rf.j_lo;
            hmax_rel = hmax - rf.href;
            exit_ok = allow_exit && (rf.X <= hmax_rel);
            const float tJ = (float)rf.j_hi * a.T.delta_f;
            const float rb = fmaxf(rise_bound(rf, tJ), 0.25f * rf.B * rf.B * rf.inv_rho);
            G = 3.0f * kGuardRel * (rf.guard0 + fabsf(hmax_rel) + rb);
            if (rf.j_hi < rf.j_lo) {
                finish_ray(a, r, rf, best, bestj, 0, 0);
                r = -1;
            }
        }
        if (__ballot_sync(kFull, r >= 0) == 0) {
            if (!open) break;
            continue;
        }
        if (r < 0) continue;
        float rise;
        const float c = leaf_cost(a.T, rf, j, &rise);
        if (kCount) ++nl;
        if (c < best) {
            best = c;
            bestj = j;
        }
        bool done = (j >= rf.j_hi);
        if (!done && exit_ok && (j & 3) == 0) {
            const float t = __fmul_rn((float)j, a.T.delta_f);
            const float g = (((rf.X + rise) - hmax_rel) - G) / t;
            done = (g >= best);
        }
        ++j;
        if (done) {
            finish_ray(a, r, rf, best, bestj, 0, nl);
            r = -1;
        }
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

cudaError_t launch_dp_forward(const FwdArgs& a, int block, cudaStream_t s) {
    const int grid = pool_grid(a);
    if (a.O.counters)
        dp_forward_kernel<true><<<grid, block, 0, s>>>(a);
    else
        dp_forward_kernel<false><<<grid, block, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_uniform_forward(const FwdArgs& a, int block, cudaStream_t s) {
    const int grid = pool_grid(a);
    if (a.O.counters)
        uniform_forward_kernel<true><<<grid, block, 0, s>>>(a);
    else
        uniform_forward_kernel<false><<<grid, block, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_backward(const BwdArgs& a, int block, cudaStream_t s) {
    int64_t n = a.R.mode == 0 ? (int64_t)a.T.nx * a.T.ny : a.R.n;
    backward_kernel<<<resident_grid(backward_kernel, block, n), block, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace ss
