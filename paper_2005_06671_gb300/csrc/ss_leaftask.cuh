// Leaf samples as warp-wide tasks: the per-warp ring of sample tasks, each
// ray's leaf fields and running minimum in shared memory, the task pass and
// the bound of a block of samples.  Shared by the single-tile task descent
// (ss_task.cuh) and the batched kernel (batch.cu).
#pragma once

#include "ss_walk.cuh"

namespace ss {

// Ring of sample tasks per warp: 256 slots for grid rays on gnomonic tiles
// (leaf blocks of <= 4 samples, seed windows of <= 3), 512 otherwise (listed
// rays: leaf blocks of <= 8, windows of <= 5).  A lane can push one leaf block
// per walk step and kServiceSlots tasks when it draws a ray.
template <bool kGrid, bool kStereo>
struct TaskCfg {
    static constexpr int kRing = (kGrid && !kStereo) ? 256 : 512;
    static constexpr int kServiceSlots = kRing / 32;
    static constexpr int kMaxLeafLog = (kGrid && !kStereo) ? 2 : 3;   // 2^Lk <= (kRing - 31) / 32
    static constexpr int kRayWords = (kGrid && !kStereo) ? 3 : 4;      // float4 per ray
};
constexpr int kTaskWarps = 8;      // warps of a 256-thread block

template <bool kGrid, bool kStereo>
struct TaskWarp {
    using Cfg = TaskCfg<kGrid, kStereo>;
    float4 ray[32][Cfg::kRayWords];   // leaf fields of each lane's ray
    unsigned long long key[32];       // running minimum of each lane's ray
    uint32_t task[Cfg::kRing];        // (j << 5) | lane of the ray; j = 0: empty slot
};

// Order-preserving map of float bits to uint32 (for costs that are not NaN).
__device__ __forceinline__ uint32_t cost_order(float c) {
    const uint32_t b = __float_as_uint(c);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float cost_of_order(uint32_t o) {
    return __uint_as_float((o & 0x80000000u) ? (o & 0x7fffffffu) : ~o);
}
// (c + 0 turns a -0 cost into +0, which compares equal to it as a float)
__device__ __forceinline__ unsigned long long pack_key(float c, int32_t j) {
    return ((unsigned long long)cost_order(__fadd_rn(c, 0.0f)) << 32) | (uint32_t)j;
}
// +inf with no sample (j = -1): above every key a usable sample can make
constexpr unsigned long long kKeyNone = 0xff800000ffffffffull;
__device__ __forceinline__ float key_cost(unsigned long long k) {
    return cost_of_order((uint32_t)(k >> 32));
}
__device__ __forceinline__ int32_t key_j(unsigned long long k) { return (int32_t)(uint32_t)k; }

template <bool kGrid, bool kStereo>
__device__ __forceinline__ void store_leaf_ray(TaskWarp<kGrid, kStereo>& W, int slot,
                                               const RayF& r) {
    W.ray[slot][0] = make_float4(r.au_hi, r.au_lo, r.av_hi, r.av_lo);
    W.ray[slot][1] = make_float4(r.b, r.href, r.B, r.inv_2rho);
    W.ray[slot][2] = make_float4(r.inv_rho2, __int_as_float(r.iu0), __int_as_float(r.iv0), r.X);
    if constexpr (TaskCfg<kGrid, kStereo>::kRayWords > 3)
        W.ray[slot][3] = make_float4(r.u0, r.v0, r.bu, r.bv);
}

// The fields leaf_cost reads, the sums au, av rounded as in the setup.
template <bool kGrid, bool kStereo>
__device__ __forceinline__ void load_leaf_ray(const TaskWarp<kGrid, kStereo>& W, int slot,
                                              RayF& r) {
    const float4 p = W.ray[slot][0], q = W.ray[slot][1], s = W.ray[slot][2];
    r.au_hi = p.x;
    r.au_lo = p.y;
    r.av_hi = p.z;
    r.av_lo = p.w;
    r.b = q.x;
    r.href = q.y;
    r.B = q.z;
    r.inv_2rho = q.w;
    r.inv_rho2 = s.x;
    r.iu0 = __float_as_int(s.y);
    r.iv0 = __float_as_int(s.z);
    r.X = s.w;
    if constexpr (TaskCfg<kGrid, kStereo>::kRayWords > 3) {
        const float4 t = W.ray[slot][3];
        r.u0 = t.x;
        r.v0 = t.y;
        r.bu = t.z;
        r.bv = t.w;
    } else {
        r.u0 = (float)r.iu0;
        r.v0 = (float)r.iv0;
        r.bu = r.bv = 0.0f;
    }
    r.au = __fadd_rn(r.au_hi, r.au_lo);
    r.av = __fadd_rn(r.av_hi, r.av_lo);
}

// One pass over up to 32 queued tasks (warp-collective).
template <bool kGrid, bool kPoly, bool kStereo>
__device__ __forceinline__ void task_pass(const Tile& T, TaskWarp<kGrid, kStereo>& W,
                                          int32_t& head, int32_t& count, int lane) {
    constexpr int kMask = TaskCfg<kGrid, kStereo>::kRing - 1;
    const int n = min(32, count);
    if (lane < n) {
        const uint32_t t = W.task[(head + lane) & kMask];
        const int32_t j = (int32_t)(t >> 5);
        if (j > 0) {
            const int slot = (int)(t & 31u);
            RayF q;
            load_leaf_ray(W, slot, q);
            float rise;
            const float c = leaf_cost<kGrid, kPoly, kStereo>(T, q, j, rise);
            if (c < INFINITY) atomicMin(&W.key[slot], pack_key(c, j));
        }
    }
    head = (head + n) & kMask;
    count -= n;
    __syncwarp();
}

// Lower bound of the costs of samples [ja, jb] (a block probe of the exact
// descent, as in probe(): maximum-mipmap value over the block's texel
// footprint, guard for every float32 rounding), both footprint ends from
// block_end (their error is within pos_eps).
template <bool kGrid, bool kPoly, bool kStereo>
__device__ __forceinline__ float block_bound(const Tile& T, const LevelTab& L, int32_t levels,
                                             const RayF& r, int32_t ja, int32_t jb) {
    const float fa = (float)ja, fb = (float)jb;
    const float ta = __fmul_rn(fa, T.delta_f), tb = __fmul_rn(fb, T.delta_f);
    float xa, ya, xb, yb;
    block_end<kStereo>(T, r, fa, ta, kStereo ? rise_of<kPoly>(r, ta) : 0.0f, xa, ya);
    block_end<kStereo>(T, r, fb, tb, kStereo ? rise_of<kPoly>(r, tb) : 0.0f, xb, yb);
    float e = r.pos_eps;
    if (kStereo) {   // the arc bulges from its chord by at most its sagitta
        const float dx = xb - xa, dy = yb - ya;
        e += (dx * dx + dy * dy) * r.inv8r;
    }
    const int32_t x0 = max(__float2int_rd(fminf(xa, xb) - e), 0);
    const int32_t x1 = min(__float2int_rd(fmaxf(xa, xb) + e), T.nx - 2) + 1;
    const int32_t y0 = max(__float2int_rd(fminf(ya, yb) - e), 0);
    const int32_t y1 = min(__float2int_rd(fmaxf(ya, yb) + e), T.ny - 2) + 1;
    const int32_t ext = max(x1 - x0, y1 - y0);
    int32_t m = ext <= 1 ? 0 : 31 - __clz(ext);
    m += (((x1 >> m) - (x0 >> m)) > 1 || ((y1 >> m) - (y0 >> m)) > 1) ? 1 : 0;
    m = min(m, levels - 1);
    const uint32_t pm = L.pitch[m];
    const float* p = cell_ptr(L.ptr[m], pm, x0 >> m, y0 >> m);
    const uint32_t dx = (uint32_t)((x1 >> m) - (x0 >> m));
    const uint32_t dy = (uint32_t)((y1 >> m) - (y0 >> m)) * pm;
    const float V = fmaxf(fmaxf(__ldg(p), __ldg(p + dx)), fmaxf(__ldg(p + dy), __ldg(p + dy + dx))) -
                    r.href;
    const float tstar = !(r.tv > ta) ? ta : fminf(r.tv, tb);
    const float rise = rise_of<kPoly>(r, tstar);
    const float num0 = __fsub_rn(kGrid ? rise : __fadd_rn(r.X, rise), V);
    const float num = __fsub_rn(num0, fmaf(kGuardRel, fabsf(V), r.gconst));
    return __fmul_rn(num, inv_t(T, !(num >= 0.0f) ? fa : fb));
}

}  // namespace ss
