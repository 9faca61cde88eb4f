// Exact descent with warp-wide leaf tasks (the default launch of
// ss_shadow_forward for exact walks with column seeds: grid and listed rays,
// both mappings).
//
// The single-ray walk of dp_forward_kernel runs bound probes and leaf samples
// through one code path, so a warp whose lanes mix the two pays for both on
// every step.  Here the walk only bounds blocks; a leaf block that cannot be
// pruned (2^(kleaf+1) samples) is not evaluated by its lane but pushed, one
// task per sample, into a per-warp ring in shared memory, and the warp
// evaluates 32 tasks at a time, one per lane, whatever ray each belongs to.
// A ray's leaf fields live in shared memory next to its running minimum, a
// 64-bit key (orderable cost bits << 32 | sample index) that tasks lower with
// atomicMin: the smallest cost wins and, among equal costs, the smallest index,
// whatever order the tasks run in.  A walk prunes with the minimum known when
// it bounds a block; pending tasks can only lower it, so a block is pruned
// only when no sample in it can equal or beat the final minimum: the result is
// the same as dp_forward_kernel's and uniform stepping's, bit for bit (the
// tasks call the same leaf function).
//
// Scheduling follows dp_forward_kernel's column seeds: grid rays are drawn row
// by row over the block's rectangle, listed rays as LW columns of consecutive
// ids; a drawn ray pushes the samples of its seed window (around where its
// column's last finished ray has its argmin) and its first leaf block as
// tasks, and the warp evaluates them before walking.
#pragma once

#include "ss_forward.cuh"

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

template <bool kCount, bool kGrid, bool kPoly, bool kStereo>
__global__ void __launch_bounds__(256, SS_FWD_MIN_BLOCKS) dp_task_kernel(const FwdArgs a) {
    using Cfg = TaskCfg<kGrid, kStereo>;
    constexpr int kMask = Cfg::kRing - 1;
    __shared__ LevelTab s_lev;
    __shared__ int32_t s_next;
    __shared__ int32_t s_seed[kColSeedMaxW];                   // column seeds: argmin
    __shared__ float s_su[kColSeedMaxW], s_sv[kColSeedMaxW];   // and that ray's origin
    __shared__ TaskWarp<kGrid, kStereo> s_tw[kTaskWarps];
    if (threadIdx.x < kMaxLevels) {
        s_lev.ptr[threadIdx.x] = a.P.ptr[threadIdx.x];
        s_lev.pitch[threadIdx.x] = (uint32_t)a.P.pitch[threadIdx.x];
    }
    const ChunkRange P = block_pool(a, &s_next);
    // Draw order.  Grid rays: row by row over the block's rectangle (seed table
    // = its columns).  Listed rays: the run of ids read as LW columns of LH
    // consecutive ids, drawn row by row.
    const int32_t LW = P.rect ? 0 : min(kListSeedCols, P.cnt);
    const int32_t LH = LW > 0 ? (P.cnt + LW - 1) / LW : 0;
    const int32_t n_order = LW > 0 ? LW * LH : P.cnt;
    for (int i = threadIdx.x; i < (P.rect ? P.w : LW); i += blockDim.x) {
        s_seed[i] = -1;
        s_su[i] = s_sv[i] = 0.0f;
    }
    const int lane = threadIdx.x & 31;
    TaskWarp<kGrid, kStereo>& W = s_tw[threadIdx.x >> 5];
    W.key[lane] = kKeyNone;
    __syncthreads();
    const float span = a.stats[0] - a.stats[1];
    const int32_t levels = a.P.levels;
    const int32_t Lk = a.kleaf + 1;            // leaf blocks hold 2^Lk samples
    const int32_t sw = a.seed_w;
    // seed windows become tasks when they fit the slots of a drawn ray
    const bool win_tasks = 2 * sw + 1 + (1 << Lk) <= Cfg::kServiceSlots;
    int32_t head = 0, count = 0;               // the ring (same values in every lane)

    int32_t r = -1;              // local index of the lane's ray, -1 = none
    bool done = false, open = true;
    RayF rf;
    int32_t s0 = 0, k = 0, nb = 0, nl = 0;
    float best = INFINITY;
    while (true) {
        unsigned act = __ballot_sync(kFull, r >= 0 && !done);
        const unsigned want = __ballot_sync(kFull, (r < 0 || done) && open);
        if (act == 0 || __popc(want) >= a.refill_min) {
            while (count > 0) task_pass<kGrid, kPoly, kStereo>(a.T, W, head, count, lane);
            if (done) {
                const unsigned long long key = W.key[lane];
                const int32_t bj = key_j(key);
                finish_ray<kStereo, true>(a.T, a.R, a.O, chunk_ray(P, a.T.nx, r), key_cost(key),
                                          bj, nb, nl);
                if (bj > 0) {
                    const int32_t c = seed_col(P, r, LH);
                    s_seed[c] = bj;
                    if (kGrid) {
                        s_su[c] = rf.u0;
                        s_sv[c] = rf.v0;
                    }
                }
                done = false;
                r = -1;
            }
            bool fresh = false;
            int32_t prev_j = -1;
            float su = 0.0f, sv = 0.0f;
            if (open) {
                const int32_t ns = draw_strip(n_order, &s_next, r, open);
                if (ns >= 0 && r < 0) {
                    // listed rays: virtual column ns % LW, row ns / LW (the last
                    // row is padded: ids past the run draw nothing)
                    const int32_t e = LW > 0 ? (ns % LW) * LH + ns / LW : ns;
                    if (e < P.cnt) {
                        r = e;
                        fresh = true;
                        const int32_t c = LW > 0 ? ns % LW : seed_col(P, r, LH);
                        prev_j = s_seed[c];
                        su = s_su[c];
                        sv = s_sv[c];
                    }
                }
            }
            // a drawn ray: setup; its seed window and first leaf block become
            // tasks (sparse samples in the lane without a near neighbour)
            int32_t wa = 1, wb = 0, la = 1, lb = 0;
            if (fresh) {
                setup_ray<kGrid, false, kStereo>(a.T, a.R, chunk_ray(P, a.T.nx, r), span, rf);
                store_leaf_ray(W, lane, rf);
                nb = nl = 0;
                unsigned long long key = kKeyNone;
                const bool near = prev_j > 0;
                const int32_t jc = !near  ? -1
                                   : kGrid ? seed_centre(rf, prev_j, su - rf.u0, sv - rf.v0)
                                           : prev_j;
                if (near && win_tasks) {
                    wa = max(rf.j_lo, jc - sw);
                    wb = min(rf.j_hi, jc + sw);
                }
                if (wb < wa) {   // no window of usable samples: seeds in the lane
                    int32_t sj, n_seed;
                    const float sc = seed_ray<kGrid, kPoly, kStereo>(a.T, rf, near, jc, sw, true,
                                                                     sj, n_seed);
                    if (sj > 0 && sc < INFINITY) key = pack_key(sc, sj);
                    if (kCount) nl = n_seed;
                }
                W.key[lane] = key;
                la = max(rf.j_lo, 1);
                lb = min(rf.j_hi, 1 << Lk);
                s0 = 1 << Lk;
                k = Lk;
                done = rf.j_hi <= s0;   // no sample after the first leaf block (or none at all)
            }
            const int32_t nw = max(wb - wa + 1, 0), nlf = max(lb - la + 1, 0);
            const unsigned em = __ballot_sync(kFull, nw + nlf > 0);
            if (nw + nlf > 0) {
                const int32_t base = head + count + __popc(em & lanemask_lt()) * Cfg::kServiceSlots;
                for (int i = 0; i < nw + nlf; ++i) {
                    const int32_t j = i < nw ? wa + i : la + (i - nw);
                    W.task[(base + i) & kMask] = ((uint32_t)j << 5) | (uint32_t)lane;
                }
                for (int i = nw + nlf; i < Cfg::kServiceSlots; ++i)
                    W.task[(base + i) & kMask] = (uint32_t)lane;   // empty
                if (kCount) nl += nw + nlf;
            }
            count += __popc(em) * Cfg::kServiceSlots;
            __syncwarp();
            while (count > 0) task_pass<kGrid, kPoly, kStereo>(a.T, W, head, count, lane);
            if (r >= 0) best = key_cost(W.key[lane]);
            act = __ballot_sync(kFull, r >= 0 && !done);
            if (act == 0) {
                if (!__any_sync(kFull, r >= 0) && !open) break;
                continue;
            }
        }
        // one bound probe per walking lane; a leaf block that cannot be pruned
        // becomes tasks
        int32_t ea = 1, eb = 0;
        if (r >= 0 && !done) {
            const int32_t s1 = s0 + 1;
            int32_t ja = max(s1, rf.j_lo);
            int32_t jb = min(s0 + (1 << k), rf.j_hi);
            const bool valid = ja <= jb;
            ja = valid ? ja : rf.j_lo;
            jb = valid ? jb : rf.j_lo;
            const float v = block_bound<kGrid, kPoly, kStereo>(a.T, s_lev, levels, rf, ja, jb);
            const bool pass = valid && !(v > best);
            if (kCount) nb += valid ? 1 : 0;
            const bool descend = pass && k > Lk;
            if (pass && k == Lk) {
                ea = ja;
                eb = jb;
            }
            const int32_t s_adv = s0 + (1 << k);
            s0 = descend ? s0 : s_adv;
            k = descend ? k - 1 : max(__ffs(s_adv) - 1, Lk);
            done = !descend && s_adv >= rf.j_hi;
        }
        const int32_t ne = eb - ea + 1;
        const unsigned em = __ballot_sync(kFull, ne > 0);
        if (em) {
            if (ne > 0) {
                const int32_t base = head + count + (__popc(em & lanemask_lt()) << Lk);
                for (int i = 0; i < (1 << Lk); ++i) {
                    const int32_t j = i < ne ? ea + i : 0;
                    W.task[(base + i) & kMask] = ((uint32_t)j << 5) | (uint32_t)lane;
                }
                if (kCount) nl += ne;
            }
            count += __popc(em) << Lk;
            __syncwarp();
            if (count >= 32) {
                do {
                    task_pass<kGrid, kPoly, kStereo>(a.T, W, head, count, lane);
                } while (count >= 32);
                if (r >= 0) best = key_cost(W.key[lane]);
            }
        }
    }
}

}  // namespace ss
