// Forward kernels (exact max-mip descent, light-only descent, uniform
// stepping, and the FP64 re-evaluation of penumbra rays), templated on the
// tile mapping; fwd_gnomonic.cu and fwd_stereo.cu each instantiate one mapping
// so the two compile in parallel.
//
// Work decomposition: one thread walks one shadow ray at a time; each block
// owns a contiguous range of ray ids (grid mode: row-major texels, so a warp's
// rays are neighbours whose samples touch neighbouring texels) and its lanes
// draw rays from that range as they finish.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "ss_launch.h"
#include "ss_walk.cuh"
#include "ss_strip.cuh"

namespace ss {

// Minimum resident 256-thread blocks per SM for the forward kernels (caps
// registers at 65536 / (256 * SS_FWD_MIN_BLOCKS)).
#ifndef SS_FWD_MIN_BLOCKS
#define SS_FWD_MIN_BLOCKS 4
#endif

// Scheduling of the exact descent and uniform stepping (the light-only descent
// parks set-up rays first, see dp_light_kernel).  Block b owns rays
// [b*rays_per_block, ...) (the grid oversubscribes the SMs so the hardware
// block scheduler balances them).  Each lane walks one ray.  A lane whose ray
// is finished keeps its result in registers and waits; once at least
// refill_min lanes of the warp are waiting (or all are), the warp services
// them together: finished rays are written, and the waiting lanes draw the
// next rays of the block pool (one shared-memory atomic per warp).
__device__ __forceinline__ ChunkRange block_pool(const FwdArgs& a, int32_t* s_next) {
    if (threadIdx.x == 0) *s_next = 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) report_nonfinite_heights(a.stats, a.O.status);
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

// Draw strips for this warp's lanes with r < 0 (one shared-memory atomic per
// warp); returns the new strip index or -1.
__device__ __forceinline__ int32_t draw_strip(int32_t n_strips, int32_t* s_next, int32_t r,
                                              bool& open) {
    const unsigned idle = __ballot_sync(kFull, r < 0);
    const int nidle = __popc(idle);
    int base = 0;
    if ((threadIdx.x & 31) == 0 && nidle > 0) base = atomicAdd(s_next, nidle);
    base = __shfl_sync(kFull, base, 0);
    if (base + nidle >= n_strips) open = false;
    if (r >= 0) return -1;
    const int my = base + __popc(idle & lanemask_lt());
    return my < n_strips ? my : -1;
}

// Seed-table column of local ray r >= 0: its column in a rectangular chunk, or
// its virtual column (LH consecutive ids each) in a run of listed rays.
__device__ __forceinline__ int32_t seed_col(const ChunkRange& P, int32_t r, int32_t LH) {
    return (int32_t)(P.rect ? (uint32_t)r % (uint32_t)P.w : (uint32_t)r / (uint32_t)LH);
}

// ---------------------------------------------------------------- descent
// Exact walks (light-only walks: dp_light_kernel below).
// Column seeds (grid rays in rectangles of at most kColSeedMaxW columns, the
// default): lanes draw single rays row by row across the block's rectangle and
// each ray starts from the lowest of its own samples within +-seed_w of where
// the argmin of the last finished ray of its column (a shared-memory table of
// argmin and origin, typically one or two rows above) lies along this ray
// (seed_centre).  Single-ray draws keep the block's tail to one ray per lane;
// a ray drawn before any ray of its column has finished takes the sparse
// samples of seed_geo instead.
//
// Strips: the block's rays are cut into strips of a.strip neighbouring rays
// (down a column of the block's rectangle for rectangular grid chunks, else
// consecutive ids).  A lane walks its strip's rays in order, each seeded from
// the previous ray's argmin, the first from sparse samples.  Neighbouring rays
// are parallel and one texel apart, so their minima sit at nearly the same
// terrain point and the walk prunes from the start (a seed is a sample cost,
// an upper bound of the minimum, so the result is unchanged).
// Each loop iteration is one probe of the exact descent (walk_step) per
// walking lane.  Lanes whose ray is done wait until refill_min of them are
// (or all are); the warp then writes their results and sets up their next
// rays together (next ray of the strip, or a new strip from the block pool).
template <bool kCount, bool kGrid, bool kPoly, bool kStereo>
__global__ void __launch_bounds__(256, SS_FWD_MIN_BLOCKS) dp_forward_kernel(const FwdArgs a) {
    __shared__ LevelTab s_lev;
    __shared__ int32_t s_next;
    if (threadIdx.x < kMaxLevels) {
        s_lev.ptr[threadIdx.x] = a.P.ptr[threadIdx.x];
        s_lev.pitch[threadIdx.x] = (uint32_t)a.P.pitch[threadIdx.x];
    }
    __shared__ int32_t s_seed[kColSeedMaxW];   // column seeds: argmin of a finished ray
    __shared__ float s_su[kColSeedMaxW], s_sv[kColSeedMaxW];   // and that ray's origin
    const ChunkRange P = block_pool(a, &s_next);
    // Column seeds.  Grid rectangles: columns of the rectangle.  Runs of ids
    // (listed rays): the run is read as LW columns of LH consecutive ids each,
    // drawn row by row, so an id is drawn a round after the id before it.
    const bool colseed = a.colseed != 0;
    const int32_t LW = (colseed && !P.rect) ? min(kListSeedCols, P.cnt) : 0;
    const int32_t LH = LW > 0 ? (P.cnt + LW - 1) / LW : 0;
    if (colseed)
        for (int i = threadIdx.x; i < (P.rect ? P.w : LW); i += blockDim.x) {
            s_seed[i] = -1;
            s_su[i] = s_sv[i] = 0.0f;
        }
    __syncthreads();
    const float span = a.stats[0] - a.stats[1];
    const int32_t kleaf = a.kleaf, levels = a.P.levels;
    const int32_t S = colseed ? 1 : a.strip;
    const int32_t n_strips = LW > 0 ? LW * LH : strip_count(P, S);

    const int32_t stride = P.rect ? P.w : 1;   // local index step along a strip
    int32_t r = -1;              // local index of the current ray, -1 = none
    int32_t left = 0;            // rays of the strip after the current one
    bool done = false, open = true;
    RayF rf;
    Walk w;
    w.best = INFINITY;
    w.bestj = -1;
    while (true) {
        unsigned act = __ballot_sync(kFull, r >= 0 && !done);
        const unsigned want = __ballot_sync(kFull, (r < 0 || done) && (left > 0 || open));
        if (act == 0 || __popc(want) >= a.refill_min) {
            bool fresh = false;
            int32_t prev_j = -1;     // a neighbour's argmin, and its origin:
            float su = 0.0f, sv = 0.0f;
            if (done) {
                finish_ray<kStereo, true>(a.T, a.R, a.O, chunk_ray(P, a.T.nx, r), w.best, w.bestj,
                                    w.nb, w.nl);
                if (colseed && w.bestj > 0) {
                    const int32_t c = seed_col(P, r, LH);
                    s_seed[c] = w.bestj;
                    if (kGrid) {
                        s_su[c] = rf.u0;
                        s_sv[c] = rf.v0;
                    }
                }
                done = false;
                if (left > 0) {
                    prev_j = w.bestj;
                    su = rf.u0;
                    sv = rf.v0;
                    r += stride;
                    --left;
                    fresh = true;
                } else {
                    r = -1;
                }
            }
            if (open) {
                const int32_t ns = draw_strip(n_strips, &s_next, r, open);
                if (ns >= 0 && r < 0) {
                    if (LW > 0) {            // virtual column ns % LW, row ns / LW
                        const int32_t e = (ns % LW) * LH + ns / LW;
                        if (e < P.cnt) {
                            r = e;
                            left = 0;
                            fresh = true;
                            prev_j = s_seed[ns % LW];
                            su = s_su[ns % LW];
                            sv = s_sv[ns % LW];
                        }
                    } else {
                        const Strip st = strip_of(P, S, ns);
                        r = st.first;
                        left = st.count - 1;
                        fresh = true;
                        if (colseed) {                   // a ray above in this column
                            const int32_t c = seed_col(P, r, LH);
                            prev_j = s_seed[c];
                            su = s_su[c];
                            sv = s_sv[c];
                        }
                    }
                }
            }
            if (fresh) {
                setup_ray<kGrid, false, kStereo>(a.T, a.R, chunk_ray(P, a.T.nx, r), span, rf);
                const bool near = prev_j > 0;
                const int32_t jc = !near ? -1
                                   : kGrid ? seed_centre(rf, prev_j, su - rf.u0, sv - rf.v0)
                                           : prev_j;
                int32_t sj, n_seed;
                // seeded modes: a ray with no finished neighbour takes sparse samples
                const float sc = seed_ray<kGrid, kPoly, kStereo>(a.T, rf, near, jc, a.seed_w,
                                                                 colseed || S > 1, sj, n_seed);
                if (sj > 0) {
                    walk_begin_seeded<false>(w, rf, kleaf, sc, sj);
                    if (kCount) w.nl = n_seed;
                } else {
                    walk_begin<false>(w, rf, kleaf);
                }
                if (rf.j_hi < rf.j_lo) done = true;   // no usable sample: written next service
            }
            act = __ballot_sync(kFull, r >= 0 && !done);
            if (act == 0) {
                if (!__any_sync(kFull, (r >= 0) || left > 0) && !open) break;
                continue;
            }
        }
        if (r < 0 || done) continue;
        done = walk_step<kCount, kGrid, kPoly, false, kStereo>(a.T, s_lev, levels, kleaf, rf, w);
    }
}

// ------------------------------------------------------- light-only descent
// Light-only walks are short (~30 probes per ray against ~130 for an exact
// walk), so the per-ray setup weighs more, and it is what this kernel
// amortises.  Each warp keeps a queue of up to kQSlots rays that are already
// set up, parked in shared memory.  When the queue cannot serve the lanes
// waiting for a ray, the warp refills it in one pass: one shared-memory atomic
// draws up to kQSlots rays (in the block's draw order) and every lane sets up
// one of them.  A lane that finishes a ray then only writes its light, loads
// the next parked ray and evaluates its seed samples (column seeds, read at
// that moment so that they are as recent as possible).
//
// (Measured on GB300, 4096^2 grid: 10.2 -> 7.8 ms; 6 M polar view rays: 54 ->
// 35 ms.  Exact walks stay with dp_forward_kernel: parking rays a row ahead
// makes their column seeds older, which costs an exact walk more probes than
// the shared setup saves.)

// Set up ray `ray` and park it in queue slot `slot`.  Not inlined: the walking
// lanes' state stays in registers around the call instead of competing with
// the setup's FP64 temporaries.
template <bool kGrid, bool kStereo>
static __device__ __noinline__ void park_ray(const FwdArgs& a, int64_t ray, float span,
                                             uint32_t (*q)[kQSlots], int slot) {
    RayF t;
    setup_ray<kGrid, true, kStereo>(a.T, a.R, ray, span, t);
    RayPack<kGrid, true, kStereo>::store(q, slot, t);
}

template <bool kCount, bool kGrid, bool kPoly, bool kStereo>
__global__ void __launch_bounds__(256, SS_FWD_MIN_BLOCKS)
dp_light_kernel(const __grid_constant__ FwdArgs a) {
    using Pack = RayPack<kGrid, true, kStereo>;
    constexpr int kWr = Pack::kWords;          // word of the parked ray's local index
    __shared__ LevelTab s_lev;
    __shared__ int32_t s_next;
    __shared__ int32_t s_seed[kColSeedMaxW];   // column seeds: argmin of a finished ray
    __shared__ float s_su[kColSeedMaxW], s_sv[kColSeedMaxW];   // and that ray's origin
    __shared__ uint32_t s_q[8][kWr + 1][kQSlots];
    if (threadIdx.x < kMaxLevels) {
        s_lev.ptr[threadIdx.x] = a.P.ptr[threadIdx.x];
        s_lev.pitch[threadIdx.x] = (uint32_t)a.P.pitch[threadIdx.x];
    }
    const ChunkRange P = block_pool(a, &s_next);
    // Draw order.  Grid rectangles: row by row (the seed of a ray is the last
    // finished ray of its column of the rectangle).  Runs of ids (listed rays
    // with column seeds): LW columns of LH consecutive ids each, row by row.
    const bool colseed = a.colseed != 0;
    const int32_t LW = (colseed && !P.rect) ? min(kListSeedCols, P.cnt) : 0;
    const int32_t LH = LW > 0 ? (P.cnt + LW - 1) / LW : 0;
    const int32_t n_order = LW > 0 ? LW * LH : P.cnt;
    if (colseed)
        for (int i = threadIdx.x; i < (P.rect ? P.w : LW); i += blockDim.x) {
            s_seed[i] = -1;
            s_su[i] = s_sv[i] = 0.0f;
        }
    __syncthreads();
    const float span = a.stats[0] - a.stats[1];
    const int32_t kleaf = a.kleaf, levels = a.P.levels;
    const int lane = threadIdx.x & 31;
    uint32_t (*q)[kQSlots] = s_q[threadIdx.x >> 5];

    int32_t r = -1;              // local index of the current ray, -1 = none
    bool done = false, open = true;
    int32_t qh = 0, qn = 0;      // queue head slot and length (warp-uniform)
    RayF rf;
    Walk w;
    w.best = INFINITY;
    w.bestj = -1;
    while (true) {
        const unsigned act = __ballot_sync(kFull, r >= 0 && !done);
        const int n_idle = 32 - __popc(act);
        if (act == 0 || ((open || qn > 0) && n_idle >= a.refill_min)) {
            if (done) {
                finish_ray<kStereo, true>(a.T, a.R, a.O, chunk_ray(P, a.T.nx, r), w.best, w.bestj,
                                          w.nb, w.nl);
                if (colseed && w.bestj > 0) {
                    const int32_t c = seed_col(P, r, LH);
                    s_seed[c] = w.bestj;
                    if (kGrid) {
                        s_su[c] = rf.u0;
                        s_sv[c] = rf.v0;
                    }
                }
                done = false;
                r = -1;
            }
            if (qn < n_idle && open) {
                // refill the queue: up to kQSlots - qn rays, one per lane
                const int want = kQSlots - qn;
                int base = 0;
                if (lane == 0) base = atomicAdd(&s_next, want);
                base = __shfl_sync(kFull, base, 0);
                if (base + want >= n_order) open = false;
                const int m = max(0, min(want, n_order - base));
                if (lane < m) {
                    const int32_t o = base + lane;
                    // listed rays: virtual column o % LW
                    const int32_t e = LW > 0 ? (o % LW) * LH + o / LW : o;
                    const int slot = (qh + qn + lane) % kQSlots;
                    if (e < P.cnt)
                        park_ray<kGrid, kStereo>(a, chunk_ray(P, a.T.nx, e), span, q, slot);
                    q[kWr][slot] = (uint32_t)(e < P.cnt ? e : -1);   // -1: padding of the last row
                }
                qn += m;
                __syncwarp();
            }
            // idle lanes take parked rays in queue order
            const unsigned idle = ~__ballot_sync(kFull, r >= 0);
            const int k = __popc(idle & lanemask_lt());
            const int take = min(__popc(idle), qn);
            if (r < 0 && k < take) {
                const int slot = (qh + k) % kQSlots;
                r = (int32_t)q[kWr][slot];
                if (r >= 0) {
                    Pack::load(q, slot, rf);
                    const int32_t c = seed_col(P, r, LH);
                    const int32_t prev_j = colseed ? s_seed[c] : -1;
                    const bool near = prev_j > 0;
                    const int32_t jc =
                        !near   ? -1
                        : kGrid ? seed_centre(rf, prev_j, s_su[c] - rf.u0, s_sv[c] - rf.v0)
                                : prev_j;
                    int32_t sj, n_seed;
                    const float sc = seed_ray<kGrid, kPoly, kStereo>(a.T, rf, near, jc, a.seed_w,
                                                                     false, sj, n_seed);
                    if (sj > 0) {
                        walk_begin_seeded<true>(w, rf, kleaf, sc, sj);
                        if (kCount) w.nl = n_seed;
                    } else {
                        walk_begin<true>(w, rf, kleaf);
                    }
                    if (rf.j_hi < rf.j_lo) done = true;   // no usable sample: written next service
                }
            }
            qh = (qh + take) % kQSlots;
            qn -= take;
            __syncwarp();
            if (__ballot_sync(kFull, r >= 0 && !done) == 0) {
                if (!open && qn == 0 && !__any_sync(kFull, r >= 0)) break;
                continue;
            }
        }
        if (r < 0 || done) continue;
        done = walk_step<kCount, kGrid, kPoly, true, kStereo>(a.T, s_lev, levels, kleaf, rf, w);
    }
}

// ---------------------------------------------------------------- uniform
// Every usable sample in order, same scheduling as the descent.  Early exit
// (exact): with H(t) = h_p + rise(t) convex and H(0) = h_p <= max h,
// g(t) = (H(t) - max h - G)/t is non-decreasing and bounds every later
// sample's cost from below; once g(t_j) >= best no later sample can win.
// G = 3 guards covers the float32 rounding of both sides.
template <bool kCount, bool kGrid, bool kPoly, bool kLight, bool kStereo>
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
                finish_ray<kStereo>(a.T, a.R, a.O, chunk_ray(P, a.T.nx, r), best, bestj, 0, nl);
                r = -1;
                done = false;
            }
            if (open) {
                const int32_t nr = draw(P, &s_next, r, open);
                if (nr >= 0 && r < 0) {
                    r = nr;
                    setup_ray<kGrid, kLight, kStereo>(a.T, a.R, chunk_ray(P, a.T.nx, r), span, rf);
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
                        finish_ray<kStereo>(a.T, a.R, a.O, chunk_ray(P, a.T.nx, r), best, bestj, 0, 0);
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
        const float c = leaf_cost<kGrid, kPoly, kStereo>(a.T, rf, j, rise);
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

static int pool_grid(const FwdArgs& a) {
    const int64_t n = a.R.mode == 0 ? (int64_t)a.T.nx * a.T.ny : a.R.n;
    return (int)chunk_count(n, a.T.nx, a.T.ny, (int32_t)a.rays_per_block,
                            a.R.mode == 0 ? a.tile_w : 0);
}

// ---------------------------------------------------------------- refine
// FP64 re-evaluation of the rays the descent left pending (penumbra rays, a
// few percent).  A block gathers the pending rays of its kRefineRounds x 256
// ids into shared memory, then every thread takes one: full warps of FP64 work
// instead of a lane or two inside the walk's services.
constexpr int kRefineRounds = 8;

template <bool kStereo>
__global__ void __launch_bounds__(256) refine_kernel(const FwdArgs a) {
    __shared__ int64_t s_ray[256 * kRefineRounds];
    __shared__ int32_t s_cnt;
    const int64_t n = ray_count(a.T, a.R);
    const int64_t base = (int64_t)blockIdx.x * 256 * kRefineRounds;
    if (threadIdx.x == 0) s_cnt = 0;
    __syncthreads();
    for (int k = 0; k < kRefineRounds; ++k) {
        const int64_t r = base + (int64_t)k * 256 + threadIdx.x;
        if (r < n && a.O.light[r] == kLightPending) s_ray[atomicAdd(&s_cnt, 1)] = r;
    }
    __syncthreads();
    const int cnt = s_cnt;
    for (int i = threadIdx.x; i < cnt; i += 256) {
        const int64_t r = s_ray[i];
        float light, cost;
        refine_ray(a.T, a.R, r, a.O.argmin[r], kStereo, light, cost);
        a.O.light[r] = light;
        if (a.O.cost) a.O.cost[r] = cost;
    }
}

#define SS_FWD_CASE(C, G, P, L) \
    case ((C) << 3) | ((G) << 2) | ((P) << 1) | (L): return Launch<C, G, P, L, kStereo>::go(a, grid, block, s);

// runtime flags -> the kernel instance (counters, grid mode, rise series, light-only)
template <bool kStereo, template <bool, bool, bool, bool, bool> class Launch>
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

// defined in ss_task.cuh
template <bool kCount, bool kGrid, bool kPoly, bool kStereo>
__global__ void __launch_bounds__(256, SS_FWD_MIN_BLOCKS) dp_task_kernel(const FwdArgs a);

// The task descent (ss_task.cuh) serves exact walks with column seeds: grid
// rays in rectangles (leaf blocks of <= 4 samples on gnomonic tiles, <= 8 on
// stereographic ones), listed rays in runs (<= 8).  (Polar view, 6.0 M rays on
// the 16384^2 stereographic tile, 32 rays per lane: 28.5 ms against 37.5 ms for
// the single-lane walk, once the float32 range search took the FP64 crossings
// out of the setup; with them the tasks had measured slower, 70 against 65 ms.)
inline bool use_task_descent(const FwdArgs& a, bool grid, bool stereo, bool light) {
    return !light && a.colseed && (!grid || a.tile_w > 0) &&
           a.kleaf <= (grid && !stereo ? 1 : 2) && !(a.flags & 0x10u);   // SS_FLAG_LANE_LEAVES
}

template <bool C, bool G, bool P, bool L, bool S>
struct DpLaunch {
    static cudaError_t go(const FwdArgs& a, int grid, int block, cudaStream_t s) {
        bool tasks = false;
        if constexpr (!L) {
            if (use_task_descent(a, G, S, L)) {
                dp_task_kernel<C, G, P, S><<<grid, block, 0, s>>>(a);
                tasks = true;
            }
        }
        if (tasks)
            ;
        else if (L)
            dp_light_kernel<C, G, P, S><<<grid, block, 0, s>>>(a);
        else
            dp_forward_kernel<C, G, P, S><<<grid, block, 0, s>>>(a);
        const int64_t n = a.R.mode == 0 ? (int64_t)a.T.nx * a.T.ny : a.R.n;
        const int64_t rb = ((n + 256 * kRefineRounds - 1) / (256 * kRefineRounds));
        refine_kernel<S><<<(unsigned)rb, 256, 0, s>>>(a);
        return cudaGetLastError();
    }
};

template <bool C, bool G, bool P, bool L, bool S>
struct UniLaunch {
    static cudaError_t go(const FwdArgs& a, int grid, int block, cudaStream_t s) {
        uniform_forward_kernel<C, G, P, L, S><<<grid, block, 0, s>>>(a);
        return cudaGetLastError();
    }
};

}  // namespace ss
