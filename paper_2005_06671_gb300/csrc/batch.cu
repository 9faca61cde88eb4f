// Batched forward: many (heightfield tile, sun) instances of uneven sizes in one
// persistent launch with a device-side work queue.
//
// The instances' rays are cut into chunks (32 * rays_per_thread rays, or
// rectangles of them); chunks of one instance are consecutive in the queue.
// A grid of resident blocks (occupancy x SMs) pulls chunks with one global
// atomicAdd per chunk and per warp; each warp keeps a copy of its current
// instance's descriptor in shared memory and walks each ray with the same
// exact descent as the single-tile forward (walk_step), refilling idle lanes
// from its chunk: by default ray by ray row-major over a rectangular chunk,
// each ray seeded from the argmin of its column's last finished ray (a small
// per-warp table), or with strips of neighbouring rays (as in the single-tile
// kernel).  A warp switches instance only once all its lanes are idle,
// so lanes never mix instances.  No device-side wait: the queue is a counter.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "ss_batch.h"
#include "ss_walk.cuh"
#include "ss_strip.cuh"
#include "ss_leaftask.cuh"

namespace ss {

// Minimum resident 256-thread blocks per SM of the batched kernel (it carries
// queue state on top of the walk: 80 registers at 3 blocks).
#ifndef SS_BATCH_MIN_BLOCKS
#define SS_BATCH_MIN_BLOCKS 3
#endif

namespace {

// upper_bound over the chunk prefix sums: instance that owns chunk q
__device__ __forceinline__ int32_t owner(const int64_t* prefix, int32_t n, int64_t q) {
    int32_t lo = 0, hi = n;   // prefix[lo] <= q < prefix[hi]
    while (hi - lo > 1) {
        const int32_t mid = (lo + hi) >> 1;
        if (__ldg(prefix + mid) <= q) lo = mid; else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ void load_desc(BatchItemDesc* dst, const BatchItemDesc* src) {
    const int lane = threadIdx.x & 31;
    const uint32_t* s = reinterpret_cast<const uint32_t*>(src);
    uint32_t* d = reinterpret_cast<uint32_t*>(dst);
    constexpr int kWords = sizeof(BatchItemDesc) / 4;
    for (int i = lane; i < kWords; i += 32) d[i] = __ldg(s + i);
    __syncwarp();
}

// Warp-uniform scheduling state, kept in shared memory next to the warp's
// instance descriptor so the lanes' registers hold only the walk.
struct LaneRay {
    int64_t ray;        // the lane's ray: id within the warp's instance
    int32_t slot;       // its column in the seed table, or -1
    int32_t pad;
};

struct WarpSched {
    ChunkRange C;       // current chunk of `cur`
    int64_t stash;      // a grabbed chunk of another instance, or -1
    int32_t c_next;     // next undrawn strip of C
    int32_t n_strips;   // strips of C
    int32_t colseed;    // C is drawn ray by ray with column seeds
    int32_t cur;        // instance of this warp, or -1
    int32_t open;       // the queue may still have chunks
    float span;         // height span of `cur`
};

template <bool kCount, bool kLight>
__global__ void __launch_bounds__(256, SS_BATCH_MIN_BLOCKS) batch_dp_kernel(const BatchArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    BatchItemDesc& D = reinterpret_cast<BatchItemDesc*>(smem)[wid];
    WarpSched& S = reinterpret_cast<WarpSched*>(
        smem + (size_t)(blockDim.x >> 5) * sizeof(BatchItemDesc))[wid];
    // column seeds of this warp's chunk: argmin of the last finished ray per
    // column, and that ray's origin
    int32_t* seeds = reinterpret_cast<int32_t*>(
        smem + (size_t)(blockDim.x >> 5) * (sizeof(BatchItemDesc) + sizeof(WarpSched))) +
        wid * 3 * kBatchSeedW;
    float* seed_u = reinterpret_cast<float*>(seeds + kBatchSeedW);
    float* seed_v = seed_u + kBatchSeedW;
    // Each lane's ray as an id within the instance, and its seed column: a warp
    // moves to its next chunk (same instance) while other lanes still walk rays
    // of the previous one, so a lane's ray must not be kept as an index into
    // the warp's current chunk.
    LaneRay& L = reinterpret_cast<LaneRay*>(
        smem + (size_t)(blockDim.x >> 5) *
                   (sizeof(BatchItemDesc) + sizeof(WarpSched) + 3 * kBatchSeedW * sizeof(int32_t)))
        [threadIdx.x];
    const Rays grid_rays = { 0, 0, nullptr, nullptr, nullptr };
    if (lane == 0) {
        S.C.cnt = 0;
        S.stash = -1;
        S.c_next = 0;
        S.n_strips = 0;
        S.colseed = 0;
        S.cur = -1;
        S.open = 1;
        S.span = 0.0f;
    }
    __syncwarp();

    int32_t r = -1;              // >= 0 while this lane holds a ray (id in L.ray)
    int32_t left = 0;            // rays of this lane's strip after the current one
    bool done = false;
    RayF rf;
    Walk w;
    w.best = INFINITY;
    w.bestj = -1;
    while (true) {
        unsigned act = __ballot_sync(kFull, r >= 0 && !done);
        const bool more = S.open || S.stash >= 0 || S.c_next < S.n_strips;
        const unsigned want = __ballot_sync(kFull, (r < 0 || done) && (left > 0 || more));
        if (act == 0 || __popc(want) >= a.refill_min) {
            // finished rays are written; a lane with more rays in its strip moves
            // to the next one, seeded from this ray's argmin (same instance)
            if (done) {
                finish_ray(D.T, grid_rays, D.O, L.ray, w.best, w.bestj, w.nb, w.nl);
                if (L.slot >= 0 && w.bestj > 0) {
                    seeds[L.slot] = w.bestj;
                    seed_u[L.slot] = rf.u0;
                    seed_v[L.slot] = rf.v0;
                }
                done = false;
                int32_t prev_j = -1;
                const float su = rf.u0, sv = rf.v0;
                if (left > 0) {          // next ray of the strip: a row down, or the next id
                    prev_j = w.bestj;
                    L.ray += D.tile_w > 0 ? (int64_t)D.T.nx : 1;
                    L.slot = -1;
                    --left;
                } else {
                    r = -1;
                }
                if (r >= 0) {
                    setup_ray<true, kLight>(D.T, grid_rays, L.ray, S.span, rf);
                    const bool near = prev_j > 0;
                    const int32_t jc =
                        near ? seed_centre(rf, prev_j, su - rf.u0, sv - rf.v0) : -1;
                    int32_t sj, n_seed;
                    const float sc =
                        D.poly
                            ? seed_ray<true, true, false>(D.T, rf, near, jc, a.seed_w, false, sj,
                                                          n_seed)
                            : seed_ray<true, false, false>(D.T, rf, near, jc, a.seed_w, false, sj,
                                                           n_seed);
                    if (sj > 0) {
                        walk_begin_seeded<kLight>(w, rf, a.kleaf, sc, sj);
                        if (kCount) w.nl = n_seed;
                    } else {
                        walk_begin<kLight>(w, rf, a.kleaf);
                    }
                    if (rf.j_hi < rf.j_lo) done = true;   // written at the next service
                }
            }
            // draw strips for idle lanes, taking chunks from the queue as needed
            while (true) {
                const unsigned idle = __ballot_sync(kFull, r < 0);
                if (idle == 0) break;
                const int32_t c_next = S.c_next, nst = S.n_strips;
                if (c_next < nst) {
                    const int32_t my = c_next + __popc(idle & lanemask_lt());
                    if (r < 0 && my < nst) {
                        const Strip st = strip_of(S.C, S.colseed ? 1 : a.strip, my);
                        r = st.first;
                        left = st.count - 1;
                        L.ray = chunk_ray(S.C, D.T.nx, r);
                        L.slot = S.colseed ? r % S.C.w : -1;
                        setup_ray<true, kLight>(D.T, grid_rays, L.ray, S.span, rf);
                        const int32_t pj = S.colseed ? seeds[L.slot] : -1;
                        const bool near = pj > 0;
                        const int32_t jc = near ? seed_centre(rf, pj, seed_u[L.slot] - rf.u0,
                                                              seed_v[L.slot] - rf.v0)
                                                : -1;
                        // seeded modes: a ray with no finished neighbour takes sparse samples
                        const bool geo = !kLight && (S.colseed || a.strip > 1);
                        int32_t sj, n_seed;
                        const float sc =
                            D.poly
                                ? seed_ray<true, true, false>(D.T, rf, near, jc, a.seed_w, geo,
                                                              sj, n_seed)
                                : seed_ray<true, false, false>(D.T, rf, near, jc, a.seed_w, geo,
                                                               sj, n_seed);
                        if (sj > 0) {
                            walk_begin_seeded<kLight>(w, rf, a.kleaf, sc, sj);
                            if (kCount) w.nl = n_seed;
                        } else {
                            walk_begin<kLight>(w, rf, a.kleaf);
                        }
                        if (rf.j_hi < rf.j_lo) done = true;   // written at the next service
                    }
                    __syncwarp();
                    if (lane == 0) S.c_next = min(c_next + __popc(idle), nst);
                    __syncwarp();
                    continue;
                }
                // current chunk exhausted: take the stashed or the next chunk
                int64_t q = S.stash;
                if (q < 0) {
                    if (!S.open) break;
                    long long got = 0;
                    if (lane == 0) got = (long long)atomicAdd(a.counter, 1ULL);
                    q = (int64_t)__shfl_sync(kFull, got, 0);
                    if (q >= a.total_chunks) {
                        __syncwarp();
                        if (lane == 0) S.open = 0;
                        __syncwarp();
                        break;
                    }
                }
                const int32_t item = owner(a.chunk_prefix, a.n_items, q);
                if (item != S.cur) {
                    const bool walking = __ballot_sync(kFull, r >= 0) != 0;
                    __syncwarp();
                    if (walking) {   // lanes still walk (or hold results of) the current instance
                        if (lane == 0) S.stash = q;
                        __syncwarp();
                        break;
                    }
                    load_desc(&D, a.items + item);
                    if (lane == 0) {
                        S.cur = item;
                        S.span = __ldg(D.stats) - __ldg(D.stats + 1);
                        report_nonfinite_heights(D.stats, D.O.status);
                    }
                }
                __syncwarp();
                if (lane == 0) {
                    S.stash = -1;
                    S.C = chunk_range(q - __ldg(a.chunk_prefix + item), D.n_rays, D.T.nx, D.T.ny,
                                      a.chunk_rays, D.tile_w);
                    S.colseed = a.colseed && S.C.rect && S.C.w <= kBatchSeedW;
                    S.n_strips = strip_count(S.C, S.colseed ? 1 : a.strip);
                    S.c_next = 0;
                }
                for (int i = lane; i < kBatchSeedW; i += 32) {
                    seeds[i] = -1;
                    seed_u[i] = seed_v[i] = 0.0f;
                }
                __syncwarp();
            }
            act = __ballot_sync(kFull, r >= 0 && !done);
            if (act == 0) {
                if (!__any_sync(kFull, r >= 0) && !S.open && S.stash < 0 && S.c_next >= S.n_strips)
                    break;
                continue;
            }
        }
        if (r < 0 || done) continue;
        done = D.poly ? walk_step<kCount, true, true, kLight>(D.T, D.L, D.levels, a.kleaf, rf, w)
                      : walk_step<kCount, true, false, kLight>(D.T, D.L, D.levels, a.kleaf, rf, w);
    }
}

// Exact walks of the batch with leaf samples as warp-wide tasks (as
// dp_task_kernel, ss_task.cuh): a lane's walk only bounds blocks; a leaf block
// that cannot be pruned is pushed, one task per sample, into the warp's ring,
// and the warp evaluates 32 tasks at a time with the instance's leaf function;
// each ray's running minimum is a 64-bit key in shared memory.  Scheduling,
// chunks, strips and column seeds are batch_dp_kernel's; a drawn ray's seed
// window and first leaf block become tasks (sparse seeds stay in the lane), and
// the ring is drained before rays are written and before the warp moves to
// another instance (a warp switches instance only when all its lanes are idle).
template <bool kCount>
__global__ void __launch_bounds__(256, SS_BATCH_MIN_BLOCKS) batch_task_kernel(const BatchArgs a) {
    using Cfg = TaskCfg<true, false>;
    constexpr int kMask = Cfg::kRing - 1;
    extern __shared__ __align__(16) unsigned char smem[];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nw = blockDim.x >> 5;
    TaskWarp<true, false>& TW = reinterpret_cast<TaskWarp<true, false>*>(smem)[wid];
    unsigned char* rest = smem + (size_t)nw * sizeof(TaskWarp<true, false>);
    BatchItemDesc& D = reinterpret_cast<BatchItemDesc*>(rest)[wid];
    WarpSched& S = reinterpret_cast<WarpSched*>(rest + (size_t)nw * sizeof(BatchItemDesc))[wid];
    int32_t* seeds = reinterpret_cast<int32_t*>(
        rest + (size_t)nw * (sizeof(BatchItemDesc) + sizeof(WarpSched))) + wid * 3 * kBatchSeedW;
    float* seed_u = reinterpret_cast<float*>(seeds + kBatchSeedW);
    float* seed_v = seed_u + kBatchSeedW;
    LaneRay& L = reinterpret_cast<LaneRay*>(
        rest + (size_t)nw * (sizeof(BatchItemDesc) + sizeof(WarpSched) +
                             3 * kBatchSeedW * sizeof(int32_t)))[threadIdx.x];
    const Rays grid_rays = { 0, 0, nullptr, nullptr, nullptr };
    if (lane == 0) {
        S.C.cnt = 0;
        S.stash = -1;
        S.c_next = 0;
        S.n_strips = 0;
        S.colseed = 0;
        S.cur = -1;
        S.open = 1;
        S.span = 0.0f;
    }
    TW.key[lane] = kKeyNone;
    __syncwarp();
    const int32_t Lk = a.kleaf + 1;     // leaf blocks hold 2^Lk samples
    const int32_t sw = a.seed_w;
    int32_t head = 0, count = 0;        // the ring (same values in every lane)

    int32_t r = -1;              // >= 0 while this lane holds a ray (id in L.ray)
    int32_t left = 0;            // rays of this lane's strip after the current one
    bool done = false;
    RayF rf;
    int32_t s0 = 0, k = 0, nb = 0, nl = 0;
    float best = INFINITY;

    auto drain = [&]() {
        if (D.poly)
            while (count > 0) task_pass<true, true, false>(D.T, TW, head, count, lane);
        else
            while (count > 0) task_pass<true, false, false>(D.T, TW, head, count, lane);
    };
    // a lane's new ray: setup, its seed window (around where a neighbour's argmin
    // lies along it) and first leaf block as pending tasks [wa, wb], [la, lb],
    // or sparse seeds in the lane
    int32_t wa = 1, wb = 0, la = 1, lb = 0;
    auto start_ray = [&](int32_t prev_j, float su, float sv, bool geo) {
        setup_ray<true, false>(D.T, grid_rays, L.ray, S.span, rf);
        store_leaf_ray(TW, lane, rf);
        nb = nl = 0;
        unsigned long long key = kKeyNone;
        const bool near = prev_j > 0;
        const int32_t jc = near ? seed_centre(rf, prev_j, su - rf.u0, sv - rf.v0) : -1;
        wa = 1;
        wb = 0;
        if (near) {
            wa = max(rf.j_lo, jc - sw);
            wb = min(rf.j_hi, jc + sw);
        }
        if (wb < wa) {
            int32_t sj, n_seed;
            const float sc = D.poly
                                 ? seed_ray<true, true, false>(D.T, rf, near, jc, sw, geo, sj, n_seed)
                                 : seed_ray<true, false, false>(D.T, rf, near, jc, sw, geo, sj,
                                                                n_seed);
            if (sj > 0 && sc < INFINITY) key = pack_key(sc, sj);
            if (kCount) nl = n_seed;
        }
        TW.key[lane] = key;
        la = max(rf.j_lo, 1);
        lb = min(rf.j_hi, 1 << Lk);
        s0 = 1 << Lk;
        k = Lk;
        done = rf.j_hi <= s0;
    };

    while (true) {
        unsigned act = __ballot_sync(kFull, r >= 0 && !done);
        const bool more = S.open || S.stash >= 0 || S.c_next < S.n_strips;
        const unsigned want = __ballot_sync(kFull, (r < 0 || done) && (left > 0 || more));
        if (act == 0 || __popc(want) >= a.refill_min) {
            drain();
            wa = 1;
            wb = 0;
            la = 1;
            lb = 0;
            if (done) {
                const unsigned long long key = TW.key[lane];
                const int32_t bj = key_j(key);
                finish_ray(D.T, grid_rays, D.O, L.ray, key_cost(key), bj, nb, nl);
                if (L.slot >= 0 && bj > 0) {
                    seeds[L.slot] = bj;
                    seed_u[L.slot] = rf.u0;
                    seed_v[L.slot] = rf.v0;
                }
                done = false;
                const float su = rf.u0, sv = rf.v0;
                if (left > 0) {          // next ray of the strip: a row down, or the next id
                    L.ray += D.tile_w > 0 ? (int64_t)D.T.nx : 1;
                    L.slot = -1;
                    --left;
                    start_ray(bj, su, sv, false);
                } else {
                    r = -1;
                }
            }
            // draw strips for idle lanes, taking chunks from the queue as needed
            while (true) {
                const unsigned idle = __ballot_sync(kFull, r < 0);
                if (idle == 0) break;
                const int32_t c_next = S.c_next, nst = S.n_strips;
                if (c_next < nst) {
                    const int32_t my = c_next + __popc(idle & lanemask_lt());
                    if (r < 0 && my < nst) {
                        const Strip st = strip_of(S.C, S.colseed ? 1 : a.strip, my);
                        r = st.first;
                        left = st.count - 1;
                        L.ray = chunk_ray(S.C, D.T.nx, r);
                        L.slot = S.colseed ? r % S.C.w : -1;
                        const int32_t pj = S.colseed ? seeds[L.slot] : -1;
                        start_ray(pj, pj > 0 ? seed_u[L.slot] : 0.0f,
                                  pj > 0 ? seed_v[L.slot] : 0.0f, S.colseed || a.strip > 1);
                    }
                    __syncwarp();
                    if (lane == 0) S.c_next = min(c_next + __popc(idle), nst);
                    __syncwarp();
                    continue;
                }
                // current chunk exhausted: take the stashed or the next chunk
                int64_t q = S.stash;
                if (q < 0) {
                    if (!S.open) break;
                    long long got = 0;
                    if (lane == 0) got = (long long)atomicAdd(a.counter, 1ULL);
                    q = (int64_t)__shfl_sync(kFull, got, 0);
                    if (q >= a.total_chunks) {
                        __syncwarp();
                        if (lane == 0) S.open = 0;
                        __syncwarp();
                        break;
                    }
                }
                const int32_t item = owner(a.chunk_prefix, a.n_items, q);
                if (item != S.cur) {
                    const bool walking = __ballot_sync(kFull, r >= 0) != 0;
                    __syncwarp();
                    if (walking) {   // lanes still walk (or hold results of) the current instance
                        if (lane == 0) S.stash = q;
                        __syncwarp();
                        break;
                    }
                    load_desc(&D, a.items + item);
                    if (lane == 0) {
                        S.cur = item;
                        S.span = __ldg(D.stats) - __ldg(D.stats + 1);
                        report_nonfinite_heights(D.stats, D.O.status);
                    }
                }
                __syncwarp();
                if (lane == 0) {
                    S.stash = -1;
                    S.C = chunk_range(q - __ldg(a.chunk_prefix + item), D.n_rays, D.T.nx, D.T.ny,
                                      a.chunk_rays, D.tile_w);
                    S.colseed = a.colseed && S.C.rect && S.C.w <= kBatchSeedW;
                    S.n_strips = strip_count(S.C, S.colseed ? 1 : a.strip);
                    S.c_next = 0;
                }
                for (int i = lane; i < kBatchSeedW; i += 32) {
                    seeds[i] = -1;
                    seed_u[i] = seed_v[i] = 0.0f;
                }
                __syncwarp();
            }
            // the new rays' seed windows and first leaf blocks, then walk
            const int32_t nwin = max(wb - wa + 1, 0), nlf = max(lb - la + 1, 0);
            const unsigned em = __ballot_sync(kFull, nwin + nlf > 0);
            if (nwin + nlf > 0) {
                const int32_t base = head + count + __popc(em & lanemask_lt()) * Cfg::kServiceSlots;
                for (int i = 0; i < Cfg::kServiceSlots; ++i) {
                    const int32_t j = i < nwin ? wa + i : (i - nwin < nlf ? la + (i - nwin) : 0);
                    TW.task[(base + i) & kMask] = ((uint32_t)j << 5) | (uint32_t)lane;
                }
                if (kCount) nl += nwin + nlf;
            }
            count += __popc(em) * Cfg::kServiceSlots;
            __syncwarp();
            drain();
            if (r >= 0) best = key_cost(TW.key[lane]);
            act = __ballot_sync(kFull, r >= 0 && !done);
            if (act == 0) {
                if (!__any_sync(kFull, r >= 0) && !S.open && S.stash < 0 && S.c_next >= S.n_strips)
                    break;
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
            const float v = D.poly ? block_bound<true, true, false>(D.T, D.L, D.levels, rf, ja, jb)
                                   : block_bound<true, false, false>(D.T, D.L, D.levels, rf, ja, jb);
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
                    TW.task[(base + i) & kMask] = ((uint32_t)j << 5) | (uint32_t)lane;
                }
                if (kCount) nl += ne;
            }
            count += __popc(em) << Lk;
            __syncwarp();
            if (count >= 32) {
                if (D.poly) {
                    do {
                        task_pass<true, true, false>(D.T, TW, head, count, lane);
                    } while (count >= 32);
                } else {
                    do {
                        task_pass<true, false, false>(D.T, TW, head, count, lane);
                    } while (count >= 32);
                }
                if (r >= 0) best = key_cost(TW.key[lane]);
            }
        }
    }
}

template <typename K>
int resident_blocks(K kernel, int block, size_t smem) {
    int per_sm = 0, dev = 0, sms = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, smem) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        sms = 1;
    return per_sm * sms;
}

}  // namespace

size_t batch_workspace_bytes(int32_t n_items) {
    return kBatchHeader + align256((size_t)n_items * sizeof(BatchItemDesc)) +
           align256((size_t)(n_items + 1) * sizeof(int64_t));
}

void batch_layout(void* ws, int32_t n_items, unsigned long long** counter, BatchItemDesc** items,
                  int64_t** prefix) {
    unsigned char* b = static_cast<unsigned char*>(ws);
    *counter = reinterpret_cast<unsigned long long*>(b);
    *items = reinterpret_cast<BatchItemDesc*>(b + kBatchHeader);
    *prefix = reinterpret_cast<int64_t*>(b + kBatchHeader +
                                         align256((size_t)n_items * sizeof(BatchItemDesc)));
}

cudaError_t launch_batch_forward(const BatchArgs& a, int block, bool count, cudaStream_t s) {
    const size_t smem = (size_t)(block / 32) *
                            (sizeof(BatchItemDesc) + sizeof(WarpSched) + 3 * kBatchSeedW * sizeof(int32_t)) +
                        (size_t)block * sizeof(LaneRay);
    // exact walks with leaf tasks: seed windows of <= 3 and leaf blocks of <= 4
    // samples fit a drawn ray's ring slots
    const size_t tsmem = smem + (size_t)(block / 32) * sizeof(TaskWarp<true, false>);
    if (!a.light_only && !a.lane_leaves && a.kleaf <= 1 && a.seed_w <= 1 &&
        tsmem <= 48 * 1024) {
        if (count)
            batch_task_kernel<true><<<resident_blocks(batch_task_kernel<true>, block, tsmem), block,
                                      tsmem, s>>>(a);
        else
            batch_task_kernel<false><<<resident_blocks(batch_task_kernel<false>, block, tsmem),
                                       block, tsmem, s>>>(a);
        return cudaGetLastError();
    }
    if (count) {
        if (a.light_only)
            batch_dp_kernel<true, true><<<resident_blocks(batch_dp_kernel<true, true>, block, smem), block, smem, s>>>(a);
        else
            batch_dp_kernel<true, false><<<resident_blocks(batch_dp_kernel<true, false>, block, smem), block, smem, s>>>(a);
    } else {
        if (a.light_only)
            batch_dp_kernel<false, true><<<resident_blocks(batch_dp_kernel<false, true>, block, smem), block, smem, s>>>(a);
        else
            batch_dp_kernel<false, false><<<resident_blocks(batch_dp_kernel<false, false>, block, smem), block, smem, s>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace ss
