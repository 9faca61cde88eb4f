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
