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
#include "ss_leaftask.cuh"

namespace ss {

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
        // lanes that want a ray: the others, while the pool is open (open is
        // warp-uniform: only draw_strip, run by every lane, changes it)
        const unsigned want = open ? ~act : 0u;
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
