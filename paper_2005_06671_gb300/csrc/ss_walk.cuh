// Per-ray pieces shared by the single-tile and batched forward kernels:
// setup of a ray's float32 state, one step of the exact descent, and the
// final write of a ray's outputs.
#pragma once

#include "ss_device.cuh"

namespace ss {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ int64_t ray_count(const Tile& T, const Rays& R) {
    return R.mode == 0 ? (int64_t)T.nx * T.ny : R.n;
}

// cos(eps_p) of ray r's origin in float32 (relative error ~1e-7), enough to
// decide whether its light is saturated.
__device__ __forceinline__ float cos_elev_f32(const Tile& T, const Rays& R, int64_t r,
                                              bool stereo) {
    float u, v;
    if (R.mode == 0) {
        int32_t iu, iv;
        grid_uv(T, r, iu, iv);
        u = (float)iu;
        v = (float)iv;
    } else {
        u = R.uv[2 * r];
        v = R.uv[2 * r + 1];
    }
    const float g = T.g_f, Rs = T.R_f;
    const float X = (u - T.cx_f) * g, Y = (v - T.cy_f) * g;
    float se;
    if (!stereo) {
        se = (X * T.sx_f + Y * T.sy_f + Rs * T.sz_f) * rsqrtf(X * X + Y * Y + Rs * Rs);
    } else {   // n = (2x, 2y, 1 - x^2 - y^2) / (1 + x^2 + y^2), (x, y) = (X, Y) / 2R
        const float k = 0.5f / Rs, x = X * k, y = Y * k, q = x * x + y * y;
        se = (2.0f * x * T.sx_f + 2.0f * y * T.sy_f + (1.0f - q) * T.sz_f) / (1.0f + q);
    }
    return sqrtf(fmaxf(0.0f, 1.0f - se * se));
}

// FP64 re-evaluation of ray r's argmin sample (rays whose light is not
// saturated): the cost in FP64, the disc formula (Eq. discfrac) in float32
// (error < 1e-7 in light).
__device__ __forceinline__ void refine_ray(const Tile& T, const Rays& R, int64_t r,
                                           int32_t bestj, bool stereo, float& light, float& cost) {
    double up, vp, hp, href, ow[4];
    int32_t oi0, oj0;
    ray_origin(T, R, r, up, vp, hp, href, oi0, oj0, ow);
    Geom64 G;
    geom64_any(T, up, vp, hp, G, stereo);
    const double c = leaf_cost64(T, G, bestj, stereo);
    const float se = (float)G.sin_e;
    const float d = (float)c * sqrtf(fmaxf(0.0f, 1.0f - se * se)) / T.alpha_f;
    light = disc_light32(d);
    cost = (float)c;
}

// Light value marking a ray whose FP64 re-evaluation is left to refine_kernel.
constexpr float kLightPending = -1.0f;

// Final value of one ray: the FP64 re-evaluation of its argmin sample unless
// the light is certainly saturated (|c*| cos(eps) >= 1.001 alpha), then the
// disc-occlusion formula (Eq. discfrac).  kDefer: leave the re-evaluation to
// refine_kernel (light = kLightPending), so that the walk's warp services
// carry no FP64 re-evaluation with a lane or two active.
template <bool kStereo = false, bool kDefer = false>
__device__ __forceinline__ void finish_ray(const Tile& T, const Rays& R, const Outputs& O,
                                           int64_t r, float best, int32_t bestj, int32_t nb,
                                           int32_t nl) {
    float light, cost;
    bool write_cost = true;
    if (bestj < 0) {
        light = 1.0f;
        cost = INFINITY;
    } else if (fabsf(best) * cos_elev_f32(T, R, r, kStereo) >= 1.001f * T.alpha_f) {
        light = best > 0.0f ? 1.0f : 0.0f;
        cost = best;
    } else if (kDefer) {
        light = kLightPending;
        cost = 0.0f;
        write_cost = false;
    } else {
        refine_ray(T, R, r, bestj, kStereo, light, cost);
    }
    O.light[r] = light;
    O.argmin[r] = bestj;
    if (O.cost && write_cost) O.cost[r] = cost;
    if (O.counters) {
        O.counters[2 * r] = nb;
        O.counters[2 * r + 1] = nl;
    }
}

template <bool kGrid, bool kLight = false, bool kStereo = false>
__device__ __forceinline__ void setup_ray(const Tile& T, const Rays& R, int64_t r, float span,
                                          RayF& rf) {
    double up, vp, hp, href;
    float uf, vf;
    if (kGrid) {
        int32_t u, v;
        grid_uv(T, r, u, v);
        if (!kStereo) {   // no FP64 on the common path
            float se;
            make_rayf_gnomonic_grid(T, u, v, T.h[(int64_t)v * T.pitch + u], span, rf, se);
            if (kLight) {
                const float ce = sqrtf(fmaxf(0.0f, 1.0f - se * se));
                rf.c_sat = ce > 0.0f ? 1.002f * T.alpha_f / ce : INFINITY;
            }
            return;
        }
        uf = (float)u;
        vf = (float)v;
        up = (double)u;
        vp = (double)v;
        hp = href = (double)T.h[(int64_t)v * T.pitch + u];
    } else {
        uf = R.uv[2 * r];
        vf = R.uv[2 * r + 1];
        if (R.status && !(isfinite(uf) && isfinite(vf) && (!R.lift || isfinite(R.lift[r]))))
            atomicOr(R.status, kDevNonfiniteRay);
        if (!kStereo) {
            double ow[4];
            int32_t oi0, oj0;
            ray_origin(T, R, r, up, vp, hp, href, oi0, oj0, ow);
        }
    }
    float se;
    if (!kStereo) {
        make_rayf_gnomonic<kGrid>(T, up, vp, uf, vf, hp, href, span, rf, se);
    } else {
        // origin and local frame in float-float (stereographic, see geom_stereo_df)
        float hr;
        const DF hpd = kGrid ? DF{ (float)hp, 0.0f }
                             : origin_height_df(T, uf, vf, R.lift ? R.lift[r] : 0.0f, hr);
        if (kGrid) hr = (float)href;
        Geom64 G;
        geom_stereo_df(T, uf, vf, hpd, G);
        make_rayf<true>(T, G, (double)hr, span, rf);
        if (kGrid) rf.X = 0.0f;
        se = (float)G.sin_e;
    }
    if (kLight) {   // saturation threshold of the light (with a 0.2% margin)
        const float ce = sqrtf(fmaxf(0.0f, 1.0f - se * se));
        rf.c_sat = ce > 0.0f ? 1.002f * T.alpha_f / ce : INFINITY;
    }
}

// A set-up ray parked in shared memory (one 32-bit word per field, word-major:
// q[word][slot], so that lanes writing or reading different slots hit
// different banks).  Only the fields the walk reads for this kernel instance
// are kept; iu0/iv0 (grid rays), au, av and the gnomonic inv_rho2 are
// recomputed on load by the same operations as in the setup.
constexpr int kQSlots = 32;

template <bool kGrid, bool kLight, bool kStereo>
struct RayPack {
    static constexpr int kWords = 15 + (kGrid ? 0 : 3) + (kStereo ? 4 : 0) + (kLight ? 1 : 0);

    __device__ static __forceinline__ void store(uint32_t (*q)[kQSlots], int s, const RayF& r) {
        int k = 0;
        q[k++][s] = __float_as_uint(r.u0);
        q[k++][s] = __float_as_uint(r.v0);
        q[k++][s] = __float_as_uint(r.au_hi);
        q[k++][s] = __float_as_uint(r.au_lo);
        q[k++][s] = __float_as_uint(r.av_hi);
        q[k++][s] = __float_as_uint(r.av_lo);
        q[k++][s] = __float_as_uint(r.b);
        q[k++][s] = __float_as_uint(r.B);
        q[k++][s] = __float_as_uint(r.inv_2rho);
        q[k++][s] = __float_as_uint(r.href);
        q[k++][s] = __float_as_uint(r.tv);
        q[k++][s] = __float_as_uint(r.gconst);
        q[k++][s] = __float_as_uint(r.pos_eps);
        q[k++][s] = (uint32_t)r.j_lo;
        q[k++][s] = (uint32_t)r.j_hi;
        if (!kGrid) {
            q[k++][s] = __float_as_uint(r.X);
            q[k++][s] = (uint32_t)r.iu0;
            q[k++][s] = (uint32_t)r.iv0;
        }
        if (kStereo) {
            q[k++][s] = __float_as_uint(r.inv_rho2);
            q[k++][s] = __float_as_uint(r.bu);
            q[k++][s] = __float_as_uint(r.bv);
            q[k++][s] = __float_as_uint(r.inv8r);
        }
        if (kLight) q[k++][s] = __float_as_uint(r.c_sat);
    }

    __device__ static __forceinline__ void load(const uint32_t (*q)[kQSlots], int s, RayF& r) {
        int k = 0;
        r.u0 = __uint_as_float(q[k++][s]);
        r.v0 = __uint_as_float(q[k++][s]);
        r.au_hi = __uint_as_float(q[k++][s]);
        r.au_lo = __uint_as_float(q[k++][s]);
        r.av_hi = __uint_as_float(q[k++][s]);
        r.av_lo = __uint_as_float(q[k++][s]);
        r.b = __uint_as_float(q[k++][s]);
        r.B = __uint_as_float(q[k++][s]);
        r.inv_2rho = __uint_as_float(q[k++][s]);
        r.href = __uint_as_float(q[k++][s]);
        r.tv = __uint_as_float(q[k++][s]);
        r.gconst = __uint_as_float(q[k++][s]);
        r.pos_eps = __uint_as_float(q[k++][s]);
        r.j_lo = (int32_t)q[k++][s];
        r.j_hi = (int32_t)q[k++][s];
        if (!kGrid) {
            r.X = __uint_as_float(q[k++][s]);
            r.iu0 = (int32_t)q[k++][s];
            r.iv0 = (int32_t)q[k++][s];
        } else {
            r.X = 0.0f;
            r.iu0 = (int32_t)r.u0;   // grid origins are texel centres
            r.iv0 = (int32_t)r.v0;
        }
        if (kStereo) {
            r.inv_rho2 = __uint_as_float(q[k++][s]);
            r.bu = __uint_as_float(q[k++][s]);
            r.bv = __uint_as_float(q[k++][s]);
            r.inv8r = __uint_as_float(q[k++][s]);
        } else {
            r.inv_rho2 = inv_rho2_of(r.inv_2rho);
            r.bu = r.bv = r.inv8r = 0.0f;
        }
        r.c_sat = kLight ? __uint_as_float(q[k++][s]) : 0.0f;
        r.au = __fadd_rn(r.au_hi, r.au_lo);
        r.av = __fadd_rn(r.av_hi, r.av_lo);
        r.guard0 = 0.0f;   // (not read by the descent)
    }
};




// Grid-mode rays grouped into chunks of `chunk` rays: with tile_w == 0 the
// chunks are runs of consecutive ray ids (row-major texels); with tile_w > 0
// (chunk a multiple of tile_w) they are tile_w x (chunk / tile_w) rectangles
// of texels in row-major order of rectangles, smaller at the right and bottom
// edges.  A chunk's rays are drawn in row-major order within it.
struct ChunkRange {
    int64_t lo;       // first ray id (linear chunks)
    int32_t cnt;      // rays in the chunk
    int32_t x0, y0, w;   // rectangle origin and width (rectangular chunks)
    int32_t rect;
};

__host__ __device__ __forceinline__ int64_t chunk_count(int64_t n, int32_t nx, int32_t ny,
                                                        int32_t chunk, int32_t tile_w) {
    if (tile_w <= 0) return (n + chunk - 1) / chunk;
    const int32_t th = chunk / tile_w;
    return (int64_t)((nx + tile_w - 1) / tile_w) * ((ny + th - 1) / th);
}

__device__ __forceinline__ ChunkRange chunk_range(int64_t c, int64_t n, int32_t nx, int32_t ny,
                                                  int32_t chunk, int32_t tile_w) {
    ChunkRange C;
    if (tile_w <= 0) {
        C.rect = 0;
        C.lo = c * chunk;
        const int64_t left = n - C.lo;
        C.cnt = (int32_t)(left < chunk ? left : chunk);
        C.x0 = C.y0 = C.w = 0;
    } else {
        const int32_t th = chunk / tile_w, rx = (nx + tile_w - 1) / tile_w;
        const int32_t bx = (int32_t)(c % rx), by = (int32_t)(c / rx);
        C.rect = 1;
        C.lo = 0;
        C.x0 = bx * tile_w;
        C.y0 = by * th;
        C.w = min(tile_w, nx - C.x0);
        C.cnt = C.w * min(th, ny - C.y0);
    }
    return C;
}

__device__ __forceinline__ int64_t chunk_ray(const ChunkRange& C, int32_t nx, int32_t i) {
    if (!C.rect) return C.lo + i;
    const int32_t q = (int32_t)((uint32_t)i / (uint32_t)C.w);   // i >= 0
    return (int64_t)(C.y0 + q) * nx + C.x0 + (i - q * C.w);
}

// Lane state of the descent over one ray.
struct Walk {
    float best;
    int32_t bestj, s0, k, nb, nl;
};

// While best is +inf every block on the left spine of the tree is split without
// a bound being able to prune it, so the walk starts directly with the first
// run of leaves (same order, same result).  In light-only mode best starts at
// +c_sat, which can prune from the root, so the walk starts at the root.
template <bool kLight = false>
__device__ __forceinline__ void walk_begin(Walk& w, const RayF& rf, int32_t kleaf) {
    w.bestj = -1;
    w.s0 = w.nb = w.nl = 0;
    if (kLight) {
        w.best = rf.c_sat;
        const int32_t K = rf.j_hi <= 1 ? 0 : 32 - __clz(rf.j_hi - 1);   // 2^K >= j_hi
        w.k = K > kleaf ? K : 0;
    } else {
        w.best = INFINITY;
        w.k = 0;
    }
}

// Seeded start: best is already the cost of sample seed_j (an upper bound of
// the minimum); the walk still visits every sample whose cost could be lower
// or equal at a smaller index.  It starts with the first run of leaves, as an
// unseeded walk does: every block on the left spine contains the first
// samples, whose bound (divided by the smallest t) is almost never above best,
// so probing them first would only add failed bounds.  Light-only walks start
// at the root, where +c_sat can prune a whole lit ray.
template <bool kLight = false>
__device__ __forceinline__ void walk_begin_seeded(Walk& w, const RayF& rf, int32_t kleaf,
                                                  float seed, int32_t seed_j) {
    w.s0 = w.nb = w.nl = 0;
    const int32_t K = rf.j_hi <= 1 ? 0 : 32 - __clz(rf.j_hi - 1);   // 2^K >= j_hi
    w.k = (kLight && K > kleaf) ? K : 0;
    const bool use = !kLight || seed < rf.c_sat;
    w.best = use ? seed : rf.c_sat;
    w.bestj = use ? seed_j : -1;
}

// Best of the ray's own samples within +-sw of index j0 (clipped to
// [j_lo, j_hi]); j_out = -1 when none is usable.  Smallest index on ties.
template <bool kGrid, bool kPoly, bool kStereo>
__device__ __forceinline__ float seed_near(const Tile& T, const RayF& rf, int32_t j0, int32_t sw,
                                           int32_t& j_out) {
    float best = INFINITY;
    j_out = -1;
    const int32_t lo = max(rf.j_lo, j0 - sw), hi = min(rf.j_hi, j0 + sw);
    for (int32_t j = lo; j <= hi; ++j) {
        float rise;
        const float c = leaf_cost<kGrid, kPoly, kStereo>(T, rf, j, rise);
        if (c < best) {
            best = c;
            j_out = j;
        }
    }
    return best;
}

// Seed of a ray with no finished neighbour (the first row of a block's
// rectangle): the best of its samples j_lo - 1 + 2^k, k = 0, 1, ..., and j_hi
// (about log2 of the range: 12 samples for 3000).  Near samples are dense and
// far ones sparse, like the walk's blocks; in a CPU simulation of the 4096^2
// workload such a seed cut an unseeded walk from 336 to 163 probes (the 12
// samples included).  n_out: samples evaluated.  Smallest index on ties.
template <bool kGrid, bool kPoly, bool kStereo>
__device__ __forceinline__ float seed_geo(const Tile& T, const RayF& rf, int32_t& j_out,
                                          int32_t& n_out) {
    float best = INFINITY;
    j_out = -1;
    n_out = 0;
    if (rf.j_hi < rf.j_lo) return best;
    for (int32_t d = 1; d <= (1 << 30); d <<= 1) {
        const int32_t j = min(rf.j_lo - 1 + d, rf.j_hi);
        float rise;
        const float c = leaf_cost<kGrid, kPoly, kStereo>(T, rf, j, rise);
        ++n_out;
        if (c < best) {
            best = c;
            j_out = j;
        }
        if (j >= rf.j_hi) break;
    }
    return best;
}

// Where this ray meets the terrain point of a parallel neighbouring ray's
// argmin j_src: p + j a = p_src + j_src a gives j = j_src + d.a / |a|^2,
// d = p_src - p (texels), a the per-sample step of this ray at its origin.
// A neighbour one row up along a ray running down the columns is two samples
// ahead (0.5-texel steps), so a window around j_src alone would miss it.
// (Grid rays.  Listed rays keep the window at j_src: on the polar view the
// centring saved 5% of the probes but measured 4% slower.)
__device__ __forceinline__ int32_t seed_centre(const RayF& rf, int32_t j_src, float du, float dv) {
    const float a2 = rf.au * rf.au + rf.av * rf.av;
    const float sh = a2 > 0.0f ? __fdividef(du * rf.au + dv * rf.av, a2) : 0.0f;
    return j_src + (int32_t)rintf(fminf(fmaxf(sh, -1.0e6f), 1.0e6f));
}

// Seed of a newly drawn ray: with a finished neighbour (`near`), its samples
// within +-sw of jc (seed_centre of the neighbour's argmin); else, or when
// that window holds no usable sample, the sparse samples of seed_geo when
// `geo`; else none (j_out = -1).  n_out: samples evaluated (the probe counters
// include them).
template <bool kGrid, bool kPoly, bool kStereo>
__device__ __forceinline__ float seed_ray(const Tile& T, const RayF& rf, bool near, int32_t jc,
                                          int32_t sw, bool geo, int32_t& j_out, int32_t& n_out) {
    float best = INFINITY;
    j_out = -1;
    n_out = 0;
    if (near) {
        n_out = max(0, min(rf.j_hi, jc + sw) - max(rf.j_lo, jc - sw) + 1);
        best = seed_near<kGrid, kPoly, kStereo>(T, rf, jc, sw, j_out);
    }
    if (j_out < 0 && geo) {
        int32_t n_geo;
        best = seed_geo<kGrid, kPoly, kStereo>(T, rf, j_out, n_geo);
        n_out += n_geo;
    }
    return best;
}

// One probe of the exact descent and the state update; true when finished.
// Stackless depth-first walk over aligned sample blocks [s0+1, s0+2^k]: a
// block's bound is compared with the running minimum; blocks that cannot win
// are skipped, the others split; blocks of <= 2^kleaf samples are evaluated
// sample by sample.  After a block the walk continues at s0 += 2^k with
// k = ctz(s0), the next block in near-to-far order, so samples are evaluated
// in increasing j and a strict '<' keeps the smallest j among equal costs.
// Blocks are clipped to [j_lo, j_hi].
template <bool kCount, bool kGrid, bool kPoly, bool kLight = false, bool kStereo = false>
__device__ __forceinline__ bool walk_step(const Tile& T, const LevelTab& L, int32_t levels,
                                          int32_t kleaf, const RayF& rf, Walk& w) {
    const bool leaf = (w.k == 0);
    const int32_t s1 = w.s0 + 1;
    int32_t ja = leaf ? s1 : max(s1, rf.j_lo);
    int32_t jb = leaf ? s1 : min(w.s0 + (1 << w.k), rf.j_hi);
    const bool valid = leaf ? (s1 >= rf.j_lo) : (ja <= jb);
    ja = valid ? ja : rf.j_lo;
    jb = valid ? jb : rf.j_lo;
    const float v = probe<kGrid, kPoly, kStereo>(T, L, levels, rf, ja, jb, leaf);
    // a seeded walk may meet a sample as good as the seed at a smaller index
    const bool improve = valid && leaf && (v < w.best || (v == w.best && ja < w.bestj));
    w.best = improve ? v : w.best;
    w.bestj = improve ? ja : w.bestj;
    const bool descend = valid && !leaf && !(v > w.best);
    if (kCount) {
        w.nl += (valid && leaf) ? 1 : 0;
        w.nb += (valid && !leaf) ? 1 : 0;
    }
    const int32_t s_adv = w.s0 + (1 << w.k);
    const int32_t k_adv = __ffs(s_adv) - 1;
    w.s0 = descend ? w.s0 : s_adv;
    w.k = descend ? ((w.k - 1 > kleaf) ? w.k - 1 : 0) : ((k_adv <= kleaf) ? 0 : k_adv);
    const bool end = !descend && (s_adv >= rf.j_hi);
    return kLight ? (end || w.best <= -rf.c_sat) : end;
}

}  // namespace ss
