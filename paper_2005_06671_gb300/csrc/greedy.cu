// The paper's greedy descent (Algorithm 1 with the ray length T of Eq. maxstep
// and the interval concatenation of Sec. 3.3 "Long shadows"): an approximation
// of the minimum, reproduced so that its error against the exact descent can be
// measured on the same GPU.  One thread per ray, FP64 (3 tip samples per level,
// N' levels per run, a handful of runs: ~45 samples per ray).
//
// Per run r (starting at distance a_r along the ray):
//   T_r: the ray parameter closest to the line through the sphere's centre and
//        the texel point 2^(N'-1) texels from the run start's texel image along
//        the sun's texture-plane direction (s_x, s_y);
//   t_0 = 1; level k = 0 .. N'-1 reads mip level m = N'-1-k at the tips
//        t_k, t_k - 2^-(k+1), t_k - 2^-k (distance a_r + t T_r), keeping the
//        smallest Delta = H - M (H = tip height over the sphere, M = the level-m
//        texel containing the tip's texel image; the first one on ties); tips at
//        t <= 0 or off the tile are not read; then t_{k+1} = t* + 2^-(k+1), or
//        t_k - 2^-k when no tip was read;
//   J_r = Delta* / (a_r + t* T_r) of the last level.
// The ray's cost is the smallest J_r; light = F(clamp(J cos(eps_p)/alpha, -1, 1)).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "ss_launch.h"
#include "ss_walk.cuh"

namespace ss {

namespace {

struct GreedyArgs {
    Tile T;
    Pyramid P;
    Rays R;
    const float* stats;   // (global max, global min) of the heights
    float* light;
    float* cost;
    float* t_star;
    int32_t n_runs;
    int32_t levels[kGreedyMaxRuns];
};

__device__ __forceinline__ void cross3(const double a[3], const double b[3], double c[3]) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

__device__ __forceinline__ double dot3(const double a[3], const double b[3]) {
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

// Eq. maxstep for a run starting at point Rs: length of the run
__device__ double run_length(const Tile& T, const double Rs[3], const double s[3], int32_t m0) {
    double u0, v0;
    if (!texel_image64(T, Rs, u0, v0)) return -1.0;
    const double ln = sqrt(s[0] * s[0] + s[1] * s[1]);
    if (!(ln > 0.0)) return -1.0;
    const double span = ldexp(1.0, m0);
    double e[3];
    texel_dir64(T, u0 + span * s[0] / ln, v0 + span * s[1] / ln, e);
    const double c[3] = { -Rs[0], -Rs[1], -Rs[2] };
    double ce[3], se[3];
    cross3(c, e, ce);
    cross3(s, e, se);
    const double den = dot3(se, se);
    if (!(den > 0.0)) return -1.0;
    return dot3(ce, se) / den;
}

// one tip: true and delta = H - M when its texel image lies in the tile
__device__ __forceinline__ bool tip(const Tile& T, const Pyramid& P, const double p[3],
                                    const double s[3], double dist, int32_t m, double& delta) {
    const double q[3] = { p[0] + dist * s[0], p[1] + dist * s[1], p[2] + dist * s[2] };
    double u, v;
    if (!texel_image64(T, q, u, v) || !in_tile64(T, u, v)) return false;
    const double cell = ldexp(1.0, m);
    const int32_t w = ((T.nx - 1) >> m) + 1, h = ((T.ny - 1) >> m) + 1;
    const int32_t I = min(max((int32_t)floor((u + 0.5) / cell), 0), w - 1);
    const int32_t J = min(max((int32_t)floor((v + 0.5) / cell), 0), h - 1);
    const double M = (double)P.ptr[m][(int64_t)J * P.pitch[m] + I];
    delta = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2]) - T.R - M;
    return true;
}

__global__ void __launch_bounds__(256) greedy_kernel(const GreedyArgs a) {
    const Tile& T = a.T;
    const int64_t n = ray_count(T, a.R);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const double s[3] = { T.sx, T.sy, T.sz };
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += stride) {
        double up, vp, hp, href, ow[4];
        int32_t oi0, oj0;
        ray_origin(T, a.R, r, up, vp, hp, href, oi0, oj0, ow);
        double nv[3];
        texel_dir64(T, up, vp, nv);
        const double rho = T.R + hp;
        const double p[3] = { rho * nv[0], rho * nv[1], rho * nv[2] };
        double bestJ = INFINITY, bestd = -1.0, start = 0.0;
        for (int32_t run = 0; run < a.n_runs; ++run) {
            const int32_t Np = a.levels[run];
            const double Rs[3] = { p[0] + start * s[0], p[1] + start * s[1], p[2] + start * s[2] };
            const double Tr = run_length(T, Rs, s, Np - 1);
            if (!(Tr > 0.0)) break;
            double tk = 1.0, dstar = INFINITY, ts = -1.0;
            for (int32_t k = 0; k < Np; ++k) {
                const int32_t m = min(Np - 1 - k, a.P.levels - 1);
                const double step = ldexp(1.0, -(k + 1));
                dstar = INFINITY;
                ts = -1.0;
                for (int i = 0; i < 3; ++i) {
                    if (i > 0) tk -= step;
                    double dl;
                    if (tk > 0.0 && tip(T, a.P, p, s, start + tk * Tr, m, dl) && dl < dstar) {
                        dstar = dl;
                        ts = tk;
                    }
                }
                if (ts > -1.0) tk = ts + step;
            }
            if (ts > -1.0) {
                const double dist = start + ts * Tr;
                const double J = dstar / dist;
                if (J < bestJ) {
                    bestJ = J;
                    bestd = dist;
                }
            }
            start += Tr;
        }
        float light = 1.0f;
        if (bestd > 0.0) {
            const double se = dot3(nv, s);
            const double ce = sqrt(fmax(0.0, 1.0 - se * se));
            light = (float)disc_light64(bestJ * ce / T.alpha);
        }
        a.light[r] = light;
        if (a.cost) a.cost[r] = (float)bestJ;
        if (a.t_star) a.t_star[r] = (float)bestd;
    }
}

// ------------------------------------------------- float32 greedy descent
// The same algorithm at the arithmetic of the paper's shader (float32), on
// gnomonic tiles: tip heights in the ray's local frame (origin height minus a
// reference texel, plus the cancellation-free rise), tip texel images from the
// ray's float32 slope (as the exact descent's block ends), the run length of
// Eq. maxstep in float32 in the tile-centre frame.  FP64 only where a tip's
// level-m texel is ambiguous: when its float32 image lies within its error
// margin of a cell edge or of the tile's border, the FP64 image decides.
// An approximation of the same approximation: reported beside the FP64 kernel,
// which keeps decision identity with the oracle.

// Eq. maxstep in float32: run start Rs = P0 + rs (P0 = (0, 0, R), the tile
// centre's point on the sphere; rs a few km, kept to ~1 mm)
__device__ float run_length_f32(const Tile& T, const float rs[3], const float s[3], int32_t m0) {
    const float R = T.R_f, kx = T.R_f / T.g_f;
    const float qz = R + rs[2];
    if (!(qz > 0.0f)) return -1.0f;
    const float u0 = kx * rs[0] / qz + T.cx_f, v0 = kx * rs[1] / qz + T.cy_f;
    const float ln = sqrtf(s[0] * s[0] + s[1] * s[1]);
    if (!(ln > 0.0f)) return -1.0f;
    const float span = ldexpf(1.0f, m0);
    const float X = (u0 + span * s[0] / ln - T.cx_f) * T.g_f;
    const float Y = (v0 + span * s[1] / ln - T.cy_f) * T.g_f;
    const float im = rsqrtf(X * X + Y * Y + R * R);
    const float e[3] = { X * im, Y * im, R * im };
    // c = -(P0 + rs); c x e = -(P0 x e) - rs x e, with P0 x e = R (-e_y, e_x, 0)
    const float ce[3] = { R * e[1] - (rs[1] * e[2] - rs[2] * e[1]),
                          -R * e[0] - (rs[2] * e[0] - rs[0] * e[2]),
                          -(rs[0] * e[1] - rs[1] * e[0]) };
    const float se[3] = { s[1] * e[2] - s[2] * e[1], s[2] * e[0] - s[0] * e[2],
                          s[0] * e[1] - s[1] * e[0] };
    const float den = se[0] * se[0] + se[1] * se[1] + se[2] * se[2];
    if (!(den > 0.0f)) return -1.0f;
    return (ce[0] * se[0] + ce[1] * se[1] + ce[2] * se[2]) / den;
}

// A tip the float32 margin leaves ambiguous, for grid rays: its texel image
// u = u_p + Au j/(1 + b j), j = dist/delta, in float-float (relative error
// ~1e-13, ~1e-9 texel), the same map geom64 evaluates in FP64.  Returns false
// (FP64 decides) when the position is within 1e-6 texel of a tile edge or of
// the cell edge that decides the mip texel.
__device__ __forceinline__ bool tip_df(const Tile& T, const RayF& rf, float dist, float cell,
                                       int32_t w, int32_t h, bool& have, DF A[3], bool& in,
                                       int32_t& I, int32_t& J) {
    if (!have) {
        gnomonic_grid_df(T, rf.u0, rf.v0, rf.href, A[0], A[1], A[2]);
        have = true;
    }
    const DF jd = df_div(DF{ dist, 0.0f }, DF{ T.delta_hi, T.delta_lo });
    const DF den = df_add(DF{ 1.0f, 0.0f }, df_mul(A[2], jd));
    if (!(den.hi > 0.25f)) return false;   // (far along the ray: FP64 decides)
    const DF tau = df_div(jd, den);
    const DF U = df_add(DF{ rf.u0, 0.0f }, df_mul(A[0], tau));
    const DF V = df_add(DF{ rf.v0, 0.0f }, df_mul(A[1], tau));
    // every decision is the sign of a float-float difference: hi may be an
    // integer (or an edge) exactly while lo carries the other side
    constexpr float kE2 = 1e-6f;
    const float lim[4] = { 0.0f, (float)(T.nx - 1), 0.0f, (float)(T.ny - 1) };
    float d[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        d[e] = df_add(e < 2 ? U : V, DF{ -lim[e], 0.0f }).hi;
        if (fabsf(d[e]) < kE2) return false;
    }
    in = d[0] > 0.0f && d[1] < 0.0f && d[2] > 0.0f && d[3] < 0.0f;
    const float ic = 1.0f / cell;   // a power of two: exact scaling
    const DF fu = df_add(U, DF{ 0.5f, 0.0f }), fv = df_add(V, DF{ 0.5f, 0.0f });
    const DF su = { fu.hi * ic, fu.lo * ic }, sv = { fv.hi * ic, fv.lo * ic };
    const float nu = rintf(su.hi), nv = rintf(sv.hi);
    const float du = df_add(su, DF{ -nu, 0.0f }).hi, dv = df_add(sv, DF{ -nv, 0.0f }).hi;
    if (fabsf(du) < kE2 * ic || fabsf(dv) < kE2 * ic) return false;
    // floor(x) = n - 1 below the nearest integer n, n above it
    I = min(max((int32_t)nu - (du < 0.0f ? 1 : 0), 0), w - 1);
    J = min(max((int32_t)nv - (dv < 0.0f ? 1 : 0), 0), h - 1);
    return true;
}

// Three resident blocks per SM (80 registers): 4096^2, N' = {5,5,5}, GB300:
// 6.39 ms against 8.61 ms at 96 registers (two blocks) and 6.91 ms at four.
#ifndef SS_GREEDY_MIN_BLOCKS
#define SS_GREEDY_MIN_BLOCKS 3
#endif
template <bool kGrid>
__global__ void __launch_bounds__(256, SS_GREEDY_MIN_BLOCKS) greedy_f32_kernel(const GreedyArgs a) {
    const Tile& T = a.T;
    const int64_t n = ray_count(T, a.R);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const float s[3] = { T.sx_f, T.sy_f, T.sz_f };
    const double sd[3] = { T.sx, T.sy, T.sz };
    const float span = a.stats[0] - a.stats[1];
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += stride) {
        RayF rf;
        setup_ray<kGrid, false, false>(T, a.R, r, span, rf);
        // origin relative to P0 (p = rho n, n = (X, Y, R)/m, m = |(X, Y, R)|):
        // p_z - R = (R/m)(rho - m) = (R/m)(h_p - (X^2 + Y^2)/(m + R)), no
        // cancellation; the FP64 origin only for ambiguous tips
        const float Xp = (rf.u0 - T.cx_f) * T.g_f, Yp = (rf.v0 - T.cy_f) * T.g_f;
        const float rho = 0.5f / rf.inv_2rho;
        const float im = rsqrtf(Xp * Xp + Yp * Yp + T.R_f * T.R_f);
        const float m = 1.0f / im;
        const float hp = rf.href + rf.X;
        float p0[3];
        p0[0] = rho * Xp * im;
        p0[1] = rho * Yp * im;
        p0[2] = T.R_f * im * (hp - (Xp * Xp + Yp * Yp) / (m + T.R_f));
        bool have64 = false, have_df = false;
        double p64[3] = { 0.0, 0.0, 0.0 };
        DF Adf[3];   // grid rays: float-float Au, Av, b (on the first ambiguous tip)
        const float amax = fmaxf(fabsf(rf.au), fabsf(rf.av));
        float bestJ = INFINITY, bestd = -1.0f, start = 0.0f;
        for (int32_t run = 0; run < a.n_runs; ++run) {
            const int32_t Np = a.levels[run];
            const float rs[3] = { p0[0] + start * s[0], p0[1] + start * s[1],
                                  p0[2] + start * s[2] };
            const float Tr = run_length_f32(T, rs, s, Np - 1);
            if (!(Tr > 0.0f)) break;
            float tk = 1.0f, dstar = INFINITY, ts = -1.0f;
            for (int32_t k = 0; k < Np; ++k) {
                const int32_t mlev = min(Np - 1 - k, a.P.levels - 1);
                const float step = ldexpf(1.0f, -(k + 1));
                const float cell = ldexpf(1.0f, mlev);
                const int32_t w = ((T.nx - 1) >> mlev) + 1, h = ((T.ny - 1) >> mlev) + 1;
                dstar = INFINITY;
                ts = -1.0f;
                for (int i = 0; i < 3; ++i) {
                    if (i > 0) tk -= step;
                    if (!(tk > 0.0f)) continue;
                    const float dist = start + tk * Tr;
                    const float jf = dist / T.delta_f;
                    float u, v;
                    block_end<false>(T, rf, jf, 0.0f, 0.0f, u, v);
                    const float E = 1e-3f + 5e-7f * (float)(T.nx + T.ny) + 8e-7f * amax * jf;
                    const float fu = (u + 0.5f) / cell, fv = (v + 0.5f) / cell;
                    const float eu = E / cell;
                    const bool amb = fabsf(fu - rintf(fu)) < eu || fabsf(fv - rintf(fv)) < eu ||
                                     fabsf(u) < E || fabsf(u - (float)(T.nx - 1)) < E ||
                                     fabsf(v) < E || fabsf(v - (float)(T.ny - 1)) < E;
                    bool in;
                    int32_t I, J;
                    if (!amb) {
                        in = u >= 0.0f && u <= (float)(T.nx - 1) && v >= 0.0f &&
                             v <= (float)(T.ny - 1);
                        I = min(max((int32_t)floorf(fu), 0), w - 1);
                        J = min(max((int32_t)floorf(fv), 0), h - 1);
                    } else if (kGrid && tip_df(T, rf, dist, cell, w, h, have_df, Adf, in, I, J)) {
                        // settled in float-float
                    } else {
                        if (!have64) {
                            double up, vp, hp, href, ow[4];
                            int32_t oi0, oj0;
                            ray_origin(T, a.R, r, up, vp, hp, href, oi0, oj0, ow);
                            double nv[3];
                            texel_dir64(T, up, vp, nv);
                            const double rhod = T.R + hp;
                            for (int c = 0; c < 3; ++c) p64[c] = rhod * nv[c];
                            have64 = true;
                        }
                        const double dd = (double)dist;
                        const double q[3] = { p64[0] + dd * sd[0], p64[1] + dd * sd[1],
                                              p64[2] + dd * sd[2] };
                        double ud, vd;
                        in = texel_image64(T, q, ud, vd) && in_tile64(T, ud, vd);
                        const double celld = (double)cell;
                        I = min(max((int32_t)floor((ud + 0.5) / celld), 0), w - 1);
                        J = min(max((int32_t)floor((vd + 0.5) / celld), 0), h - 1);
                    }
                    if (!in) continue;
                    const float M = __ldg(a.P.ptr[mlev] + (int64_t)J * a.P.pitch[mlev] + I);
                    const float dl = (rf.X + rise_of<false>(rf, dist)) - (M - rf.href);
                    if (dl < dstar) {
                        dstar = dl;
                        ts = tk;
                    }
                }
                if (ts > -1.0f) tk = ts + step;
            }
            if (ts > -1.0f) {
                const float dist = start + ts * Tr;
                const float J = dstar / dist;
                if (J < bestJ) {
                    bestJ = J;
                    bestd = dist;
                }
            }
            start += Tr;
        }
        float light = 1.0f;
        if (bestd > 0.0f) light = disc_light32(bestJ * cos_elev_f32(T, a.R, r, false) / T.alpha_f);
        a.light[r] = light;
        if (a.cost) a.cost[r] = bestJ;
        if (a.t_star) a.t_star[r] = bestd;
    }
}

}  // namespace

cudaError_t launch_greedy(const Tile& T, const Pyramid& P, const Rays& R, const int32_t* levels,
                          int32_t n_runs, float* light, float* cost, float* t_star,
                          cudaStream_t s, const float* stats, bool f32) {
    GreedyArgs a{};
    a.T = T;
    a.P = P;
    a.R = R;
    a.stats = stats;
    a.light = light;
    a.cost = cost;
    a.t_star = t_star;
    a.n_runs = n_runs;
    for (int i = 0; i < n_runs && i < kGreedyMaxRuns; ++i) a.levels[i] = levels[i];
    const int64_t n = R.mode == 0 ? (int64_t)T.nx * T.ny : R.n;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, greedy_kernel, 256, 0) !=
            cudaSuccess || per_sm < 1)
        per_sm = 1;
    const int64_t cap = (int64_t)device_sm_count() * per_sm, want = (n + 255) / 256;
    const int grid = (int)(want < cap ? (want < 1 ? 1 : want) : cap);
    if (!f32)
        greedy_kernel<<<grid, 256, 0, s>>>(a);
    else if (R.mode == 0)
        greedy_f32_kernel<true><<<grid, 256, 0, s>>>(a);
    else
        greedy_f32_kernel<false><<<grid, 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace ss
