// View rays of a camera against the bilinear terrain: the terrain points a
// camera sees, which are the origins of the shadow rays (Sec. 4: view rays are
// intersected with the displaced terrain, and the maximum mipmap lets a ray
// skip what it passes above).
//
// Per pixel:
//   d = unit(forward + a right + b up), x(tau) = C + tau d, samples tau_k = k step;
//   the hit is the first sample whose texel image is in the tile and lies on or
//   below the terrain (|x| - R - h <= 0, decided in FP64); when the sample
//   before it is in the tile too the crossing is refined in FP64: bisection
//   until the bracket lies in one bilinear cell, then the single root of the
//   quadratic F there (see refine_crossing).
// Sample blocks are walked near-to-far like the shadow descent (aligned blocks
// of 2^k samples, next block at s0 += 2^k) in float32: a block is skipped when
// the ray's lowest height over it exceeds the maximum-mipmap value over its
// texel footprint by more than the float32 rounding, or when the footprint
// misses the tile; a sample is tested in FP64 unless float32 shows it clearly
// above or below the terrain or off the tile.  So the first sample found below
// the terrain is the first one overall, the same sample as an FP64 march.
//
// A second pass gathers each block's hits and refines them with full warps.
// Then the hits are compacted in pixel order (per-block counts, one scan block,
// a scatter), so the ray list is deterministic.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <cmath>

#include "ss_launch.h"

namespace ss {

namespace {

constexpr int kViewBlock = 256;
constexpr int kViewLeaf = 2;          // blocks of <= 4 samples are tested sample by sample

struct Cam {
    double C[3], f[3], r[3], u[3];
    double tan_x, tan_y;
    int32_t W, H;
    // per launch (host): 2/W, 2/H; |C|^2, |C|; the float32 ray state's camera terms
    double inv_w2, inv_h2, cc, cn;
    float cxf, cyf, czf, alt, zsum, inv_2cn, two_r_g;
};

struct ViewArgs {
    Tile T;
    Pyramid P;
    Cam cam;
    double step, inv_step;
    int64_t K;
    const float* stats;       // (global max, global min) of the heights
    float2* pix_uv;           // per pixel: hit texel coords, NaN when none
    int32_t* hit_k;           // per pixel: first sample below the terrain, -1 when none
    int32_t* block_count;     // per block of kViewBlock pixels
    int64_t* block_off;       // exclusive prefix of block_count
    int32_t n_blocks;
    float* uv_out;
    int32_t* pixel_out;
    int64_t* count_out;
};

// sample at distance tau: in-tile flag, and whether it is on or below the terrain
__device__ __forceinline__ bool below(const Tile& T, const double C[3], const double d[3],
                                      double tau, bool& inside, double& u, double& v) {
    const double x[3] = { C[0] + tau * d[0], C[1] + tau * d[1], C[2] + tau * d[2] };
    inside = texel_image64(T, x, u, v) && in_tile64(T, u, v);
    if (!inside) return false;
    int32_t i0, j0;
    double w[4];
    const double hb = fetch_bilinear64(T.h, T.pitch, T.nx, T.ny, u, v, &i0, &j0, w);
    const double H = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]) - T.R;
    return H - hb <= 0.0;
}

// below() for the bisection of the crossing: one square root and one division
// (|x| serves both the height and the stereographic image; 1/g folded into the
// scale).  Its roundings differ from below()'s only at the 1e-16 relative
// level, and the bisection stops at a bracket of 2^-kViewHalvings of the step,
// below the FP64 resolution of |x| - R at the lunar radius (~1e-10 m), so the
// float32 hit coordinates are those of the full 48-halving bisection.
constexpr int kViewHalvings = 36;

__device__ __forceinline__ bool below_fast(const Tile& T, const double C[3], const double d[3],
                                           double tau) {
    const double x[3] = { C[0] + tau * d[0], C[1] + tau * d[1], C[2] + tau * d[2] };
    const double m = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
    double k;
    if (T.proj == 0) {
        if (!(x[2] > 0.0)) return false;
        k = (T.R * T.inv_g) / x[2];
    } else {
        const double den = m + x[2];
        if (!(den > 0.0)) return false;
        k = (2.0 * T.R * T.inv_g) / den;
    }
    const double u = x[0] * k + T.cx, v = x[1] * k + T.cy;
    if (!in_tile64(T, u, v)) return false;
    int32_t i0, j0;
    double w[4];
    const double hb = fetch_bilinear64(T.h, T.pitch, T.nx, T.ny, u, v, &i0, &j0, w);
    return (m - T.R) - hb <= 0.0;
}

// below_fast's arithmetic, keeping the value F = (|x| - R) - h and the texel
// image: below_fast(tau) == (in && f <= 0), bit for bit.
struct ViewPt {
    double tau, f, u, v;
    bool in;
};

__device__ __forceinline__ ViewPt view_pt(const Tile& T, const double C[3], const double d[3],
                                          double tau) {
    ViewPt p;
    p.tau = tau;
    p.f = 0.0;
    p.u = p.v = 0.0;
    p.in = false;
    const double x[3] = { C[0] + tau * d[0], C[1] + tau * d[1], C[2] + tau * d[2] };
    const double m = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
    double k;
    if (T.proj == 0) {
        if (!(x[2] > 0.0)) return p;
        k = (T.R * T.inv_g) / x[2];
    } else {
        const double den = m + x[2];
        if (!(den > 0.0)) return p;
        k = (2.0 * T.R * T.inv_g) / den;
    }
    p.u = x[0] * k + T.cx;
    p.v = x[1] * k + T.cy;
    if (!in_tile64(T, p.u, p.v)) return p;
    p.in = true;
    int32_t i0, j0;
    double w[4];
    const double hb = fetch_bilinear64(T.h, T.pitch, T.nx, T.ny, p.u, p.v, &i0, &j0, w);
    p.f = (m - T.R) - hb;
    return p;
}

// the bilinear cell fetch_bilinear64 reads for in-tile point p
__device__ __forceinline__ bool same_cell(const Tile& T, const ViewPt& a, const ViewPt& b) {
    const int32_t ia = min(max((int32_t)floor(a.u), 0), T.nx - 2);
    const int32_t ib = min(max((int32_t)floor(b.u), 0), T.nx - 2);
    const int32_t ja = min(max((int32_t)floor(a.v), 0), T.ny - 2);
    const int32_t jb = min(max((int32_t)floor(b.v), 0), T.ny - 2);
    return ia == ib && ja == jb;
}

// maximum of the heights over texel box [x0, x1] x [y0, y1] (inclusive, clamped
// to the tile), read as <= 2x2 cells of the coarsest level whose cells cover it
__device__ __forceinline__ float box_max(const Tile& T, const Pyramid& P, int32_t x0, int32_t x1,
                                         int32_t y0, int32_t y1) {
    const int32_t ext = max(x1 - x0, y1 - y0);
    int32_t m = ext <= 1 ? 0 : 31 - __clz(ext);
    m += (((x1 >> m) - (x0 >> m)) > 1 || ((y1 >> m) - (y0 >> m)) > 1) ? 1 : 0;
    m = min(m, P.levels - 1);
    const float* base = P.ptr[m];
    const int64_t pm = P.pitch[m];
    const int32_t cx0 = x0 >> m, cx1 = x1 >> m, cy0 = y0 >> m, cy1 = y1 >> m;
    const float a = base[(int64_t)cy0 * pm + cx0], b = base[(int64_t)cy0 * pm + cx1];
    const float c = base[(int64_t)cy1 * pm + cx0], e = base[(int64_t)cy1 * pm + cx1];
    return fmaxf(fmaxf(a, b), fmaxf(c, e));
}

// float32 state of one view ray.  The camera is taken relative to the tile
// centre's point on the sphere, P0 = (0, 0, R) (a few km, so float32 keeps it
// to a few mm); the ray height over the sphere is the camera altitude plus
// rise(tau) = |C + tau d| - |C| in the cancellation-free form of the shadow
// rays (rise_of), so heights carry ~1e-2 m of rounding and texel positions
// ~2e-3 texel (5 m texels) over the ray's 150 km.
struct ViewRayF {
    float cx, cy, cz;        // C - P0
    float dx, dy, dz;        // unit direction
    float alt;               // |C| - R
    float two_r_g;           // 2R/g (stereographic) or R/g (gnomonic)
    float zsum;              // |C| + R: |x| + x_z = zsum + rise + cz + tau dz
    RayF rise;               // B = 2 C.d, inv_2rho = 1/(2|C|): rise_of's fields
};

// texel coordinates of the ray point at tau (rise = rise(tau)); false when the
// point has no image (gnomonic: not in front of the plane; stereographic: near
// the antipode)
__device__ __forceinline__ bool view_image_f(const Tile& T, const ViewRayF& q, float tau,
                                             float rise, float& u, float& v) {
    const float x = q.cx + tau * q.dx, y = q.cy + tau * q.dy;
    float den;
    if (T.proj == 0) {
        den = T.R_f + (q.cz + tau * q.dz);              // x_z
    } else {
        den = q.zsum + (rise + (q.cz + tau * q.dz));    // |x| + x_z
    }
    if (!(den > 1.0f)) return false;
    const float k = q.two_r_g / den;
    u = x * k + T.cx_f;
    v = y * k + T.cy_f;
    return true;
}

// unit direction of pixel pix's view ray
__device__ __forceinline__ void pixel_dir(const Cam& cm, int64_t pix, double d[3]) {
    const int64_t i = pix % cm.W, j = pix / cm.W;
    const double aa = (((double)i + 0.5) * cm.inv_w2 - 1.0) * cm.tan_x;
    const double bb = (1.0 - ((double)j + 0.5) * cm.inv_h2) * cm.tan_y;
#pragma unroll
    for (int k = 0; k < 3; ++k) d[k] = cm.f[k] + aa * cm.r[k] + bb * cm.u[k];
    const double idn = 1.0 / sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
#pragma unroll
    for (int k = 0; k < 3; ++k) d[k] *= idn;
}

// Pass 1: per pixel, the first sample below the terrain (hit_k, -1 when none).
__global__ void __launch_bounds__(kViewBlock) view_hit_kernel(const ViewArgs a) {
    const int64_t npix = (int64_t)a.cam.W * a.cam.H;
    const int64_t pix = (int64_t)blockIdx.x * kViewBlock + threadIdx.x;
    if (pix < npix) {
        const Tile& T = a.T;
        const Cam& cm = a.cam;
        double d[3];
        pixel_dir(cm, pix, d);
        const double* C = cm.C;
        int64_t hit_k = -1;
        // samples that can reach the highest height: tau in [tau_in, tau_out]
        const double hmax = (double)a.stats[0];
        const double Rm = T.R + hmax;
        const double cd = C[0] * d[0] + C[1] * d[1] + C[2] * d[2];
        const double disc = cd * cd - (cm.cc - Rm * Rm);
        int64_t k0 = 1, k1 = 0;
        if (disc >= 0.0) {
            const double sq = sqrt(disc);
            const double tau_in = -cd - sq, tau_out = -cd + sq;
            if (tau_out >= 0.0) {
                // (the one-sample margins cover the rounding of the reciprocal)
                k0 = tau_in > 0.0 ? (int64_t)floor(tau_in * a.inv_step) - 1 : 1;
                k0 = k0 < 1 ? 1 : k0;
                k1 = (int64_t)ceil(tau_out * a.inv_step) + 1;
                k1 = k1 > a.K ? a.K : k1;
            }
        }
        // image circle of the ray (stereographic): 1/(8 r) in texels^-1
        float inv8r = 0.0f;
        if (T.proj != 0) {
            const double N[3] = { C[1] * d[2] - C[2] * d[1], C[2] * d[0] - C[0] * d[2],
                                  C[0] * d[1] - C[1] * d[0] };
            const double nn = sqrt(N[0] * N[0] + N[1] * N[1] + N[2] * N[2]);
            inv8r = nn > 0.0 ? (float)(fabs(N[2]) / nn * T.g / (16.0 * T.R)) : 0.0f;
        }
        ViewRayF q;
        q.cx = cm.cxf;
        q.cy = cm.cyf;
        q.cz = cm.czf;
        q.dx = (float)d[0];
        q.dy = (float)d[1];
        q.dz = (float)d[2];
        q.alt = cm.alt;
        q.two_r_g = cm.two_r_g;
        q.zsum = cm.zsum;
        q.rise.B = (float)(2.0 * cd);
        q.rise.inv_2rho = cm.inv_2cn;
        const float stepf = (float)a.step;
        const float tv = (float)(-cd);   // closest approach to the centre
        // float32 guards: a block is skipped when its lowest ray height is above
        // the maximum height under its footprint by more than kBlockGuard (the
        // rounding of the float32 height is ~1e-2 m); a sample is ruled out
        // when it is above the bilinear terrain by more than kLeafGuard plus a
        // share of its cell's height range (position error <= 2e-3 texel), and
        // is a hit when it is below by as much; anything closer is decided in
        // FP64 (below()), as before.
        constexpr float kBlockGuard = 0.05f, kLeafGuard = 0.05f, kPosMargin = 0.01f;
        const float nxm = (float)(T.nx - 1), nym = (float)(T.ny - 1);
        if (k0 <= k1) {
            const int64_t b0 = k0 - 1, n = k1 - b0;
            int32_t kk = 0;
            while (((int64_t)1 << kk) < n) ++kk;
            int64_t s0 = 0;
            int32_t k = kk;
            while (s0 < n) {
                const int64_t ja = b0 + s0 + 1;
                const int64_t jb = min(b0 + s0 + ((int64_t)1 << k), k1);
                bool descend = false;
                if (k <= kViewLeaf) {
                    for (int64_t qj = ja; qj <= jb; ++qj) {
                        const float t = (float)qj * stepf;
                        const float rs = rise_of<false>(q.rise, t);
                        float u, v;
                        bool decide = true;   // false: certainly no hit at this sample
                        bool hit = false;     // certainly a hit (below by more than the guard)
                        if (view_image_f(T, q, t, rs, u, v)) {
                            const bool out = u < -kPosMargin || u > nxm + kPosMargin ||
                                             v < -kPosMargin || v > nym + kPosMargin;
                            const bool in = u >= kPosMargin && u <= nxm - kPosMargin &&
                                            v >= kPosMargin && v <= nym - kPosMargin;
                            if (out) {
                                decide = false;
                            } else if (in) {
                                const int32_t i0 = min((int32_t)floorf(u), T.nx - 2);
                                const int32_t j0 = min((int32_t)floorf(v), T.ny - 2);
                                const float fu = u - (float)i0, fv = v - (float)j0;
                                const float* p = T.h + (int64_t)j0 * T.pitch + i0;
                                const float h00 = __ldg(p), h10 = __ldg(p + 1);
                                const float h01 = __ldg(p + T.pitch), h11 = __ldg(p + T.pitch + 1);
                                const float top = h00 + fu * (h10 - h00);
                                const float bot = h01 + fu * (h11 - h01);
                                const float hb = top + fv * (bot - top);
                                const float rng = fmaxf(fmaxf(h00, h10), fmaxf(h01, h11)) -
                                                  fminf(fminf(h00, h10), fminf(h01, h11));
                                const float gap = (q.alt + rs) - hb, gd = kLeafGuard + 0.01f * rng;
                                decide = !(gap > gd);
                                hit = gap < -gd;
                            }
                        }
                        if (hit) {
                            hit_k = qj;
                            break;
                        }
                        if (decide) {
                            bool ins;
                            double uu, vv;
                            if (below(T, C, d, (double)qj * a.step, ins, uu, vv)) {
                                hit_k = qj;
                                break;
                            }
                        }
                    }
                    if (hit_k >= 0) break;
                } else {
                    const float ta = (float)ja * stepf, tb = (float)jb * stepf;
                    float ua, va, ub, vb;
                    if (!view_image_f(T, q, ta, rise_of<false>(q.rise, ta), ua, va) ||
                        !view_image_f(T, q, tb, rise_of<false>(q.rise, tb), ub, vb)) {
                        descend = true;
                    } else {
                        const float du = ub - ua, dv = vb - va;
                        const float e = kPosMargin + (du * du + dv * dv) * inv8r;
                        const float lo_u = fminf(ua, ub) - e, hi_u = fmaxf(ua, ub) + e;
                        const float lo_v = fminf(va, vb) - e, hi_v = fmaxf(va, vb) + e;
                        const bool misses = hi_u < 0.0f || lo_u > nxm || hi_v < 0.0f || lo_v > nym;
                        if (!misses) {
                            const int32_t x0 = max(__float2int_rd(lo_u), 0);
                            const int32_t x1 = min(__float2int_rd(hi_u) + 1, T.nx - 1);
                            const int32_t y0 = max(__float2int_rd(lo_v), 0);
                            const int32_t y1 = min(__float2int_rd(hi_v) + 1, T.ny - 1);
                            const float M = box_max(T, a.P, x0, x1, y0, y1);
                            const float tc = fminf(fmaxf(tv, ta), tb);
                            const float Hmin = q.alt + rise_of<false>(q.rise, tc);
                            descend = !(Hmin - M > kBlockGuard);
                        }
                    }
                }
                if (descend) {
                    --k;
                } else {
                    s0 += (int64_t)1 << k;
                    k = s0 == 0 ? kk : min(__ffsll(s0) - 1, kk);
                }
            }
        }
        a.hit_k[pix] = (int32_t)hit_k;
    }
}

// The crossing of F in [lo, hi] (F(lo) > 0 in the tile, F(hi) <= 0): the upper
// end of a bracket of the crossing.  The halvings of the bisection run until
// both ends lie in one bilinear cell: up to there the choices are the
// bisection's own (below_fast's arithmetic).  Inside one cell the terrain
// along the ray is a quadratic in tau (bilinear along a line; the image arc
// bends by ~1e-8 texel over a cell) and so is the ray's height (to ~1e-12 m),
// so F has exactly one root in a bracket where it changes sign: F at the
// midpoint and the quadratic through the three values place it, and one more
// value confirms a bracket [r - eps, r] or [r, r + eps] around the estimate r,
// eps = 8 x the FP64 rounding of F (2e-9 m) over the slope |F'| (at least
// 2^-36 of the step, the bisection's own bracket).  The upper end then lies
// within eps of the crossing, below 1/3 of a float32 step of texel
// coordinates >= 0.25.  Near-tangent crossings (eps above 2^-22 of the step),
// points near the tile's low edges and failed confirmations finish with
// halvings to 2^-kViewHalvings of the step, as before.
__device__ __noinline__ double refine_crossing(const Tile& T, const double C[3], const double d[3],
                                               ViewPt lo, double hi_t, double step) {
    double lo_t = lo.tau;
    ViewPt hi = view_pt(T, C, d, hi_t);
    const double tol = ldexp(step, -kViewHalvings);
    if (!(lo.in && lo.f > 0.0 && hi.in && hi.f <= 0.0)) {
        // (below()'s and below_fast's roundings disagree at an end): plain halvings
        for (int it = 0; it < kViewHalvings; ++it) {
            const double mid = lo_t + 0.5 * (hi_t - lo_t);
            if (below_fast(T, C, d, mid))
                hi_t = mid;
            else
                lo_t = mid;
        }
        return hi_t;
    }
    int it = 0;
    for (; it < kViewHalvings && !same_cell(T, lo, hi); ++it) {
        const ViewPt m = view_pt(T, C, d, lo.tau + 0.5 * (hi.tau - lo.tau));
        if (m.in && m.f <= 0.0)
            hi = m;
        else
            lo = m;
        if (!lo.in) break;   // (the ray left the tile between samples)
    }
    if (it < kViewHalvings && lo.in && same_cell(T, lo, hi)) {
        const double t0 = lo.tau, h = hi.tau - lo.tau;
        const ViewPt m = view_pt(T, C, d, t0 + 0.5 * h);
        // quadratic F(t0 + s h) = A + B s + Cq s^2 through s = 0, 1/2, 1
        const double A = lo.f, Cq = 2.0 * (lo.f + hi.f - 2.0 * m.f), B = hi.f - lo.f - Cq;
        if (m.in && same_cell(T, lo, m)) {
            if (m.f <= 0.0)
                hi = m;
            else
                lo = m;
        }
        const double l0 = (lo.tau - t0) / h, l1 = (hi.tau - t0) / h;   // bracket in s
        double s = -1.0;
        if (fabs(Cq) <= 1e-12 * fabs(B)) {
            if (B != 0.0) s = -A / B;
        } else {
            const double disc = B * B - 4.0 * A * Cq;
            if (disc >= 0.0) {
                const double q = -0.5 * (B + copysign(sqrt(disc), B));
                const double s1 = q / Cq, s2 = q != 0.0 ? A / q : -1.0;
                s = (s1 >= l0 && s1 <= l1) ? s1 : s2;
            }
        }
        const double r = t0 + s * h;
        const double slope = fabs((B + 2.0 * Cq * s) / h);
        const double eps = fmax(tol, 1.6e-8 / slope);
        const bool low_edge = fmin(lo.u, lo.v) < 0.25 || fmin(hi.u, hi.v) < 0.25;
        if (s >= l0 && s <= l1 && r > lo.tau && r <= hi.tau && slope > 0.0 &&
            eps <= ldexp(step, -22) && !low_edge) {
            const ViewPt pr = view_pt(T, C, d, r);
            if (pr.in && same_cell(T, lo, pr)) {
                if (pr.f <= 0.0) {           // crossing in (lo, r]
                    hi = pr;
                    if (r - eps <= lo.tau) return hi.tau;
                    const ViewPt pc = view_pt(T, C, d, r - eps);
                    if (pc.in && pc.f > 0.0) return hi.tau;
                    if (pc.in) hi = pc;
                } else {                     // crossing in (r, hi]
                    lo = pr;
                    if (r + eps >= hi.tau) return hi.tau;
                    const ViewPt pc = view_pt(T, C, d, r + eps);
                    if (pc.in && pc.f <= 0.0) return pc.tau;
                    if (pc.in) lo = pc;
                }
            }
        }
    }
    // halvings of whatever bracket is left, down to the bisection's resolution
    double a_t = lo.tau, b_t = hi.tau;
    for (int k = 0; k < 2 * kViewHalvings && b_t - a_t > tol; ++k) {
        const double mid = a_t + 0.5 * (b_t - a_t);
        if (below_fast(T, C, d, mid))
            b_t = mid;
        else
            a_t = mid;
    }
    return b_t;
}

// Pass 2: the hits of a block of pixels, gathered in shared memory so that
// full warps run the FP64 bisection of the crossing (a pass-1 warp has a hit in
// only some of its lanes); writes every pixel's texel coordinates (NaN without
// a hit) and the block's hit count.
__global__ void __launch_bounds__(kViewBlock) view_refine_kernel(const ViewArgs a) {
    __shared__ int32_t s_pix[kViewBlock];
    __shared__ int32_t s_cnt;
    const int64_t npix = (int64_t)a.cam.W * a.cam.H;
    const int64_t base = (int64_t)blockIdx.x * kViewBlock;
    const int64_t pix = base + threadIdx.x;
    if (threadIdx.x == 0) s_cnt = 0;
    __syncthreads();
    const bool mine = pix < npix && a.hit_k[pix] >= 0;
    if (pix < npix && !mine) a.pix_uv[pix] = make_float2(NAN, NAN);
    if (mine) s_pix[atomicAdd(&s_cnt, 1)] = threadIdx.x;
    __syncthreads();
    const int cnt = s_cnt;
    if (threadIdx.x == 0) a.block_count[blockIdx.x] = cnt;
    if ((int)threadIdx.x < cnt) {
        const Tile& T = a.T;
        const int64_t p = base + s_pix[threadIdx.x];
        const int64_t hit_k = a.hit_k[p];
        double d[3];
        pixel_dir(a.cam, p, d);
        const double* C = a.cam.C;
        double hi = (double)hit_k * a.step;
        // the sample before the hit, evaluated once: its in-tile state decides
        // whether the crossing is refined, its F starts the refinement
        if (hit_k > 1) {
            const ViewPt lo = view_pt(T, C, d, (double)(hit_k - 1) * a.step);
            if (lo.in) hi = refine_crossing(T, C, d, lo, hi, a.step);
        }
        const double xh[3] = { C[0] + hi * d[0], C[1] + hi * d[1], C[2] + hi * d[2] };
        double hu, hv;
        // the point lies between two samples of the tile: it has an image
        texel_image64(T, xh, hu, hv);
        a.pix_uv[p] = make_float2((float)hu, (float)hv);
    }
}

// exclusive prefix of the per-block counts (one block of 1024 threads)
__global__ void __launch_bounds__(1024) view_scan_kernel(const ViewArgs a) {
    __shared__ int64_t part[1024];
    const int t = threadIdx.x;
    const int per = (a.n_blocks + 1023) / 1024;
    const int lo = min(t * per, a.n_blocks), hi = min(lo + per, a.n_blocks);
    int64_t s = 0;
    for (int b = lo; b < hi; ++b) s += a.block_count[b];
    part[t] = s;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {   // inclusive Hillis-Steele scan
        const int64_t v = t >= o ? part[t - o] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    int64_t run = t > 0 ? part[t - 1] : 0;
    for (int b = lo; b < hi; ++b) {
        a.block_off[b] = run;
        run += a.block_count[b];
    }
    if (t == 1023) *a.count_out = part[1023];
}

// scatter the hits of each block to their place in pixel order
__global__ void __launch_bounds__(kViewBlock) view_compact_kernel(const ViewArgs a) {
    __shared__ int32_t warp_base[kViewBlock / 32];
    const int64_t npix = (int64_t)a.cam.W * a.cam.H;
    const int64_t pix = (int64_t)blockIdx.x * kViewBlock + threadIdx.x;
    float2 uv = make_float2(NAN, NAN);
    if (pix < npix) uv = a.pix_uv[pix];
    const bool hit = !isnan(uv.x);
    const unsigned m = __ballot_sync(0xffffffffu, hit);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) warp_base[w] = __popc(m);
    __syncthreads();
    if (threadIdx.x == 0) {
        int32_t s = 0;
        for (int k = 0; k < kViewBlock / 32; ++k) {
            const int32_t c = warp_base[k];
            warp_base[k] = s;
            s += c;
        }
    }
    __syncthreads();
    if (hit) {
        const int64_t o = a.block_off[blockIdx.x] + warp_base[w] +
                          __popc(m & ((1u << lane) - 1u));
        a.uv_out[2 * o] = uv.x;
        a.uv_out[2 * o + 1] = uv.y;
        if (a.pixel_out) a.pixel_out[o] = (int32_t)pix;
    }
}

}  // namespace

int64_t view_blocks(int32_t width, int32_t height) {
    return ((int64_t)width * height + kViewBlock - 1) / kViewBlock;
}

size_t view_workspace_bytes(int32_t width, int32_t height) {
    const int64_t npix = (int64_t)width * height, nb = view_blocks(width, height);
    return (size_t)(npix * 8 + nb * 4 + 256 + nb * 8 + 256 + npix * 4 + 256);
}

cudaError_t launch_view_rays(const Tile& T, const Pyramid& P, const ViewCamera& vc, double step,
                             int64_t K, const float* stats, float* uv, int32_t* pixel,
                             int64_t* count, void* workspace, cudaStream_t s) {
    ViewArgs a{};
    a.T = T;
    a.P = P;
    for (int k = 0; k < 3; ++k) {
        a.cam.C[k] = vc.pos[k];
        a.cam.f[k] = vc.forward[k];
        a.cam.r[k] = vc.right[k];
        a.cam.u[k] = vc.up[k];
    }
    a.cam.tan_x = vc.tan_x;
    a.cam.tan_y = vc.tan_y;
    a.cam.W = vc.width;
    a.cam.H = vc.height;
    a.cam.inv_w2 = 2.0 / (double)vc.width;
    a.cam.inv_h2 = 2.0 / (double)vc.height;
    a.cam.cc = vc.pos[0] * vc.pos[0] + vc.pos[1] * vc.pos[1] + vc.pos[2] * vc.pos[2];
    a.cam.cn = std::sqrt(a.cam.cc);
    a.cam.cxf = (float)vc.pos[0];
    a.cam.cyf = (float)vc.pos[1];
    a.cam.czf = (float)(vc.pos[2] - T.R);
    a.cam.alt = (float)(a.cam.cn - T.R);
    a.cam.zsum = (float)(a.cam.cn + T.R);
    a.cam.inv_2cn = (float)(0.5 / a.cam.cn);
    a.cam.two_r_g = (float)((T.proj == 0 ? 1.0 : 2.0) * T.R / T.g);
    a.step = step;
    a.inv_step = 1.0 / step;
    a.K = K;
    a.stats = stats;
    const int64_t npix = (int64_t)vc.width * vc.height, nb = view_blocks(vc.width, vc.height);
    unsigned char* ws = static_cast<unsigned char*>(workspace);
    a.pix_uv = reinterpret_cast<float2*>(ws);
    size_t off = (size_t)npix * 8;
    a.block_count = reinterpret_cast<int32_t*>(ws + off);
    off += (size_t)nb * 4;
    off = (off + 255) & ~(size_t)255;
    a.block_off = reinterpret_cast<int64_t*>(ws + off);
    off += (size_t)nb * 8;
    off = (off + 255) & ~(size_t)255;
    a.hit_k = reinterpret_cast<int32_t*>(ws + off);
    a.n_blocks = (int32_t)nb;
    a.uv_out = uv;
    a.pixel_out = pixel;
    a.count_out = count;
    view_hit_kernel<<<(unsigned)nb, kViewBlock, 0, s>>>(a);
    view_refine_kernel<<<(unsigned)nb, kViewBlock, 0, s>>>(a);
    view_scan_kernel<<<1, 1024, 0, s>>>(a);
    view_compact_kernel<<<(unsigned)nb, kViewBlock, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace ss
