// Device-side building blocks shared by the forward (descent and uniform),
// backward and batched kernels.
//
// Per ray, FP64 is used once to set up a local frame (Sec. 3.1 shadow ray
// p + t s; the gnomonic tile mapping of Sec. 3.2 / Appendix, under which the
// ray's texel image is the straight line u(t) = u_p + A t'/(1 + b t')); every
// sample is then evaluated in float32:
//
//   t_j   = j * delta
//   rise  = |p + t s| - |p| = t (2 rho sin_e + t) / (rho + sqrt(rho^2 + t (2 rho sin_e + t)))
//   c_j   = ((h_p - h_ref) + rise - bilinear(H - h_ref)(u_j, v_j)) / t_j
//
// with rho = R + h_p and h_ref a texel value next to the origin, so no float32
// quantity is ever of the size of R (|p + t s| - R in float32 at R = 1737 km
// would carry ~0.1 m of rounding).  Sample positions are formed from an exact
// integer part and a float32 fraction.  The same leaf function serves the
// descent and the uniform kernel, so both see bit-identical sample values.
#pragma once

#ifdef SS_RANGE_CHECK
#include <cstdio>
#endif
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

namespace ss {

constexpr int kMaxLevels = 18;     // 2^17 > SS_MAX_DIM
constexpr float kPosEps = 1e-3f;   // texel margin of footprint boxes
constexpr float kGuardRel = 1.9073486328125e-06f;  // 2^-19 = 32 float32 unit roundoffs

// Maximum mipmap as seen by a kernel; level 0 is the heightfield itself.
struct Pyramid {
    const float* ptr[kMaxLevels];
    int64_t pitch[kMaxLevels];
    int32_t levels;
};

// Scalar launch parameters of one (tile, sun) instance.
struct Tile {
    const float* h;
    int64_t pitch;
    int32_t nx, ny;
    int32_t proj;
    int32_t J;                 // floor(max_len / delta)
    double g, R, cx, cy;       // texel size, radius, tile centre in texel coords
    double sx, sy, sz;         // sun direction
    double delta;              // sample spacing (m)
    double inv_gR;             // 1 / (g R)
    double inv_R;              // 1 / R
    double inv_g;              // 1 / g
    double alpha;              // sun angular radius
    float delta_f;             // (float)delta
    float inv_delta_f;         // (float)(1/delta)
    float sz_f;                // (float)sz
    float alpha_f;
    float sx_f, sy_f, R_f;     // (float)sx, (float)sy, (float)R
    float g_f, cx_f, cy_f;     // (float)g, (float)cx, (float)cy (converted once, on the host)
    // float-float (hi + lo) copies for the grid-ray setup (df_* below)
    float g_hi, g_lo, R_lo, RR_hi, RR_lo, delta_hi, delta_lo, igR_hi, igR_lo;
    float Rsx_hi, Rsx_lo, Rsy_hi, Rsy_lo, sz_lo, szR_f;
    // and for the stereographic setup: sx, sy (low words), 2R/g
    float sx_lo, sy_lo, k2_hi, k2_lo;
};

struct Rays {
    int32_t mode;              // 0 grid, 1 list
    int64_t n;
    const float* uv;
    const float* lift;
    uint32_t* status;          // device status word for non-finite listed inputs, or null
};

struct Outputs {
    float* light;
    int32_t* argmin;
    float* cost;
    int32_t* counters;
    uint32_t* status;          // device status word (kDev* bits), or null
};

// Bits of the device status word (the C ABI's SS_DEV_* values).
constexpr uint32_t kDevNonfiniteHeight = 0x1u;
constexpr uint32_t kDevNonfiniteRay = 0x2u;
constexpr uint32_t kDevNonfiniteGrad = 0x4u;

// Word 2 of a maximum mipmap's stats block: the number of non-finite heights.
__device__ __forceinline__ void report_nonfinite_heights(const float* stats, uint32_t* status) {
    if (status && __float_as_uint(__ldg(stats + 2)) != 0u) atomicOr(status, kDevNonfiniteHeight);
}

// FP64 per-ray geometry (setup, final re-evaluation, backward).
struct Geom64 {
    double up, vp;             // origin texel coordinates
    double hp, href;           // origin height, reference texel height
    double rho, inv_rho;       // R + h_p and its reciprocal
    double sin_e;              // sun elevation over the radial normal at p
    double nhat[3];            // radial unit normal at p
    double Au, Av, b;          // gnomonic: u_j = u_p + Au * j/(1 + b j), same for v
    double Bu, Bv, inv_a0;     // stereographic: u_j = u_p + (Au j - Bu w)/(1 + w inv_a0),
                               //   w = rise(t_j) + t_j s_z, a0 = |p| + p_z
    double nz_cross;           // stereographic: |z of unit(p x s)| (image circle curvature)
    int32_t oi0, oj0;          // origin bilinear base texel
    double ow[4];              // origin bilinear weights (i0,j0),(i0+1,j0),(i0,j0+1),(i0+1,j0+1)
};

// float32 per-ray state of the hot loop (kept small: it lives in registers
// for the whole walk of a ray).
struct RayF {
    int32_t iu0, iv0;          // integer part of the origin position
    float u0, v0;              // origin position (exact: integer or the input float)
    float au_hi, au_lo, av_hi, av_lo;  // per-sample slope split so that j*a_hi is exact
    float au, av;              // au_hi + au_lo, av_hi + av_lo (rounded once)
    float b;                   // projective coefficient
    float B;                   // 2 rho sin_e
    float inv_2rho, inv_rho2;  // 1/(2 rho), 1/rho^2
    float X;                   // h_p - h_ref (0 in grid mode)
    float href;
    float tv;                  // distance of the lowest ray point (sin_e < 0), else -1
    float guard0;              // |X| + height span of the tile
    float gconst;              // 2^-19 (guard0 + 2 max|rise bound| over the ray)
    float pos_eps;             // footprint margin covering float32 block-end positions
    float c_sat;               // light-only mode: 1.002 alpha / cos(eps_p)
    float bu, bv;              // stereographic: texels per metre of w (see Geom64)
    float inv8r;               // stereographic: 1/(8 r) of the image circle (texels^-1)
    int32_t j_lo, j_hi;        // usable sample range (empty when j_lo > j_hi)
};

// ------------------------------------------------------------------ helpers
__device__ __forceinline__ double fetch_bilinear64(const float* __restrict__ h, int64_t pitch,
                                                   int nx, int ny, double u, double v,
                                                   int32_t* i0o, int32_t* j0o, double w[4]) {
    int32_t i0 = (int32_t)floor(u), j0 = (int32_t)floor(v);
    i0 = min(max(i0, 0), nx - 2);
    j0 = min(max(j0, 0), ny - 2);
    double fu = u - (double)i0, fv = v - (double)j0;
    const float* r0 = h + (int64_t)j0 * pitch + i0;
    double h00 = r0[0], h10 = r0[1], h01 = r0[pitch], h11 = r0[pitch + 1];
    w[0] = (1.0 - fu) * (1.0 - fv);
    w[1] = fu * (1.0 - fv);
    w[2] = (1.0 - fu) * fv;
    w[3] = fu * fv;
    *i0o = i0;
    *j0o = j0;
    return w[0] * h00 + w[1] * h10 + w[2] * h01 + w[3] * h11;
}

// Split a into hi + lo with hi carrying at most 8 significant bits, so that
// j * hi is exact in float32 for j < 2^16.
__device__ __forceinline__ void split8(double a, float& hi, float& lo) {
    float af = (float)a;
    hi = __int_as_float(__float_as_int(af) & (int)0xFFFF0000u);
    lo = (float)(a - (double)hi);
}

// Per-ray part of the float32 guard of a block bound: 2^-19 (guard0 + 2 R_max)
// with R_max >= |t (B + t)| / rho for every t in [0, t(j_hi)] (which bounds
// both |rise| and rise_bound), with 0.1% slack for its own rounding.
__device__ __forceinline__ void set_gconst(const Tile& T, RayF& r) {
    const float tm = (float)max(r.j_hi, 1) * T.delta_f;
    const float w1 = fabsf(tm * (r.B + tm));
    const float w2 = r.B < 0.0f ? 0.25f * r.B * r.B : 0.0f;
    const float rmax = fmaxf(w1, w2) * (2.0f * r.inv_2rho) * 1.001f;
    r.gconst = kGuardRel * (r.guard0 + 2.0f * rmax);
}

// Texel of grid ray r: r < nx ny <= 2^32 (the host checks pitch ny <= 2^32),
// so a 32-bit unsigned division is exact.
__device__ __forceinline__ void grid_uv(const Tile& T, int64_t r, int32_t& u, int32_t& v) {
    const uint32_t rr = (uint32_t)r, q = rr / (uint32_t)T.nx;
    v = (int32_t)q;
    u = (int32_t)(rr - q * (uint32_t)T.nx);
}

// Origin height (FP64) of ray r.
__device__ __forceinline__ void ray_origin(const Tile& T, const Rays& R, int64_t r,
                                           double& up, double& vp, double& hp, double& href,
                                           int32_t& oi0, int32_t& oj0, double ow[4]) {
    if (R.mode == 0) {
        int32_t u, v;
        grid_uv(T, r, u, v);
        up = (double)u;
        vp = (double)v;
        float hv = T.h[v * T.pitch + u];
        hp = hv;
        href = hv;
        oi0 = (int32_t)(u < T.nx - 2 ? u : T.nx - 2);
        oj0 = (int32_t)(v < T.ny - 2 ? v : T.ny - 2);
        ow[0] = ow[1] = ow[2] = ow[3] = 0.0;
        ow[(u - oi0) + 2 * (v - oj0)] = 1.0;
    } else {
        up = (double)R.uv[2 * r];
        vp = (double)R.uv[2 * r + 1];
        hp = fetch_bilinear64(T.h, T.pitch, T.nx, T.ny, up, vp, &oi0, &oj0, ow);
        href = (double)T.h[(int64_t)oj0 * T.pitch + oi0];
        if (R.lift) hp += (double)R.lift[r];
    }
}

// FP64 local frame of a ray whose origin is at texel coords (up, vp), height hp.
__device__ __forceinline__ void geom64(const Tile& T, double up, double vp, double hp,
                                       Geom64& G) {
    const double Xp = (up - T.cx) * T.g, Yp = (vp - T.cy) * T.g;
    const double m2 = Xp * Xp + Yp * Yp + T.R * T.R;
    const double im = rsqrt(m2);              // 1/|(X, Y, R)|
    const double m = m2 * im;
    G.up = up;
    G.vp = vp;
    G.hp = hp;
    G.nhat[0] = Xp * im;
    G.nhat[1] = Yp * im;
    G.nhat[2] = T.R * im;
    G.sin_e = (Xp * T.sx + Yp * T.sy + T.R * T.sz) * im;
    G.rho = T.R + hp;
    G.inv_rho = 1.0 / G.rho;
    const double f = T.delta * m * G.inv_rho; // sample index -> t' along the ray
    const double k = f * T.inv_gR;
    G.Au = k * (T.R * T.sx - T.sz * Xp);
    G.Av = k * (T.R * T.sy - T.sz * Yp);
    G.b = f * T.sz * T.inv_R;
}

// Polar stereographic tile (centred on the pole, plane z = R, projection from
// the antipode): direction n = (4RX, 4RY, 4R^2 - r^2)/(4R^2 + r^2).  A point q
// maps to X = 2R q_x/(|q| + q_z); with q = p + t s, |q| = |p| + rise(t):
//   X(t) - X_p = (t (2R s_x/a0) - w (2R p_x/a0^2)) / (1 + w/a0),
//   a0 = |p| + p_z, w = rise(t) + t s_z,
// which is free of cancellation.  The image of the ray is an arc of a circle
// of radius 2R / |z of unit(p x s)| (great circles map to circles).
__device__ __forceinline__ void geom64_stereo(const Tile& T, double up, double vp, double hp,
                                              Geom64& G) {
    const double Xp = (up - T.cx) * T.g, Yp = (vp - T.cy) * T.g;
    const double fr = 4.0 * T.R * T.R, r2 = Xp * Xp + Yp * Yp;
    const double inv_den = 1.0 / (fr + r2);
    G.up = up;
    G.vp = vp;
    G.hp = hp;
    G.nhat[0] = 4.0 * T.R * Xp * inv_den;
    G.nhat[1] = 4.0 * T.R * Yp * inv_den;
    G.nhat[2] = (fr - r2) * inv_den;
    G.sin_e = G.nhat[0] * T.sx + G.nhat[1] * T.sy + G.nhat[2] * T.sz;
    G.rho = T.R + hp;
    G.inv_rho = 1.0 / G.rho;
    // a0 = rho (1 + n_z) = rho 2 fr / (fr + r2)
    G.inv_a0 = G.inv_rho * (fr + r2) / (2.0 * fr);
    const double k = 2.0 * T.R / T.g;
    G.Au = T.delta * k * T.sx * G.inv_a0;
    G.Av = T.delta * k * T.sy * G.inv_a0;
    G.Bu = k * G.rho * G.nhat[0] * G.inv_a0 * G.inv_a0;
    G.Bv = k * G.rho * G.nhat[1] * G.inv_a0 * G.inv_a0;
    G.b = 0.0;
    const double cx = G.nhat[1] * T.sz - G.nhat[2] * T.sy;
    const double cy = G.nhat[2] * T.sx - G.nhat[0] * T.sz;
    const double cz = G.nhat[0] * T.sy - G.nhat[1] * T.sx;
    const double cn = sqrt(cx * cx + cy * cy + cz * cz);
    G.nz_cross = cn > 0.0 ? fabs(cz) / cn : 0.0;
}

// Either mapping; `stereo` is a compile-time constant in the forward kernels
// (one mapping per instance) and T.proj != 0 in the backward kernel.
__device__ __forceinline__ void geom64_any(const Tile& T, double up, double vp, double hp,
                                           Geom64& G, bool stereo) {
    if (!stereo)
        geom64(T, up, vp, hp, G);
    else
        geom64_stereo(T, up, vp, hp, G);
}

// FP64 rise |p + t s| - |p| without cancellation
__device__ __forceinline__ double rise64(const Geom64& G, double t) {
    const double w = t * (2.0 * G.rho * G.sin_e + t);
    return w / (G.rho + sqrt(G.rho * G.rho + w));
}

// FP64 texel position of the point of the ray at distance t (either mapping)
__device__ __forceinline__ void pos64(const Tile& T, const Geom64& G, double jd, double t,
                                      double& U, double& V, bool stereo) {
    if (!stereo) {
        const double tau = jd / (1.0 + G.b * jd);
        U = G.up + G.Au * tau;
        V = G.vp + G.Av * tau;
    } else {
        const double w = rise64(G, t) + t * T.sz;
        const double den = 1.0 + w * G.inv_a0;
        U = G.up + (G.Au * jd - G.Bu * w) / den;
        V = G.vp + (G.Av * jd - G.Bv * w) / den;
    }
}

__device__ __forceinline__ double cos_elev(const Geom64& G) {
    return sqrt(fmax(0.0, 1.0 - G.sin_e * G.sin_e));
}

// Sample index at which u_p + a j/(1 + b j) reaches boundary B (j = (B - u_p) /
// (a - b (B - u_p))); +inf when it never does.
__device__ __forceinline__ double cross_j(double p0, double a, double b, double B) {
    const double d = B - p0;
    const double den = a - b * d;
    return (den != 0.0 && d / den >= 0.0) ? d / den : INFINITY;
}

// Usable sample range: texel image inside [0,nx-1]x[0,ny-1], intersected with
// [1, J].  The image is a straight texel line traversed monotonically, so the
// usable samples are one run; origins inside the tile (grid mode, usual list
// mode) only need the exit, one division per axis.
__device__ __forceinline__ void sample_range(const Tile& T, const Geom64& G, int32_t& j_lo,
                                             int32_t& j_hi) {
    const double p0[2] = { G.up, G.vp }, a[2] = { G.Au, G.Av };
    const double hi[2] = { (double)(T.nx - 1), (double)(T.ny - 1) };
    const bool inside = p0[0] >= 0.0 && p0[0] <= hi[0] && p0[1] >= 0.0 && p0[1] <= hi[1];
    double jl = 0.0, jh = INFINITY;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        if (inside) {
            if (a[k] != 0.0) jh = fmin(jh, cross_j(p0[k], a[k], G.b, a[k] > 0.0 ? hi[k] : 0.0));
        } else if (a[k] == 0.0) {
            if (p0[k] < 0.0 || p0[k] > hi[k]) jh = -1.0;   // never enters
        } else {
            const double j0 = cross_j(p0[k], a[k], G.b, 0.0);
            const double j1 = cross_j(p0[k], a[k], G.b, hi[k]);
            const bool below = (a[k] > 0.0) ? (p0[k] < 0.0) : (p0[k] > hi[k]);
            const bool above = (a[k] > 0.0) ? (p0[k] > hi[k]) : (p0[k] < 0.0);
            if (above) jh = -1.0;                         // moving away from the tile
            const double enter = below ? (a[k] > 0.0 ? j0 : j1) : 0.0;
            const double leave = a[k] > 0.0 ? j1 : j0;
            jl = fmax(jl, enter);
            jh = fmin(jh, leave);
        }
    }
    if (!(jh >= jl) || jh < 1.0) {
        j_lo = 1;
        j_hi = 0;
        return;
    }
    j_lo = (int32_t)fmax(1.0, ceil(jl));
    j_hi = (int32_t)fmin((double)T.J, floor(jh));
}

// (stereographic tiles only)
// Exit sample of a ray whose origin lies in the tile (gnomonic): along each
// axis the image p0 + a j/(1 + b j) leaves [0, n-1] once.  A float32 estimate
// of the crossing is confirmed (or moved by a step or two) with the exact FP64
// test  a j <= d (1 + b j)  (a > 0; >= for a < 0; d = bound - p0), which needs
// no division.  Returns false (caller falls back to sample_range) when the
// projective denominator could vanish within the ray or the estimate is off.
__device__ __forceinline__ bool exit_fast(const Tile& T, double up, double vp, double Au,
                                          double Av, double b, int32_t& j_hi) {
    const double J = (double)T.J;
    if (!(1.0 + b * J > 0.25)) return false;   // 1 + b j > 0 on [0, J] (linear in j)
    int32_t jh = T.J;
    const double p0s[2] = { up, vp }, as[2] = { Au, Av };
    const double hi[2] = { (double)(T.nx - 1), (double)(T.ny - 1) };
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const double a = as[k];
        if (a == 0.0) continue;
        const double d = (a > 0.0 ? hi[k] : 0.0) - p0s[k];
        const float den = (float)a - (float)b * (float)d;
        const float jf = den != 0.0f ? (float)d / den : INFINITY;
        // the float estimate is within ~3e-7 jf of the crossing: when that
        // leaves no doubt about floor(jf) (or about jf >= J), it is the answer
        const float margin = 1e-6f * fabsf(jf) + 1e-3f;
        // the image reaches the bound at j = d / den >= 0 when den has the sign
        // of the slope (of d); otherwise it never does (or den is ~0): exact test
        if ((a > 0.0f ? den > 0.0f : den < 0.0f) && jf >= 0.0f) {
            if (jf >= (float)T.J + margin) {
                continue;                            // no exit before J on this axis
            }
            const float fl = floorf(jf), fr = jf - fl;
            if (fr > margin && fr < 1.0f - margin && jf < (float)T.J) {
                jh = min(jh, (int32_t)fl);
                continue;
            }
        }
        int32_t jc = !(jf < (float)T.J) ? T.J : (jf < 0.0f ? 0 : (int32_t)floorf(jf));
        // in(j): sample j's image is on the tile side of this bound
#define SS_IN(j) (a > 0.0 ? (a * (double)(j) <= d * fma(b, (double)(j), 1.0)) \
                          : (a * (double)(j) >= d * fma(b, (double)(j), 1.0)))
        int steps = 0;
        while (jc < T.J && SS_IN(jc + 1) && steps < 3) { ++jc; ++steps; }
        while (jc >= 1 && !SS_IN(jc) && steps < 3) { --jc; ++steps; }
        const bool ok = (jc == 0 || SS_IN(jc)) && (jc == T.J || !SS_IN(jc + 1));
#undef SS_IN
        if (!ok) return false;
        jh = min(jh, jc);
    }
    j_hi = jh;
    return true;
}

// ------------------------------------------------------- float-float (df)
// A value carried as an unevaluated sum hi + lo of two floats (about 48
// significant bits), built from the error-free transformations of Dekker and
// Knuth: TwoSum, and TwoProd through the fused multiply-add.  Every operation
// below is an explicitly rounded intrinsic, so the compiler can neither
// contract nor reorder it (that would break the error-free steps).  Relative
// error of add/mul ~2^-44; used where the grid-ray setup needs more than
// float32 (the per-sample slope) without the GB300's slow FP64 pipe.
struct DF {
    float hi, lo;
};

__device__ __forceinline__ DF df_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return DF{ s, e };
}

__device__ __forceinline__ DF df_fast_two_sum(float a, float b) {   // |a| >= |b|
    const float s = __fadd_rn(a, b);
    return DF{ s, __fsub_rn(b, __fsub_rn(s, a)) };
}

__device__ __forceinline__ DF df_add(DF x, DF y) {
    const DF s = df_two_sum(x.hi, y.hi);
    return df_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo)));
}

__device__ __forceinline__ DF df_neg(DF x) { return DF{ -x.hi, -x.lo }; }

__device__ __forceinline__ DF df_mul(DF x, DF y) {
    const float p = __fmul_rn(x.hi, y.hi);
    float e = __fmaf_rn(x.hi, y.hi, -p);
    e = __fmaf_rn(x.hi, y.lo, __fmaf_rn(x.lo, y.hi, e));
    return df_fast_two_sum(p, e);
}

__device__ __forceinline__ DF df_mul_f(DF x, float y) {
    const float p = __fmul_rn(x.hi, y);
    const float e = __fmaf_rn(x.lo, y, __fmaf_rn(x.hi, y, -p));
    return df_fast_two_sum(p, e);
}

// sqrt(x), x > 0: float seed and one Newton correction, r + (x - r^2) / (2 r)
__device__ __forceinline__ DF df_sqrt(DF x) {
    const float r = __fsqrt_rn(x.hi);
    const float p = __fmul_rn(r, r);
    const float pe = __fmaf_rn(r, r, -p);
    const float res = __fadd_rn(__fsub_rn(__fsub_rn(x.hi, p), pe), x.lo);
    return df_fast_two_sum(r, __fdiv_rn(res, __fmul_rn(2.0f, r)));
}

// x / y: float quotient and one correction, q + (x - q y) / y
__device__ __forceinline__ DF df_div(DF x, DF y) {
    const float q = __fdiv_rn(x.hi, y.hi);
    const DF qy = df_mul_f(y, q);
    const DF rem = df_add(x, df_neg(qy));
    return df_fast_two_sum(q, __fdiv_rn(rem.hi, y.hi));
}

__device__ __forceinline__ double df_to_double(DF x) { return (double)x.hi + (double)x.lo; }

// geom64_stereo's fields from float-float arithmetic (relative error ~1e-13
// against its ~1e-16): the divisions, the square root and the products run on
// the float32 pipes, and the FP64 values are assembled from the two words.
// (u, v): origin texel coordinates (float); hp: origin height.
__device__ __forceinline__ void geom_stereo_df(const Tile& T, float uf, float vf, DF hp,
                                               Geom64& G) {
    const DF g = { T.g_hi, T.g_lo };
    const DF Xp = df_mul(g, df_two_sum(uf, -T.cx_f));
    const DF Yp = df_mul(g, df_two_sum(vf, -T.cy_f));
    const DF fr = { 4.0f * T.RR_hi, 4.0f * T.RR_lo };   // 4 R^2 (exact scaling)
    const DF r2 = df_add(df_mul(Xp, Xp), df_mul(Yp, Yp));
    const DF den = df_add(fr, r2);
    const DF iden = df_div(DF{ 1.0f, 0.0f }, den);
    const DF R4 = { 4.0f * T.R_f, 4.0f * T.R_lo };
    const DF nx = df_mul(df_mul(R4, Xp), iden), ny = df_mul(df_mul(R4, Yp), iden);
    const DF nz = df_mul(df_add(fr, df_neg(r2)), iden);
    const DF sx = { T.sx_f, T.sx_lo }, sy = { T.sy_f, T.sy_lo }, sz = { T.sz_f, T.sz_lo };
    const DF se = df_add(df_add(df_mul(nx, sx), df_mul(ny, sy)), df_mul(nz, sz));
    const DF rho = df_add(DF{ T.R_f, T.R_lo }, hp);
    const DF irho = df_div(DF{ 1.0f, 0.0f }, rho);
    // a0 = rho (1 + n_z) = 2 fr rho / (fr + r2)
    const DF ia0 = df_div(df_mul(irho, den), DF{ 2.0f * fr.hi, 2.0f * fr.lo });
    const DF k2 = { T.k2_hi, T.k2_lo };
    const DF dk = df_mul(DF{ T.delta_hi, T.delta_lo }, k2);
    const DF kr = df_mul(df_mul(k2, rho), df_mul(ia0, ia0));
    G.up = (double)uf;
    G.vp = (double)vf;
    G.hp = df_to_double(hp);
    G.nhat[0] = df_to_double(nx);
    G.nhat[1] = df_to_double(ny);
    G.nhat[2] = df_to_double(nz);
    G.sin_e = df_to_double(se);
    G.rho = df_to_double(rho);
    G.inv_rho = df_to_double(irho);
    G.inv_a0 = df_to_double(ia0);
    G.Au = df_to_double(df_mul(df_mul(dk, sx), ia0));
    G.Av = df_to_double(df_mul(df_mul(dk, sy), ia0));
    G.Bu = df_to_double(df_mul(kr, nx));
    G.Bv = df_to_double(df_mul(kr, ny));
    G.b = 0.0;
    // |z of unit(n x s)| (image circle curvature; a float32 bound is enough)
    const float cxf = ny.hi * sz.hi - nz.hi * sy.hi, cyf = nz.hi * sx.hi - nx.hi * sz.hi;
    const float czf = nx.hi * sy.hi - ny.hi * sx.hi;
    const float cnf = sqrtf(cxf * cxf + cyf * cyf + czf * czf);
    G.nz_cross = cnf > 0.0f ? (double)(fabsf(czf) / cnf) : 0.0;
}

// Origin of listed ray r in float-float: the bilinear height at its (u, v)
// (fetch_bilinear64's cell and weights) plus its lift; href = the cell's base
// texel height.
__device__ __forceinline__ DF origin_height_df(const Tile& T, float uf, float vf, float lift,
                                               float& href) {
    int32_t i0 = (int32_t)floorf(uf), j0 = (int32_t)floorf(vf);
    i0 = min(max(i0, 0), T.nx - 2);
    j0 = min(max(j0, 0), T.ny - 2);
    const float fu = uf - (float)i0, fv = vf - (float)j0;   // exact
    const DF gu = df_two_sum(1.0f, -fu), gv = df_two_sum(1.0f, -fv);
    const float* p = T.h + (int64_t)j0 * T.pitch + i0;
    const float h00 = p[0], h10 = p[1], h01 = p[T.pitch], h11 = p[T.pitch + 1];
    DF acc = df_mul_f(df_mul(gu, gv), h00);
    acc = df_add(acc, df_mul_f(df_mul(DF{ fu, 0.0f }, gv), h10));
    acc = df_add(acc, df_mul_f(df_mul(gu, DF{ fv, 0.0f }), h01));
    acc = df_add(acc, df_mul_f(DF{ __fmul_rn(fu, fv), __fmaf_rn(fu, fv, -__fmul_rn(fu, fv)) },
                               h11));
    href = h00;
    return df_add(acc, DF{ lift, 0.0f });
}

// 1/rho^2 from 1/(2 rho) (gnomonic setup; recomputed when a parked ray is loaded)
__device__ __forceinline__ float inv_rho2_of(float inv_2rho) {
    return __fmul_rn(__fmul_rn(4.0f, inv_2rho), inv_2rho);
}

// exit_fast for a grid ray (origin (u, v) inside the tile) with float-float
// slope and projective coefficient: the same float estimate, and the same
// exact FP64 test (from the float-float values) when the estimate is in doubt.
__device__ __forceinline__ bool exit_fast_df(const Tile& T, float u, float v, DF Au, DF Av, DF b,
                                             int32_t& j_hi) {
    if (!(1.0f + b.hi * (float)T.J > 0.25f)) return false;   // 1 + b j > 0 on [0, J]
    int32_t jh = T.J;
    const float p0s[2] = { u, v };
    const DF as[2] = { Au, Av };
    const float hi[2] = { (float)(T.nx - 1), (float)(T.ny - 1) };
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const float a = as[k].hi;
        if (a == 0.0f) continue;
        const float d = (a > 0.0f ? hi[k] : 0.0f) - p0s[k];    // exact: integers
        const float den = a - b.hi * d;
        const float jf = den != 0.0f ? d / den : INFINITY;
        const float margin = 1e-6f * fabsf(jf) + 1e-3f;
        // the image reaches the bound at j = d / den >= 0 when den has the sign
        // of the slope (of d); otherwise it never does (or den is ~0): exact test
        if ((a > 0.0f ? den > 0.0f : den < 0.0f) && jf >= 0.0f) {
            if (jf >= (float)T.J + margin) continue;
            const float fl = floorf(jf), fr = jf - fl;
            if (fr > margin && fr < 1.0f - margin && jf < (float)T.J) {
                jh = min(jh, (int32_t)fl);
                continue;
            }
        }
        const double ad = df_to_double(as[k]), bd = df_to_double(b), dd = (double)d;
        int32_t jc = !(jf < (float)T.J) ? T.J : (jf < 0.0f ? 0 : (int32_t)floorf(jf));
#define SS_IN(j) (ad > 0.0 ? (ad * (double)(j) <= dd * fma(bd, (double)(j), 1.0)) \
                           : (ad * (double)(j) >= dd * fma(bd, (double)(j), 1.0)))
        int steps = 0;
        while (jc < T.J && SS_IN(jc + 1) && steps < 3) { ++jc; ++steps; }
        while (jc >= 1 && !SS_IN(jc) && steps < 3) { --jc; ++steps; }
        const bool ok = (jc == 0 || SS_IN(jc)) && (jc == T.J || !SS_IN(jc + 1));
#undef SS_IN
        if (!ok) return false;
        jh = min(jh, jc);
    }
    j_hi = jh;
    return true;
}

// Split a float-float value like split8: hi keeps 8 significant bits (j * hi
// exact for j < 2^16), lo the rest rounded once.
__device__ __forceinline__ void split8_df(DF a, float& hi, float& lo) {
    hi = __int_as_float(__float_as_int(a.hi) & (int)0xFFFF0000u);
    lo = __fadd_rn(__fsub_rn(a.hi, hi), a.lo);   // a.hi - hi is exact
}

// Setup of a grid ray (origin at texel (u, v), height h) on a gnomonic tile
// without FP64 on the common path: the per-sample slope and the projective
// coefficient in float-float (the same formulas as make_rayf_gnomonic:
// m = |(X, Y, R)|, f = delta m / (R + h), a = f (R s_xy - s_z (X, Y)) / (g R),
// b = f s_z / R), the exit sample from the float estimate; FP64 only when
// that estimate is in doubt or the exit cannot be found that way.
// The gnomonic map of a grid ray from texel (u, v) at height h in float-float:
// u_j = u + Au j/(1 + b j) (and v), as geom64 computes it in FP64.
__device__ __forceinline__ void gnomonic_grid_df(const Tile& T, float uf, float vf, float h,
                                                 DF& Au, DF& Av, DF& b) {
    const DF g = { T.g_hi, T.g_lo };
    const DF Xp = df_mul_f(g, __fsub_rn(uf, T.cx_f));   // u - cx exact (half-integers)
    const DF Yp = df_mul_f(g, __fsub_rn(vf, T.cy_f));
    const DF m2 = df_add(df_add(df_mul(Xp, Xp), df_mul(Yp, Yp)), DF{ T.RR_hi, T.RR_lo });
    const DF rho = df_add(DF{ T.R_f, T.R_lo }, DF{ h, 0.0f });
    const DF f = df_mul(DF{ T.delta_hi, T.delta_lo }, df_div(df_sqrt(m2), rho));
    const DF k = df_mul(f, DF{ T.igR_hi, T.igR_lo });
    const DF sz = { T.sz_f, T.sz_lo };
    Au = df_mul(k, df_add(DF{ T.Rsx_hi, T.Rsx_lo }, df_neg(df_mul(sz, Xp))));
    Av = df_mul(k, df_add(DF{ T.Rsy_hi, T.Rsy_lo }, df_neg(df_mul(sz, Yp))));
    b = df_mul_f(f, T.szR_f);
}

__device__ __forceinline__ void make_rayf_gnomonic_grid(const Tile& T, int32_t u, int32_t v,
                                                        float h, float span, RayF& r,
                                                        float& sin_e) {
    const float uf = (float)u, vf = (float)v;
    DF Au, Av, b;
    gnomonic_grid_df(T, uf, vf, h, Au, Av, b);
    const float Xf = (uf - T.cx_f) * T.g_f, Yf = (vf - T.cy_f) * T.g_f;
    const float imf = rsqrtf(Xf * Xf + Yf * Yf + T.R_f * T.R_f);
    const float se = (Xf * T.sx_f + Yf * T.sy_f + T.R_f * T.sz_f) * imf;
    const float rhof = T.R_f + h;
    sin_e = se;
    r.iu0 = u;
    r.iv0 = v;
    r.u0 = uf;
    r.v0 = vf;
    split8_df(Au, r.au_hi, r.au_lo);
    split8_df(Av, r.av_hi, r.av_lo);
    r.b = b.hi;
    r.B = 2.0f * rhof * se;
    r.inv_2rho = 0.5f / rhof;
    r.inv_rho2 = inv_rho2_of(r.inv_2rho);
    r.X = 0.0f;
    r.href = h;
    r.tv = se < 0.0f ? -rhof * se : -1.0f;
    r.guard0 = span;
    r.bu = r.bv = r.inv8r = 0.0f;
    r.au = __fadd_rn(r.au_hi, r.au_lo);
    r.av = __fadd_rn(r.av_hi, r.av_lo);
    r.j_lo = 1;
    if (!exit_fast_df(T, uf, vf, Au, Av, b, r.j_hi)) {
        Geom64 G;
        G.up = (double)u;
        G.vp = (double)v;
        G.Au = df_to_double(Au);
        G.Av = df_to_double(Av);
        G.b = df_to_double(b);
        sample_range(T, G, r.j_lo, r.j_hi);
    }
    const float amax = fmaxf(fabsf(r.au), fabsf(r.av));
    r.pos_eps = 1e-3f + 5e-7f * (float)(T.nx + T.ny) + 8e-7f * amax * (float)max(r.j_hi, 1);
    set_gconst(T, r);
}

// Float32 ray setup for gnomonic tiles.  FP64 only where float32 is not
// enough: the per-sample slope (a j must be good to ~1e-7 texel at j ~ 10^4)
// and the usable range; the sun elevation over p and the rise coefficients in
// float32 (their ~1e-7 errors shift all of a ray's costs together, and rays
// in the penumbra are re-evaluated in FP64 at the end).
template <bool kGrid>
__device__ __forceinline__ void make_rayf_gnomonic(const Tile& T, double up, double vp, float uf,
                                                   float vf, double hp, double href, float span,
                                                   RayF& r, float& sin_e) {
    const double Xp = (up - T.cx) * T.g, Yp = (vp - T.cy) * T.g;
    const double m2 = Xp * Xp + Yp * Yp + T.R * T.R;
    // 1/sqrt(m2) and 1/rho from float seeds and one Newton step each (relative
    // error ~1e-14, far below what the positions need; no FP64 division)
    double im = (double)rsqrtf((float)m2);
    im = im * fma(-0.5 * m2, im * im, 1.5);
    const double rho = T.R + hp;
    double ir = (double)__frcp_rn((float)rho);
    ir = ir * fma(-rho, ir, 2.0);
    const double f = T.delta * (m2 * im) * ir;
    const double k = f * T.inv_gR;
    const double Au = k * (T.R * T.sx - T.sz * Xp), Av = k * (T.R * T.sy - T.sz * Yp);
    const double b = f * T.sz * T.inv_R;
    const float Xf = (uf - T.cx_f) * T.g_f, Yf = (vf - T.cy_f) * T.g_f;
    const float imf = rsqrtf(Xf * Xf + Yf * Yf + T.R_f * T.R_f);
    const float se = (Xf * T.sx_f + Yf * T.sy_f + T.R_f * T.sz_f) * imf;
    const float rhof = T.R_f + (float)hp;
    sin_e = se;
    r.iu0 = (int32_t)floorf(uf);
    r.iv0 = (int32_t)floorf(vf);
    r.u0 = uf;
    r.v0 = vf;
    split8(Au, r.au_hi, r.au_lo);
    split8(Av, r.av_hi, r.av_lo);
    r.b = (float)b;
    r.B = 2.0f * rhof * se;
    r.inv_2rho = 0.5f / rhof;
    r.inv_rho2 = inv_rho2_of(r.inv_2rho);
    r.X = kGrid ? 0.0f : (float)(hp - href);
    r.href = (float)href;
    r.tv = se < 0.0f ? -rhof * se : -1.0f;
    r.guard0 = fabsf(r.X) + span;
    r.bu = r.bv = r.inv8r = 0.0f;
    r.au = __fadd_rn(r.au_hi, r.au_lo);
    r.av = __fadd_rn(r.av_hi, r.av_lo);
    const bool inside = up >= 0.0 && up <= (double)(T.nx - 1) && vp >= 0.0 &&
                        vp <= (double)(T.ny - 1);
    r.j_lo = 1;
    if (!(inside && exit_fast(T, up, vp, Au, Av, b, r.j_hi))) {
        Geom64 G;
        G.up = up;
        G.vp = vp;
        G.Au = Au;
        G.Av = Av;
        G.b = b;
        sample_range(T, G, r.j_lo, r.j_hi);
    }
    const float amax = fmaxf(fabsf(r.au), fabsf(r.av));
    r.pos_eps = 1e-3f + 5e-7f * (float)(T.nx + T.ny) + 8e-7f * amax * (float)max(r.j_hi, 1);
    set_gconst(T, r);
}

__device__ __forceinline__ bool inside64(const Tile& T, const Geom64& G, int32_t j) {
    double U, V;
    pos64(T, G, (double)j, (double)j * T.delta, U, V, true);
    return U >= 0.0 && U <= (double)(T.nx - 1) && V >= 0.0 && V <= (double)(T.ny - 1);
}

#ifdef SS_RANGE_CHECK
static __device__ unsigned int g_range_mismatch, g_range_reentry;
#endif

// Polar stereographic usable range: the first run of in-tile samples.  The
// ray's directions sweep a great circle (plane N . n = 0, N = p x s); the
// preimage of a tile edge X = X_B is the small circle E . n = e0 with
// E = (2R, 0, -X_B), e0 = X_B (likewise for Y).  Their intersections give the
// crossing points exactly (a quadratic), each mapped back to its ray distance
// t = -((p x n) . (s x n)) / |s x n|^2; the run is bounded by the first
// crossings, then its end samples are confirmed with the FP64 position.
// (kept out of line: its FP64 scratch would otherwise crowd the walk's registers)
static __device__ __noinline__ void sample_range_stereo(const Tile& T, const Geom64& G,
                                                    int32_t& j_lo, int32_t& j_hi) {
    const double p[3] = { G.rho * G.nhat[0], G.rho * G.nhat[1], G.rho * G.nhat[2] };
    const double sv[3] = { T.sx, T.sy, T.sz };
    const double N[3] = { p[1] * sv[2] - p[2] * sv[1], p[2] * sv[0] - p[0] * sv[2],
                          p[0] * sv[1] - p[1] * sv[0] };
    const double Xlo = (0.0 - T.cx) * T.g, Xhi = ((double)(T.nx - 1) - T.cx) * T.g;
    const double Ylo = (0.0 - T.cy) * T.g, Yhi = ((double)(T.ny - 1) - T.cy) * T.g;
    double tc[8];
    int nc = 0;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const bool xedge = e < 2;
        const double B = xedge ? (e == 0 ? Xlo : Xhi) : (e == 2 ? Ylo : Yhi);
        const double E[3] = { xedge ? 2.0 * T.R : 0.0, xedge ? 0.0 : 2.0 * T.R, -B };
        const double e0 = B;
        const double d[3] = { N[1] * E[2] - N[2] * E[1], N[2] * E[0] - N[0] * E[2],
                              N[0] * E[1] - N[1] * E[0] };
        const double dd = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        if (!(dd > 0.0)) continue;
        const double NN = N[0] * N[0] + N[1] * N[1] + N[2] * N[2];
        const double NE = N[0] * E[0] + N[1] * E[1] + N[2] * E[2];
        double x0[3];
        for (int i = 0; i < 3; ++i) x0[i] = e0 * (NN * E[i] - NE * N[i]) / dd;
        const double bq = x0[0] * d[0] + x0[1] * d[1] + x0[2] * d[2];
        const double cq = x0[0] * x0[0] + x0[1] * x0[1] + x0[2] * x0[2] - 1.0;
        const double disc = bq * bq - dd * cq;
        if (!(disc >= 0.0)) continue;
        const double sq = sqrt(disc);
        for (int k = 0; k < 2; ++k) {
            const double lam = (-bq + (k ? sq : -sq)) / dd;
            const double n[3] = { x0[0] + lam * d[0], x0[1] + lam * d[1], x0[2] + lam * d[2] };
            if (!(1.0 + n[2] > 0.0)) continue;
            const double other = 2.0 * T.R * (xedge ? n[1] : n[0]) / (1.0 + n[2]);
            const double olo = xedge ? Ylo : Xlo, ohi = xedge ? Yhi : Xhi;
            if (other < olo || other > ohi) continue;
            const double pn[3] = { p[1] * n[2] - p[2] * n[1], p[2] * n[0] - p[0] * n[2],
                                   p[0] * n[1] - p[1] * n[0] };
            const double sn[3] = { sv[1] * n[2] - sv[2] * n[1], sv[2] * n[0] - sv[0] * n[2],
                                   sv[0] * n[1] - sv[1] * n[0] };
            const double s2 = sn[0] * sn[0] + sn[1] * sn[1] + sn[2] * sn[2];
            if (!(s2 > 0.0)) continue;
            const double t = -(pn[0] * sn[0] + pn[1] * sn[1] + pn[2] * sn[2]) / s2;
            const double lam2 = (p[0] + t * sv[0]) * n[0] + (p[1] + t * sv[1]) * n[1] +
                                (p[2] + t * sv[2]) * n[2];
            if (t > 0.0 && lam2 > 0.0 && nc < 8) tc[nc++] = t;
        }
    }
    // sort the crossing distances (at most 8)
    for (int i = 1; i < nc; ++i)
        for (int k = i; k > 0 && tc[k] < tc[k - 1]; --k) {
            const double tmp = tc[k];
            tc[k] = tc[k - 1];
            tc[k - 1] = tmp;
        }
    // Between consecutive crossings the in/out status is constant (tested at the
    // interval's midpoint).  The run starts in the first inside interval that
    // holds a sample and extends over later inside intervals until an outside
    // interval that holds a sample (an excursion between two samples does not
    // split the run: both samples are in the tile).
    const double tmax = (double)T.J * T.delta;
    int32_t run_lo = -1, run_hi = -1;
#ifdef SS_RANGE_CHECK
    bool run_ended = false;
#endif
    double lo_t = 0.0;
    for (int i = 0; i <= nc; ++i) {
        const double hi_t = i < nc ? fmin(tc[i], tmax) : tmax;
        if (hi_t > lo_t) {
            const int32_t lo = (int32_t)fmax(1.0, ceil(lo_t / T.delta));
            const int32_t hi = (int32_t)fmin((double)T.J, floor(hi_t / T.delta));
            const double tm = 0.5 * (lo_t + hi_t);
            double U, V;
            pos64(T, G, tm / T.delta, tm, U, V, true);
            const bool in = U >= 0.0 && U <= (double)(T.nx - 1) && V >= 0.0 &&
                            V <= (double)(T.ny - 1);
            if (lo <= hi) {
                if (in) {
#ifdef SS_RANGE_CHECK
                    if (run_ended) {   // test builds: samples in the tile after the run
                        const unsigned k = atomicAdd(&g_range_reentry, 1u);
                        if (k < 8u || (k & (k - 1u)) == 0u)
                            printf("re-entry %u up=%.9g vp=%.9g run [%d,%d] again at %d\n", k + 1u,
                                   G.up, G.vp, run_lo, run_hi, lo);
                        break;
                    }
#endif
                    if (run_lo < 0) run_lo = lo;
                    run_hi = hi;
                } else if (run_lo >= 0) {
#ifdef SS_RANGE_CHECK
                    run_ended = true;   // (test builds look on for a re-entry)
#else
                    break;
#endif
                }
            }
        }
        if (hi_t >= tmax) break;
        lo_t = hi_t;
    }
    if (run_lo < 0) {
        j_lo = 1;
        j_hi = 0;
        return;
    }
    // confirm the ends with the FP64 positions (a crossing within rounding of a sample)
    int32_t lo = run_lo, hi = run_hi;
    if (!inside64(T, G, lo) && lo < hi) ++lo;
    if (lo > 1 && inside64(T, G, lo - 1)) --lo;
    if (!inside64(T, G, hi) && hi > lo) --hi;
    if (hi < T.J && inside64(T, G, hi + 1)) ++hi;
    if (!inside64(T, G, lo)) {
        j_lo = 1;
        j_hi = 0;
        return;
    }
    j_lo = lo;
    j_hi = hi;
}


static __device__ __noinline__ bool sample_range_stereo_f32(const Tile& T, const Geom64& G,
                                                         const RayF& r, int32_t& j_lo,
                                                         int32_t& j_hi);

template <bool kStereo>
__device__ __forceinline__ void make_rayf(const Tile& T, const Geom64& G, double href,
                                          float span, RayF& r) {
    double iu = floor(G.up), iv = floor(G.vp);
    r.iu0 = (int32_t)iu;
    r.iv0 = (int32_t)iv;
    r.u0 = (float)G.up;
    r.v0 = (float)G.vp;
    split8(G.Au, r.au_hi, r.au_lo);
    split8(G.Av, r.av_hi, r.av_lo);
    r.b = (float)G.b;
    r.B = (float)(2.0 * G.rho * G.sin_e);
    r.inv_2rho = (float)(0.5 * G.inv_rho);
    r.inv_rho2 = (float)(G.inv_rho * G.inv_rho);
    r.X = (float)(G.hp - href);
    r.href = (float)href;
    r.tv = G.sin_e < 0.0 ? (float)(-G.rho * G.sin_e) : -1.0f;
    r.guard0 = fabsf(r.X) + span;
    if (!kStereo) {
        sample_range(T, G, r.j_lo, r.j_hi);
        r.bu = r.bv = r.inv8r = 0.0f;
    } else {
        r.b = (float)G.inv_a0;
        r.bu = (float)G.Bu;
        r.bv = (float)G.Bv;
        r.inv8r = (float)(G.nz_cross * T.g / (16.0 * T.R));
        r.au = __fadd_rn(r.au_hi, r.au_lo);
        r.av = __fadd_rn(r.av_hi, r.av_lo);
        if (!sample_range_stereo_f32(T, G, r, r.j_lo, r.j_hi))
            sample_range_stereo(T, G, r.j_lo, r.j_hi);
#ifdef SS_RANGE_CHECK
        {   // test builds: the float32 search against the FP64 one
            int32_t a = 1, b = 0;
            sample_range_stereo(T, G, a, b);
            if ((a <= b || r.j_lo <= r.j_hi) && (a != r.j_lo || b != r.j_hi) &&
                atomicAdd(&g_range_mismatch, 1u) < 8u)
                printf("range mismatch up=%.9g vp=%.9g f32 [%d,%d] fp64 [%d,%d]\n", G.up, G.vp,
                       r.j_lo, r.j_hi, a, b);
        }
#endif
    }
    r.au = __fadd_rn(r.au_hi, r.au_lo);
    r.av = __fadd_rn(r.av_hi, r.av_lo);
    // float32 block-end positions u0 + a*tau err by <= ulp(coordinate) plus
    // ~3 ulp of a*tau; the margin takes 4x that, plus 1e-3 texel
    float amax = fmaxf(fabsf((float)G.Au), fabsf((float)G.Av));
    r.pos_eps = 1e-3f + 5e-7f * (float)(T.nx + T.ny) + 8e-7f * amax * (float)max(r.j_hi, 1);
    if (kStereo) {
        // the stereographic end positions also carry w * B with |w| <= 2 t
        const float bmax = fmaxf(fabsf(r.bu), fabsf(r.bv));
        r.pos_eps += 8e-7f * bmax * 2.0f * (float)((double)max(r.j_hi, 1) * T.delta);
    }
    set_gconst(T, r);
}

// ------------------------------------------------------------ float32 leaf
// Every operation that produces a sample value is an explicitly rounded
// intrinsic (__fadd_rn, __fmul_rn, __fmaf_rn, ...), which the compiler never
// contracts or reorders: the value is the same bits in every kernel and
// inlining context that evaluates it.  Template flags only remove operations
// that are exact no-ops for the specialised case (x + 0, grid origins).
//   kGrid: rays start at texel centres (fractional origin 0, X = 0).
//   kPoly: the rise series converges for every ray of the launch.
struct Pos {
    int32_t i;
    float f;
};

__device__ __forceinline__ float corr_of(const RayF& r, float jf) {
    float jb = __fmul_rn(jf, r.b);
    return __fdividef(__fmul_rn(jf, jb), __fadd_rn(1.0f, jb));   // j - j/(1 + b j)
}

// Texel coordinate of sample j along one axis: integer part exact, fraction
// accurate to ~1e-7 texel.  The offset from the origin is j*a (a = a_hi + a_lo,
// j*a_hi exact) minus a small correction that carries the curvature of the
// mapping: a * corr (gnomonic, corr = j - j/(1 + b j)) or corr itself
// (stereographic, in texels).  Base clamped to [0, n-2] (the fraction absorbs it).
template <bool kGrid, bool kStereo>
__device__ __forceinline__ Pos axis_pos(int32_t i0, float u0, float a_hi, float a_lo, float a,
                                        float corr, float jf, int32_t n) {
    float p = __fmul_rn(jf, a_hi);       // exact: a_hi has <= 8 significant bits
    float kp = floorf(p);
    float fp = __fsub_rn(p, kp);         // exact
    float tail = kStereo ? __fmaf_rn(jf, a_lo, -corr)
                         : __fmaf_rn(jf, a_lo, -__fmul_rn(a, corr));
    float s = kGrid ? __fadd_rn(fp, tail)
                    : __fadd_rn(__fadd_rn(__fsub_rn(u0, (float)i0), fp), tail);
    float fs = floorf(s);
    int32_t i = i0 + __float2int_rz(kp) + __float2int_rz(fs);
    float f = __fsub_rn(s, fs);
    int32_t ic = min(max(i, 0), n - 2);
    f = __fadd_rn(f, (float)(i - ic));
    Pos P;
    P.i = ic;
    P.f = f;
    return P;
}

__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// rise(t) = |p + t s| - |p| = w / (rho + sqrt(rho^2 + w)), w = t (2 rho sin_e + t),
// without cancellation.  With x = w / rho^2 this is (w / 2 rho) * 2/(1 + sqrt(1 + x))
// = (w / 2 rho) (1 - x/4 + x^2/8 - 5x^3/64 + 7x^4/128 - ...); the host selects
// the series (kPoly) only when |x| <= 1/32 for every ray (truncation < 1e-9
// relative), else the closed form is used.
template <bool kPoly>
__device__ __forceinline__ float rise_of(const RayF& r, float t) {
    float w = __fmul_rn(t, __fadd_rn(r.B, t));
    if (!kPoly) {
        float rho = __fdiv_rn(0.5f, r.inv_2rho);
        return __fdiv_rn(w, __fadd_rn(rho, __fsqrt_rn(__fmaf_rn(rho, rho, w))));
    }
    float x = __fmul_rn(w, r.inv_rho2);
    float p = __fmaf_rn(x, 0.0546875f, -0.078125f);
    p = __fmaf_rn(x, p, 0.125f);
    p = __fmaf_rn(x, p, -0.25f);
    p = __fmaf_rn(x, p, 1.0f);
    return __fmul_rn(__fmul_rn(w, r.inv_2rho), p);
}

// upper bound of |rise(t)| without a square root: |w| / rho
__device__ __forceinline__ float rise_bound(const RayF& r, float t) {
    return fabsf(t * (r.B + t)) * (2.0f * r.inv_2rho);
}

__device__ __forceinline__ float bilerp_rn(float d00, float d10, float d01, float d11, float fu,
                                           float fv) {
    float top = __fmaf_rn(fu, __fsub_rn(d10, d00), d00);
    float bot = __fmaf_rn(fu, __fsub_rn(d11, d01), d01);
    return __fmaf_rn(fv, __fsub_rn(bot, top), top);
}

// Corrections of sample j's offset along u and v (see axis_pos):
//   gnomonic:      j - j/(1 + b j) for both axes (axis_pos scales it by a)
//   stereographic: w (B + j a / a0) / (1 + w / a0) texels, w = rise(t_j) + t_j s_z
template <bool kStereo>
__device__ __forceinline__ void axis_corr(const Tile& T, const RayF& r, float jf, float t,
                                          float rise, float& cu, float& cv) {
    if (!kStereo) {
        cu = cv = corr_of(r, jf);
    } else {
        const float au = r.au, av = r.av;
        const float w = __fadd_rn(rise, __fmul_rn(t, T.sz_f));
        const float q = __fdividef(w, __fmaf_rn(w, r.b, 1.0f));   // r.b = 1/a0
        cu = __fmul_rn(q, __fmaf_rn(__fmul_rn(jf, au), r.b, r.bu));
        cv = __fmul_rn(q, __fmaf_rn(__fmul_rn(jf, av), r.b, r.bv));
    }
}

// 1/t_j: delta^-1 times the hardware reciprocal of j (deterministic, <= 2 ulp)
__device__ __forceinline__ float inv_t(const Tile& T, float jf) {
    return __fmul_rn(T.inv_delta_f, rcp_approx(jf));
}

// Element offsets stay below 2^32 (the host checks pitch * ny <= 2^32).
__device__ __forceinline__ const float* cell_ptr(const float* base, uint32_t pitch, int32_t x,
                                                 int32_t y) {
    return base + ((uint32_t)y * pitch + (uint32_t)x);
}

// Cost of sample j (float32); the uniform kernel's sample value.  probe() with
// leaf == true returns the same bits.
template <bool kGrid, bool kPoly, bool kStereo>
__device__ __forceinline__ float leaf_cost(const Tile& T, const RayF& r, int32_t j,
                                           float& rise) {
    const float jf = (float)j;
    const float t = __fmul_rn(jf, T.delta_f);
    const float rise_s = kStereo ? rise_of<kPoly>(r, t) : 0.0f;
    float cu, cv;
    axis_corr<kStereo>(T, r, jf, t, rise_s, cu, cv);
    const Pos pu = axis_pos<kGrid, kStereo>(r.iu0, r.u0, r.au_hi, r.au_lo, r.au, cu, jf, T.nx);
    const Pos pv = axis_pos<kGrid, kStereo>(r.iv0, r.v0, r.av_hi, r.av_lo, r.av, cv, jf, T.ny);
    const uint32_t pitch = (uint32_t)T.pitch;
    const float* p = cell_ptr(T.h, pitch, pu.i, pv.i);
    const float d00 = __fsub_rn(__ldg(p), r.href), d10 = __fsub_rn(__ldg(p + 1), r.href);
    const float d01 = __fsub_rn(__ldg(p + pitch), r.href);
    const float d11 = __fsub_rn(__ldg(p + pitch + 1), r.href);
    rise = kStereo ? rise_s : rise_of<kPoly>(r, t);
    const float hb = bilerp_rn(d00, d10, d01, d11, pu.f, pv.f);
    const float h = kGrid ? rise : __fadd_rn(r.X, rise);
    return __fmul_rn(__fsub_rn(h, hb), inv_t(T, jf));
}

// float32 texel position of sample j for block footprints (error <= pos_eps);
// rise = rise(t_j) (used by the stereographic mapping only)
template <bool kStereo>
__device__ __forceinline__ void block_end(const Tile& T, const RayF& r, float jf, float t,
                                          float rise, float& u, float& v) {
    const float au = r.au, av = r.av;
    if (!kStereo) {
        float tau = __fdividef(jf, __fmaf_rn(jf, r.b, 1.0f));
        u = __fmaf_rn(au, tau, r.u0);
        v = __fmaf_rn(av, tau, r.v0);
    } else {
        const float w = __fadd_rn(rise, __fmul_rn(t, T.sz_f));
        const float id = __fdividef(1.0f, __fmaf_rn(w, r.b, 1.0f));
        u = __fmaf_rn(__fmaf_rn(jf, au, -__fmul_rn(w, r.bu)), id, r.u0);
        v = __fmaf_rn(__fmaf_rn(jf, av, -__fmul_rn(w, r.bv)), id, r.v0);
    }
}

// ------------------------------------------- stereographic range, float32
// The first run of in-tile samples (what sample_range_stereo finds with FP64
// crossings) from float32 positions, certified so that the result is the same:
//  * a sample whose float32 position (block_end, exact-formula rise) is more
//    than E inside every edge is inside, more than E outside an edge is
//    outside; E is the walk's footprint margin taken at j = J (a bound of the
//    float32 position error over the whole ray) plus the rounding of the
//    margin itself;
//  * the ray's image is a circle arc of radius rc = 1/(8 inv8r) texels, and the
//    samples between two samples lie on the arc between them, within
//    L^2/(4 rc) of its chord (length L, L < rc); the chord is as far inside
//    the tile as its nearer end, so when both ends are inside by more than
//    E + L^2/(4 rc) every sample between them is inside (certified).
// A bisection keeps jl, the last sample known to continue the run from sample
// 1, and jh, a sample the certificate does not reach from jl; at jh = jl + 1
// sample jh is classified alone (FP64 when within E of an edge): outside ends
// the run, inside starts another pass from it.  Returns false (the caller
// runs the FP64 search) when sample 1 is not inside or after kRangePasses
// passes (rays that run along an edge).
constexpr int kRangePasses = 4;

struct RangePt {
    float u, v, m;   // float32 position, distance inside the nearest edge
};

__device__ __forceinline__ RangePt range_pt(const Tile& T, const RayF& r, int32_t j) {
    RangePt p;
    const float jf = (float)j;
    const float t = __fmul_rn(jf, T.delta_f);
    block_end<true>(T, r, jf, t, rise_of<false>(r, t), p.u, p.v);
    p.m = fminf(fminf(p.u, (float)(T.nx - 1) - p.u), fminf(p.v, (float)(T.ny - 1) - p.v));
    return p;
}

__device__ __forceinline__ bool range_cert(const RayF& r, const RangePt& a, const RangePt& b,
                                           float E) {
    const float du = b.u - a.u, dv = b.v - a.v;
    const float L = sqrtf(du * du + dv * dv) + 3.0f * E;   // exact chord length bound
    if (L * r.inv8r >= 0.125f) return false;               // chord not shorter than rc
    const float sag = 2.02f * r.inv8r * L * L;             // L^2 / (4 rc), 1% margin
    return fminf(a.m, b.m) - sag > E;
}

static __device__ __noinline__ bool sample_range_stereo_f32(const Tile& T, const Geom64& G,
                                                         const RayF& r, int32_t& j_lo,
                                                         int32_t& j_hi) {
    const int32_t J = T.J;
    if (J < 1) return false;
    const float amax = fmaxf(fabsf(r.au), fabsf(r.av)), bmax = fmaxf(fabsf(r.bu), fabsf(r.bv));
    const float E = 2e-3f + 5e-7f * (float)(T.nx + T.ny) + 8e-7f * amax * (float)J +
                    8e-7f * bmax * 2.0f * ((float)J * T.delta_f);
    RangePt pl = range_pt(T, r, 1);
    if (!(pl.m > E) && (pl.m < -E || !inside64(T, G, 1))) return false;
    int32_t jl = 1;
    for (int pass = 0; pass < kRangePasses; ++pass) {
        if (jl == J) break;
        int32_t jh = J;
        RangePt ph = range_pt(T, r, J);
        if (range_cert(r, pl, ph, E)) {
            jl = J;
            break;
        }
        while (jh - jl > 1) {
            const int32_t jm = jl + ((jh - jl) >> 1);
            const RangePt pm = range_pt(T, r, jm);
            if (range_cert(r, pl, pm, E)) {
                jl = jm;
                pl = pm;
            } else {
                jh = jm;
                ph = pm;
            }
        }
        const bool in = ph.m > E ? true : ph.m < -E ? false : inside64(T, G, jh);
        if (!in) {
            j_lo = 1;
            j_hi = jl;
            return true;
        }
        jl = jh;
        pl = ph;
    }
    if (jl != J) return false;
    j_lo = 1;
    j_hi = J;
    return true;
}

// Levels of the maximum mipmap as a kernel sees them (shared memory copy).
struct LevelTab {
    const float* ptr[kMaxLevels];
    uint32_t pitch[kMaxLevels];
};

// One probe of the descent, a single code path for both kinds so that a warp
// whose lanes mix them stays converged:
//  * leaf: the cost of sample ja, bit-identical to leaf_cost();
//  * block [ja, jb]: a lower bound of every leaf cost in it, through the
//    maximum mipmap (Eq. optimumk2: the clearance over an interval is at least
//    the ray's lowest height there minus the maximum terrain height below it).
//    M = max over the 2x2 cells, at the coarsest level whose cells cover the
//    texel footprint box of the block's samples (the float32 end positions
//    widened by pos_eps); the guard 2^-19 (|X| + |rise| + |M - h_ref| + span)
//    covers every float32 rounding of the leaf and of the bound, so no sample
//    that could win is skipped.
template <bool kGrid, bool kPoly, bool kStereo>
__device__ __forceinline__ float probe(const Tile& T, const LevelTab& L, int32_t levels,
                                       const RayF& r, int32_t ja, int32_t jb, bool leaf) {
    const float fa = (float)ja, fb = (float)jb;
    // stereographic positions need the rise at both ends first
    const float sa = kStereo ? __fmul_rn(fa, T.delta_f) : 0.0f;
    const float sb = kStereo ? __fmul_rn(fb, T.delta_f) : 0.0f;
    const float rise_a = kStereo ? rise_of<kPoly>(r, sa) : 0.0f;
    // leaf position (the sample's bilinear cell)
    float cu, cv;
    axis_corr<kStereo>(T, r, fa, sa, rise_a, cu, cv);
    const Pos ua = axis_pos<kGrid, kStereo>(r.iu0, r.u0, r.au_hi, r.au_lo, r.au, cu, fa, T.nx);
    const Pos va = axis_pos<kGrid, kStereo>(r.iv0, r.v0, r.av_hi, r.av_lo, r.av, cv, fa, T.ny);
    // block footprint box from both ends (stereographic: plus the arc's sagitta);
    // the near end is the leaf position (i + f, more accurate than block_end)
    const float xa = __fadd_rn((float)ua.i, ua.f), ya = __fadd_rn((float)va.i, va.f);
    float xb, yb;
    block_end<kStereo>(T, r, fb, sb, kStereo ? rise_of<kPoly>(r, sb) : 0.0f, xb, yb);
    float e = r.pos_eps;
    if (kStereo) {
        const float dx = xb - xa, dy = yb - ya;
        e += (dx * dx + dy * dy) * r.inv8r;
    }
    // clamped before the +1, so no conversion result can overflow
    int32_t x0 = max(__float2int_rd(fminf(xa, xb) - e), 0);
    int32_t x1 = min(__float2int_rd(fmaxf(xa, xb) + e), T.nx - 2) + 1;
    int32_t y0 = max(__float2int_rd(fminf(ya, yb) - e), 0);
    int32_t y1 = min(__float2int_rd(fmaxf(ya, yb) + e), T.ny - 2) + 1;
    const int32_t ext = max(x1 - x0, y1 - y0);
    int32_t m = ext <= 1 ? 0 : 31 - __clz(ext);
    m += (((x1 >> m) - (x0 >> m)) > 1 || ((y1 >> m) - (y0 >> m)) > 1) ? 1 : 0;
    m = min(m, levels - 1);
    m = leaf ? 0 : m;
    x0 = leaf ? ua.i : x0;
    y0 = leaf ? va.i : y0;
    x1 = leaf ? ua.i + 1 : x1;
    y1 = leaf ? va.i + 1 : y1;
    const uint32_t pm = L.pitch[m];
    const float* p = cell_ptr(L.ptr[m], pm, x0 >> m, y0 >> m);
    const uint32_t dx = (uint32_t)((x1 >> m) - (x0 >> m));
    const uint32_t dy = (uint32_t)((y1 >> m) - (y0 >> m)) * pm;
    const float d00 = __fsub_rn(__ldg(p), r.href);
    const float d10 = __fsub_rn(__ldg(p + dx), r.href);
    const float d01 = __fsub_rn(__ldg(p + dy), r.href);
    const float d11 = __fsub_rn(__ldg(p + dy + dx), r.href);
    const float ta = __fmul_rn(fa, T.delta_f), tb = __fmul_rn(fb, T.delta_f);
    const float tstar = (leaf || !(r.tv > ta)) ? ta : fminf(r.tv, tb);
    const float rise = rise_of<kPoly>(r, tstar);             // = rise(ta) for a leaf
    const float V = leaf ? bilerp_rn(d00, d10, d01, d11, ua.f, va.f)
                         : fmaxf(fmaxf(d00, d10), fmaxf(d01, d11));
    const float h = kGrid ? rise : __fadd_rn(r.X, rise);
    const float num0 = __fsub_rn(h, V);
    // |rise| and rise_bound(tb) are both below the ray's largest rise bound
    const float guard = fmaf(kGuardRel, fabsf(V), r.gconst);
    const float num = leaf ? num0 : __fsub_rn(num0, guard);
    const float den_j = (leaf || !(num >= 0.0f)) ? fa : fb;
    return __fmul_rn(num, inv_t(T, den_j));
}

// ------------------------------------------------------ FP64 re-evaluation
__device__ __forceinline__ double leaf_cost64(const Tile& T, const Geom64& G, int32_t j,
                                              bool stereo, double* U = nullptr,
                                              double* V = nullptr) {
    const double jd = (double)j;
    const double t = jd * T.delta;
    double u, v;
    pos64(T, G, jd, t, u, v, stereo);
    if (U) *U = u;
    if (V) *V = v;
    int32_t i0, j0;
    double w[4];
    const double hb = fetch_bilinear64(T.h, T.pitch, T.nx, T.ny, u, v, &i0, &j0, w);
    return ((G.hp - hb) + rise64(G, t)) / t;
}

// ------------------------------------------------ FP64 mapping helpers
// unit direction of texel coordinates (u, v) under the tile's mapping
__device__ __forceinline__ void texel_dir64(const Tile& T, double u, double v, double n[3]) {
    const double X = (u - T.cx) * T.g, Y = (v - T.cy) * T.g;
    if (T.proj == 0) {
        const double im = rsqrt(X * X + Y * Y + T.R * T.R);
        n[0] = X * im;
        n[1] = Y * im;
        n[2] = T.R * im;
    } else {
        const double fr = 4.0 * T.R * T.R, r2 = X * X + Y * Y, id = 1.0 / (fr + r2);
        n[0] = 4.0 * T.R * X * id;
        n[1] = 4.0 * T.R * Y * id;
        n[2] = (fr - r2) * id;
    }
}

// texel image of the direction of point x; false without an image (gnomonic:
// not in front of the plane; stereographic: the antipode)
__device__ __forceinline__ bool texel_image64(const Tile& T, const double x[3], double& u,
                                              double& v) {
    double X, Y;
    if (T.proj == 0) {
        if (!(x[2] > 0.0)) return false;
        const double k = T.R / x[2];
        X = x[0] * k;
        Y = x[1] * k;
    } else {
        const double m = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
        const double den = m + x[2];
        if (!(den > 0.0)) return false;
        const double k = 2.0 * T.R / den;
        X = x[0] * k;
        Y = x[1] * k;
    }
    u = X / T.g + T.cx;
    v = Y / T.g + T.cy;
    return true;
}

__device__ __forceinline__ bool in_tile64(const Tile& T, double u, double v) {
    return u >= 0.0 && u <= (double)(T.nx - 1) && v >= 0.0 && v <= (double)(T.ny - 1);
}

__device__ __forceinline__ float disc_light32(float d) {
    if (!(d > -1.0f)) return 0.0f;
    if (!(d < 1.0f)) return 1.0f;
    return (3.14159265358979f - acosf(d) + d * sqrtf(1.0f - d * d)) * 0.318309886183791f;
}

__device__ __forceinline__ double disc_light64(double d) {
    if (d <= -1.0) return 0.0;
    if (d >= 1.0) return 1.0;
    return (M_PI - acos(d) + d * sqrt(1.0 - d * d)) / M_PI;
}

}  // namespace ss
