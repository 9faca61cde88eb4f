/*
 * FP64 restatement of the paper's greedy descent (Algorithm 1, "Fast Soft
 * Shadow Algorithm", with the ray length T of Eq. maxstep and the interval
 * concatenation of Sec. 3.3 "Long shadows").
 *
 * TEST INFRASTRUCTURE ONLY (same rules as shadow_oracle.c).
 *
 * This is the paper's approximate method, reproduced to measure its error
 * against the exact minimum; it is not the exact descent.  Steps per ray, in
 * the paper's order and notation (readings of the parts the paper leaves open
 * are marked R-n):
 *   origin p (as in shadow_oracle.c), sun direction s, runs r = 0, 1, ... with
 *   N'_r levels each; run r starts at distance a_r along the ray (a_0 = 0,
 *   a_{r+1} = a_r + T_r).
 *   T_r (Eq. maxstep): with R = p + a_r s, E = the texel image of R moved by
 *     2^(N'_r - 1) texels along the unit texture-plane direction of (s_x, s_y),
 *     e = the direction of E on the sphere (R-1: texel units and the tile's own
 *     mapping stand for the paper's normalised texture plane), T_r is the
 *     parameter of R + T s closest to the line through the centre along e:
 *     T = ((-R x e) . (s x e)) / |s x e|^2.
 *   Normalised parameter t in [0, 1] over [a_r, a_r + T_r]; t_0 = 1;
 *   for k = 0 .. N'-1, mip level m = N'-1-k:
 *     Delta* = +inf (R-2: heights in metres, so "1" becomes +inf), t* = -1;
 *     the ray tip at t_k, t_k - 2^-(k+1), t_k - 2^-k (the DDA steps, in that
 *     order) is sampled: H = |q| - R, M = the level-m maximum-mipmap texel that
 *     contains the tip's texel image (R-3: point sampling, level-m texel
 *     I = floor((u + 0.5) / 2^m)); Delta = H - M; strict < keeps the first;
 *     R-4: tips at t <= 0 or with no texel image in [0,nx-1]x[0,ny-1] are not
 *     sampled;
 *     if t* > -1: t_{k+1} = t* + 2^-(k+1), else t_{k+1} = t_k - 2^-k (the value
 *     the DDA left in t_k).
 *   The run's result is the last level's (Delta*, t*): J_r = Delta* / (a_r +
 *   t* T_r) (R-5: the final division by the distance, Alg. 1's last step,
 *   gives a clearance angle in radians).
 *   R-6: the ray's cost is the minimum J_r over the runs (first run on ties);
 *   light = F(clamp(J cos(eps_p) / alpha, -1, 1)) as for the exact method, and
 *   1 when no run sampled anything (J = +inf).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

#define OG_PROJ_GNOMONIC 0

typedef struct {
    const double* h;             /* heights [ny][pitch] (FP64 copy) */
    int64_t pitch;
    int32_t nx, ny;
    double g, R;
    int32_t proj;
    const float* lev[32];        /* level m of the maximum mipmap, dense rows */
    int32_t lw[32], lh[32];
    int32_t nlev;
} og_tile;

static void og_dir(const og_tile* t, double u, double v, double n[3]) {
    double X = (u - 0.5 * (t->nx - 1)) * t->g, Y = (v - 0.5 * (t->ny - 1)) * t->g;
    if (t->proj == OG_PROJ_GNOMONIC) {
        double m = sqrt(X * X + Y * Y + t->R * t->R);
        n[0] = X / m; n[1] = Y / m; n[2] = t->R / m;
    } else {
        double r2 = X * X + Y * Y, fr = 4.0 * t->R * t->R;
        n[0] = 4.0 * t->R * X / (fr + r2);
        n[1] = 4.0 * t->R * Y / (fr + r2);
        n[2] = (fr - r2) / (fr + r2);
    }
}

static int og_image(const og_tile* t, const double q[3], double* u, double* v) {
    double X, Y;
    if (t->proj == OG_PROJ_GNOMONIC) {
        if (!(q[2] > 0.0)) return 0;
        X = t->R * q[0] / q[2];
        Y = t->R * q[1] / q[2];
    } else {
        double m = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2]), den = m + q[2];
        if (!(den > 0.0)) return 0;
        X = 2.0 * t->R * q[0] / den;
        Y = 2.0 * t->R * q[1] / den;
    }
    *u = X / t->g + 0.5 * (t->nx - 1);
    *v = Y / t->g + 0.5 * (t->ny - 1);
    return 1;
}

static double og_bilinear(const og_tile* t, double u, double v) {
    int64_t i0 = (int64_t)floor(u), j0 = (int64_t)floor(v);
    if (i0 > t->nx - 2) i0 = t->nx - 2;
    if (j0 > t->ny - 2) j0 = t->ny - 2;
    if (i0 < 0) i0 = 0;
    if (j0 < 0) j0 = 0;
    double fu = u - (double)i0, fv = v - (double)j0;
    const double* r0 = t->h + j0 * t->pitch;
    const double* r1 = r0 + t->pitch;
    return (1.0 - fu) * (1.0 - fv) * r0[i0] + fu * (1.0 - fv) * r0[i0 + 1] +
           (1.0 - fu) * fv * r1[i0] + fu * fv * r1[i0 + 1];
}

static void og_cross(const double a[3], const double b[3], double c[3]) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

static double og_dot(const double a[3], const double b[3]) {
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

/* Eq. maxstep: ray length of one run starting at R (see the header) */
static double og_maxstep(const og_tile* t, const double Rs[3], const double s[3], int32_t m0) {
    double u0, v0;
    if (!og_image(t, Rs, &u0, &v0)) return -1.0;
    double lx = s[0], ly = s[1], ln = sqrt(lx * lx + ly * ly);
    if (!(ln > 0.0)) return -1.0;
    double span = ldexp(1.0, m0);
    double e[3];
    og_dir(t, u0 + span * lx / ln, v0 + span * ly / ln, e);
    double c[3] = { -Rs[0], -Rs[1], -Rs[2] }, cb[3], ab[3];
    og_cross(c, e, cb);
    og_cross(s, e, ab);
    double den = og_dot(ab, ab);
    if (!(den > 0.0)) return -1.0;
    return og_dot(cb, ab) / den;
}

/* one tip sample: 1 and *delta = H - M when the tip has an in-tile image */
static int og_sample(const og_tile* t, const double p[3], const double s[3], double dist,
                     int32_t m, double* delta) {
    double q[3] = { p[0] + dist * s[0], p[1] + dist * s[1], p[2] + dist * s[2] };
    double u, v;
    if (!og_image(t, q, &u, &v)) return 0;
    if (!(u >= 0.0 && u <= (double)(t->nx - 1) && v >= 0.0 && v <= (double)(t->ny - 1))) return 0;
    double cell = ldexp(1.0, m);
    int64_t I = (int64_t)floor((u + 0.5) / cell), Jv = (int64_t)floor((v + 0.5) / cell);
    if (I > t->lw[m] - 1) I = t->lw[m] - 1;
    if (Jv > t->lh[m] - 1) Jv = t->lh[m] - 1;
    if (I < 0) I = 0;
    if (Jv < 0) Jv = 0;
    double M = (double)t->lev[m][Jv * t->lw[m] + I];
    double H = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2]) - t->R;
    *delta = H - M;
    return 1;
}

static void og_ray(const og_tile* t, const double s[3], double alpha, const int32_t* levels,
                   int32_t n_runs, double u, double v, double lift, double* light, double* cost,
                   double* tstar_out) {
    double n[3];
    og_dir(t, u, v, n);
    double hp = og_bilinear(t, u, v) + lift;
    double p[3] = { (t->R + hp) * n[0], (t->R + hp) * n[1], (t->R + hp) * n[2] };
    double bestJ = INFINITY, bestd = -1.0, a = 0.0;
    for (int32_t r = 0; r < n_runs; ++r) {
        int32_t Np = levels[r];
        double Rs[3] = { p[0] + a * s[0], p[1] + a * s[1], p[2] + a * s[2] };
        double T = og_maxstep(t, Rs, s, Np - 1);
        if (!(T > 0.0)) break;
        double tk = 1.0, dstar = INFINITY, ts = -1.0;
        for (int32_t k = 0; k < Np; ++k) {
            int32_t m = Np - 1 - k;
            dstar = INFINITY;
            ts = -1.0;
            double step = ldexp(1.0, -(k + 1));
            for (int i = 0; i < 3; ++i) {
                if (i > 0) tk -= step;
                double d;
                if (tk > 0.0 && og_sample(t, p, s, a + tk * T, m, &d) && d < dstar) {
                    dstar = d;
                    ts = tk;
                }
            }
            if (ts > -1.0) tk = ts + ldexp(1.0, -(k + 1));
        }
        if (ts > -1.0) {
            double dist = a + ts * T;
            double J = dstar / dist;
            if (J < bestJ) {
                bestJ = J;
                bestd = dist;
            }
        }
        a += T;
    }
    *cost = bestJ;
    *tstar_out = bestd;
    if (!(bestd > 0.0)) {
        *light = 1.0;
        return;
    }
    double se = n[0] * s[0] + n[1] * s[1] + n[2] * s[2];
    double ce = sqrt(fmax(0.0, 1.0 - se * se));
    double dd = bestJ * ce / alpha;
    if (dd > 1.0) dd = 1.0;
    if (dd < -1.0) dd = -1.0;
    *light = (M_PI - acos(dd) + dd * sqrt(1.0 - dd * dd)) / M_PI;
}

int32_t or_maxmip(const float* h, int32_t nx, int32_t ny, int64_t pitch, float* out);

/*
 * heights: float32 [ny][nx] (the mipmap is built from them) and the same values
 * in FP64 (h64) for the origin's bilinear height; levels[n_runs] = N' per run.
 * mode 0: one ray per texel centre; mode 1: n listed origins uv (+ lift).
 * Outputs per ray: light, cost J (rad, +inf when nothing sampled), t* (m, -1).
 */
void og_greedy(const float* h, const double* h64, int32_t nx, int32_t ny, double g, double R,
               int32_t proj, double elev, double az, double alpha, const int32_t* levels,
               int32_t n_runs, int32_t mode, int64_t n, const float* uv, const float* lift,
               double* light, double* cost, double* tstar) {
    og_tile t;
    t.h = h64;
    t.pitch = nx;
    t.nx = nx;
    t.ny = ny;
    t.g = g;
    t.R = R;
    t.proj = proj;
    int64_t total = 0;
    for (int32_t w = nx, hh = ny; w > 1 || hh > 1; w = (w + 1) / 2, hh = (hh + 1) / 2)
        total += (int64_t)((w + 1) / 2) * ((hh + 1) / 2);
    float* mip = (float*)malloc(sizeof(float) * (size_t)(total > 0 ? total : 1));
    t.nlev = or_maxmip(h, nx, ny, nx, mip);
    t.lev[0] = h;
    t.lw[0] = nx;
    t.lh[0] = ny;
    const float* cur = mip;
    for (int32_t l = 1; l < t.nlev && l < 32; ++l) {
        t.lw[l] = (t.lw[l - 1] + 1) / 2;
        t.lh[l] = (t.lh[l - 1] + 1) / 2;
        t.lev[l] = cur;
        cur += (int64_t)t.lw[l] * t.lh[l];
    }
    double s[3] = { cos(elev) * sin(az), cos(elev) * cos(az), sin(elev) };
    int64_t nr = mode == 0 ? (int64_t)nx * ny : n;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t r = 0; r < nr; ++r) {
        double u, v, l = 0.0;
        if (mode == 0) {
            u = (double)(r % nx);
            v = (double)(r / nx);
        } else {
            u = (double)uv[2 * r];
            v = (double)uv[2 * r + 1];
            l = lift ? (double)lift[r] : 0.0;
        }
        og_ray(&t, s, alpha, levels, n_runs, u, v, l, &light[r], &cost[r], &tstar[r]);
    }
    free(mip);
}
