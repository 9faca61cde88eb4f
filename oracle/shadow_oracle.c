/*
 * FP64 brute-force oracle for soft shadows on a heightfield draped on a sphere.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's
 * CPU-baseline / reference leg may load this library.  It shares no code, header,
 * table or constant with the CUDA path, and never calls it.
 *
 * What it computes (the plain definition, every sample evaluated, no pruning and
 * no early exit):
 *   - Shadow ray R(t) = p + t*L from the surface point p toward the light centre
 *     (Sec. 3.1, "Soft Shadow Theory").
 *   - Per-sample clearance Delta h = H(t) - h(t) and cost Delta h / t; the ray's
 *     cost is the minimum over samples, J* = Delta h* / t* (Eq. shadowfrac and
 *     the final step of Algorithm 1).  Reading: the minimum is taken of
 *     Delta h / t, in radians, not of Delta h alone (Eq. cost).
 *   - Disc occlusion: the sun is a disc of angular radius r_L; the horizon chord
 *     sits at normalised distance d from the disc centre and the lit fraction is
 *     the circular-segment area (pi - acos d + d sqrt(1-d^2)) / pi (Eq. discfrac).
 *     Reading: d = clamp(J* cos(eps_p) / r_L, -1, 1) with eps_p the sun elevation
 *     over the radial normal at p (Eq. discsegment is garbled in the source).
 *   - Maximum mipmap: each level texel is the maximum of the level-0 texels it
 *     covers (Sec. 3.2, "Maximum mipmaps").
 *   - Texture mapping: gnomonic (a 3-D line maps to a straight texture line,
 *     Sec. 3.2 and the Appendix) or polar stereographic.
 *   - Analytic gradient of sum_r gL_r * light_r with respect to the heights and
 *     the sun direction, at each ray's argmin sample (subgradient of the min).
 *
 * Geometry (all lengths in metres):
 *   sphere centre at the origin; tile frame x = grid +u (columns), y = grid +v
 *   (rows), z = tile-centre direction.  Texel (u, v) has plane coordinates
 *   X = (u - (nx-1)/2) g, Y = (v - (ny-1)/2) g.
 *   gnomonic:          unit direction n = (X, Y, R) / |(X, Y, R)|
 *   polar stereographic: n = (4RX, 4RY, 4R^2 - X^2 - Y^2) / (4R^2 + X^2 + Y^2)
 *   sun: s = (cos e sin a, cos e cos a, sin e), elevation e and azimuth a (from
 *   grid +y toward +x) in the tile-centre frame.
 *   samples t_j = j * delta, j = 1..floor(Lmax / delta), delta = step_texels * g.
 *   A sample is used when its texel coordinates lie in [0,nx-1] x [0,ny-1] and
 *   the ray has not left the tile before it: only the first run of in-tile
 *   samples counts (reading: a shadow ray is followed until its image leaves
 *   the heightfield; for gnomonic tiles, where the image is a straight line,
 *   that run is every in-tile sample; on polar stereographic tiles the image
 *   is a circle arc that could re-enter, and re-entries are not followed).
 *   Bilinear: base = min(floor(u), nx-2), frac = u - base.
 *   Ties: the smallest j among equal costs.  No usable sample: cost = +inf,
 *   argmin = -1, light = 1.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_PROJ_GNOMONIC 0
#define OR_PROJ_STEREO 1

typedef struct {
    const double* h;   /* heights [ny][pitch] */
    int32_t nx, ny;
    int64_t pitch;
    double g, R;
    int32_t proj;
} or_tile;

typedef struct {
    double elev, az, alpha;
} or_sun;

/* ---- small vector helpers -------------------------------------------------- */
static double dot3(const double* a, const double* b) { return a[0]*b[0] + a[1]*b[1] + a[2]*b[2]; }
static double norm3(const double* a) { return sqrt(dot3(a, a)); }

static void sun_dir(const or_sun* s, double out[3]) {
    out[0] = cos(s->elev) * sin(s->az);
    out[1] = cos(s->elev) * cos(s->az);
    out[2] = sin(s->elev);
}

/* texel coordinates -> unit direction on the sphere */
static void texel_to_dir(const or_tile* t, double u, double v, double n[3]) {
    double X = (u - 0.5 * (t->nx - 1)) * t->g;
    double Y = (v - 0.5 * (t->ny - 1)) * t->g;
    if (t->proj == OR_PROJ_GNOMONIC) {
        double m = sqrt(X * X + Y * Y + t->R * t->R);
        n[0] = X / m; n[1] = Y / m; n[2] = t->R / m;
    } else {
        double r2 = X * X + Y * Y, fr = 4.0 * t->R * t->R;
        n[0] = 4.0 * t->R * X / (fr + r2);
        n[1] = 4.0 * t->R * Y / (fr + r2);
        n[2] = (fr - r2) / (fr + r2);
    }
}

/* point q (any length) -> texel coordinates of its direction; returns 0 if it
 * has no image (behind the gnomonic plane / at the stereographic pole). */
static int point_to_texel(const or_tile* t, const double q[3], double* u, double* v) {
    double X, Y;
    if (t->proj == OR_PROJ_GNOMONIC) {
        if (!(q[2] > 0.0)) return 0;
        X = t->R * q[0] / q[2];
        Y = t->R * q[1] / q[2];
    } else {
        double m = norm3(q);
        double den = m + q[2];
        if (!(den > 0.0)) return 0;
        X = 2.0 * t->R * q[0] / den;
        Y = 2.0 * t->R * q[1] / den;
    }
    *u = X / t->g + 0.5 * (t->nx - 1);
    *v = Y / t->g + 0.5 * (t->ny - 1);
    return 1;
}

/* d(u,v)/dq (2x3) of point_to_texel */
static void point_to_texel_jac(const or_tile* t, const double q[3], double J[2][3]) {
    if (t->proj == OR_PROJ_GNOMONIC) {
        double k = t->R / t->g;
        J[0][0] = k / q[2]; J[0][1] = 0.0;        J[0][2] = -k * q[0] / (q[2] * q[2]);
        J[1][0] = 0.0;      J[1][1] = k / q[2];   J[1][2] = -k * q[1] / (q[2] * q[2]);
    } else {
        double m = norm3(q);
        double den = m + q[2];
        double k = 2.0 * t->R / t->g;
        double dden[3] = { q[0] / m, q[1] / m, q[2] / m + 1.0 };
        for (int i = 0; i < 3; ++i) {
            J[0][i] = k * ((i == 0 ? den : 0.0) - q[0] * dden[i]) / (den * den);
            J[1][i] = k * ((i == 1 ? den : 0.0) - q[1] * dden[i]) / (den * den);
        }
    }
}

static int inside(const or_tile* t, double u, double v) {
    return u >= 0.0 && u <= (double)(t->nx - 1) && v >= 0.0 && v <= (double)(t->ny - 1);
}

/* bilinear interpolation; also returns base texel, weights and the gradient */
typedef struct { int64_t i0, j0; double w[4]; double du, dv; double h; } or_bil;

static void bilinear(const or_tile* t, double u, double v, or_bil* b) {
    int64_t i0 = (int64_t)floor(u), j0 = (int64_t)floor(v);
    if (i0 > t->nx - 2) i0 = t->nx - 2;
    if (j0 > t->ny - 2) j0 = t->ny - 2;
    if (i0 < 0) i0 = 0;
    if (j0 < 0) j0 = 0;
    double fu = u - (double)i0, fv = v - (double)j0;
    const double* r0 = t->h + j0 * t->pitch;
    const double* r1 = r0 + t->pitch;
    double h00 = r0[i0], h10 = r0[i0 + 1], h01 = r1[i0], h11 = r1[i0 + 1];
    b->i0 = i0; b->j0 = j0;
    b->w[0] = (1.0 - fu) * (1.0 - fv);   /* (i0,   j0)   */
    b->w[1] = fu * (1.0 - fv);           /* (i0+1, j0)   */
    b->w[2] = (1.0 - fu) * fv;           /* (i0,   j0+1) */
    b->w[3] = fu * fv;                   /* (i0+1, j0+1) */
    b->h = b->w[0] * h00 + b->w[1] * h10 + b->w[2] * h01 + b->w[3] * h11;
    b->du = (1.0 - fv) * (h10 - h00) + fv * (h11 - h01);
    b->dv = (1.0 - fu) * (h01 - h00) + fu * (h11 - h10);
}

/* lit fraction of a unit disc cut by a chord at signed distance d (Eq. discfrac) */
double or_disc_light(double d) {
    if (d <= -1.0) return 0.0;
    if (d >= 1.0) return 1.0;
    return (M_PI - acos(d) + d * sqrt(1.0 - d * d)) / M_PI;
}

/* ---- one ray ---------------------------------------------------------------- */
typedef struct {
    double n[3];      /* unit radial direction at the origin */
    double p[3];      /* origin point */
    double hp;        /* origin height */
    or_bil ob;        /* origin bilinear (weights of h_p) */
} or_origin;

static void make_origin(const or_tile* t, double u, double v, double lift, or_origin* o) {
    texel_to_dir(t, u, v, o->n);
    bilinear(t, u, v, &o->ob);
    o->hp = o->ob.h + lift;
    double rho = t->R + o->hp;
    for (int i = 0; i < 3; ++i) o->p[i] = rho * o->n[i];
}

static int64_t n_samples(double lmax, double delta) {
    if (!(delta > 0.0) || !(lmax > 0.0)) return 0;
    return (int64_t)floor(lmax / delta);
}

/* cost of sample j; returns 0 when the sample has no texel in the tile */
static int sample_cost(const or_tile* t, const or_origin* o, const double s[3],
                       double tj, double* cost) {
    double q[3] = { o->p[0] + tj * s[0], o->p[1] + tj * s[1], o->p[2] + tj * s[2] };
    double u, v;
    if (!point_to_texel(t, q, &u, &v) || !inside(t, u, v)) return 0;
    or_bil b;
    bilinear(t, u, v, &b);
    double H = norm3(q) - t->R;
    *cost = (H - b.h) / tj;
    return 1;
}

/* cost2 (may be NULL): the runner-up, the smallest cost over the usable
 * samples other than the argmin (+inf with fewer than two), so that a caller
 * can tell a unique minimum from a tie. */
static void ray_forward(const or_tile* t, const or_sun* sun, const double s[3],
                        double lmax, double step_texels, double u, double v, double lift,
                        double* light, int64_t* argmin, double* cost, double* cost2) {
    or_origin o;
    make_origin(t, u, v, lift, &o);
    double delta = step_texels * t->g;
    int64_t J = n_samples(lmax, delta);
    double best = INFINITY, second = INFINITY;
    int64_t bj = -1;
    int seen = 0;
    for (int64_t j = 1; j <= J; ++j) {
        double c;
        if (sample_cost(t, &o, s, (double)j * delta, &c)) {
            seen = 1;
            if (c < best) {
                second = best;
                best = c;
                bj = j;
            } else if (c < second) {
                second = c;
            }
        } else if (seen) {
            break;   /* the ray has left the tile: it is not followed further */
        }
    }
    double se = dot3(o.n, s);
    double ce = sqrt(fmax(0.0, 1.0 - se * se));
    *argmin = bj;
    *cost = best;
    if (cost2) *cost2 = second;
    if (bj < 0) { *light = 1.0; return; }
    double d = best * ce / sun->alpha;
    if (d > 1.0) d = 1.0;
    if (d < -1.0) d = -1.0;
    *light = or_disc_light(d);
}

static void ray_origin_coords(const or_tile* t, int32_t mode, int64_t r, const float* uv,
                              const float* lift, double* u, double* v, double* l) {
    if (mode == 0) {
        *u = (double)(r % t->nx);
        *v = (double)(r / t->nx);
        *l = 0.0;
    } else {
        *u = (double)uv[2 * r];
        *v = (double)uv[2 * r + 1];
        *l = lift ? (double)lift[r] : 0.0;
    }
}

/* sun direction of elevation e and azimuth a (tile-centre frame) */
void or_sun_vector(double elev, double az, double* out) {
    or_sun sun = { elev, az, 0.0 };
    sun_dir(&sun, out);
}

/* ---- exported API --------------------------------------------------------------
 * heights: double [ny][pitch]; mode 0 = one ray per texel centre (n = nx*ny, ray r
 * at (r % nx, r / nx)); mode 1 = list of n origins uv[2n] (floats, texel coords)
 * with optional lift[n] (metres above the bilinear surface).  */
void or_shadow(const double* h, int32_t nx, int32_t ny, int64_t pitch, double g, double R,
               int32_t proj, double elev, double az, double alpha, double lmax,
               double step_texels, int32_t mode, int64_t n, const float* uv,
               const float* lift, double* light, int64_t* argmin, double* cost) {
    or_tile t = { h, nx, ny, pitch, g, R, proj };
    or_sun sun = { elev, az, alpha };
    double s[3];
    sun_dir(&sun, s);
    int64_t nr = (mode == 0) ? (int64_t)nx * ny : n;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t r = 0; r < nr; ++r) {
        double u, v, l;
        ray_origin_coords(&t, mode, r, uv, lift, &u, &v, &l);
        ray_forward(&t, &sun, s, lmax, step_texels, u, v, l, &light[r], &argmin[r], &cost[r],
                    NULL);
    }
}

/* The same forward with the light direction given as a 3-vector s (used as
 * is, not normalised: q = p + t s, sin(eps_p) = n_p . s) instead of elevation
 * and azimuth, so that the light can be differentiated along each component of
 * s as a free vector; and with the runner-up cost of every ray (cost2, may be
 * NULL; see ray_forward). */
void or_shadow_svec(const double* h, int32_t nx, int32_t ny, int64_t pitch, double g, double R,
                    int32_t proj, const double* svec, double alpha, double lmax,
                    double step_texels, int32_t mode, int64_t n, const float* uv,
                    const float* lift, double* light, int64_t* argmin, double* cost,
                    double* cost2) {
    or_tile t = { h, nx, ny, pitch, g, R, proj };
    or_sun sun = { 0.0, 0.0, alpha };
    const double s[3] = { svec[0], svec[1], svec[2] };
    int64_t nr = (mode == 0) ? (int64_t)nx * ny : n;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t r = 0; r < nr; ++r) {
        double u, v, l;
        ray_origin_coords(&t, mode, r, uv, lift, &u, &v, &l);
        ray_forward(&t, &sun, s, lmax, step_texels, u, v, l, &light[r], &argmin[r], &cost[r],
                    cost2 ? &cost2[r] : NULL);
    }
}

/* every sample's cost along one ray (NaN where the sample is outside the tile) */
int64_t or_ray_costs(const double* h, int32_t nx, int32_t ny, int64_t pitch, double g,
                     double R, int32_t proj, double elev, double az, double lmax,
                     double step_texels, double u, double v, double lift,
                     double* costs, int64_t max_out) {
    or_tile t = { h, nx, ny, pitch, g, R, proj };
    or_sun sun = { elev, az, 0.0 };
    double s[3];
    sun_dir(&sun, s);
    or_origin o;
    make_origin(&t, u, v, lift, &o);
    double delta = step_texels * g;
    int64_t J = n_samples(lmax, delta);
    int seen = 0, left = 0;
    for (int64_t j = 1; j <= J && j <= max_out; ++j) {
        double c;
        int ok = !left && sample_cost(&t, &o, s, (double)j * delta, &c);
        if (ok) seen = 1;
        else if (seen) left = 1;
        costs[j - 1] = ok ? c : NAN;
    }
    return J;
}

/* Texel coordinates (u, v) of the image of sample j[r] of every ray, with the
 * light direction given as a 3-vector (as or_shadow_svec): out_uv[2r],
 * out_uv[2r+1]; NaN when j[r] < 1 or the point has no image.  Lets a caller
 * find the bilinear cell (and so the texels) a ray's argmin sample reads. */
void or_sample_uv(const double* h, int32_t nx, int32_t ny, int64_t pitch, double g, double R,
                  int32_t proj, const double* svec, double step_texels, int32_t mode, int64_t n,
                  const float* uv, const float* lift, const int64_t* j, double* out_uv) {
    or_tile t = { h, nx, ny, pitch, g, R, proj };
    const double s[3] = { svec[0], svec[1], svec[2] };
    const double delta = step_texels * g;
    int64_t nr = (mode == 0) ? (int64_t)nx * ny : n;
    for (int64_t r = 0; r < nr; ++r) {
        out_uv[2 * r] = out_uv[2 * r + 1] = NAN;
        if (j[r] < 1) continue;
        double u, v, l;
        ray_origin_coords(&t, mode, r, uv, lift, &u, &v, &l);
        or_origin o;
        make_origin(&t, u, v, l, &o);
        const double tj = (double)j[r] * delta;
        const double q[3] = { o.p[0] + tj * s[0], o.p[1] + tj * s[1], o.p[2] + tj * s[2] };
        double uq, vq;
        if (point_to_texel(&t, q, &uq, &vq)) {
            out_uv[2 * r] = uq;
            out_uv[2 * r + 1] = vq;
        }
    }
}

/* per-ray radial sine of the sun elevation, n_p . s */
void or_sin_elev(const double* h, int32_t nx, int32_t ny, int64_t pitch, double g, double R,
                 int32_t proj, double elev, double az, int32_t mode, int64_t n,
                 const float* uv, double* out) {
    or_tile t = { h, nx, ny, pitch, g, R, proj };
    or_sun sun = { elev, az, 0.0 };
    double s[3];
    sun_dir(&sun, s);
    int64_t nr = (mode == 0) ? (int64_t)nx * ny : n;
    for (int64_t r = 0; r < nr; ++r) {
        double u, v, l, nn[3];
        ray_origin_coords(&t, mode, r, uv, NULL, &u, &v, &l);
        texel_to_dir(&t, u, v, nn);
        out[r] = dot3(nn, s);
    }
}

/*
 * Analytic gradient of  L = sum_r gL[r] * light[r]  at the given per-ray argmin
 * (1-based sample index, -1 = none).  Accumulates dL/dh into grad_h [ny][pitch]
 * and writes grad_sun[5] = (dL/d elev, dL/d az, dL/ds_x, dL/ds_y, dL/ds_z), the
 * last three with s treated as a free 3-vector.  grad_h_abs and grad_h_cnt
 * (both [ny][pitch], may be NULL) accumulate, per texel, the sum of the absolute
 * values of the non-zero per-ray contributions and their number, the scale of
 * the rounding of a float32 accumulation of the same terms.
 *
 * light = F(d), d = c cos(eps)/alpha (clamped: zero gradient outside (-1, 1)),
 * F'(d) = (2/pi) sqrt(1 - d^2).
 * c = (H(t*) - h(q*)) / t*, q* = p + t* s, H = |q*| - R, p = (R + h_p) n_p,
 * h(q*) bilinear at the texel image of q*, h_p bilinear at the origin (+ lift).
 */
void or_grad(const double* h, int32_t nx, int32_t ny, int64_t pitch, double g, double R,
             int32_t proj, double elev, double az, double alpha, double step_texels,
             int32_t mode, int64_t n, const float* uv, const float* lift,
             const int64_t* argmin, const double* gL, double* grad_h, double* grad_sun,
             double* grad_h_abs, double* grad_h_cnt) {
    or_tile t = { h, nx, ny, pitch, g, R, proj };
    or_sun sun = { elev, az, alpha };
    double s[3];
    sun_dir(&sun, s);
    double ds_de[3] = { -sin(elev) * sin(az), -sin(elev) * cos(az), cos(elev) };
    double ds_da[3] = { cos(elev) * cos(az), -cos(elev) * sin(az), 0.0 };
    double delta = step_texels * g;
    int64_t nr = (mode == 0) ? (int64_t)nx * ny : n;
    double gs[3] = { 0.0, 0.0, 0.0 };
    for (int64_t r = 0; r < nr; ++r) {
        if (argmin[r] < 0 || gL[r] == 0.0) continue;
        double u, v, l;
        ray_origin_coords(&t, mode, r, uv, lift, &u, &v, &l);
        or_origin o;
        make_origin(&t, u, v, l, &o);
        double ts = (double)argmin[r] * delta;
        double q[3] = { o.p[0] + ts * s[0], o.p[1] + ts * s[1], o.p[2] + ts * s[2] };
        double uq, vq;
        if (!point_to_texel(&t, q, &uq, &vq)) continue;
        or_bil b;
        bilinear(&t, uq, vq, &b);
        double qn = norm3(q);
        double c = (qn - R - b.h) / ts;
        double se = dot3(o.n, s);
        double ce = sqrt(fmax(0.0, 1.0 - se * se));
        double d = c * ce / alpha;
        if (!(d > -1.0 && d < 1.0)) continue;
        double dF = (2.0 / M_PI) * sqrt(1.0 - d * d);
        double gd = gL[r] * dF;              /* dL/dd */
        double gc = gd * ce / alpha;         /* dL/dc */
        double Jq[2][3];
        point_to_texel_jac(&t, q, Jq);
        /* gradient of h(q) with respect to q */
        double dhq[3];
        for (int i = 0; i < 3; ++i) dhq[i] = b.du * Jq[0][i] + b.dv * Jq[1][i];
        /* sample texels: dc/dh_k = -w_k / t* */
        int64_t idx[4] = { b.j0 * pitch + b.i0, b.j0 * pitch + b.i0 + 1,
                           (b.j0 + 1) * pitch + b.i0, (b.j0 + 1) * pitch + b.i0 + 1 };
        for (int k = 0; k < 4; ++k) {
            double x = gc * (-b.w[k] / ts);
            grad_h[idx[k]] += x;
            if (grad_h_abs && x != 0.0) { grad_h_abs[idx[k]] += fabs(x); grad_h_cnt[idx[k]] += 1.0; }
        }
        /* origin texels: dc/dh_p = (dH/dq - dh/dq) . n_p / t*  */
        double dHq[3] = { q[0] / qn, q[1] / qn, q[2] / qn };
        double dcdhp = ((dHq[0] - dhq[0]) * o.n[0] + (dHq[1] - dhq[1]) * o.n[1] +
                        (dHq[2] - dhq[2]) * o.n[2]) / ts;
        int64_t oidx[4] = { o.ob.j0 * pitch + o.ob.i0, o.ob.j0 * pitch + o.ob.i0 + 1,
                            (o.ob.j0 + 1) * pitch + o.ob.i0, (o.ob.j0 + 1) * pitch + o.ob.i0 + 1 };
        for (int k = 0; k < 4; ++k) {
            double x = gc * dcdhp * o.ob.w[k];
            grad_h[oidx[k]] += x;
            if (grad_h_abs && x != 0.0) { grad_h_abs[oidx[k]] += fabs(x); grad_h_cnt[oidx[k]] += 1.0; }
        }
        /* sun: dc/ds = (dH/dq - dh/dq) (q depends on s through t* s), plus the
         * cos(eps) factor of d: dd/ds = (c/alpha) * (-se/ce) * n_p */
        for (int i = 0; i < 3; ++i) {
            double dcds = dHq[i] - dhq[i];
            double dce = (ce > 0.0) ? (-se / ce) * o.n[i] : 0.0;
            gs[i] += gc * dcds + gd * (c / alpha) * dce;
        }
    }
    grad_sun[2] = gs[0];
    grad_sun[3] = gs[1];
    grad_sun[4] = gs[2];
    grad_sun[0] = dot3(gs, ds_de);
    grad_sun[1] = dot3(gs, ds_da);
}

/*
 * Maximum mipmap (Sec. 3.2): level 0 is the input; level l+1 has ceil(w/2) x
 * ceil(h/2) texels, each the maximum of the (up to) 2x2 level-l texels below
 * it.  Levels 1..L-1 are written densely (row pitch = level width) one after
 * another into out; returns the number of levels L (including level 0).
 */
int32_t or_maxmip(const float* h, int32_t nx, int32_t ny, int64_t pitch, float* out) {
    int32_t w = nx, hh = ny, L = 1;
    const float* src = h;
    int64_t sp = pitch;
    float* dst = out;
    while (w > 1 || hh > 1) {
        int32_t w2 = (w + 1) / 2, h2 = (hh + 1) / 2;
        for (int32_t y = 0; y < h2; ++y)
            for (int32_t x = 0; x < w2; ++x) {
                float m = src[(int64_t)(2 * y) * sp + 2 * x];
                for (int dy = 0; dy < 2; ++dy)
                    for (int dx = 0; dx < 2; ++dx) {
                        int32_t xx = 2 * x + dx, yy = 2 * y + dy;
                        if (xx < w && yy < hh) {
                            float c = src[(int64_t)yy * sp + xx];
                            if (c > m) m = c;
                        }
                    }
                dst[(int64_t)y * w2 + x] = m;
            }
        src = dst;
        sp = w2;
        dst += (int64_t)w2 * h2;
        w = w2;
        hh = h2;
        ++L;
    }
    return L;
}

int32_t or_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
