/*
 * FP64 oracle for the view rays of the polar scene: the first intersection of
 * each pixel's view ray with the bilinear terrain draped on the sphere.
 *
 * TEST INFRASTRUCTURE ONLY (same rules as shadow_oracle.c: loaded by tests/,
 * __graft_entry__.smoke() and bench.py's CPU legs only; no code shared with
 * the CUDA path).
 *
 * The surface points that receive shadow rays in the paper's renderer are the
 * terrain points seen by the camera (Sec. 4, view rays against the displaced
 * surface).  Definition used here (plain, every sample tested in order):
 *   pixel (i, j), row 0 at the top: a = (2(i + 0.5)/W - 1) tan_x,
 *   b = (1 - 2(j + 0.5)/H) tan_y, d = unit(forward + a right + b up);
 *   x(tau) = C + tau d, samples tau_k = k * step, k = 1 .. floor(max_dist / step);
 *   F(tau) = |x| - R - h(texel image of x)   (h bilinear, FP64 over float32 texels)
 *   for points whose texel image lies in [0,nx-1] x [0,ny-1];
 *   hit = the smallest k whose image is in the tile with F(tau_k) <= 0; when the
 *   image of tau_{k-1} is in the tile too, the crossing is refined by 48
 *   bisection halvings of [tau_{k-1}, tau_k] (keep the half whose upper end has
 *   an in-tile image with F <= 0); the hit point is the upper end.
 *   Output: texel coordinates (u, v) of the hit point, or NaN for no hit.
 * Samples before the ray first descends to the tile's highest height cannot
 * satisfy F <= 0; the loop starts one sample before that point (a skip that
 * does not change which sample is first), and stops once the ray is above the
 * highest height and climbing (|x| is convex in tau).
 */
#include <math.h>
#include <stdint.h>

#define OV_PROJ_GNOMONIC 0

typedef struct {
    const double* h;
    int32_t nx, ny;
    int64_t pitch;
    double g, R;
    int32_t proj;
    double hmax;
} ov_tile;

/* texel image of the direction of x; 0 when outside the tile or without image */
static int ov_image(const ov_tile* t, const double x[3], double* u, double* v) {
    double X, Y;
    if (t->proj == OV_PROJ_GNOMONIC) {
        if (!(x[2] > 0.0)) return 0;
        X = t->R * x[0] / x[2];
        Y = t->R * x[1] / x[2];
    } else {
        double m = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
        double den = m + x[2];
        if (!(den > 0.0)) return 0;
        X = 2.0 * t->R * x[0] / den;
        Y = 2.0 * t->R * x[1] / den;
    }
    *u = X / t->g + 0.5 * (double)(t->nx - 1);
    *v = Y / t->g + 0.5 * (double)(t->ny - 1);
    return *u >= 0.0 && *u <= (double)(t->nx - 1) && *v >= 0.0 && *v <= (double)(t->ny - 1);
}

static double ov_bilinear(const ov_tile* t, double u, double v) {
    int64_t i0 = (int64_t)floor(u), j0 = (int64_t)floor(v);
    if (i0 > t->nx - 2) i0 = t->nx - 2;
    if (j0 > t->ny - 2) j0 = t->ny - 2;
    if (i0 < 0) i0 = 0;
    if (j0 < 0) j0 = 0;
    double fu = u - (double)i0, fv = v - (double)j0;
    const double* r0 = t->h + j0 * t->pitch;
    const double* r1 = r0 + t->pitch;
    double top = r0[i0] + fu * (r0[i0 + 1] - r0[i0]);
    double bot = r1[i0] + fu * (r1[i0 + 1] - r1[i0]);
    return top + fv * (bot - top);
}

/* 1: in-tile point below (or on) the terrain; *uv set for in-tile points */
static int ov_below(const ov_tile* t, const double C[3], const double d[3], double tau,
                    int* in_tile, double* u, double* v) {
    double x[3] = { C[0] + tau * d[0], C[1] + tau * d[1], C[2] + tau * d[2] };
    *in_tile = ov_image(t, x, u, v);
    if (!*in_tile) return 0;
    double H = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]) - t->R;
    return H - ov_bilinear(t, *u, *v) <= 0.0;
}

static void ov_pixel(const ov_tile* t, const double C[3], const double f[3], const double r[3],
                     const double up[3], double tan_x, double tan_y, int32_t W, int32_t H,
                     int64_t pix, double step, int64_t K, double* out_u, double* out_v) {
    int64_t i = pix % W, j = pix / W;
    double a = (2.0 * ((double)i + 0.5) / (double)W - 1.0) * tan_x;
    double b = (1.0 - 2.0 * ((double)j + 0.5) / (double)H) * tan_y;
    double d[3];
    for (int k = 0; k < 3; ++k) d[k] = f[k] + a * r[k] + b * up[k];
    double dn = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    for (int k = 0; k < 3; ++k) d[k] /= dn;
    *out_u = NAN;
    *out_v = NAN;
    /* first tau with |x| <= R + hmax (smaller root of a quadratic), if any */
    double Rm = t->R + t->hmax;
    double cd = C[0] * d[0] + C[1] * d[1] + C[2] * d[2];
    double cc = C[0] * C[0] + C[1] * C[1] + C[2] * C[2];
    double disc = cd * cd - (cc - Rm * Rm);
    if (disc < 0.0) return;                     /* never reaches the highest height */
    double tau_in = -cd - sqrt(disc);
    double tau_out = -cd + sqrt(disc);
    if (tau_out < 0.0) return;
    int64_t k0 = tau_in > 0.0 ? (int64_t)floor(tau_in / step) - 1 : 1;
    if (k0 < 1) k0 = 1;
    int64_t k1 = (int64_t)ceil(tau_out / step) + 1;
    if (k1 > K) k1 = K;
    int prev_in = 0;
    for (int64_t k = k0; k <= k1; ++k) {
        double tau = (double)k * step, u, v;
        int in_tile;
        if (ov_below(t, C, d, tau, &in_tile, &u, &v)) {
            double hi = tau;
            if (prev_in && k > 1) {
                double lo = (double)(k - 1) * step;
                for (int it = 0; it < 48; ++it) {
                    double mid = lo + 0.5 * (hi - lo);
                    double um, vm;
                    int inm;
                    if (ov_below(t, C, d, mid, &inm, &um, &vm))
                        hi = mid;
                    else
                        lo = mid;
                }
            }
            double x[3] = { C[0] + hi * d[0], C[1] + hi * d[1], C[2] + hi * d[2] };
            ov_image(t, x, out_u, out_v);
            return;
        }
        prev_in = in_tile;
    }
}

/* heights double [ny][pitch]; pixels: n indices into the W x H frame (row-major) */
void ov_view_hits(const double* h, int32_t nx, int32_t ny, int64_t pitch, double g, double R,
                  int32_t proj, const double* cam_pos, const double* fwd, const double* right,
                  const double* up, double tan_x, double tan_y, int32_t W, int32_t H,
                  double step, double max_dist, int64_t n, const int64_t* pixels,
                  double* u_out, double* v_out) {
    ov_tile t = { h, nx, ny, pitch, g, R, proj, -INFINITY };
    for (int32_t y = 0; y < ny; ++y)
        for (int32_t x = 0; x < nx; ++x)
            if (h[(int64_t)y * pitch + x] > t.hmax) t.hmax = h[(int64_t)y * pitch + x];
    int64_t K = (int64_t)floor(max_dist / step);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t q = 0; q < n; ++q)
        ov_pixel(&t, cam_pos, fwd, right, up, tan_x, tan_y, W, H, pixels[q], step, K,
                 &u_out[q], &v_out[q]);
}
