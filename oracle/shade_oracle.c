/*
 * FP64 oracle for the shading epilogue: Lambertian irradiance of the terrain
 * under several disc lights (Sun, Earth), each attenuated by its lit fraction.
 *
 * TEST INFRASTRUCTURE ONLY (same rules as shadow_oracle.c).
 *
 * Sec. 3.4 treats the lights (Sun, Earth) as discs whose visible fraction s is
 * the circular-segment area; Sec. 6.3 shades with a Lambertian BRDF.  Per ray
 * origin (u, v) and light l (direction L_l from elevation/azimuth as for the
 * sun, intensity I_l, lit fraction s_l from the shadow pass):
 *   E = sum_l I_l s_l max(0, N . L_l),
 * N the unit normal of the terrain surface r(u, v) = (R + h(u, v)) n(u, v),
 * N ~ dr/du x dr/dv, dr/du = h_u n + (R + h) dn/du.
 * Readings: grid rays (texel centres) take h_u, h_v as central differences of
 * the texel values (one-sided on the border); listed origins take the gradient
 * of the bilinear interpolant in their cell (base min(floor(u), nx-2)), and
 * R + h uses the terrain height (not the lift).  dn/du, dn/dv are taken here
 * by central differences of the mapping with a step of 1e-3 texel (error
 * ~1e-9 relative), independently of any closed form.
 */
#include <math.h>
#include <stdint.h>

typedef struct {
    const double* h;
    int32_t nx, ny;
    double g, R;
    int32_t proj;
} os_tile;

static void os_dir(const os_tile* t, double u, double v, double n[3]) {
    double X = (u - 0.5 * (t->nx - 1)) * t->g, Y = (v - 0.5 * (t->ny - 1)) * t->g;
    if (t->proj == 0) {
        double m = sqrt(X * X + Y * Y + t->R * t->R);
        n[0] = X / m; n[1] = Y / m; n[2] = t->R / m;
    } else {
        double r2 = X * X + Y * Y, fr = 4.0 * t->R * t->R;
        n[0] = 4.0 * t->R * X / (fr + r2);
        n[1] = 4.0 * t->R * Y / (fr + r2);
        n[2] = (fr - r2) / (fr + r2);
    }
}

static double os_h(const os_tile* t, int64_t i, int64_t j) { return t->h[j * t->nx + i]; }

static void os_ray(const os_tile* t, int32_t mode, double u, double v, const double* L,
                   const double* I, const double* const* s_frac, int32_t n_lights, int64_t r,
                   double* E) {
    double hu, hv, h;
    if (mode == 0) {
        int64_t i = (int64_t)u, j = (int64_t)v;
        int64_t il = i > 0 ? i - 1 : i, ir = i < t->nx - 1 ? i + 1 : i;
        int64_t jl = j > 0 ? j - 1 : j, jr = j < t->ny - 1 ? j + 1 : j;
        hu = (os_h(t, ir, j) - os_h(t, il, j)) / (double)(ir - il);
        hv = (os_h(t, i, jr) - os_h(t, i, jl)) / (double)(jr - jl);
        h = os_h(t, i, j);
    } else {
        int64_t i0 = (int64_t)floor(u), j0 = (int64_t)floor(v);
        if (i0 > t->nx - 2) i0 = t->nx - 2;
        if (j0 > t->ny - 2) j0 = t->ny - 2;
        if (i0 < 0) i0 = 0;
        if (j0 < 0) j0 = 0;
        double fu = u - (double)i0, fv = v - (double)j0;
        double h00 = os_h(t, i0, j0), h10 = os_h(t, i0 + 1, j0);
        double h01 = os_h(t, i0, j0 + 1), h11 = os_h(t, i0 + 1, j0 + 1);
        hu = (1.0 - fv) * (h10 - h00) + fv * (h11 - h01);
        hv = (1.0 - fu) * (h01 - h00) + fu * (h11 - h10);
        h = (1.0 - fu) * (1.0 - fv) * h00 + fu * (1.0 - fv) * h10 + (1.0 - fu) * fv * h01 +
            fu * fv * h11;
    }
    double n[3], a[3], b[3], du[3], dv[3];
    os_dir(t, u, v, n);
    const double e = 1e-3;
    os_dir(t, u + e, v, a);
    os_dir(t, u - e, v, b);
    for (int k = 0; k < 3; ++k) du[k] = (a[k] - b[k]) / (2.0 * e);
    os_dir(t, u, v + e, a);
    os_dir(t, u, v - e, b);
    for (int k = 0; k < 3; ++k) dv[k] = (a[k] - b[k]) / (2.0 * e);
    double rho = t->R + h, ru[3], rv[3];
    for (int k = 0; k < 3; ++k) {
        ru[k] = hu * n[k] + rho * du[k];
        rv[k] = hv * n[k] + rho * dv[k];
    }
    double N[3] = { ru[1] * rv[2] - ru[2] * rv[1], ru[2] * rv[0] - ru[0] * rv[2],
                    ru[0] * rv[1] - ru[1] * rv[0] };
    double nn = sqrt(N[0] * N[0] + N[1] * N[1] + N[2] * N[2]);
    double out = 0.0;
    for (int32_t l = 0; l < n_lights; ++l) {
        double c = (N[0] * L[3 * l] + N[1] * L[3 * l + 1] + N[2] * L[3 * l + 2]) / nn;
        out += I[l] * s_frac[l][r] * (c > 0.0 ? c : 0.0);
    }
    *E = out;
}

/* heights double [ny][nx]; lights: elevation/azimuth (rad), intensity and the
 * per-ray lit fraction s_frac[l][n]; mode 0 grid rays, 1 listed uv. */
void os_shade(const double* h, int32_t nx, int32_t ny, double g, double R, int32_t proj,
              int32_t mode, int64_t n, const float* uv, int32_t n_lights, const double* elev,
              const double* az, const double* intensity, const double* const* s_frac,
              double* E) {
    os_tile t = { h, nx, ny, g, R, proj };
    double L[3 * 8];
    for (int32_t l = 0; l < n_lights && l < 8; ++l) {
        L[3 * l] = cos(elev[l]) * sin(az[l]);
        L[3 * l + 1] = cos(elev[l]) * cos(az[l]);
        L[3 * l + 2] = sin(elev[l]);
    }
    int64_t nr = mode == 0 ? (int64_t)nx * ny : n;
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < nr; ++r) {
        double u = mode == 0 ? (double)(r % nx) : (double)uv[2 * r];
        double v = mode == 0 ? (double)(r / nx) : (double)uv[2 * r + 1];
        os_ray(&t, mode, u, v, L, intensity, s_frac, n_lights, r, &E[r]);
    }
}
