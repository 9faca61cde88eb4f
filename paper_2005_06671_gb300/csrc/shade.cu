// Shading epilogue: Lambertian irradiance of the terrain under several disc
// lights (Sec. 3.4: Sun and Earth as discs with their lit fractions; Sec. 6.3:
// Lambertian BRDF),
//   E = sum_l I_l s_l max(0, N . L_l),
// N the unit normal of the surface r(u, v) = (R + h) n(u, v):
//   N ~ (h_u n + A) x (h_v n + B) = A x B + h_u (n x B) + h_v (A x n),
//   A = (R + h) dn/du, B = (R + h) dn/dv   (tangent vectors of length ~g),
// with the mapping's derivatives in closed form:
//   gnomonic  n = w/|w|, w = (X, Y, R):  dn/du = g (e_x - n n_x) / |w|
//   stereo    n = (2x, 2y, 1 - q)/(1 + q), (x, y) = (X, Y)/2R, q = x^2 + y^2:
//             dn/dx = (2(1 + q - 2x^2), -4xy, -4x)/(1 + q)^2, dx/du = g/2R.
// h_u, h_v: central differences of the texel values for grid rays (one-sided
// on the border), the bilinear gradient in the origin's cell for listed rays.
// float32 throughout (an elementwise pass: a few loads and ~80 flops per ray).
// Bound: HBM (lit fractions in, irradiance out, heights once).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "ss_launch.h"

namespace ss {

namespace {

struct ShadeArgs {
    const float* h;
    int64_t pitch;
    int32_t nx, ny, proj, mode;
    int64_t n;
    const float* uv;
    float g, R, cx, cy;
    int32_t n_lights;
    float L[kShadeMaxLights][3];
    float I[kShadeMaxLights];
    const float* lit[kShadeMaxLights];
    float* E;
};

__device__ __forceinline__ void cross3f(const float a[3], const float b[3], float c[3]) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

__global__ void __launch_bounds__(256) shade_kernel(const ShadeArgs a) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < a.n; r += stride) {
        float u, v, hu, hv, h;
        if (a.mode == 0) {
            const int32_t j = (int32_t)(r / a.nx), i = (int32_t)(r - (int64_t)j * a.nx);
            const int32_t il = i > 0 ? i - 1 : i, ir = i < a.nx - 1 ? i + 1 : i;
            const int32_t jl = j > 0 ? j - 1 : j, jr = j < a.ny - 1 ? j + 1 : j;
            const float* row = a.h + (int64_t)j * a.pitch;
            // spans are 1 or 2 texels: halving is exact, so this equals the division
            hu = (__ldg(row + ir) - __ldg(row + il)) * (ir - il == 2 ? 0.5f : 1.0f);
            hv = (__ldg(a.h + (int64_t)jr * a.pitch + i) - __ldg(a.h + (int64_t)jl * a.pitch + i)) *
                 (jr - jl == 2 ? 0.5f : 1.0f);
            h = __ldg(row + i);
            u = (float)i;
            v = (float)j;
        } else {
            u = a.uv[2 * r];
            v = a.uv[2 * r + 1];
            const int32_t i0 = min(max((int32_t)floorf(u), 0), a.nx - 2);
            const int32_t j0 = min(max((int32_t)floorf(v), 0), a.ny - 2);
            const float fu = u - (float)i0, fv = v - (float)j0;
            const float* p = a.h + (int64_t)j0 * a.pitch + i0;
            const float h00 = __ldg(p), h10 = __ldg(p + 1);
            const float h01 = __ldg(p + a.pitch), h11 = __ldg(p + a.pitch + 1);
            hu = (1.0f - fv) * (h10 - h00) + fv * (h11 - h01);
            hv = (1.0f - fu) * (h01 - h00) + fu * (h11 - h10);
            h = (1.0f - fu) * (1.0f - fv) * h00 + fu * (1.0f - fv) * h10 +
                (1.0f - fu) * fv * h01 + fu * fv * h11;
        }
        const float X = (u - a.cx) * a.g, Y = (v - a.cy) * a.g;
        const float rho = a.R + h;
        float n[3], A[3], B[3];
        if (a.proj == 0) {
            const float im = rsqrtf(X * X + Y * Y + a.R * a.R);
            n[0] = X * im;
            n[1] = Y * im;
            n[2] = a.R * im;
            const float k = rho * a.g * im;
            A[0] = k * (1.0f - n[0] * n[0]);
            A[1] = -k * n[1] * n[0];
            A[2] = -k * n[2] * n[0];
            B[0] = -k * n[0] * n[1];
            B[1] = k * (1.0f - n[1] * n[1]);
            B[2] = -k * n[2] * n[1];
        } else {
            const float i2R = 0.5f / a.R, x = X * i2R, y = Y * i2R, q = x * x + y * y;
            const float iq = 1.0f / (1.0f + q);
            n[0] = 2.0f * x * iq;
            n[1] = 2.0f * y * iq;
            n[2] = (1.0f - q) * iq;
            const float k = rho * a.g * i2R * iq * iq;
            A[0] = k * 2.0f * (1.0f + q - 2.0f * x * x);
            A[1] = -k * 4.0f * x * y;
            A[2] = -k * 4.0f * x;
            B[0] = -k * 4.0f * x * y;
            B[1] = k * 2.0f * (1.0f + q - 2.0f * y * y);
            B[2] = -k * 4.0f * y;
        }
        float AB[3], nB[3], An[3];
        cross3f(A, B, AB);
        cross3f(n, B, nB);
        cross3f(A, n, An);
        float N[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) N[k] = AB[k] + hu * nB[k] + hv * An[k];
        const float inv = rsqrtf(N[0] * N[0] + N[1] * N[1] + N[2] * N[2]);
        float E = 0.0f;
        for (int l = 0; l < a.n_lights; ++l) {
            const float c = (N[0] * a.L[l][0] + N[1] * a.L[l][1] + N[2] * a.L[l][2]) * inv;
            E += a.I[l] * __ldg(a.lit[l] + r) * fmaxf(c, 0.0f);
        }
        a.E[r] = E;
    }
}

}  // namespace

cudaError_t launch_shade(const Tile& T, const Rays& R, const ShadeLight* lights, int32_t n_lights,
                         float* E, cudaStream_t s) {
    ShadeArgs a{};
    a.h = T.h;
    a.pitch = T.pitch;
    a.nx = T.nx;
    a.ny = T.ny;
    a.proj = T.proj;
    a.mode = R.mode;
    a.n = R.mode == 0 ? (int64_t)T.nx * T.ny : R.n;
    a.uv = R.uv;
    a.g = (float)T.g;
    a.R = (float)T.R;
    a.cx = (float)T.cx;
    a.cy = (float)T.cy;
    a.n_lights = n_lights;
    for (int l = 0; l < n_lights; ++l) {
        const double ce = cos(lights[l].elevation_rad);
        a.L[l][0] = (float)(ce * sin(lights[l].azimuth_rad));
        a.L[l][1] = (float)(ce * cos(lights[l].azimuth_rad));
        a.L[l][2] = (float)sin(lights[l].elevation_rad);
        a.I[l] = (float)lights[l].intensity;
        a.lit[l] = lights[l].lit;
    }
    a.E = E;
    // one ray per thread (grid-stride only beyond 2^31 threads): every load of a
    // ray is independent, so many rays in flight keep HBM busy
    const int64_t want = (a.n + 255) / 256, cap = (int64_t)1 << 23;
    const int grid = (int)(want < cap ? (want < 1 ? 1 : want) : cap);
    shade_kernel<<<grid, 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace ss
