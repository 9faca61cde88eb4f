// Backward kernel and the launchers of all single-tile kernels.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "ss_launch.h"
#include "ss_walk.cuh"

namespace ss {

// ---------------------------------------------------------------- backward
// d light / d (heights, sun) at the forward argmin, FP64 per ray (only rays in
// the penumbra have a non-zero gradient).  Heights: atomicAdd (float32);
// sun: block reduction in FP64, then one atomicAdd per block and component.

// Gradient contributions of ray r (argmin j >= 1, dL/dlight gl != 0): height
// texels by atomicAdd, the sun components accumulated into gs.
__device__ __forceinline__ void backward_ray(const BwdArgs& a, int64_t r, int32_t j, float gl,
                                             double gs[5]) {
    double up, vp, hp, href, ow[4];
    int32_t oi0, oj0;
    ray_origin(a.T, a.R, r, up, vp, hp, href, oi0, oj0, ow);
    Geom64 G;
    geom64_any(a.T, up, vp, hp, G, a.T.proj != 0);
    double U, V;
    double c = leaf_cost64(a.T, G, j, a.T.proj != 0, &U, &V);
    const double cos_e = cos_elev(G);
    double d = c * cos_e / a.T.alpha;
    if (!(d > -1.0 && d < 1.0)) return;
    double gd = (double)gl * (2.0 / M_PI) * sqrt(1.0 - d * d);   // dL/dd
    double gc = gd * cos_e / a.T.alpha;                         // dL/dc
    double t = (double)j * a.T.delta;
    // sample texels and the bilinear gradient at (U, V)
    int32_t i0 = (int32_t)floor(U), j0 = (int32_t)floor(V);
    i0 = min(max(i0, 0), a.T.nx - 2);
    j0 = min(max(j0, 0), a.T.ny - 2);
    double fu = U - i0, fv = V - j0;
    const float* hr = a.T.h + (int64_t)j0 * a.T.pitch + i0;
    double h00 = hr[0], h10 = hr[1], h01 = hr[a.T.pitch], h11 = hr[a.T.pitch + 1];
    double du = (1.0 - fv) * (h10 - h00) + fv * (h11 - h01);
    double dv = (1.0 - fu) * (h01 - h00) + fu * (h11 - h10);
    double w[4] = { (1.0 - fu) * (1.0 - fv), fu * (1.0 - fv), (1.0 - fu) * fv, fu * fv };
    float* gp = a.grad_h + (int64_t)j0 * a.grad_pitch + i0;
    atomicAdd(gp, (float)(-gc * w[0] / t));
    atomicAdd(gp + 1, (float)(-gc * w[1] / t));
    atomicAdd(gp + a.grad_pitch, (float)(-gc * w[2] / t));
    atomicAdd(gp + a.grad_pitch + 1, (float)(-gc * w[3] / t));
    // texel-coordinate Jacobians dU/dq, dV/dq at the sample point q = p + t s
    const double q[3] = { G.rho * G.nhat[0] + t * a.T.sx, G.rho * G.nhat[1] + t * a.T.sy,
                          G.rho * G.nhat[2] + t * a.T.sz };
    const double qn = sqrt(G.rho * G.rho + t * (2.0 * G.rho * G.sin_e + t));   // |q|
    double JU[3], JV[3];
    if (a.T.proj == 0) {        // U = (R/g) q_x / q_z + c_x
        const double kq = a.T.R / a.T.g;
        JU[0] = kq / q[2]; JU[1] = 0.0; JU[2] = -kq * q[0] / (q[2] * q[2]);
        JV[0] = 0.0; JV[1] = kq / q[2]; JV[2] = -kq * q[1] / (q[2] * q[2]);
    } else {                    // U = (2R/g) q_x / (|q| + q_z) + c_x
        const double kq = 2.0 * a.T.R / a.T.g, D = qn + q[2], iD = 1.0 / D;
        double dD[3] = { q[0] / qn, q[1] / qn, q[2] / qn + 1.0 };
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            JU[i] = kq * ((i == 0 ? iD : 0.0) - q[0] * dD[i] * iD * iD);
            JV[i] = kq * ((i == 1 ? iD : 0.0) - q[1] * dD[i] * iD * iD);
        }
    }
    // origin height: moves the ray's origin (and every q) along n_p
    const double dHdhp = (G.rho + t * G.sin_e) / qn;
    const double dUdhp = JU[0] * G.nhat[0] + JU[1] * G.nhat[1] + JU[2] * G.nhat[2];
    const double dVdhp = JV[0] * G.nhat[0] + JV[1] * G.nhat[1] + JV[2] * G.nhat[2];
    const double dcdhp = (dHdhp - (du * dUdhp + dv * dVdhp)) / t;
    float* go = a.grad_h + (int64_t)oj0 * a.grad_pitch + oi0;
    const double go_s = gc * dcdhp;
    if (ow[0] != 0.0) atomicAdd(go, (float)(go_s * ow[0]));
    if (ow[1] != 0.0) atomicAdd(go + 1, (float)(go_s * ow[1]));
    if (ow[2] != 0.0) atomicAdd(go + a.grad_pitch, (float)(go_s * ow[2]));
    if (ow[3] != 0.0) atomicAdd(go + a.grad_pitch + 1, (float)(go_s * ow[3]));
    // sun direction: dc/ds = q/|q| - grad_q h(texel image of q)
    double ce_term = cos_e > 0.0 ? (-G.sin_e / cos_e) : 0.0;
    double gsv[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        double dcds = q[i] / qn - (du * JU[i] + dv * JV[i]);
        gsv[i] = gc * dcds + gd * (c / a.T.alpha) * ce_term * G.nhat[i];
    }
    gs[0] += gsv[0] * a.ds_de[0] + gsv[1] * a.ds_de[1] + gsv[2] * a.ds_de[2];
    gs[1] += gsv[0] * a.ds_da[0] + gsv[1] * a.ds_da[1] + gsv[2] * a.ds_da[2];
    gs[2] += gsv[0];
    gs[3] += gsv[1];
    gs[4] += gsv[2];
}

// Most rays are skipped (saturated light, zero dL/dlight), so a block first
// gathers the rays of kBwdRounds x blockDim ids that need the FP64 work into
// shared memory, then every thread takes one: full warps of FP64 work instead
// of a lane or two per warp (GB300 runs FP64 at 1/64 of the FP32 rate).
constexpr int kBwdRounds = 8;

__global__ void __launch_bounds__(256) backward_kernel(const BwdArgs a) {
    __shared__ int64_t s_ray[256 * kBwdRounds];
    __shared__ int32_t s_cnt;
    const int64_t n = ray_count(a.T, a.R);
    double gs[5] = { 0.0, 0.0, 0.0, 0.0, 0.0 };
    const int64_t chunk = (int64_t)blockDim.x * kBwdRounds;
    for (int64_t base = (int64_t)blockIdx.x * chunk; base < n; base += (int64_t)gridDim.x * chunk) {
        if (threadIdx.x == 0) s_cnt = 0;
        __syncthreads();
        // all loads of the round first (independent, in flight together), then the tests
        int32_t jj[kBwdRounds];
        float gg[kBwdRounds], cc[kBwdRounds];
#pragma unroll
        for (int k = 0; k < kBwdRounds; ++k) {
            const int64_t r = base + (int64_t)k * blockDim.x + threadIdx.x;
            const bool in = r < n;
            jj[k] = in ? a.argmin[r] : 0;
            gg[k] = in ? a.grad_light[r] : 0.0f;
            cc[k] = (in && a.cost) ? a.cost[r] : 0.0f;
        }
#pragma unroll
        for (int k = 0; k < kBwdRounds; ++k) {
            const int64_t r = base + (int64_t)k * blockDim.x + threadIdx.x;
            if (jj[k] < 1 || gg[k] == 0.0f) continue;
            // the forward's float32 cost rules out rays whose light is certainly
            // saturated (the same test the forward uses before its FP64 re-evaluation)
            if (a.cost && fabsf(cc[k]) * cos_elev_f32(a.T, a.R, r, a.T.proj != 0) >=
                              1.001f * a.T.alpha_f)
                continue;
            s_ray[atomicAdd(&s_cnt, 1)] = r;
        }
        __syncthreads();
        const int cnt = s_cnt;
        for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
            const int64_t r = s_ray[i];
            backward_ray(a, r, a.argmin[r], a.grad_light[r], gs);
        }
        __syncthreads();   // s_ray and s_cnt are reused by the next chunk
    }
    // block reduction of the sun gradient
    __shared__ double red[5][8];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        double v = gs[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) red[k][threadIdx.x >> 5] = v;
    }
    __syncthreads();
    if (threadIdx.x < 5) {
        double v = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[threadIdx.x][w];
        if (v != 0.0) atomicAdd(a.grad_sun + threadIdx.x, v);
    }
}

// ---------------------------------------------------------------- launchers
static int g_sm_count = 0;

int device_sm_count() {
    if (g_sm_count == 0) {
        int dev = 0, n = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess)
            g_sm_count = n;
        else
            g_sm_count = 1;
    }
    return g_sm_count;
}

// Grid-stride kernels: one wave of resident blocks (occupancy x SMs), fewer
// when there is not enough work.
template <typename K>
static int resident_grid(K kernel, int block, int64_t n_threads) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, 0) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    int64_t cap = (int64_t)device_sm_count() * per_sm;
    int64_t want = (n_threads + block - 1) / block;
    if (want < 1) want = 1;
    return (int)(want < cap ? want : cap);
}

cudaError_t launch_dp_forward_gnomonic(const FwdArgs& a, int block, cudaStream_t s);
cudaError_t launch_dp_forward_stereo(const FwdArgs& a, int block, cudaStream_t s);
cudaError_t launch_uniform_forward_gnomonic(const FwdArgs& a, int block, cudaStream_t s);
cudaError_t launch_uniform_forward_stereo(const FwdArgs& a, int block, cudaStream_t s);

cudaError_t launch_dp_forward(const FwdArgs& a, int block, cudaStream_t s) {
    return a.T.proj == 0 ? launch_dp_forward_gnomonic(a, block, s)
                         : launch_dp_forward_stereo(a, block, s);
}

cudaError_t launch_uniform_forward(const FwdArgs& a, int block, cudaStream_t s) {
    return a.T.proj == 0 ? launch_uniform_forward_gnomonic(a, block, s)
                         : launch_uniform_forward_stereo(a, block, s);
}

cudaError_t launch_backward(const BwdArgs& a, int block, cudaStream_t s) {
    int64_t n = a.R.mode == 0 ? (int64_t)a.T.nx * a.T.ny : a.R.n;
    backward_kernel<<<resident_grid(backward_kernel, block, n), block, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace ss
