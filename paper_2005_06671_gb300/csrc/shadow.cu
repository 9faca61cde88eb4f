// Backward kernel and the launchers of all single-tile kernels.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <type_traits>

#include "ss_launch.h"
#include "ss_walk.cuh"

namespace ss {

// ---------------------------------------------------------------- backward
// d light / d (heights, sun) at the forward argmin, FP64 per ray (only rays in
// the penumbra have a non-zero gradient).  backward_ray computes one ray's
// contributions (up to 8 texels and the 5 sun components) and hands them to a
// sink:
//   AtomicSink  heights by float32 atomicAdd; sun summed in FP64 per thread,
//               then one FP64 atomicAdd per block and component;
//   ScanSink    deterministic pass 1: counts contributions per texel (integer
//               atomics) and keeps the largest |contribution| and count;
//   FixedSink   deterministic pass 2: contributions rounded to integers at a
//               power-of-two scale and summed in 64-bit integers (exact,
//               order-free), the sun components likewise.

template <class Sink>
__device__ __forceinline__ void backward_ray(const BwdArgs& a, int64_t r, int32_t j, float gl,
                                             Sink& sink) {
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
    sink.texel(i0, j0, -gc * w[0] / t);
    sink.texel(i0 + 1, j0, -gc * w[1] / t);
    sink.texel(i0, j0 + 1, -gc * w[2] / t);
    sink.texel(i0 + 1, j0 + 1, -gc * w[3] / t);
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
    const double go_s = gc * dcdhp;
    if (ow[0] != 0.0) sink.texel(oi0, oj0, go_s * ow[0]);
    if (ow[1] != 0.0) sink.texel(oi0 + 1, oj0, go_s * ow[1]);
    if (ow[2] != 0.0) sink.texel(oi0, oj0 + 1, go_s * ow[2]);
    if (ow[3] != 0.0) sink.texel(oi0 + 1, oj0 + 1, go_s * ow[3]);
    // sun direction: dc/ds = q/|q| - grad_q h(texel image of q)
    double ce_term = cos_e > 0.0 ? (-G.sin_e / cos_e) : 0.0;
    double gsv[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        double dcds = q[i] / qn - (du * JU[i] + dv * JV[i]);
        gsv[i] = gc * dcds + gd * (c / a.T.alpha) * ce_term * G.nhat[i];
    }
    double gs[5];
    gs[0] = gsv[0] * a.ds_de[0] + gsv[1] * a.ds_de[1] + gsv[2] * a.ds_de[2];
    gs[1] = gsv[0] * a.ds_da[0] + gsv[1] * a.ds_da[1] + gsv[2] * a.ds_da[2];
    gs[2] = gsv[0];
    gs[3] = gsv[1];
    gs[4] = gsv[2];
    sink.sun(gs);
}

// Deterministic mode: header at the start of the workspace, then the per-texel
// counts (uint32, dense nx * ny) and sums (int64).
struct DetHeader {
    unsigned long long max_h;     // largest |texel contribution| (bits of a double >= 0)
    unsigned long long max_s;     // largest |sun component| (bits of a double >= 0)
    unsigned int max_cnt;         // largest per-texel count
    unsigned int pad;
    unsigned long long n_rays;    // rays that contributed
    double scale_h, inv_h;        // 2^S and 2^-S of the texel sums
    double scale_s, inv_s;        // likewise for the sun sums
    long long sun[5];             // the sun sums
};
constexpr size_t kDetHeader = 256;
static_assert(sizeof(DetHeader) <= kDetHeader, "deterministic header");

struct DetWs {
    DetHeader* hdr;
    unsigned int* cnt;
    long long* acc;
};

__host__ __device__ inline size_t det_cnt_offset() { return kDetHeader; }
__host__ __device__ inline size_t det_acc_offset(int64_t n_texels) {
    return (kDetHeader + (size_t)n_texels * 4 + 255) & ~(size_t)255;
}

struct AtomicSink {
    const BwdArgs& a;
    double gs[5];
    __device__ explicit AtomicSink(const BwdArgs& args) : a(args) {
#pragma unroll
        for (int k = 0; k < 5; ++k) gs[k] = 0.0;
    }
    __device__ void texel(int32_t x, int32_t y, double v) {
        atomicAdd(a.grad_h + (int64_t)y * a.grad_pitch + x, (float)v);
    }
    __device__ void sun(const double g[5]) {
#pragma unroll
        for (int k = 0; k < 5; ++k) gs[k] += g[k];
    }
    __device__ void flush() {   // block reduction, one atomic per component
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
};

struct ScanSink {
    const BwdArgs& a;
    DetWs ws;
    double mh, ms;
    unsigned int mc;
    unsigned long long nr;
    __device__ ScanSink(const BwdArgs& args, DetWs w) : a(args), ws(w), mh(0.0), ms(0.0), mc(0),
                                                        nr(0) {}
    __device__ void texel(int32_t x, int32_t y, double v) {
        const unsigned int c = atomicAdd(ws.cnt + (int64_t)y * a.T.nx + x, 1u) + 1u;
        mc = max(mc, c);
        mh = fmax(mh, fabs(v));
    }
    __device__ void sun(const double g[5]) {
#pragma unroll
        for (int k = 0; k < 5; ++k) ms = fmax(ms, fabs(g[k]));
        ++nr;
    }
    __device__ void flush() {   // warp maxima, one atomic per warp
        unsigned long long bh = (unsigned long long)__double_as_longlong(mh);
        unsigned long long bs = (unsigned long long)__double_as_longlong(ms);
        unsigned int c = mc;
        unsigned long long n = nr;
        for (int o = 16; o > 0; o >>= 1) {
            bh = max(bh, __shfl_down_sync(0xffffffffu, bh, o));
            bs = max(bs, __shfl_down_sync(0xffffffffu, bs, o));
            c = max(c, __shfl_down_sync(0xffffffffu, c, o));
            n += __shfl_down_sync(0xffffffffu, n, o);
        }
        if ((threadIdx.x & 31) == 0 && n > 0) {
            atomicMax(&ws.hdr->max_h, bh);
            atomicMax(&ws.hdr->max_s, bs);
            atomicMax(&ws.hdr->max_cnt, c);
            atomicAdd(&ws.hdr->n_rays, n);
        }
    }
};

struct FixedSink {
    const BwdArgs& a;
    DetWs ws;
    double sh, ss;
    long long acc[5];
    __device__ FixedSink(const BwdArgs& args, DetWs w) : a(args), ws(w) {
        sh = ws.hdr->scale_h;
        ss = ws.hdr->scale_s;
#pragma unroll
        for (int k = 0; k < 5; ++k) acc[k] = 0;
    }
    __device__ void texel(int32_t x, int32_t y, double v) {
        const long long q = __double2ll_rn(v * sh);
        if (q != 0)
            atomicAdd(reinterpret_cast<unsigned long long*>(ws.acc + (int64_t)y * a.T.nx + x),
                      (unsigned long long)q);
    }
    __device__ void sun(const double g[5]) {
#pragma unroll
        for (int k = 0; k < 5; ++k) acc[k] += __double2ll_rn(g[k] * ss);
    }
    __device__ void flush() {   // exact integer warp sums, one atomic per warp
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            long long v = acc[k];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if ((threadIdx.x & 31) == 0 && v != 0)
                atomicAdd(reinterpret_cast<unsigned long long*>(&ws.hdr->sun[k]),
                          (unsigned long long)v);
        }
    }
};

template <int kMode>
__device__ __forceinline__ auto make_sink(const BwdArgs& a, const DetWs& ws) {
    if constexpr (kMode == 0) return AtomicSink(a);
    else if constexpr (kMode == 1) return ScanSink(a, ws);
    else return FixedSink(a, ws);
}

// Most rays are skipped (saturated light, zero dL/dlight), so a block first
// gathers the rays of kBwdRounds x blockDim ids that need the FP64 work into
// shared memory, then every thread takes one: full warps of FP64 work instead
// of a lane or two per warp (GB300 runs FP64 at 1/64 of the FP32 rate).
// (The order of the gathered rays varies from run to run; the deterministic
// sinks do not depend on it.)
constexpr int kBwdRounds = 8;

template <int kMode>   // 0 atomic, 1 deterministic scan, 2 deterministic sums
__global__ void __launch_bounds__(256) backward_kernel(const __grid_constant__ BwdArgs a,
                                                       const DetWs ws) {
    __shared__ int64_t s_ray[256 * kBwdRounds];
    __shared__ int32_t s_cnt;
    const int64_t n = ray_count(a.T, a.R);
    typename std::conditional<kMode == 0, AtomicSink,
                              typename std::conditional<kMode == 1, ScanSink, FixedSink>::type>::type
        sink = make_sink<kMode>(a, ws);
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
            if (!isfinite(gg[k])) {   // reported, and the ray is skipped
                if (a.status && kMode != 2) atomicOr(a.status, kDevNonfiniteGrad);
                continue;
            }
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
            backward_ray(a, r, a.argmin[r], a.grad_light[r], sink);
        }
        __syncthreads();   // s_ray and s_cnt are reused by the next chunk
    }
    sink.flush();
}

// Scales of the deterministic sums (one thread): the largest power of two 2^S
// with (largest |value|) (largest count) 2^S < 2^62, so that no partial sum of
// rounded values can leave the int64 range.
__device__ __forceinline__ void det_scale(double m, double n, double& scale, double& inv) {
    if (!(m > 0.0) || !(n > 0.0)) {
        scale = 1.0;
        inv = 1.0;
        return;
    }
    int e;
    frexp(m * n, &e);   // m n < 2^e
    const int S = min(62 - e, 1000);
    scale = ldexp(1.0, S);
    inv = ldexp(1.0, -S);
}

__global__ void det_scale_kernel(DetHeader* h) {
    det_scale(__longlong_as_double((long long)h->max_h), (double)h->max_cnt, h->scale_h,
              h->inv_h);
    det_scale(__longlong_as_double((long long)h->max_s), (double)h->n_rays, h->scale_s,
              h->inv_s);
}

// grad_h += sum 2^-S per texel that received contributions; grad_sun likewise
__global__ void det_finish_kernel(const BwdArgs a, const DetWs ws) {
    const int64_t n = (int64_t)a.T.nx * a.T.ny;
    const double inv = ws.hdr->inv_h;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        if (ws.cnt[k] == 0u) continue;
        const int64_t y = k / a.T.nx, x = k - y * a.T.nx;
        a.grad_h[y * a.grad_pitch + x] += (float)((double)ws.acc[k] * inv);
    }
    if (blockIdx.x == 0 && threadIdx.x < 5)
        a.grad_sun[threadIdx.x] += (double)ws.hdr->sun[threadIdx.x] * ws.hdr->inv_s;
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

size_t backward_det_workspace_bytes(int32_t nx, int32_t ny) {
    const int64_t n = (int64_t)nx * ny;
    return det_acc_offset(n) + (size_t)n * 8;
}

cudaError_t launch_backward(const BwdArgs& a, int block, cudaStream_t s) {
    int64_t n = a.R.mode == 0 ? (int64_t)a.T.nx * a.T.ny : a.R.n;
    const DetWs none{ nullptr, nullptr, nullptr };
    backward_kernel<0><<<resident_grid(backward_kernel<0>, block, n), block, 0, s>>>(a, none);
    return cudaGetLastError();
}

// Deterministic backward: zero the workspace, pass 1 (counts and maxima), the
// scales, pass 2 (integer sums), then the sums added to grad_h / grad_sun.
cudaError_t launch_backward_det(const BwdArgs& a, int block, void* workspace, cudaStream_t s) {
    const int64_t n = a.R.mode == 0 ? (int64_t)a.T.nx * a.T.ny : a.R.n;
    const int64_t nt = (int64_t)a.T.nx * a.T.ny;
    unsigned char* base = static_cast<unsigned char*>(workspace);
    const DetWs ws{ reinterpret_cast<DetHeader*>(base),
                    reinterpret_cast<unsigned int*>(base + det_cnt_offset()),
                    reinterpret_cast<long long*>(base + det_acc_offset(nt)) };
    cudaError_t e = cudaMemsetAsync(workspace, 0, backward_det_workspace_bytes(a.T.nx, a.T.ny), s);
    if (e != cudaSuccess) return e;
    backward_kernel<1><<<resident_grid(backward_kernel<1>, block, n), block, 0, s>>>(a, ws);
    det_scale_kernel<<<1, 1, 0, s>>>(ws.hdr);
    backward_kernel<2><<<resident_grid(backward_kernel<2>, block, n), block, 0, s>>>(a, ws);
    det_finish_kernel<<<resident_grid(det_finish_kernel, 256, nt), 256, 0, s>>>(a, ws);
    return cudaGetLastError();
}

}  // namespace ss
