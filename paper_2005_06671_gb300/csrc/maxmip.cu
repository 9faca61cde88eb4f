// Maximum-mipmap builder (Sec. 3.2 "Maximum mipmaps": each level texel is the
// maximum of the texels it covers one level down).
//
// One pass reads a 64x64 tile of its input level with coalesced float4 loads
// into shared memory and writes the up-to-6 coarser levels of that tile
// (32x32 ... 1x1) from shared memory, so level 0 is read from HBM exactly once
// and every coarser level is written once.  Passes repeat on the last level
// written until the pyramid reaches 1x1 (4096^2: 2 passes; 16384^2: 3).
// Children outside the level are ignored (treated as -inf).  Max is exact, so
// the result is bit-identical to any other evaluation order.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "ss_launch.h"

namespace ss {

namespace {

constexpr int kTile = 64;
constexpr int kPassLevels = 6;   // 64 -> 1

struct MipPass {
    const float* in;
    int64_t in_pitch;
    int32_t in_w, in_h;
    int32_t nlev;                       // levels written by this pass (<= 6)
    float* out[kPassLevels];
    int64_t out_pitch[kPassLevels];
    int32_t out_w[kPassLevels], out_h[kPassLevels];
    float* stats;                       // (max, min)
    int32_t write_min;                  // pass 0: fold the tile minimum into stats[1]
    int32_t write_max;                  // last pass: store the 1x1 level into stats[0]
};

__device__ __forceinline__ void atomic_min_float(float* addr, float v) {
    // Float ordering on the bit patterns: non-negative floats order as signed
    // ints, negative floats order inversely as unsigned ints.
    if (v >= 0.0f)
        atomicMin(reinterpret_cast<int*>(addr), __float_as_int(v));
    else
        atomicMax(reinterpret_cast<unsigned int*>(addr), __float_as_uint(v));
}

template <bool kVec4>
__global__ void __launch_bounds__(256) mip_pass_kernel(const MipPass a) {
    __shared__ __align__(16) float buf0[kTile * kTile];
    __shared__ __align__(16) float buf1[(kTile / 2) * (kTile / 2)];
    const int tid = threadIdx.x;
    const int x0 = blockIdx.x * kTile, y0 = blockIdx.y * kTile;
    float tmin = INFINITY;
    if (kVec4) {
        // 64 rows x 16 float4; in_pitch % 4 == 0 and 16-byte aligned base
#pragma unroll
        for (int it = 0; it < 4; ++it) {
            int idx = it * 256 + tid;
            int row = idx >> 4, c4 = idx & 15;
            int y = y0 + row, x = x0 + c4 * 4;
            float4 v = make_float4(-INFINITY, -INFINITY, -INFINITY, -INFINITY);
            if (y < a.in_h) {
                const float* src = a.in + (int64_t)y * a.in_pitch + x;
                if (x + 3 < a.in_w) {
                    v = __ldg(reinterpret_cast<const float4*>(src));
                } else {
                    if (x < a.in_w) v.x = __ldg(src);
                    if (x + 1 < a.in_w) v.y = __ldg(src + 1);
                    if (x + 2 < a.in_w) v.z = __ldg(src + 2);
                }
            }
            reinterpret_cast<float4*>(buf0)[row * (kTile / 4) + c4] = v;
            if (a.write_min) {
                if (y < a.in_h) {
                    if (x < a.in_w) tmin = fminf(tmin, v.x);
                    if (x + 1 < a.in_w) tmin = fminf(tmin, v.y);
                    if (x + 2 < a.in_w) tmin = fminf(tmin, v.z);
                    if (x + 3 < a.in_w) tmin = fminf(tmin, v.w);
                }
            }
        }
    } else {
#pragma unroll 4
        for (int it = 0; it < 16; ++it) {
            int idx = it * 256 + tid;
            int row = idx >> 6, col = idx & 63;
            int y = y0 + row, x = x0 + col;
            float v = -INFINITY;
            if (y < a.in_h && x < a.in_w) {
                v = __ldg(a.in + (int64_t)y * a.in_pitch + x);
                tmin = fminf(tmin, v);
            }
            buf0[row * kTile + col] = v;
        }
    }
    __syncthreads();
    if (a.write_min) {
        for (int o = 16; o > 0; o >>= 1) tmin = fminf(tmin, __shfl_down_sync(0xffffffffu, tmin, o));
        __shared__ float wmin[8];
        if ((tid & 31) == 0) wmin[tid >> 5] = tmin;
        __syncthreads();
        if (tid == 0) {
            float m = wmin[0];
            for (int w = 1; w < 8; ++w) m = fminf(m, wmin[w]);
            if (m < INFINITY) atomic_min_float(a.stats + 1, m);
        }
    }
    // successive 2x2 reductions in shared memory: src (size s) -> dst (size s/2)
    float* src = buf0;
    float* dst = buf1;
    int s = kTile;
    for (int l = 0; l < a.nlev; ++l) {
        const int h2 = s >> 1;
        for (int idx = tid; idx < h2 * h2; idx += 256) {
            int oy = idx / h2, ox = idx - oy * h2;
            const float* p = src + (2 * oy) * s + 2 * ox;
            float m = fmaxf(fmaxf(p[0], p[1]), fmaxf(p[s], p[s + 1]));
            dst[idx] = m;
            int gx = (x0 >> (l + 1)) + ox, gy = (y0 >> (l + 1)) + oy;
            if (gx < a.out_w[l] && gy < a.out_h[l]) {
                a.out[l][(int64_t)gy * a.out_pitch[l] + gx] = m;
                if (a.write_max && l == a.nlev - 1 && a.out_w[l] == 1 && a.out_h[l] == 1)
                    a.stats[0] = m;
            }
        }
        __syncthreads();
        float* t = src;   // ping-pong: the level just read becomes the next destination
        src = dst;
        dst = t;
        s = h2;
    }
}

}  // namespace

bool mip_layout(int32_t nx, int32_t ny, MipLayout* L) {
    if (nx < 1 || ny < 1 || nx > 65536 || ny > 65536) return false;
    int32_t w = nx, h = ny, l = 0;
    int64_t cur = 0;
    L->w[0] = nx;
    L->h[0] = ny;
    L->pitch[0] = 0;
    L->offset[0] = 0;
    while (w > 1 || h > 1) {
        w = (w + 1) / 2;
        h = (h + 1) / 2;
        ++l;
        if (l >= kMaxLevels) return false;
        L->w[l] = w;
        L->h[l] = h;
        L->pitch[l] = ((int64_t)w + 3) / 4 * 4;
        cur = (cur + 63) / 64 * 64;
        L->offset[l] = cur;
        cur += L->pitch[l] * h;
    }
    L->levels = l + 1;
    L->stats_offset = (cur + 63) / 64 * 64;
    L->total_elems = L->stats_offset + 64;
    return true;
}

cudaError_t launch_build_maxmip(const float* h, int32_t nx, int32_t ny, int64_t pitch,
                                float* mip, const MipLayout& L, cudaStream_t s) {
    float* stats = mip + L.stats_offset;
    // stats[1] starts at a large positive float (bytes 0x7f7f7f7f = 3.39e38)
    cudaError_t e = cudaMemsetAsync(stats + 1, 0x7f, sizeof(float), s);
    if (e != cudaSuccess) return e;
    if (L.levels == 1) {
        // 1x1 heightfield: max = min = the single value
        e = cudaMemcpyAsync(stats, h, sizeof(float), cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return e;
        return cudaMemcpyAsync(stats + 1, h, sizeof(float), cudaMemcpyDeviceToDevice, s);
    }
    int32_t lin = 0;   // input level of the pass
    bool first = true;
    while (lin < L.levels - 1) {
        MipPass a{};
        a.in = lin == 0 ? h : mip + L.offset[lin];
        a.in_pitch = lin == 0 ? pitch : L.pitch[lin];
        a.in_w = L.w[lin];
        a.in_h = L.h[lin];
        a.nlev = L.levels - 1 - lin < kPassLevels ? L.levels - 1 - lin : kPassLevels;
        for (int k = 0; k < a.nlev; ++k) {
            a.out[k] = mip + L.offset[lin + 1 + k];
            a.out_pitch[k] = L.pitch[lin + 1 + k];
            a.out_w[k] = L.w[lin + 1 + k];
            a.out_h[k] = L.h[lin + 1 + k];
        }
        a.stats = stats;
        a.write_min = first ? 1 : 0;
        a.write_max = (lin + a.nlev == L.levels - 1) ? 1 : 0;
        dim3 grid((a.in_w + kTile - 1) / kTile, (a.in_h + kTile - 1) / kTile);
        bool vec = (a.in_pitch % 4 == 0) && ((reinterpret_cast<uintptr_t>(a.in) & 15) == 0);
        if (vec)
            mip_pass_kernel<true><<<grid, 256, 0, s>>>(a);
        else
            mip_pass_kernel<false><<<grid, 256, 0, s>>>(a);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        lin += a.nlev;
        first = false;
    }
    return cudaSuccess;
}

}  // namespace ss
