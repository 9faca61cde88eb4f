// Maximum-mipmap builder (Sec. 3.2 "Maximum mipmaps": each level texel is the
// maximum of the texels it covers one level down).
//
// One pass reads a 64x64 tile of its input level with coalesced float4 loads
// and writes the up-to-6 coarser levels of that tile (32x32 ... 1x1): level 1
// straight from registers, the rest from shared memory, so level 0 is read
// from HBM exactly once and every coarser level is written once.  Passes repeat on the last level
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
    float* stats;                       // (max, min, non-finite count as uint32)
    int32_t write_min;                  // pass 0: fold the tile minimum into stats[1] and
                                        // count its non-finite texels into stats[2]
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

// One 64x64 input tile per block.  Thread t owns input rows 2(t/8), 2(t/8)+1
// and columns 8(t%8) .. 8(t%8)+7: it loads them as four float4 (a warp reads
// eight full 256-byte row segments), reduces them in registers to four
// level-1 texels (one float4 store), and leaves the 32x32 level-1 tile in
// shared memory for the coarser levels.
template <bool kVec4>
__global__ void __launch_bounds__(256) mip_pass_kernel(const MipPass a) {
    __shared__ __align__(16) float lv1[32 * 32];
    __shared__ __align__(16) float lv2[16 * 16];
    __shared__ float wmin[8];
    __shared__ uint32_t wbad[8];
    const int tid = threadIdx.x;
    const int x0 = blockIdx.x * kTile, y0 = blockIdx.y * kTile;
    const int rp = tid >> 3, cb = tid & 7;
    const int y = y0 + 2 * rp, x = x0 + 8 * cb;
    float v[2][8];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int yy = y + r;
        const bool row_ok = yy < a.in_h;
        const float* src = a.in + (int64_t)yy * a.in_pitch + x;
        if (kVec4 && row_ok && x + 7 < a.in_w) {
            const float4 p0 = __ldg(reinterpret_cast<const float4*>(src));
            const float4 p1 = __ldg(reinterpret_cast<const float4*>(src + 4));
            v[r][0] = p0.x; v[r][1] = p0.y; v[r][2] = p0.z; v[r][3] = p0.w;
            v[r][4] = p1.x; v[r][5] = p1.y; v[r][6] = p1.z; v[r][7] = p1.w;
        } else {
#pragma unroll
            for (int c = 0; c < 8; ++c)
                v[r][c] = (row_ok && x + c < a.in_w) ? __ldg(src + c) : -INFINITY;
        }
    }
    if (a.write_min) {
        float m = INFINITY;
        uint32_t bad = 0;   // non-finite texels (fminf/fmaxf skip NaN; infinities count too)
#pragma unroll
        for (int r = 0; r < 2; ++r)
#pragma unroll
            for (int c = 0; c < 8; ++c)
                if (y + r < a.in_h && x + c < a.in_w) {
                    m = fminf(m, v[r][c]);
                    bad += isfinite(v[r][c]) ? 0u : 1u;
                }
        for (int o = 16; o > 0; o >>= 1) m = fminf(m, __shfl_down_sync(0xffffffffu, m, o));
        bad = __reduce_add_sync(0xffffffffu, bad);
        if ((tid & 31) == 0) {
            wmin[tid >> 5] = m;
            wbad[tid >> 5] = bad;
        }
    }
    // level 1 from registers: texels (x0/2 + 4cb + k, y0/2 + rp), k = 0..3
    float4 o1;
    o1.x = fmaxf(fmaxf(v[0][0], v[0][1]), fmaxf(v[1][0], v[1][1]));
    o1.y = fmaxf(fmaxf(v[0][2], v[0][3]), fmaxf(v[1][2], v[1][3]));
    o1.z = fmaxf(fmaxf(v[0][4], v[0][5]), fmaxf(v[1][4], v[1][5]));
    o1.w = fmaxf(fmaxf(v[0][6], v[0][7]), fmaxf(v[1][6], v[1][7]));
    reinterpret_cast<float4*>(lv1)[rp * 8 + cb] = o1;
    {
        const int gx = (x0 >> 1) + 4 * cb, gy = (y0 >> 1) + rp;
        if (gy < a.out_h[0]) {
            float* dst = a.out[0] + (int64_t)gy * a.out_pitch[0] + gx;
            if (gx + 3 < a.out_w[0]) {
                *reinterpret_cast<float4*>(dst) = o1;   // level pitches are multiples of 4
            } else {
                if (gx < a.out_w[0]) dst[0] = o1.x;
                if (gx + 1 < a.out_w[0]) dst[1] = o1.y;
                if (gx + 2 < a.out_w[0]) dst[2] = o1.z;
            }
        }
        if (a.write_max && a.nlev == 1 && a.out_w[0] == 1 && a.out_h[0] == 1 && gx == 0 && gy == 0)
            a.stats[0] = o1.x;
    }
    __syncthreads();
    if (a.write_min && tid == 0) {
        float m = wmin[0];
        uint32_t bad = wbad[0];
        for (int w = 1; w < 8; ++w) {
            m = fminf(m, wmin[w]);
            bad += wbad[w];
        }
        if (m < INFINITY) atomic_min_float(a.stats + 1, m);
        if (bad) atomicAdd(reinterpret_cast<unsigned int*>(a.stats + 2), bad);
    }
    // levels 2.. (16x16 -> 1x1) through shared memory, sizes known at compile time
    float* src = lv1;
    float* dst = lv2;
#pragma unroll
    for (int l = 1; l < kPassLevels; ++l) {
        if (l >= a.nlev) break;
        const int s = kTile >> l, h2 = s >> 1;   // input size s, output size h2
        if (tid < h2 * h2) {
            const int oy = tid / h2, ox = tid - oy * h2;
            const float* p = src + (2 * oy) * s + 2 * ox;
            const float m = fmaxf(fmaxf(p[0], p[1]), fmaxf(p[s], p[s + 1]));
            dst[tid] = m;
            const int gx = (x0 >> (l + 1)) + ox, gy = (y0 >> (l + 1)) + oy;
            if (gx < a.out_w[l] && gy < a.out_h[l]) {
                a.out[l][(int64_t)gy * a.out_pitch[l] + gx] = m;
                if (a.write_max && l == a.nlev - 1 && a.out_w[l] == 1 && a.out_h[l] == 1)
                    a.stats[0] = m;
            }
        }
        __syncthreads();
        float* t = src;
        src = dst;
        dst = t;
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
    // stats[1] starts at a large positive float (bytes 0x7f7f7f7f = 3.39e38),
    // the non-finite count stats[2] at 0
    cudaError_t e = cudaMemsetAsync(stats + 1, 0x7f, sizeof(float), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(stats + 2, 0, sizeof(float), s);
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
