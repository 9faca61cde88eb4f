// Strips of neighbouring rays within a chunk of rays (see the descent kernels):
// down a column of a rectangular chunk, or runs of consecutive ids.
#pragma once

#include "ss_walk.cuh"

namespace ss {

struct Strip {
    int32_t first, count;
};

__device__ __forceinline__ int32_t strip_count(const ChunkRange& P, int32_t S) {
    if (!P.rect) return (P.cnt + S - 1) / S;
    const int32_t h = P.cnt / P.w;
    return P.w * ((h + S - 1) / S);
}

__device__ __forceinline__ Strip strip_of(const ChunkRange& P, int32_t S, int32_t s) {
    Strip st;
    if (!P.rect) {
        st.first = s * S;
        st.count = min(S, P.cnt - st.first);
    } else {
        const int32_t h = P.cnt / P.w, c = s % P.w, b = s / P.w;
        st.first = b * S * P.w + c;
        st.count = min(S, h - b * S);
    }
    return st;
}

}  // namespace ss
