// Device helpers shared by the CLUE kernels: the fp32 distance, the monotone
// bin map and the search-window half-width.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "clue_internal.h"

namespace clue {

constexpr unsigned FULL_MASK = 0xffffffffu;

// Squared distance in fp32, every operation rounded on its own (no FMA):
// dx = xj - xi, dy = yj - yi, dx*dx + dy*dy.  It is exactly symmetric in i, j.
__device__ __forceinline__ float sq_dist(float xi, float yi, float xj, float yj) {
    const float dx = __fsub_rn(xj, xi);
    const float dy = __fsub_rn(yj, yi);
    return __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
}

// Bin of coordinate v on an axis of nb bins starting at lo, floor((v-lo)/s)
// clamped to [0, nb-1].  Every step is monotone non-decreasing in v, so
// v1 <= v2 implies bin(v1) <= bin(v2); out-of-range coordinates land in the
// edge bins (Sec. 2.1's grid is fixed, hits outside it are kept).
__device__ __forceinline__ int axis_bin(float v, float lo, float inv_s, int nb) {
    float t = floorf(__fmul_rn(__fsub_rn(v, lo), inv_s));
    t = fminf(fmaxf(t, 0.0f), (float)(nb - 1));
    return (int)t;
}

// Half-width of the square search window (Eq. 1) of radius d around a hit at
// coordinate v, given dr = fl(d * (1 + 2^-12)).  A pair that passes the fp32
// test d2 < fl(d*d) is closer than d (1 + 3u) per axis (u = 2^-24); the margin
// d 2^-12 + |v| 2^-20 exceeds that excess plus the rounding of v -/+ half, so
// by monotonicity of axis_bin every true neighbour lies in a window bin.
__device__ __forceinline__ float win_half(float dr, float v) {
    return __fadd_rn(dr, __fmul_rn(fabsf(v), 0x1p-20f));
}

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

template <typename T>
__device__ __forceinline__ T warp_incl_scan(T v) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T u = __shfl_up_sync(FULL_MASK, v, o);
        if (lane_id() >= o) v += u;
    }
    return v;
}

}  // namespace clue
