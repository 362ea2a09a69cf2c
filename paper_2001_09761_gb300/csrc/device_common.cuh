// Device helpers shared by the CLUE kernels: the fp32 distance, the monotone
// bin map and the search-window half-width.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "clue_internal.h"

namespace clue {

constexpr unsigned FULL_MASK = 0xffffffffu;

// An event's weight range: [0] the min of max(biased exponent, 1), [1] the
// min of 255 - biased exponent, over its finite nonzero weights (all ones:
// none yet).  A CTA gathers its tile's range in shared memory: a warp-wide
// minimum, one shared atomic per warp (every lane of the warp calls it;
// `active` lanes contribute w) ...
__device__ __forceinline__ void weight_range_add(unsigned *s_w, float w, bool active) {
    const unsigned bits = __float_as_uint(w) & 0x7fffffffu;
    const unsigned eb = bits >> 23;
    const bool nz = active && bits != 0u && eb < 255u;
    const unsigned lo = __reduce_min_sync(FULL_MASK, nz ? max(eb, 1u) : 0xffffffffu);
    const unsigned hi = __reduce_min_sync(FULL_MASK, nz ? 255u - eb : 0xffffffffu);
    if ((threadIdx.x & 31) == 0 && lo != 0xffffffffu) {
        atomicMin(&s_w[0], lo);
        atomicMin(&s_w[1], hi);
    }
}

// The same for a (lo, hi) pair a thread has already reduced over its own
// weights (all ones: none).
__device__ __forceinline__ void weight_range_add_bounds(unsigned *s_w, unsigned lo, unsigned hi) {
    lo = __reduce_min_sync(FULL_MASK, lo);
    hi = __reduce_min_sync(FULL_MASK, hi);
    if ((threadIdx.x & 31) == 0 && lo != 0xffffffffu) {
        atomicMin(&s_w[0], lo);
        atomicMin(&s_w[1], hi);
    }
}

// ... and one thread folds it into the event's after a barrier, with an atomic
// only where it lowers the value held (which only falls, so a stale read
// costs at most a redundant atomic).
__device__ __forceinline__ void weight_range_flush(uint32_t *wexp_e, const unsigned *s_w) {
    if (s_w[0] < __ldcg(&wexp_e[0])) atomicMin(&wexp_e[0], s_w[0]);
    if (s_w[1] < __ldcg(&wexp_e[1])) atomicMin(&wexp_e[1], s_w[1]);
}

// The flat kernel's 64-bit fixed point for one event (see rho_stage): on when
// the event's weights span few enough binary orders; scale = 2^(150 - g)
// turns a weight into an exact integer, unit = 2^(g - 150) turns it back, and
// a window of T candidates is exact while bitlen(T) <= budget.
struct FixedW {
    bool on;
    float scale, unit;
    int budget;
};

__device__ __forceinline__ FixedW fixed_weights(const uint32_t *wexp_e, int chi) {
    const unsigned g = wexp_e[0], e = 255u - wexp_e[1];
    FixedW f;
    f.on = chi == 0 && g >= 24u && g <= 254u && e >= g && 25u + (e - g) <= 63u;
    f.scale = f.on ? __uint_as_float((277u - g) << 23) : 0.0f;
    f.unit = f.on ? __uint_as_float((g - 23u) << 23) : 0.0f;
    f.budget = f.on ? 39 - (int)(e - g) : 0;
    return f;
}

// The sorted record of a hit: (x, y, w, id), or under the fixed point
// (x, y, low and high words of the integer weight w 2^(150 - g)).
__device__ __forceinline__ float4 sorted_record(const float4 &r, const FixedW &f) {
    if (!f.on) return r;
    const long long iw = __float2ll_rz(__fmul_rn(r.z, f.scale));
    return make_float4(r.x, r.y, __int_as_float((int)(unsigned)iw), __int_as_float((int)(iw >> 32)));
}

__device__ __forceinline__ long long fixed_weight_of(const float4 &h) {
    return (long long)(((unsigned long long)__float_as_uint(h.w) << 32) | __float_as_uint(h.z));
}

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

// exp(a) for a <= 0 in fp32, from the mathematics: Cody and Waite's
// reduction (W. J. Cody, W. Waite, "Software Manual for the Elementary
// Functions", 1980) a = k ln2 + r with ln2 = L1 + L2 (L1 short, so k L1 is
// exact), |r| <= ln2 / 2, exp(r) by its Taylor series to degree 7 (Horner),
// exp(a) = 2^k exp(r).  Each step is one round-to-nearest fp32 operation in a
// fixed order, so the result is reproducible bit for bit on any IEEE machine.
// a below -87 gives 0 (the result there would be subnormal).
__device__ __forceinline__ float chi_exp(float a) {
    if (!(a > -87.0f)) return 0.0f;
    const float kf = floorf(__fadd_rn(__fmul_rn(a, 1.44269504f), 0.5f));
    const float r = __fadd_rn(__fsub_rn(a, __fmul_rn(kf, 0.693359375f)),
                              __fmul_rn(kf, 2.12194440e-4f));
    float p = 1.98412698e-4f;
    p = __fadd_rn(__fmul_rn(p, r), 1.38888889e-3f);
    p = __fadd_rn(__fmul_rn(p, r), 8.33333333e-3f);
    p = __fadd_rn(__fmul_rn(p, r), 4.16666667e-2f);
    p = __fadd_rn(__fmul_rn(p, r), 1.66666667e-1f);
    p = __fadd_rn(__fmul_rn(p, r), 0.5f);
    p = __fadd_rn(__fmul_rn(p, r), 1.0f);
    p = __fadd_rn(__fmul_rn(p, r), 1.0f);
    return __fmul_rn(p, __int_as_float(((int)kf + 127) << 23));
}

// The kernel chi(d) of Eq. 3 on squared distance d2: flat (1), Gaussian
// exp(-d2 inv) with inv = 1 / (2 s^2), exponential exp(-sqrt(d2) inv) with
// inv = 1 / s.
template <int CHI>
__device__ __forceinline__ float chi_of(float d2, float inv) {
    if (CHI == 1) return chi_exp(-__fmul_rn(d2, inv));
    if (CHI == 2) return chi_exp(-__fmul_rn(__fsqrt_rn(d2), inv));
    return 1.0f;
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
