// Steps S2 and S3: local density rho (Eq. 3, Algorithm 1) and nearest-higher
// nh / separation delta (Eq. 4, Algorithm 2): the shared arithmetic and the
// per-hit forms, which the tile kernels in density_tile.cuh use.
//
// Hits are read in grid (sorted) order.  The window of Eq. 1 is the set of
// bins met by [x +- R] x [y +- R]; bins of one grid row are adjacent in the
// sorted array, so a window row is one contiguous run.  Each sorted hit is
// one float4 (x, y, w, id), so a candidate costs one 16-byte load.
//
// rho_i is the exact sum over N_dc(i) of the terms chi(d_ij) w_j (flat chi =
// 1 unless the context asks for the Gaussian or exponential kernel that Eq. 3
// names; chi is computed by chi_exp, bit-reproducible), rounded once to the
// nearest fp32: a function of the neighbour set alone, so the window is read
// in any order.  The kernel adds the terms with an error-free transformation
// (TwoSum: s + t = s' + e exactly) into a running sum s and an error sum c,
// and proves c exact from the smallest term and the largest |s| (below);
// then s + c is the exact sum and one fp32 addition rounds it correctly.
// When the proof fails (terms over more than ~24 binary orders of magnitude,
// or an overflow) an integer accumulator recomputes the sum exactly.  With
// the flat chi the terms are the weights themselves, and an event whose
// weights span few enough binary orders (the fill records each event's
// exponent range) is summed in 64-bit fixed point instead: every weight is an
// integer multiple of the event's smallest weight's last place, so the sum is
// an exact integer, rounded once at the end.
#pragma once

#include <climits>

#include "device_common.cuh"

namespace clue {

struct Window {
    int lx, hx, ly, hy;
};

__device__ __forceinline__ Window window_of(float xi, float yi, float dr, const EventDesc &ev) {
    const float rx = win_half(dr, xi), ry = win_half(dr, yi);
    Window w;
    w.lx = axis_bin(__fsub_rn(xi, rx), ev.xmin, ev.inv_s, ev.nbx);
    w.hx = axis_bin(__fadd_rn(xi, rx), ev.xmin, ev.inv_s, ev.nbx);
    w.ly = axis_bin(__fsub_rn(yi, ry), ev.ymin, ev.inv_s, ev.nby);
    w.hy = axis_bin(__fadd_rn(yi, ry), ev.ymin, ev.inv_s, ev.nby);
    return w;
}

__device__ __forceinline__ int id_of(const float4 &h) { return __float_as_int(h.w); }

// ---- exact sum of fp32 values -------------------------------------------
//
// A finite fp32 value is an integer multiple of 2^-149 below 2^128, i.e. an
// integer below 2^277 in units of 2^-149; Wide holds such sums exactly as a
// 320-bit two's-complement integer (five 64-bit words, low word first).
struct Wide {
    unsigned long long v[5];
};

__device__ __forceinline__ void wide_add(Wide &a, float t) {
    const unsigned bits = __float_as_uint(t);
    const unsigned ex = (bits >> 23) & 0xffu;
    const unsigned long long mant = ex ? ((bits & 0x7fffffu) | 0x800000u) : (bits & 0x7fffffu);
    const int shift = ex ? (int)ex - 1 : 0;  // |t| = mant 2^(shift - 149)
    const int k = shift >> 6, o = shift & 63;
    const unsigned long long lo = mant << o;
    const unsigned long long hi = o ? mant >> (64 - o) : 0ull;
    const bool neg = bits >> 31;
    unsigned long long carry = 0ull;
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        const unsigned long long d = i == k ? lo : (i == k + 1 ? hi : 0ull);
        const unsigned long long x = a.v[i];
        if (!neg) {
            const unsigned long long s1 = x + d, s2 = s1 + carry;
            carry = (s1 < x) | (s2 < s1);
            a.v[i] = s2;
        } else {
            const unsigned long long d1 = x - d, d2 = d1 - carry;
            carry = (x < d) | (d1 < carry);
            a.v[i] = d2;
        }
    }
}

// The Wide value rounded to the nearest fp32, ties to the even significand.
inline __device__ float wide_round(const Wide &a) {
    const bool neg = a.v[4] >> 63;
    unsigned long long m[5];
    unsigned long long carry = neg ? 1ull : 0ull;  // |a| = ~a + 1 when negative
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        const unsigned long long x = neg ? ~a.v[i] : a.v[i];
        m[i] = x + carry;
        carry = (m[i] < x) ? 1ull : 0ull;
    }
    int top = -1;
#pragma unroll
    for (int i = 0; i < 5; ++i)
        if (m[i]) top = 64 * i + 63 - __clzll((long long)m[i]);
    unsigned bits;
    if (top < 0) {
        bits = 0u;
    } else if (top < 24) {
        bits = (unsigned)m[0];  // a subnormal or the lowest binade: the unit count
    } else {
        int sh = top - 23;  // the kept significand is bits [sh, top]
        auto bit = [&](int i) -> unsigned { return (unsigned)(m[i >> 6] >> (i & 63)) & 1u; };
        unsigned sig = 0u;
        for (int i = 0; i < 24; ++i) sig |= bit(sh + i) << i;
        const unsigned guard = bit(sh - 1);
        bool sticky = false;
        for (int i = 0; i < sh - 1; ++i) sticky = sticky || bit(i);
        if (guard && (sticky || (sig & 1u))) {
            if (++sig == (1u << 24)) {
                sig >>= 1;
                ++sh;
            }
        }
        bits = sh + 1 >= 255 ? 0x7f800000u : ((unsigned)(sh + 1) << 23) | (sig & 0x7fffffu);
    }
    return __uint_as_float(bits | (neg ? 0x80000000u : 0u));
}

// chi(d) w of a neighbour at squared distance d2 (flat: w).
template <int CHI>
__device__ __forceinline__ float term_of(float d2, float w, float inv) {
    if (CHI == 0) return w;
    return __fmul_rn(chi_of<CHI>(d2, inv), w);
}

// rho by the integer accumulator: the rare windows the fast path cannot prove.
// `unit` is nonzero when the records hold fixed-point weights (flat kernel),
// whose weight is then iw * unit, exactly.
template <int CHI>
__device__ __noinline__ float rho_wide(const Buffers &b, int64_t plane, int nbx, Window w,
                                       float xi, float yi, float dc2, float inv, float unit) {
    Wide acc{{0ull, 0ull, 0ull, 0ull, 0ull}};
    for (int by = w.ly; by <= w.hy; ++by) {
        const int64_t row = plane + (int64_t)by * nbx;
        const int e = b.cell_start[row + w.hx + 1];
        for (int u = b.cell_start[row + w.lx]; u < e; ++u) {
            const float4 h = b.sp[u];
            const float d2 = sq_dist(xi, yi, h.x, h.y);
            const float wj = unit != 0.0f ? __fmul_rn(__ll2float_rn(fixed_weight_of(h)), unit) : h.z;
            if (d2 < dc2) wide_add(acc, term_of<CHI>(d2, wj, inv));
        }
    }
    return wide_round(acc);
}

// Why the fast path is exact.  Let every nonzero term be a multiple of
// 2^(g - 150) (g = the biased exponent of the smallest nonzero |term|, at
// least 1).  Then every running sum s_k and every TwoSum error e_k is one too,
// and |e_k| <= ulp(s_k) / 2 <= 2^(E - 151), E the biased exponent of
// max |s_k|.  With m < 2^L terms the exact error sum, and each partial one,
// is a multiple of 2^(g - 150) below 2^(L + E - 151) <= 2^(g - 126) when
// L + E - 25 <= g: at most 24 significant bits, so an fp32 value, and
// c = fl(c + e_k) never rounds.  Then s + c is the exact sum.
//
// The fixed-point path (flat chi).  Let g be the event's smallest max(biased
// exponent, 1) over its nonzero weights and E its largest biased exponent.
// Every weight is mant 2^(max(e, 1) - 150) with mant < 2^24, so w 2^(150 - g)
// is an integer below 2^(24 + E - g): the scaling by a power of two and the
// conversion to a 64-bit integer are exact.  A window of T candidates sums
// fewer than T such integers, below 2^63 when 24 + E - g + bitlen(T) <= 63,
// so the 64-bit sum is exact.  Its conversion to fp32 rounds once (to
// nearest, ties to even) and the scaling back by 2^(g - 150) is exact while
// the result is normal, which g >= 24 ensures (a nonzero sum is at least
// 2^(g - 150)); an overflow gives inf as the correctly rounded sum would.
// Windows past the bound go to the integer accumulator.

// The running state of one hit's TwoSum density (see above).
struct TwoSumAcc {
    float s = 0.0f, c = 0.0f, smax = 0.0f;
    unsigned tmin = 0x7f800000u;  // bits of the smallest nonzero |term|
    int m = 0;
    __device__ __forceinline__ void add(float tv, bool near) {
        const float s1 = __fadd_rn(s, tv);  // TwoSum: s + tv = s1 + err exactly
        const float bb = __fsub_rn(s1, s);
        const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(s1, bb)), __fsub_rn(tv, bb));
        s = s1;
        c = __fadd_rn(c, err);
        smax = fmaxf(smax, fabsf(s1));
        const unsigned ta = __float_as_uint(tv) & 0x7fffffffu;
        tmin = ta ? min(tmin, ta) : tmin;
        m += near;
    }
    // Whether s + c is the exact sum (else the caller takes the integer
    // accumulator).
    __device__ __forceinline__ bool exact() const {
        const int g = max((int)(tmin >> 23), 1);  // 2^(g - 150): last place
        const int E = max((int)(__float_as_uint(smax) >> 23), 1);
        const int L = 32 - __clz(m);
        return E < 255 && L + E - 25 <= g;
    }
};

// rho of one sorted hit q by a walk over its window in global memory (one
// thread per hit): the general form, for tiles the staged forms do not take.
template <int CHI>
__device__ __forceinline__ float rho_of_hit(const Buffers &b, const Params &p,
                                            const EventDesc &ev, const FixedW &fw, float4 me,
                                            int lay) {
    const int64_t plane = ev.cell_off + (int64_t)lay * ev.nbx * ev.nby;
    const Window w = window_of(me.x, me.y, p.rwin_rho, ev);
    if (CHI == 0 && fw.on) {
        long long acc = 0;
        unsigned T = 0;
        for (int by = w.ly; by <= w.hy; ++by) {
            const int64_t row = plane + (int64_t)by * ev.nbx;
            const int u0 = b.cell_start[row + w.lx], e = b.cell_start[row + w.hx + 1];
            T += (unsigned)(e - u0);
            for (int u = u0; u < e; ++u) {  // branch-free body
                const float4 h = b.sp[u];
                const float d2 = sq_dist(me.x, me.y, h.x, h.y);
                acc += d2 < p.dc2 ? fixed_weight_of(h) : 0ll;
            }
        }
        return 32 - __clz(T) <= fw.budget
                   ? __fmul_rn(__ll2float_rn(acc), fw.unit)
                   : rho_wide<CHI>(b, plane, ev.nbx, w, me.x, me.y, p.dc2, p.chi_inv, fw.unit);
    }
    TwoSumAcc a;
    for (int by = w.ly; by <= w.hy; ++by) {
        const int64_t row = plane + (int64_t)by * ev.nbx;
        const int e = b.cell_start[row + w.hx + 1];
        for (int u = b.cell_start[row + w.lx]; u < e; ++u) {  // branch-free body
            const float4 h = b.sp[u];
            const float d2 = sq_dist(me.x, me.y, h.x, h.y);
            const bool near = d2 < p.dc2;
            a.add(near ? term_of<CHI>(d2, h.z, p.chi_inv) : 0.0f, near);
        }
    }
    return a.exact() ? __fadd_rn(a.s, a.c)
                     : rho_wide<CHI>(b, plane, ev.nbx, w, me.x, me.y, p.dc2, p.chi_inv, 0.0f);
}

// The (d2, j) key that starts an nh search: d2 >= 0, so its float bits order
// like its value, and starting at (bits(d_m^2), 0) folds in the strict test
// d2 < d_m^2.
__device__ __forceinline__ unsigned long long nh_none(const Params &p) {
    return (unsigned long long)__float_as_uint(p.dm2) << 32;
}

__device__ __forceinline__ unsigned long long nh_key(float d2, int j) {
    return ((unsigned long long)__float_as_uint(d2) << 32) | (unsigned)j;
}

// Sorted position u as the nh search reads it: (x, y, rho, id).  The separate
// density kernels keep it as one record; the fused kernel's rho array and the
// sorted records give it in three loads.
__device__ __forceinline__ float4 nh_record(const Buffers &b, const Params &p, int64_t u) {
    if (!p.fused) return b.spr[u];
    const float4 r = b.sp[u];
    return make_float4(r.x, r.y, b.rho[u], __int_as_float(b.sid[u]));
}

// Store rho of sorted position q (at x, y) where this run's nh reads it.
__device__ __forceinline__ void store_rho(const Buffers &b, const Params &p, int64_t q, float x,
                                          float y, float r) {
    if (p.fused)
        b.rho[q] = r;
    else
        b.spr[q] = make_float4(x, y, r, __int_as_float(b.sid[q]));
}

// nh_i by a walk over i's window in global memory (one thread per hit): over
// the window of radius d_m, the (d2, j)-lexicographic minimum among hits with
// d2 < d_m^2 and rho_j > rho_i (the minimum is order-free).
__device__ __forceinline__ unsigned long long nh_of_hit(const Buffers &b, const Params &p,
                                                       const EventDesc &ev, float xi, float yi,
                                                       float ri, int lay) {
    const int64_t plane = ev.cell_off + (int64_t)lay * ev.nbx * ev.nby;
    const Window w = window_of(xi, yi, p.rwin_nh, ev);
    unsigned long long best = nh_none(p);
    for (int by = w.ly; by <= w.hy; ++by) {
        const int64_t row = plane + (int64_t)by * ev.nbx;
        const int e = b.cell_start[row + w.hx + 1];
        for (int u = b.cell_start[row + w.lx]; u < e; ++u) {  // branch-free body
            const float4 h = nh_record(b, p, u);
            const float d2 = sq_dist(xi, yi, h.x, h.y);
            const unsigned long long k = nh_key(d2, __float_as_int(h.w));
            best = (h.z > ri && k < best) ? k : best;
        }
    }
    return best;
}

// The seed / outlier decision of Sec. 2.2 for sorted hit q (hit g), which
// needs only its rho, delta and nh: seed, outlier, or a follower of nh
// (Algorithm 3), stored as one code by hit (the scattered store this step
// cannot avoid); delta^2 and nh also go, in sorted order (coalesced), to an
// 8-byte record the intermediates export reads.
__device__ __forceinline__ void nh_store(const Buffers &b, const Params &p, int64_t q, int g,
                                         float ri, unsigned long long best) {
    const bool found = best != nh_none(p);
    const float d2v = found ? __uint_as_float((unsigned)(best >> 32))
                            : __int_as_float(0x7f800000);  // +inf (Eq. 4)
    const int nhj = found ? (int)(unsigned)best : -1;
    b.hr[q] = make_float2(d2v, __int_as_float(nhj));
    const bool seed = (ri > p.rhoc) && (d2v > p.dcs2);
    const bool outl = (ri < p.rhoc) && (d2v > p.dos2);
    const int code = seed ? CODE_SEED : outl ? CODE_OUTLIER : (nhj >= 0 ? nhj : CODE_NOISE);
    b.code[g] = code;
    if (p.chase && seed) atomicOr(&b.sbits[g >> 5], 1u << (g & 31));
    if (!p.chase && code >= 0) b.frank[g] = atomicAdd(&b.fcount[code], 1);
}

}  // namespace clue
