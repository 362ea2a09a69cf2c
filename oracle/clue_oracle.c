/*
 * CLUE oracle: a plain, slow, single-thread CPU restatement of the clustering
 * of Rovere et al., "CLUE: A Fast Parallel Clustering Algorithm for High
 * Granularity Calorimeters in High Energy Physics" (arXiv 2001.09761).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the reference the CUDA library is
 * checked against.  Only the tests, the smoke check and the benchmark's CPU
 * baseline leg may load it; the library neither includes, links nor calls it,
 * and it shares no code, header or constant with the library.
 *
 * What it computes, step by step in the paper's order:
 *   1. a fixed square grid per layer (Sec. 2.1, Eqs. 1-2), each bin listing
 *      its hits in ascending hit index;
 *   2. local density rho (Eq. 3, Algorithm 1) with the flat kernel chi = 1,
 *      or (oracle_clue_chi) the Gaussian or exponential kernel Eq. 3 names;
 *   3. nearest-higher nh and separation delta (Eq. 4, Algorithm 2);
 *   4. seed / outlier decision and follower registration (Sec. 2.2, Eq. 5,
 *      first half of Algorithm 3);
 *   5. cluster expansion by a stack, seed ids passed down the follower lists
 *      (second half of Algorithm 3).
 *
 * Readings where the paper is silent or ambiguous (each is also listed in the
 * design notes of the repository):
 *   R1  chi is flat: every j with d_ij < d_c adds w_j, j = i included.  The
 *       Gaussian and exponential kernels add fl(chi(d_ij) * w_j), chi computed
 *       by oracle_chi_exp below; the paper gives them no parameters, so their
 *       width s is an input.
 *   R2  d_ij is Euclidean in (x, y) on the same layer only, compared squared in
 *       fp32: dx = x_j - x_i, dy = y_j - y_i, d2 = dx*dx + dy*dy, every
 *       operation rounded to nearest with no fused multiply-add (this file is
 *       built with -ffp-contract=off).  Thresholds are squared once in fp32.
 *       The reported delta is sqrtf(d2).
 *   R3  every comparison is strict, as printed: d < d_c, d < d_m, rho_j > rho_i,
 *       seed iff rho > rho_c and delta > delta_c, outlier iff rho < rho_c and
 *       delta > delta_o.
 *   R4  rho_i is the exact sum of the terms over N_dc(i) (w_j, or fl(chi(d_ij)
 *       * w_j)), rounded once to the nearest fp32, ties to even.  Eq. 3 sums
 *       over a set and fixes no order; the exact sum is the one fp32 value
 *       that depends on the set alone (any fp32 addition order can differ
 *       from it, and from another order, in the last bit).
 *   R5  among nearest-higher candidates at equal d2 the smallest j wins.
 *   R7  a hit that is neither seed nor outlier and has nh = -1 (possible only
 *       when rho == rho_c) is not registered anywhere and stays noise.
 *   R8  cluster ids are 0..k-1 in ascending seed index over the whole event
 *       (all layers), as the k++ of Algorithm 3 gives.
 *   R9  noise gets cluster id -1.
 *   R10 hits outside the grid extent fall into the edge bins; the search
 *       window is widened by a tiny margin so that floating-point rounding can
 *       never drop a true neighbour (the exact d2 test decides membership, so
 *       the result does not depend on the bin size).
 *   R11 delta = +inf when nh = -1.
 *
 * Input errors (n < 0, a NaN or infinite coordinate or weight, a layer outside
 * [0, n_layers), invalid parameters) return a negative code and leave the
 * outputs unspecified.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_OK 0
#define ORACLE_ERR_ARG -1
#define ORACLE_ERR_INPUT -2
#define ORACLE_ERR_OOM -3

/* Squared distance of R2 (fp32, no contraction). */
static float sq_dist(float xi, float yi, float xj, float yj)
{
    float dx = xj - xi;
    float dy = yj - yi;
    float ax = dx * dx;
    float ay = dy * dy;
    return ax + ay;
}

/* Monotone bin index of coordinate v on an axis starting at lo with bins of
 * width s; out-of-range values land in the edge bins (R10). */
static int64_t axis_bin(double v, double lo, double s, int64_t nb)
{
    double t = floor((v - lo) / s);
    if (!(t > 0.0))
        t = 0.0;
    if (t > (double)(nb - 1))
        t = (double)(nb - 1);
    return (int64_t)t;
}

/* Half-width of the search window of radius d around coordinate v: d plus a
 * margin far larger than any rounding of the fp32 distance test (R10). */
static double window_half(double d, double v)
{
    return d * (1.0 + 1e-6) + fabs(v) * 1e-9;
}

/* exp(a) for a <= 0 in fp32, written from the mathematics: Cody and Waite's
 * reduction (W. J. Cody, W. Waite, "Software Manual for the Elementary
 * Functions", 1980) a = k ln2 + r with ln2 split into a short constant L1
 * (exact products k L1) and its remainder L2, |r| <= ln2 / 2, then
 * exp(r) by its Taylor series to degree 7 in Horner form and exp(a) =
 * 2^k exp(r).  Every operation is one fp32 rounding in a fixed order.
 * Arguments below -87 give 0 (results there would be subnormal). */
float oracle_chi_exp(float a)
{
    if (!(a > -87.0f))
        return 0.0f;
    const float kf = floorf(a * 1.44269504f + 0.5f);     /* round(a / ln2) */
    const float r = (a - kf * 0.693359375f) + kf * 2.12194440e-4f;
    float p = 1.98412698e-4f;                            /* 1/7! */
    p = p * r + 1.38888889e-3f;                          /* 1/6! */
    p = p * r + 8.33333333e-3f;                          /* 1/5! */
    p = p * r + 4.16666667e-2f;                          /* 1/4! */
    p = p * r + 1.66666667e-1f;                          /* 1/3! */
    p = p * r + 0.5f;                                    /* 1/2! */
    p = p * r + 1.0f;
    p = p * r + 1.0f;
    const int32_t bits = ((int32_t)kf + 127) << 23;      /* 2^k, -125 <= k <= 0 */
    float scale;
    memcpy(&scale, &bits, sizeof(scale));
    return p * scale;
}

/* The convolution kernel chi(d_ij) of Eq. 3 for squared distance d2:
 * kind 0 flat (1), 1 Gaussian exp(-d2 / (2 s^2)), 2 exponential exp(-d / s),
 * with s = param > 0; inv is fl(1 / fl(2 s s)) or fl(1 / s). */
static float chi_value(int32_t kind, float inv, float d2)
{
    if (kind == 1)
        return oracle_chi_exp(-(d2 * inv));
    if (kind == 2)
        return oracle_chi_exp(-(sqrtf(d2) * inv));
    return 1.0f;
}

/* Exact accumulation for R4.  A finite fp32 value is an integer multiple of
 * 2^-149 below 2^128 in magnitude, i.e. an integer below 2^277 in units of
 * 2^-149; a sum of up to 2^40 of them fits in a 320-bit two's-complement
 * integer, kept here as ten 32-bit limbs, least significant first. */
#define EXACT_LIMBS 10

static void exact_add(uint32_t acc[EXACT_LIMBS], float t)
{
    uint32_t bits;
    memcpy(&bits, &t, sizeof(bits));
    const uint32_t e = (bits >> 23) & 0xffu;
    const uint32_t frac = bits & 0x7fffffu;
    /* |t| = mant * 2^(shift - 149): subnormals have e = 0, mant = frac */
    const uint64_t mant = e ? (frac | 0x800000u) : frac;
    const int shift = e ? (int)e - 1 : 0;
    const int k = shift / 32;
    const uint64_t v = mant << (shift % 32);       /* below 2^56: limbs k, k+1 */
    const uint32_t part[2] = {(uint32_t)v, (uint32_t)(v >> 32)};
    if (!(bits >> 31)) {
        /* add |t| at limbs k, k+1, then the carry upwards */
        uint64_t carry = 0;
        for (int i = k; i < EXACT_LIMBS; ++i) {
            const uint64_t s = (uint64_t)acc[i] + (i - k < 2 ? part[i - k] : 0u) + carry;
            acc[i] = (uint32_t)s;
            carry = s >> 32;
            if (i > k && !carry)
                break;
        }
    } else {
        /* subtract |t| at limbs k, k+1, then the borrow upwards (two's
         * complement: a borrow out of the top limb wraps) */
        uint64_t borrow = 0;
        for (int i = k; i < EXACT_LIMBS; ++i) {
            const uint64_t sub = (uint64_t)(i - k < 2 ? part[i - k] : 0u) + borrow;
            borrow = (uint64_t)acc[i] < sub;
            acc[i] = (uint32_t)((uint64_t)acc[i] - sub);
            if (i > k && !borrow)
                break;
        }
    }
}

static int bit_at(const uint32_t m[EXACT_LIMBS], int i)
{
    return (int)((m[i / 32] >> (i % 32)) & 1u);
}

/* The accumulated value (units of 2^-149) rounded to the nearest fp32, ties
 * to even, +0 for an exact zero, +-inf beyond the largest finite value. */
static float exact_round(const uint32_t acc[EXACT_LIMBS])
{
    uint32_t mag[EXACT_LIMBS];
    const uint32_t neg = acc[EXACT_LIMBS - 1] >> 31;
    uint64_t carry = neg;
    for (int k = 0; k < EXACT_LIMBS; ++k) {       /* |acc| by two's complement */
        const uint64_t s = (uint64_t)(neg ? (uint32_t)~acc[k] : acc[k]) + carry;
        mag[k] = (uint32_t)s;
        carry = s >> 32;
    }
    int p = -1;                                    /* highest set bit */
    for (int k = EXACT_LIMBS - 1; k >= 0 && p < 0; --k)
        for (int b = 31; b >= 0 && mag[k]; --b)
            if ((mag[k] >> b) & 1u) {
                p = 32 * k + b;
                break;
            }
    if (p < 0)
        return 0.0f;
    uint32_t bits;
    if (p <= 23) {
        /* below 2^24 units: exactly a subnormal (or the smallest binade),
         * whose bit pattern is the unit count itself */
        bits = mag[0];
    } else {
        int sh = p - 23;                           /* keep bits [sh, p] */
        uint32_t m = 0;
        for (int b = 0; b < 24; ++b)
            m |= (uint32_t)bit_at(mag, sh + b) << b;
        const int guard = bit_at(mag, sh - 1);
        int sticky = 0;                            /* any bit below the guard bit */
        for (int k = 0; k < (sh - 1) / 32; ++k)
            sticky |= mag[k] != 0;
        sticky |= (mag[(sh - 1) / 32] & ((1u << ((sh - 1) % 32)) - 1u)) != 0;
        if (guard && (sticky || (m & 1u))) {
            m += 1;
            if (m == (1u << 24)) {
                m >>= 1;
                sh += 1;
            }
        }
        const int biased = sh + 1;                 /* value m * 2^(biased - 150) */
        bits = biased >= 255 ? 0x7f800000u : ((uint32_t)biased << 23) | (m & 0x7fffffu);
    }
    bits |= neg << 31;
    float f;
    memcpy(&f, &bits, sizeof(f));
    return f;
}

static int param_ok(float d)
{
    return isfinite(d) && d >= 0.0f && isfinite(d * d);
}

/*
 * Cluster one event of n hits.  Outputs (all length n, caller-owned):
 *   rho, delta (sqrtf of the squared separation, +inf when nh = -1),
 *   delta2 (the squared separation), nh (nearest-higher index or -1),
 *   is_seed (0/1), is_outlier (0/1), cluster_id (0..k-1 or -1).
 * Any output pointer may be NULL.  Returns ORACLE_OK or a negative code.
 */
int oracle_clue_chi(int64_t n, const float *x, const float *y, const int32_t *layer,
                    const float *w, int32_t n_layers, float x_min, float x_max,
                    float y_min, float y_max, float dc, float rhoc, float delta_c,
                    float delta_o, int32_t chi_kind, float chi_param, float *rho_out,
                    float *delta_out, float *delta2_out, int32_t *nh_out,
                    uint8_t *is_seed_out, uint8_t *is_outlier_out,
                    int32_t *cluster_id_out, int64_t *n_seeds_out)
{
    if (chi_kind < 0 || chi_kind > 2 || (chi_kind != 0 && !(chi_param > 0.0f && isfinite(chi_param))))
        return ORACLE_ERR_ARG;
    const float chi_inv = chi_kind == 1 ? 1.0f / (2.0f * (chi_param * chi_param))
                        : chi_kind == 2 ? 1.0f / chi_param : 1.0f;
    if (n < 0 || n_layers <= 0 || !(dc > 0.0f) || !param_ok(dc) || !param_ok(delta_c) ||
        !param_ok(delta_o) || !isfinite(rhoc) || !isfinite(x_min) || !isfinite(x_max) ||
        !isfinite(y_min) || !isfinite(y_max) || !(x_max > x_min) || !(y_max > y_min))
        return ORACLE_ERR_ARG;
    if (n > 0 && (!x || !y || !layer || !w))
        return ORACLE_ERR_ARG;
    for (int64_t i = 0; i < n; ++i) {
        if (!isfinite(x[i]) || !isfinite(y[i]) || !isfinite(w[i]) || layer[i] < 0 ||
            layer[i] >= n_layers)
            return ORACLE_ERR_INPUT;
    }
    if (n_seeds_out)
        *n_seeds_out = 0;
    if (n == 0)
        return ORACLE_OK;

    /* Sec. 2.2: d_m = max(delta_o, delta_c); thresholds squared once in fp32. */
    const float dm = delta_o > delta_c ? delta_o : delta_c;
    const float dc2 = dc * dc;
    const float dm2 = dm * dm;
    const float delta_c2 = delta_c * delta_c;
    const float delta_o2 = delta_o * delta_o;

    /* Step 1: fixed grid per layer, bin size max(d_c, d_m) (any size works). */
    const double s = (double)(dm > dc ? dm : dc);
    const int64_t nbx = (int64_t)ceil(((double)x_max - x_min) / s) > 0
                            ? (int64_t)ceil(((double)x_max - x_min) / s) : 1;
    const int64_t nby = (int64_t)ceil(((double)y_max - y_min) / s) > 0
                            ? (int64_t)ceil(((double)y_max - y_min) / s) : 1;
    const int64_t n_cells = (int64_t)n_layers * nbx * nby;
    if (nbx > (1 << 20) || nby > (1 << 20) || n_cells > ((int64_t)1 << 31))
        return ORACLE_ERR_ARG;

    int64_t *head = malloc(sizeof(int64_t) * (size_t)n_cells);
    int64_t *next = malloc(sizeof(int64_t) * (size_t)n);
    float *rho = malloc(sizeof(float) * (size_t)n);
    float *d2v = malloc(sizeof(float) * (size_t)n);
    int64_t *nh = malloc(sizeof(int64_t) * (size_t)n);
    int64_t *cid = malloc(sizeof(int64_t) * (size_t)n);
    int64_t *fol_head = malloc(sizeof(int64_t) * (size_t)n);
    int64_t *fol_next = malloc(sizeof(int64_t) * (size_t)n);
    int64_t *stack = malloc(sizeof(int64_t) * (size_t)n);
    uint8_t *seed = malloc((size_t)n);
    uint8_t *outl = malloc((size_t)n);
    if (!head || !next || !rho || !d2v || !nh || !cid || !fol_head || !fol_next ||
        !stack || !seed || !outl) {
        free(head); free(next); free(rho); free(d2v); free(nh); free(cid);
        free(fol_head); free(fol_next); free(stack); free(seed); free(outl);
        return ORACLE_ERR_OOM;
    }
    for (int64_t c = 0; c < n_cells; ++c)
        head[c] = -1;
    /* Register each hit in its bin; pushing in descending index order leaves
     * every bin list in ascending index order. */
    for (int64_t i = n - 1; i >= 0; --i) {
        int64_t bx = axis_bin(x[i], x_min, s, nbx);
        int64_t by = axis_bin(y[i], y_min, s, nby);
        int64_t c = ((int64_t)layer[i] * nby + by) * nbx + bx;
        next[i] = head[c];
        head[c] = i;
    }

    /* Step 2 (Eq. 3, Algorithm 1): rho_i over Omega_dc(i), the exact sum of
     * its terms rounded once (R4). */
    for (int64_t i = 0; i < n; ++i) {
        double hx = window_half(dc, x[i]), hy = window_half(dc, y[i]);
        int64_t bx0 = axis_bin((double)x[i] - hx, x_min, s, nbx);
        int64_t bx1 = axis_bin((double)x[i] + hx, x_min, s, nbx);
        int64_t by0 = axis_bin((double)y[i] - hy, y_min, s, nby);
        int64_t by1 = axis_bin((double)y[i] + hy, y_min, s, nby);
        uint32_t acc[EXACT_LIMBS] = {0};
        for (int64_t by = by0; by <= by1; ++by)
            for (int64_t bx = bx0; bx <= bx1; ++bx)
                for (int64_t j = head[((int64_t)layer[i] * nby + by) * nbx + bx]; j >= 0;
                     j = next[j]) {
                    const float d2 = sq_dist(x[i], y[i], x[j], y[j]);
                    if (d2 < dc2) {
                        const float t = chi_kind == 0 ? w[j] : chi_value(chi_kind, chi_inv, d2) * w[j];
                        exact_add(acc, t);
                    }
                }
        rho[i] = exact_round(acc);
    }

    /* Step 3 (Eq. 4, Algorithm 2): nearest-higher within d_m, ties by the
     * smaller index (R5); none gives nh = -1, delta = +inf (R11). */
    for (int64_t i = 0; i < n; ++i) {
        double hx = window_half(dm, x[i]), hy = window_half(dm, y[i]);
        int64_t bx0 = axis_bin((double)x[i] - hx, x_min, s, nbx);
        int64_t bx1 = axis_bin((double)x[i] + hx, x_min, s, nbx);
        int64_t by0 = axis_bin((double)y[i] - hy, y_min, s, nby);
        int64_t by1 = axis_bin((double)y[i] + hy, y_min, s, nby);
        float best = INFINITY;
        int64_t arg = -1;
        for (int64_t by = by0; by <= by1; ++by)
            for (int64_t bx = bx0; bx <= bx1; ++bx)
                for (int64_t j = head[((int64_t)layer[i] * nby + by) * nbx + bx]; j >= 0;
                     j = next[j]) {
                    float d2 = sq_dist(x[i], y[i], x[j], y[j]);
                    if (d2 < dm2 && rho[j] > rho[i]) {
                        if (d2 < best || (d2 == best && j < arg)) {
                            best = d2;
                            arg = j;
                        }
                    }
                }
        d2v[i] = best;
        nh[i] = arg;
    }

    /* Step 4 (Sec. 2.2, Eq. 5, Algorithm 3): seeds get ids in index order,
     * outliers are left out, everything else registers with its nh (R7). */
    int64_t k = 0, top = 0;
    for (int64_t i = 0; i < n; ++i) {
        fol_head[i] = -1;
        cid[i] = -1;
    }
    for (int64_t i = 0; i < n; ++i) {
        seed[i] = (rho[i] > rhoc) && (d2v[i] > delta_c2);
        outl[i] = (rho[i] < rhoc) && (d2v[i] > delta_o2);
        if (seed[i]) {
            cid[i] = k++;
            stack[top++] = i;
        } else if (!outl[i] && nh[i] >= 0) {
            fol_next[i] = fol_head[nh[i]];
            fol_head[nh[i]] = i;
        }
    }

    /* Step 5 (Algorithm 3): pass the ids down the follower lists. */
    while (top > 0) {
        int64_t i = stack[--top];
        for (int64_t j = fol_head[i]; j >= 0; j = fol_next[j]) {
            cid[j] = cid[i];
            stack[top++] = j;
        }
    }

    for (int64_t i = 0; i < n; ++i) {
        if (rho_out) rho_out[i] = rho[i];
        if (delta2_out) delta2_out[i] = d2v[i];
        if (delta_out) delta_out[i] = sqrtf(d2v[i]);
        if (nh_out) nh_out[i] = (int32_t)nh[i];
        if (is_seed_out) is_seed_out[i] = seed[i];
        if (is_outlier_out) is_outlier_out[i] = outl[i];
        if (cluster_id_out) cluster_id_out[i] = (int32_t)cid[i];
    }
    if (n_seeds_out)
        *n_seeds_out = k;

    free(head); free(next); free(rho); free(d2v); free(nh); free(cid);
    free(fol_head); free(fol_next); free(stack); free(seed); free(outl);
    return ORACLE_OK;
}

/* Flat-kernel CLUE (chi = 1, as Algorithm 1). */
int oracle_clue(int64_t n, const float *x, const float *y, const int32_t *layer,
                const float *w, int32_t n_layers, float x_min, float x_max,
                float y_min, float y_max, float dc, float rhoc, float delta_c,
                float delta_o, float *rho_out, float *delta_out, float *delta2_out,
                int32_t *nh_out, uint8_t *is_seed_out, uint8_t *is_outlier_out,
                int32_t *cluster_id_out, int64_t *n_seeds_out)
{
    return oracle_clue_chi(n, x, y, layer, w, n_layers, x_min, x_max, y_min, y_max, dc, rhoc,
                           delta_c, delta_o, 0, 0.0f, rho_out, delta_out, delta2_out, nh_out,
                           is_seed_out, is_outlier_out, cluster_id_out, n_seeds_out);
}
