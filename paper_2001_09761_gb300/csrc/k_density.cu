// Steps S2 and S3: local density rho (Eq. 3, Algorithm 1) and nearest-higher
// nh / separation delta (Eq. 4, Algorithm 2).
//
// One thread per hit in grid (sorted) order, so a warp covers neighbouring
// cells and its window loads hit the same lines.  The window of Eq. 1 is the
// set of bins met by [x +- R] x [y +- R]; bins of one grid row are adjacent in
// the sorted array, so a window row is one contiguous run.  Each sorted hit is
// one float4 (x, y, w, id), so a candidate costs one 16-byte load.
//
// rho is summed in fp32 in ascending hit index j over N_dc(i) of chi(d_ij) w_j
// (flat chi = 1 unless the context asks for the Gaussian or exponential kernel
// that Eq. 3 names; chi is computed by chi_exp, bit-reproducible) (the order is
// part of the result's definition, independent of the bin size): every cell
// lists its hits in ascending index, and the kernel merges the lists of the
// window's non-empty cells, adding w_j for each j that passes the distance
// test as the merge reaches it.  With the bin at least 2 R wide a window has
// at most 2 x 2 cells, merged by one loop that every lane of a warp runs
// alike (lanes that take different code paths would run one after another).
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

// r + chi(d) w for a candidate within d_c (flat: r + w exactly).
template <int CHI = 0>
__device__ __forceinline__ float add_if_near(float r, float xi, float yi, const float4 &h,
                                             float dc2, float inv = 1.0f) {
    const float d2 = sq_dist(xi, yi, h.x, h.y);
    if (CHI == 0) return d2 < dc2 ? __fadd_rn(r, h.z) : r;
    return d2 < dc2 ? __fadd_rn(r, __fmul_rn(chi_of<CHI>(d2, inv), h.z)) : r;
}

// Merge of up to K sorted cell lists given as [p[k], e[k]) (k < nk).  With
// CACHE the head hit of every list stays in registers (one load per
// candidate); without it only the head ids do (fewer registers, two loads).
template <int K, bool CACHE, int CHI>
__device__ __forceinline__ float merge_k(const float4 *__restrict__ sp, int (&p)[K],
                                         const int (&e)[K], int nk, float xi, float yi,
                                         float dc2, float inv) {
    float4 h[CACHE ? K : 1];
    int head[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const bool live = k < nk && p[k] < e[k];
        const float4 v = live ? sp[p[k]] : make_float4(0.f, 0.f, 0.f, 0.f);
        if (CACHE) h[k] = v;
        head[k] = live ? id_of(v) : INT_MAX;
    }
    float r = 0.0f;
    while (true) {
        int m = head[0], am = 0;
#pragma unroll
        for (int k = 1; k < K; ++k)
            if (head[k] < m) {
                m = head[k];
                am = k;
            }
        if (m == INT_MAX) break;
#pragma unroll
        for (int k = 0; k < K; ++k)
            if (am == k) {
                const int q = p[k]++;
                r = add_if_near<CHI>(r, xi, yi, CACHE ? h[k] : sp[q], dc2, inv);
                const bool live = q + 1 < e[k];
                if (CACHE) {
                    h[k] = live ? sp[q + 1] : h[k];
                    head[k] = live ? id_of(h[k]) : INT_MAX;
                } else {
                    head[k] = live ? id_of(sp[q + 1]) : INT_MAX;
                }
            }
    }
    return r;
}

// Windows of at most 3 x 3 cells (a bin size between d_c and 2 d_c).
template <int CHI>
__device__ __forceinline__ float rho_window9(const Buffers &b, int64_t plane, int nbx, const Window &w, float xi,
                             float yi, float dc2, float inv) {
    int p[9], e[9];
    int nk = 0;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        p[k] = e[k] = 0;
    }
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const int cx = k % 3, cy = k / 3;
        int a = 0, z = 0;
        if ((w.lx + cx <= w.hx) && (w.ly + cy <= w.hy)) {
            const int64_t c = plane + (int64_t)(w.ly + cy) * nbx + (w.lx + cx);
            a = b.cell_start[c];
            z = b.cell_start[c + 1];
        }
        const bool ne = a < z;
#pragma unroll
        for (int m = 0; m < 9; ++m)
            if (ne && m == nk) {
                p[m] = a;
                e[m] = z;
            }
        nk += ne;
    }
    return merge_k<9, false, CHI>(b.sp, p, e, nk, xi, yi, dc2, inv);
}

// Any window size: repeatedly take the smallest id above the last one taken.
// Quadratic in the window population; used only when the window spans more
// than 3 x 3 bins (a bin size near d_c plus rounding at a bin edge).
template <int CHI>
__device__ __forceinline__ float rho_select(const Buffers &b, int64_t plane, int nbx, const Window &w, float xi,
                            float yi, float dc2, float inv) {
    float r = 0.0f;
    int last = -1;
    while (true) {
        int best = INT_MAX, bq = -1;
        for (int by = w.ly; by <= w.hy; ++by)
            for (int bx = w.lx; bx <= w.hx; ++bx) {
                const int64_t c = plane + (int64_t)by * nbx + bx;
                const int e = b.cell_start[c + 1];
                for (int q = b.cell_start[c]; q < e; ++q) {
                    const int j = id_of(b.sp[q]);
                    if (j > last) {  // cells are ascending: the first one above `last`
                        if (j < best) {
                            best = j;
                            bq = q;
                        }
                        break;
                    }
                }
            }
        if (bq < 0) break;
        r = add_if_near<CHI>(r, xi, yi, b.sp[bq], dc2, inv);
        last = best;
    }
    return r;
}

// Windows of at most 2 x 2 cells.  Every lane runs the same loop (a lane
// whose window has fewer cells just has empty cursors), so lanes of a warp
// never take different code paths; a cursor keeps only its head id in a
// register and the chosen candidate is loaded once.
template <int CHI>
__device__ __forceinline__ float rho_window4(const Buffers &b, int64_t plane, int nbx,
                                             const Window &w, float xi, float yi, float dc2,
                                             float inv) {
    const float4 *__restrict__ sp = b.sp;
    const int4 *__restrict__ spi = reinterpret_cast<const int4 *>(b.sp);  // id = .w
    int p0, p1, p2, p3, e0, e1, e2, e3;
    {
        const int64_t r0 = plane + (int64_t)w.ly * nbx + w.lx;
        const bool two_x = w.hx > w.lx, two_y = w.hy > w.ly;
        p0 = b.cell_start[r0];
        e0 = b.cell_start[r0 + 1];
        p1 = e0;
        e1 = two_x ? b.cell_start[r0 + 2] : e0;
        const int64_t r1 = r0 + nbx;
        p2 = two_y ? b.cell_start[r1] : 0;
        e2 = two_y ? b.cell_start[r1 + 1] : 0;
        p3 = e2;
        e3 = (two_x && two_y) ? b.cell_start[r1 + 2] : e2;
    }
    int h0 = p0 < e0 ? spi[p0].w : INT_MAX;
    int h1 = p1 < e1 ? spi[p1].w : INT_MAX;
    int h2 = p2 < e2 ? spi[p2].w : INT_MAX;
    int h3 = p3 < e3 ? spi[p3].w : INT_MAX;
    float r = 0.0f;
    while (true) {
        const int m = min(min(h0, h1), min(h2, h3));
        if (m == INT_MAX) break;
        int q, e;
        if (m == h0) { q = p0++; e = e0; }
        else if (m == h1) { q = p1++; e = e1; }
        else if (m == h2) { q = p2++; e = e2; }
        else { q = p3++; e = e3; }
        r = add_if_near<CHI>(r, xi, yi, sp[q], dc2, inv);
        const int nx = q + 1 < e ? spi[q + 1].w : INT_MAX;
        if (m == h0) h0 = nx;
        else if (m == h1) h1 = nx;
        else if (m == h2) h2 = nx;
        else h3 = nx;
    }
    return r;
}

template <int CHI>
__global__ void __launch_bounds__(256, 1) k_rho(Buffers b, Params p) {
    for (int t = blockIdx.x; t < b.ntiles; t += gridDim.x) {
        const Tile tl = b.tiles[t];
        const EventDesc ev = b.events[tl.event];
        const int64_t nbxy = (int64_t)ev.nbx * ev.nby;
        for (int k = threadIdx.x; k < tl.len; k += blockDim.x) {
            const int q = tl.start + k;
            const float4 me = b.sp[q];
            const int64_t plane = ev.cell_off + (int64_t)b.lay_s[q] * nbxy;
            const Window w = window_of(me.x, me.y, p.rwin_rho, ev);
            const int nx = w.hx - w.lx + 1, ny = w.hy - w.ly + 1;
            float r;
            if (nx <= 2 && ny <= 2)
                r = rho_window4<CHI>(b, plane, ev.nbx, w, me.x, me.y, p.dc2, p.chi_inv);
            else if (nx <= 3 && ny <= 3)
                r = rho_window9<CHI>(b, plane, ev.nbx, w, me.x, me.y, p.dc2, p.chi_inv);
            else
                r = rho_select<CHI>(b, plane, ev.nbx, w, me.x, me.y, p.dc2, p.chi_inv);
            b.spr[q] = make_float4(me.x, me.y, r, me.w);  // x, y, rho, id for the nh step
        }
    }
}

cudaError_t launch_rho(const Buffers &b, const Params &p, const LaunchCfg &c, cudaStream_t s) {
    const int grid = b.ntiles < c.grid_cap ? b.ntiles : c.grid_cap;
    const int g = grid > 0 ? grid : 1;
    if (p.chi == 1)
        k_rho<1><<<g, c.block_density, 0, s>>>(b, p);
    else if (p.chi == 2)
        k_rho<2><<<g, c.block_density, 0, s>>>(b, p);
    else
        k_rho<0><<<g, c.block_density, 0, s>>>(b, p);
    return cudaGetLastError();
}

// nh_i: over the window of radius d_m, the (d2, j)-lexicographic minimum among
// hits with d2 < d_m^2 and rho_j > rho_i (the minimum is order-free).  The
// same thread takes the seed / outlier decision (Sec. 2.2), which needs only
// this hit's rho, delta and nh, and stores one 4-byte code by hit (the
// scattered store this step cannot avoid); delta^2 and nh also go, in sorted
// order (coalesced), to an 8-byte record the intermediates export reads (rho
// stays in the rho step's sorted records).
__global__ void __launch_bounds__(256) k_nh(Buffers b, Params p) {
    const float4 *__restrict__ sp = b.spr;  // x, y, rho, id
    for (int t = blockIdx.x; t < b.ntiles; t += gridDim.x) {
        const Tile tl = b.tiles[t];
        const EventDesc ev = b.events[tl.event];
        const int64_t nbxy = (int64_t)ev.nbx * ev.nby;
        for (int k = threadIdx.x; k < tl.len; k += blockDim.x) {
            const int q = tl.start + k;
            const float4 me = sp[q];
            const float ri = me.z;
            const int64_t plane = ev.cell_off + (int64_t)b.lay_s[q] * nbxy;
            const Window w = window_of(me.x, me.y, p.rwin_nh, ev);
            // (d2, j) packed as one unsigned key: d2 >= 0, so its float bits
            // order like its value; starting at (bits(d_m^2), 0) also folds in
            // the strict test d2 < d_m^2
            const unsigned long long none = (unsigned long long)__float_as_uint(p.dm2) << 32;
            unsigned long long best = none;
            for (int by = w.ly; by <= w.hy; ++by) {
                const int64_t row = plane + (int64_t)by * ev.nbx;
                const int e = b.cell_start[row + w.hx + 1];
                for (int u = b.cell_start[row + w.lx]; u < e; ++u) {  // branch-free body
                    const float4 h = sp[u];
                    const float d2 = sq_dist(me.x, me.y, h.x, h.y);
                    const unsigned long long k =
                        ((unsigned long long)__float_as_uint(d2) << 32) | (unsigned)id_of(h);
                    best = (h.z > ri && k < best) ? k : best;
                }
            }
            const bool found = best != none;
            const float d2v = found ? __uint_as_float((unsigned)(best >> 32))
                                    : __int_as_float(0x7f800000);  // +inf (Eq. 4)
            const int nhj = found ? (int)(unsigned)best : -1;
            b.hr[q] = make_float2(d2v, __int_as_float(nhj));
            // the decision of Sec. 2.2 needs only this hit's rho, delta and nh:
            // seed, outlier, or a follower of nh (Algorithm 3), stored by hit
            const bool seed = (ri > p.rhoc) && (d2v > p.dcs2);
            const bool outl = (ri < p.rhoc) && (d2v > p.dos2);
            const int code = seed ? CODE_SEED : outl ? CODE_OUTLIER : (nhj >= 0 ? nhj : CODE_NOISE);
            const int g = id_of(me);
            b.code[g] = code;
            if (!p.chase && code >= 0) b.frank[g] = atomicAdd(&b.fcount[code], 1);
        }
    }
}

cudaError_t launch_nh(const Buffers &b, const Params &p, const LaunchCfg &c, cudaStream_t s) {
    const int grid = b.ntiles < c.grid_cap ? b.ntiles : c.grid_cap;
    k_nh<<<grid > 0 ? grid : 1, c.block_density, 0, s>>>(b, p);
    return cudaGetLastError();
}

}  // namespace clue
