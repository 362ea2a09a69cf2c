// Steps S2 and S3: local density rho (Eq. 3, Algorithm 1) and nearest-higher
// nh / separation delta (Eq. 4, Algorithm 2).
//
// One thread per hit in grid (sorted) order, so a warp covers neighbouring
// cells and its window loads hit the same lines.  The window of Eq. 1 is the
// set of bins met by [x +- R] x [y +- R]; bins of one grid row are adjacent in
// the sorted arrays, so a window row is one contiguous run.
//
// rho is summed in fp32 in ascending hit index j over N_dc(i) (the order is
// part of the result's definition, independent of the bin size): every cell
// lists its hits in ascending index, and the kernel merges the window cells'
// lists with one cursor per cell, adding w_j for each j that passes the
// distance test as the merge reaches it.
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

// K-cursor merge over a window of at most KX x KY cells.  Cursor k follows
// cell (ly + k / KX, lx + k % KX); cells outside the window are empty.
template <int KX, int KY>
__device__ __forceinline__ float rho_merge(const Buffers &b, int64_t plane, int nbx, const Window &w,
                                           float xi, float yi, float dc2) {
    constexpr int K = KX * KY;
    int pos[K], end[K], head[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int cx = k % KX, cy = k / KX;
        const bool in = (w.lx + cx <= w.hx) && (w.ly + cy <= w.hy);
        const int64_t c = plane + (int64_t)(w.ly + cy) * nbx + (w.lx + cx);
        const int a = in ? b.cell_start[c] : 0;
        const int e = in ? b.cell_start[c + 1] : 0;
        pos[k] = a;
        end[k] = e;
        head[k] = a < e ? b.ids_s[a] : INT_MAX;
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
        int q = pos[0], qe = end[0];
#pragma unroll
        for (int k = 1; k < K; ++k)
            if (am == k) {
                q = pos[k];
                qe = end[k];
            }
        if (sq_dist(xi, yi, b.xs[q], b.ys[q]) < dc2) r = __fadd_rn(r, b.ws[q]);
        ++q;
        const int nxt = q < qe ? b.ids_s[q] : INT_MAX;
#pragma unroll
        for (int k = 0; k < K; ++k)
            if (am == k) {
                pos[k] = q;
                head[k] = nxt;
            }
    }
    return r;
}

// Any window size: repeatedly take the smallest id above the last one taken.
// Quadratic in the window population; used only when the window spans more
// than 3 x 3 bins (a bin size near d_c plus rounding at a bin edge).
__device__ float rho_select(const Buffers &b, int64_t plane, int nbx, const Window &w, float xi,
                            float yi, float dc2) {
    float r = 0.0f;
    int last = -1;
    while (true) {
        int best = INT_MAX, bq = -1;
        for (int by = w.ly; by <= w.hy; ++by)
            for (int bx = w.lx; bx <= w.hx; ++bx) {
                const int64_t c = plane + (int64_t)by * nbx + bx;
                const int e = b.cell_start[c + 1];
                for (int q = b.cell_start[c]; q < e; ++q) {
                    const int j = b.ids_s[q];
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
        if (sq_dist(xi, yi, b.xs[bq], b.ys[bq]) < dc2) r = __fadd_rn(r, b.ws[bq]);
        last = best;
    }
    return r;
}

__global__ void __launch_bounds__(512) k_rho(Buffers b, Params p) {
    for (int t = blockIdx.x; t < b.ntiles; t += gridDim.x) {
        const Tile tl = b.tiles[t];
        const EventDesc ev = b.events[tl.event];
        const int64_t nbxy = (int64_t)ev.nbx * ev.nby;
        for (int k = threadIdx.x; k < tl.len; k += blockDim.x) {
            const int q = tl.start + k;
            const float xi = b.xs[q], yi = b.ys[q];
            const int64_t plane = ev.cell_off + (int64_t)b.lay_s[q] * nbxy;
            const Window w = window_of(xi, yi, p.rwin_rho, ev);
            const int nx = w.hx - w.lx + 1, ny = w.hy - w.ly + 1;
            float r;
            if (nx <= 2 && ny <= 2)
                r = rho_merge<2, 2>(b, plane, ev.nbx, w, xi, yi, p.dc2);
            else if (nx <= 3 && ny <= 3)
                r = rho_merge<3, 3>(b, plane, ev.nbx, w, xi, yi, p.dc2);
            else
                r = rho_select(b, plane, ev.nbx, w, xi, yi, p.dc2);
            b.rho_s[q] = r;
        }
    }
}

cudaError_t launch_rho(const Buffers &b, const Params &p, const LaunchCfg &c, cudaStream_t s) {
    const int grid = b.ntiles < c.grid_cap ? b.ntiles : c.grid_cap;
    k_rho<<<grid > 0 ? grid : 1, c.block_density, 0, s>>>(b, p);
    return cudaGetLastError();
}

// nh_i: over the window of radius d_m, the (d2, j)-lexicographic minimum among
// hits with d2 < d_m^2 and rho_j > rho_i (the minimum is order-free).  Writes
// rho, delta^2 and nh back by hit index.
__global__ void __launch_bounds__(512) k_nh(Buffers b, Params p) {
    for (int t = blockIdx.x; t < b.ntiles; t += gridDim.x) {
        const Tile tl = b.tiles[t];
        const EventDesc ev = b.events[tl.event];
        const int64_t nbxy = (int64_t)ev.nbx * ev.nby;
        for (int k = threadIdx.x; k < tl.len; k += blockDim.x) {
            const int q = tl.start + k;
            const float xi = b.xs[q], yi = b.ys[q], ri = b.rho_s[q];
            const int64_t plane = ev.cell_off + (int64_t)b.lay_s[q] * nbxy;
            const Window w = window_of(xi, yi, p.rwin_nh, ev);
            float best = __int_as_float(0x7f800000);  // +inf
            int bj = INT_MAX;
            for (int by = w.ly; by <= w.hy; ++by) {
                const int64_t row = plane + (int64_t)by * ev.nbx;
                const int e = b.cell_start[row + w.hx + 1];
                for (int u = b.cell_start[row + w.lx]; u < e; ++u) {
                    if (b.rho_s[u] > ri) {
                        const float d2 = sq_dist(xi, yi, b.xs[u], b.ys[u]);
                        if (d2 < p.dm2) {
                            const int j = b.ids_s[u];
                            if (d2 < best || (d2 == best && j < bj)) {
                                best = d2;
                                bj = j;
                            }
                        }
                    }
                }
            }
            const int g = b.ids_s[q];
            b.rho[g] = ri;
            b.delta2[g] = best;
            b.nh[g] = bj == INT_MAX ? -1 : bj;
        }
    }
}

cudaError_t launch_nh(const Buffers &b, const Params &p, const LaunchCfg &c, cudaStream_t s) {
    const int grid = b.ntiles < c.grid_cap ? b.ntiles : c.grid_cap;
    k_nh<<<grid > 0 ? grid : 1, c.block_density, 0, s>>>(b, p);
    return cudaGetLastError();
}

}  // namespace clue
