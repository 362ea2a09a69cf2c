// Steps S2 and S3 tile by tile: rho (Eq. 3, Algorithm 1) and nh / delta with
// the seed / outlier decision (Eq. 4, Algorithm 2, Sec. 2.2), one CTA per tile
// of sorted hits, with the tile's candidates staged in shared memory.
//
// One thread per hit in grid order leaves half a warp idle: the windows of
// neighbouring hits hold from one to tens of candidates, and a warp runs as
// long as its longest window row by row.  Here a CTA first finds every window
// of its tile (the runs of sorted positions of its 1 to 3 grid rows) and the
// band of sorted positions all of them lie in, then
//
//  * sorted form (the band fits in shared memory, windows of at most DT_ROWS
//    rows): the band is staged once, the tile's hits are ordered by
//    descending candidate count (a counting sort in shared memory), so the
//    32 lanes of a warp take hits with near-equal windows, and each lane walks
//    its window's runs as one flat loop (no per-row reconvergence);
//  * per-hit form otherwise (windows of more rows, bands beyond the staging
//    capacity): one thread per hit, in grid order, walks its window in global
//    memory (neighbouring hits of dense regions have similar windows, so the
//    lanes of a warp stay close there too).
//
// Every form computes the same function of the neighbour sets (the exact
// density, the lexicographic minimum), so the form, the order of the hits and
// the order of the candidates never change a result.
#pragma once

#include "density_stages.cuh"

namespace clue {

constexpr int DT_ROWS = 3;       // window rows the sorted form walks
constexpr int DT_BUCKETS = 64;   // work classes of the counting sort (64+ share one)
constexpr int DT_OUT = 1 << 14;  // window starts further than this from the tile

// One hit's window for the sorted form: per row (up to DT_ROWS) the start
// relative to the tile start (16 bits) and the length (16 bits), and the
// candidate count; all in one 16-byte word.
__device__ __forceinline__ unsigned pack_row(int rel, int len) {
    return (unsigned)(unsigned short)(short)max(-DT_OUT, min(DT_OUT, rel)) |
           ((unsigned)min(len, 65535) << 16);
}
__device__ __forceinline__ int row_start(unsigned w) { return (int)(short)(w & 0xffffu); }
__device__ __forceinline__ int row_len(unsigned w) { return (int)(w >> 16); }

// Per-tile shared state: 18 KB, plus the staged band (dynamic shared memory).
struct DensityShared {
    uint4 win[TILE];                   // windows (pack_row x 3, candidate count)
    unsigned short perm[TILE];         // the tile's hits by descending window population
    int hist[DT_BUCKETS];
    int lo, hi, rows;                  // the band [lo, hi) (relative) and the most rows
    unsigned long long tsum;           // candidates over the tile's windows
};

// The tile's windows of radius parameter `dr` into sh.win (rows past DT_ROWS
// and starts past DT_OUT are flagged through sh.rows / the band, which then
// disqualify the sorted form), the band and the work histogram.  A thread
// takes the tile's hits k = threadIdx.x + u * blockDim.x, u < U, and issues
// each round of loads (records and layers, then every window row's bounds)
// for all of them before it waits on any.
template <int U>
__device__ __forceinline__ void tile_windows(const Buffers &b, const Tile &tl,
                                             const EventDesc &ev, float dr,
                                             DensityShared &sh) {
    if (threadIdx.x < DT_BUCKETS) sh.hist[threadIdx.x] = 0;
    if (threadIdx.x == 0) {
        sh.lo = INT_MAX;
        sh.hi = INT_MIN;
        sh.rows = 0;
        sh.tsum = 0ull;
    }
    __syncthreads();
    const int64_t nbxy = (int64_t)ev.nbx * ev.nby;
    int lo = INT_MAX, hi = INT_MIN, rows = 0;
    unsigned long long tsum = 0ull;
    for (int k0 = threadIdx.x; k0 < tl.len; k0 += U * blockDim.x) {
        float4 me[U];
        int lay[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int k = k0 + u * blockDim.x;
            const int q = tl.start + (k < tl.len ? k : 0);
            me[u] = b.sp[q];
            lay[u] = b.lay_s[q];
        }
        Window w[U];
        int64_t row0[U];
        int a[U][DT_ROWS], e[U][DT_ROWS];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            w[u] = window_of(me[u].x, me[u].y, dr, ev);
            row0[u] = ev.cell_off + (int64_t)lay[u] * nbxy + (int64_t)w[u].ly * ev.nbx;
#pragma unroll
            for (int r = 0; r < DT_ROWS; ++r) {
                const bool in = w[u].ly + r <= w[u].hy;
                const int64_t row = row0[u] + (in ? (int64_t)r * ev.nbx : 0);
                a[u][r] = in ? b.cell_start[row + w[u].lx] : 0;
                e[u][r] = in ? b.cell_start[row + w[u].hx + 1] : 0;
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int k = k0 + u * blockDim.x;
            if (k >= tl.len) continue;
            const int nr = w[u].hy - w[u].ly + 1;
            unsigned T = 0;
            int last = e[u][0];
#pragma unroll
            for (int r = 0; r < DT_ROWS; ++r) T += (unsigned)(e[u][r] - a[u][r]);
            for (int r = DT_ROWS; r < nr; ++r) {  // rows the sorted form does not take
                const int64_t row = row0[u] + (int64_t)r * ev.nbx;
                const int u0 = b.cell_start[row + w[u].lx];
                last = b.cell_start[row + w[u].hx + 1];
                T += (unsigned)(last - u0);
            }
            if (nr > 1 && nr <= DT_ROWS) last = nr == 2 ? e[u][1] : e[u][2];
            lo = min(lo, a[u][0] - tl.start);
            hi = max(hi, last - tl.start);
            rows = max(rows, nr);
            tsum += T;
            sh.win[k] = make_uint4(pack_row(a[u][0] - tl.start, e[u][0] - a[u][0]),
                                   pack_row(a[u][1] - tl.start, e[u][1] - a[u][1]),
                                   pack_row(a[u][2] - tl.start, e[u][2] - a[u][2]),
                                   min(T, 65535u));
            atomicAdd(&sh.hist[DT_BUCKETS - 1 - min((int)T, DT_BUCKETS - 1)], 1);
        }
    }
    lo = __reduce_min_sync(FULL_MASK, lo);
    hi = __reduce_max_sync(FULL_MASK, hi);
    rows = __reduce_max_sync(FULL_MASK, rows);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) tsum += __shfl_xor_sync(FULL_MASK, tsum, o);
    if (lane_id() == 0) {
        atomicMin(&sh.lo, lo);
        atomicMax(&sh.hi, hi);
        atomicMax(&sh.rows, rows);
        atomicAdd(&sh.tsum, tsum);
    }
    __syncthreads();
}

// Whether the sorted form takes the tile (uniform over the CTA): windows of
// at most DT_ROWS rows and a band within the launch's staging capacity.
__device__ __forceinline__ bool tile_sorted(const DensityShared &sh, int cap) {
    return sh.rows <= DT_ROWS && sh.lo >= -DT_OUT + 1 && sh.hi <= DT_OUT - 1 &&
           sh.hi - sh.lo <= cap;
}

// Counting sort of the tile's hits by descending window population (the
// histogram from tile_windows); order inside a class is arbitrary.
__device__ __forceinline__ void tile_sort(const Tile &tl, DensityShared &sh) {
    static_assert(DT_BUCKETS == 64, "one warp scans two classes per lane");
    if (threadIdx.x < 32) {
        const int v0 = sh.hist[2 * threadIdx.x], v1 = sh.hist[2 * threadIdx.x + 1];
        const int incl = warp_incl_scan(v0 + v1);
        sh.hist[2 * threadIdx.x] = incl - v0 - v1;
        sh.hist[2 * threadIdx.x + 1] = incl - v1;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < tl.len; k += blockDim.x) {
        const int T = (int)sh.win[k].w;
        const int pos = atomicAdd(&sh.hist[DT_BUCKETS - 1 - min(T, DT_BUCKETS - 1)], 1);
        sh.perm[pos] = (unsigned short)k;
    }
}

// One hit's window as a flat run of T candidates in the staged band: the
// c-th candidate is at c + base(c), base a step function of c with breaks at
// the row ends (ROWS = 2: windows of at most two rows, the usual case).
template <int ROWS>
struct FlatWin {
    int b0, b1, b2;  // band index minus c, per row
    int o1, o2;      // where rows 1 and 2 begin in c
    int T;
    __device__ __forceinline__ FlatWin(const uint4 &w, int lo) {
        const int l0 = row_len(w.x), l1 = row_len(w.y);
        o1 = l0;
        o2 = l0 + l1;
        T = (int)w.w;
        b0 = row_start(w.x) - lo;
        b1 = row_start(w.y) - lo - o1;
        b2 = row_start(w.z) - lo - o2;
    }
    __device__ __forceinline__ int at(int c) const {
        if (ROWS <= 2) return c + (c < o1 ? b0 : b1);
        return c + (c < o1 ? b0 : (c < o2 ? b1 : b2));
    }
};

// ---- rho ---------------------------------------------------------------------

// rho of the tile's hits in the sorted form (the band staged, hits ordered).
template <int CHI, int ROWS>
__device__ __forceinline__ void rho_sorted(const Buffers &b, const Params &p, const Tile &tl,
                                           const EventDesc &ev, const FixedW &fw,
                                           const DensityShared &sh, const float4 *band) {
    const bool fixed = CHI == 0 && fw.on;
    const int lo = sh.lo;
    for (int j = threadIdx.x; j < tl.len; j += blockDim.x) {
        const int k = sh.perm[j];
        const int q = tl.start + k;
        const float4 me = band[k - lo];
        const FlatWin<ROWS> f(sh.win[k], lo);
        float r;
        bool ok;
        if (fixed) {
            long long acc = 0;
#pragma unroll 2
            for (int c = 0; c < f.T; ++c) {  // branch-free body
                const float4 h = band[f.at(c)];
                const float d2 = sq_dist(me.x, me.y, h.x, h.y);
                acc += d2 < p.dc2 ? fixed_weight_of(h) : 0ll;
            }
            r = __fmul_rn(__ll2float_rn(acc), fw.unit);
            ok = 32 - __clz(f.T) <= fw.budget;
        } else {
            TwoSumAcc a;
            for (int c = 0; c < f.T; ++c) {  // branch-free body
                const float4 h = band[f.at(c)];
                const float d2 = sq_dist(me.x, me.y, h.x, h.y);
                const bool near = d2 < p.dc2;
                a.add(near ? term_of<CHI>(d2, h.z, p.chi_inv) : 0.0f, near);
            }
            r = __fadd_rn(a.s, a.c);
            ok = a.exact();
        }
        if (!ok) {  // the integer accumulator over the window in global memory
            const Window w = window_of(me.x, me.y, p.rwin_rho, ev);
            const int64_t plane = ev.cell_off + (int64_t)b.lay_s[q] * ev.nbx * ev.nby;
            r = rho_wide<CHI>(b, plane, ev.nbx, w, me.x, me.y, p.dc2, p.chi_inv,
                              fixed ? fw.unit : 0.0f);
        }
        store_rho(b, p, q, me.x, me.y, r);
    }
}

template <int CHI, int U>
__device__ __forceinline__ void rho_tile(const Buffers &b, const Params &p, int t,
                                         DensityShared &sh, float4 *band) {
    const Tile tl = b.tiles[t];
    const EventDesc ev = b.events[tl.event];
    const FixedW fw = fixed_weights(b.wexp + 2 * tl.event, CHI);  // uniform per event
    const int64_t nbxy = (int64_t)ev.nbx * ev.nby;
    tile_windows<U>(b, tl, ev, p.rwin_rho, sh);
    if (!tile_sorted(sh, p.band_cap)) {  // per-hit form
        for (int k = threadIdx.x; k < tl.len; k += blockDim.x) {
            const int q = tl.start + k;
            const float4 me = b.sp[q];
            store_rho(b, p, q, me.x, me.y, rho_of_hit<CHI>(b, p, ev, fw, me, b.lay_s[q]));
        }
        __syncthreads();
        return;
    }
    tile_sort(tl, sh);
    const int lo = sh.lo, n_band = sh.hi - sh.lo;
    for (int h = threadIdx.x; h < n_band; h += blockDim.x) band[h] = b.sp[tl.start + lo + h];
    __syncthreads();
    if (sh.rows <= 2)
        rho_sorted<CHI, 2>(b, p, tl, ev, fw, sh, band);
    else
        rho_sorted<CHI, DT_ROWS>(b, p, tl, ev, fw, sh, band);
    __syncthreads();
}

// ---- nh, delta and the decision ----------------------------------------------

// nh of the tile's hits in the sorted form (the band staged as x, y, rho, id).
template <int ROWS>
__device__ __forceinline__ void nh_sorted(const Buffers &b, const Params &p, const Tile &tl,
                                          const DensityShared &sh, const float4 *band) {
    const int lo = sh.lo;
    for (int j = threadIdx.x; j < tl.len; j += blockDim.x) {
        const int k = sh.perm[j];
        const float4 me = band[k - lo];  // x, y, rho, id
        const FlatWin<ROWS> f(sh.win[k], lo);
        unsigned long long best = nh_none(p);
#pragma unroll 2
        for (int c = 0; c < f.T; ++c) {  // branch-free body
            const float4 h = band[f.at(c)];
            const float d2 = sq_dist(me.x, me.y, h.x, h.y);
            const unsigned long long key = nh_key(d2, id_of(h));
            best = (h.z > me.z && key < best) ? key : best;
        }
        nh_store(b, p, tl.start + k, id_of(me), me.z, best);
    }
}

template <int U>
__device__ __forceinline__ void nh_tile(const Buffers &b, const Params &p, int t,
                                        DensityShared &sh, float4 *band) {
    const Tile tl = b.tiles[t];
    const EventDesc ev = b.events[tl.event];
    const int64_t nbxy = (int64_t)ev.nbx * ev.nby;
    tile_windows<U>(b, tl, ev, p.rwin_nh, sh);
    if (!tile_sorted(sh, p.band_cap)) {  // per-hit form
        for (int k = threadIdx.x; k < tl.len; k += blockDim.x) {
            const int q = tl.start + k;
            const float4 me = nh_record(b, p, q);
            nh_store(b, p, q, id_of(me), me.z, nh_of_hit(b, p, ev, me.x, me.y, me.z, b.lay_s[q]));
        }
        __syncthreads();
        return;
    }
    tile_sort(tl, sh);
    const int lo = sh.lo, n_band = sh.hi - sh.lo;
    for (int h = threadIdx.x; h < n_band; h += blockDim.x) band[h] = nh_record(b, p, tl.start + lo + h);
    __syncthreads();
    if (sh.rows <= 2)
        nh_sorted<2>(b, p, tl, sh, band);
    else
        nh_sorted<DT_ROWS>(b, p, tl, sh, band);
    __syncthreads();
}

// ---- rho, nh, delta and the decision in one pass (the fused form) ----------
//
// One CTA per tile, with the sorted form's staging done once for both steps:
// the windows of radius max(d_c, d_m) (a superset of both searches' windows;
// the exact d2 tests pick the neighbours), one ordering of the tile's hits by
// window population, one band staged.  Then rho of the tile's hits from the
// band (written to global memory for the intermediates and for other tiles);
// rho of the band's hits outside the tile (the halo, whose densities the
// tile's nh needs) by a walk over their own windows in global memory, each
// computed again by every tile whose band holds it (identical values); the
// band restaged in place as (x, y, rho, id); nh and the decision of the
// tile's hits.  So rho goes straight to nh with no pass over the batch in
// between.  A tile the sorted form does not take (a band beyond the staging
// capacity, windows of more rows) or whose halo holds more hits than the tile
// itself (dense neighbourhoods) gets only its rho here
// (rho_tile's forms) and joins a list that k_nh_rest finishes after every
// tile's rho is written.
template <int CHI, int U>
__device__ __forceinline__ void density_tile(const Buffers &b, const Params &p, int t,
                                             DensityShared &sh, float4 *band) {
    const Tile tl = b.tiles[t];
    const EventDesc ev = b.events[tl.event];
    const FixedW fw = fixed_weights(b.wexp + 2 * tl.event, CHI);  // uniform per event
    tile_windows<U>(b, tl, ev, fmaxf(p.rwin_rho, p.rwin_nh), sh);
    // fused when the band fits and its halo (whose rho is computed again here)
    // holds at most as many hits as the tile
    const bool fused = tile_sorted(sh, p.band_cap) && sh.hi - sh.lo <= 2 * tl.len;
    if (!fused) {
        __syncthreads();  // every thread has read the shared state rho_tile resets
        rho_tile<CHI, U>(b, p, t, sh, band);
        if (threadIdx.x == 0) b.rest[atomicAdd(&b.ctrl->nrest, 1)] = t;
        return;
    }
    tile_sort(tl, sh);
    const int lo = sh.lo, n_band = sh.hi - sh.lo;
    for (int h = threadIdx.x; h < n_band; h += blockDim.x) band[h] = b.sp[tl.start + lo + h];
    __syncthreads();
    if (sh.rows <= 2)
        rho_sorted<CHI, 2>(b, p, tl, ev, fw, sh, band);
    else
        rho_sorted<CHI, DT_ROWS>(b, p, tl, ev, fw, sh, band);
    __syncthreads();  // the tile's rho are written; the band's weights are no longer read
    for (int h = threadIdx.x; h < n_band; h += blockDim.x) {
        const int u = tl.start + lo + h;
        const float4 r = band[h];
        const bool in_tile = h + lo >= 0 && h + lo < tl.len;
        const float rh = in_tile ? b.rho[u] : rho_of_hit<CHI>(b, p, ev, fw, r, b.lay_s[u]);
        band[h] = make_float4(r.x, r.y, rh, __int_as_float(b.sid[u]));
    }
    __syncthreads();
    if (sh.rows <= 2)
        nh_sorted<2>(b, p, tl, sh, band);
    else
        nh_sorted<DT_ROWS>(b, p, tl, sh, band);
    __syncthreads();
}

}  // namespace clue
