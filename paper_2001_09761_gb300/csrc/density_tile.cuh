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
//    rows): the band is staged once (one bulk copy), the tile's hits are
//    ordered by descending candidate count (a counting sort in shared
//    memory), so the 32 lanes of a warp take hits with near-equal windows,
//    warps take the next 32 hits of the order as they finish the last, and
//    each lane walks its window's runs as one flat loop (no per-row
//    reconvergence);
//  * per-hit form otherwise (windows of more rows, bands beyond the staging
//    capacity): one thread per hit, in grid order, walks its window in global
//    memory (neighbouring hits of dense regions have similar windows, so the
//    lanes of a warp stay close there too).
//
// Every form computes the same function of the neighbour sets (the exact
// density, the lexicographic minimum), so the form, the order of the hits and
// the order of the candidates never change a result.
#pragma once

#include "bulk_copy.cuh"
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
    int lo2, hi2, hrows;               // the fused form's staging: the band and the halo
                                       // hits' own density windows, their most rows
    int next[2];                       // the sorted form's work counters (rho, nh)
    unsigned long long bar;            // completion of the band's bulk copy
};

// A wait on a bulk copy gives up after this much device time (a copy of the
// largest band takes microseconds).
constexpr unsigned long long STAGE_WAIT_NS = 50ull * 1000 * 1000;

// Per-CTA set-up of the staging barrier (before the CTA's first tile); the
// phase parity then goes with the CTA's threads from tile to tile.
__device__ __forceinline__ void stage_init(DensityShared &sh) {
    if (threadIdx.x == 0) bulk_bar_init(&sh.bar);
    __syncthreads();
}

// Stage n records from global `src` into the band with one bulk copy; every
// thread returns once they are there (true), or false (the same in every
// thread, the error word raised) when the wait gave up.  Called by the whole
// CTA, after a barrier that ends every earlier access to the band.
__device__ __forceinline__ bool stage_band(const Buffers &b, const float4 *src, int n,
                                           float4 *band, DensityShared &sh, unsigned &parity) {
    if (n <= 0) return true;
    if (threadIdx.x == 0) bulk_load(band, src, (unsigned)n * (unsigned)sizeof(float4), &sh.bar);
    const bool ok = bulk_bar_wait(&sh.bar, parity, STAGE_WAIT_NS);
    if (!ok) {
        bulk_bar_wait(&sh.bar, parity, STAGE_WAIT_NS);  // the copy must not outlive the CTA
        if (threadIdx.x == 0) atomicOr(&b.ctrl->err, ERRBIT_TIMEOUT);
    }
    parity ^= 1u;
    return ok;
}

// Add one to counter cnt[key] for every lane of the warp (key < 0: none) and
// return the lane's slot: the counter's old value plus the lane's rank among
// the lanes of equal key.  Lanes of equal key share one shared-memory atomic
// (neighbouring hits often fall in the same class).  All 32 lanes call it.
__device__ __forceinline__ int warp_class_add(int *cnt, int key) {
    const unsigned peers = __match_any_sync(FULL_MASK, key);
    const int leader = __ffs(peers) - 1;
    int base = 0;
    if (lane_id() == leader && key >= 0) base = atomicAdd(&cnt[key], __popc(peers));
    base = __shfl_sync(FULL_MASK, base, leader);
    return base + __popc(peers & lanemask_lt());
}

// The work class of a window of T candidates (descending T: class 0 first).
__device__ __forceinline__ int work_class(unsigned T) {
    return DT_BUCKETS - 1 - (int)min(T, (unsigned)(DT_BUCKETS - 1));
}

// The tile's windows of radius parameter `dr` into sh.win (rows past DT_ROWS
// and starts past DT_OUT are flagged through sh.rows / the band, which then
// disqualify the sorted form), the band and the work histogram.  A thread
// takes the tile's hits k = threadIdx.x + u * blockDim.x, u < U, and issues
// each round of loads (records and layers, then every window row's bounds)
// for all of them before it waits on any.  Cell indices are 32-bit (a run
// has at most 2^31 - 2 cells).  The loop runs alike in all lanes of a warp.
template <int U>
__device__ __forceinline__ void tile_windows(const Buffers &b, const Tile &tl,
                                             const EventDesc &ev, float dr,
                                             DensityShared &sh) {
    if (threadIdx.x < DT_BUCKETS) sh.hist[threadIdx.x] = 0;
    if (threadIdx.x == 0) {
        sh.lo = INT_MAX;
        sh.hi = INT_MIN;
        sh.rows = 0;
        sh.next[0] = 0;
        sh.next[1] = 0;
    }
    __syncthreads();
    const int32_t *cs = b.cell_start + ev.cell_off;  // the event's cells
    const int nbx = ev.nbx, nbxy = ev.nbx * ev.nby;
    int lo = INT_MAX, hi = INT_MIN, rows = 0;
    for (int k0 = threadIdx.x; k0 - lane_id() < tl.len; k0 += U * blockDim.x) {
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
        int row0[U];
        int a[U][DT_ROWS], e[U][DT_ROWS];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            w[u] = window_of(me[u].x, me[u].y, dr, ev);
            row0[u] = lay[u] * nbxy + w[u].ly * nbx;
#pragma unroll
            for (int r = 0; r < DT_ROWS; ++r) {
                const bool in = w[u].ly + r <= w[u].hy;
                const int row = row0[u] + (in ? r * nbx : 0);
                a[u][r] = in ? cs[row + w[u].lx] : 0;
                e[u][r] = in ? cs[row + w[u].hx + 1] : 0;
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int k = k0 + u * blockDim.x;
            int cls = -1;
            if (k < tl.len) {
                const int nr = w[u].hy - w[u].ly + 1;
                unsigned T = 0;
                int last = e[u][0];
#pragma unroll
                for (int r = 0; r < DT_ROWS; ++r) T += (unsigned)(e[u][r] - a[u][r]);
                for (int r = DT_ROWS; r < nr; ++r) {  // rows the sorted form does not take
                    const int row = row0[u] + r * nbx;
                    const int u0 = cs[row + w[u].lx];
                    last = cs[row + w[u].hx + 1];
                    T += (unsigned)(last - u0);
                }
                if (nr > 1 && nr <= DT_ROWS) last = nr == 2 ? e[u][1] : e[u][2];
                lo = min(lo, a[u][0] - tl.start);
                hi = max(hi, last - tl.start);
                rows = max(rows, nr);
                sh.win[k] = make_uint4(pack_row(a[u][0] - tl.start, e[u][0] - a[u][0]),
                                       pack_row(a[u][1] - tl.start, e[u][1] - a[u][1]),
                                       pack_row(a[u][2] - tl.start, e[u][2] - a[u][2]),
                                       min(T, 65535u));
                cls = work_class(T);
            }
            warp_class_add(sh.hist, cls);
        }
    }
    lo = __reduce_min_sync(FULL_MASK, lo);
    hi = __reduce_max_sync(FULL_MASK, hi);
    rows = __reduce_max_sync(FULL_MASK, rows);
    if (lane_id() == 0) {
        atomicMin(&sh.lo, lo);
        atomicMax(&sh.hi, hi);
        atomicMax(&sh.rows, rows);
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
    for (int k = threadIdx.x; k - lane_id() < tl.len; k += blockDim.x) {  // alike per warp
        const int pos = warp_class_add(sh.hist, k < tl.len ? work_class(sh.win[k].w) : -1);
        if (k < tl.len) sh.perm[pos] = (unsigned short)k;
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
        T = o2 + row_len(w.z);  // (w.w holds the count until the tile's rho replace it)
        b0 = row_start(w.x) - lo;
        b1 = row_start(w.y) - lo - o1;
        b2 = row_start(w.z) - lo - o2;
    }
    __device__ __forceinline__ int at(int c) const {
        if (ROWS <= 2) return c + (c < o1 ? b0 : b1);
        return c + (c < o1 ? b0 : (c < o2 ? b1 : b2));
    }
};

// The next 32 of the tile's hits in sorted order for the calling warp (its
// lanes take sorted positions j0 + lane): warps take chunks as they finish
// the last, so the heavy chunks at the front of the order spread over the
// warps and none runs on long after the rest (the phase ends at a barrier).
__device__ __forceinline__ int grab_chunk(int *next) {
    int j0 = 0;
    if (lane_id() == 0) j0 = atomicAdd(next, 32);
    return __shfl_sync(FULL_MASK, j0, 0);
}

// ---- rho ---------------------------------------------------------------------

// rho of the tile's hits in the sorted form (the band staged from sorted
// position tl.start + lo on, hits ordered).
template <int CHI, int ROWS>
__device__ __forceinline__ void rho_sorted(const Buffers &b, const Params &p, const Tile &tl,
                                           const EventDesc &ev, const FixedW &fw,
                                           DensityShared &sh, const float4 *band, int lo) {
    const bool fixed = CHI == 0 && fw.on;
    for (int j0 = grab_chunk(&sh.next[0]); j0 < tl.len; j0 = grab_chunk(&sh.next[0])) {
        const int j = j0 + lane_id();
        if (j >= tl.len) continue;  // the warp's last chunk: lanes past the tile idle
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
        sh.win[k].w = __float_as_uint(r);  // for the fused form's restaging
    }
}

template <int CHI, int U>
__device__ __forceinline__ bool rho_tile(const Buffers &b, const Params &p, int t,
                                         DensityShared &sh, float4 *band, unsigned &parity) {
    const Tile tl = b.tiles[t];
    const EventDesc ev = b.events[tl.event];
    const FixedW fw = fixed_weights(b.wexp + 2 * tl.event, CHI);  // uniform per event
    tile_windows<U>(b, tl, ev, p.rwin_rho, sh);
    if (!tile_sorted(sh, p.band_cap)) {  // per-hit form
        for (int k = threadIdx.x; k < tl.len; k += blockDim.x) {
            const int q = tl.start + k;
            const float4 me = b.sp[q];
            store_rho(b, p, q, me.x, me.y, rho_of_hit<CHI>(b, p, ev, fw, me, b.lay_s[q]));
        }
        __syncthreads();
        return true;
    }
    tile_sort(tl, sh);
    const int lo = sh.lo, n_band = sh.hi - sh.lo;
    if (!stage_band(b, b.sp + tl.start + lo, n_band, band, sh, parity)) return false;
    if (sh.rows <= 2)
        rho_sorted<CHI, 2>(b, p, tl, ev, fw, sh, band, sh.lo);
    else
        rho_sorted<CHI, DT_ROWS>(b, p, tl, ev, fw, sh, band, sh.lo);
    __syncthreads();
    return true;
}

// ---- nh, delta and the decision ----------------------------------------------

// nh of the tile's hits in the sorted form (the band staged as x, y, rho, id
// from sorted position tl.start + lo on).
template <int ROWS>
__device__ __forceinline__ void nh_sorted(const Buffers &b, const Params &p, const Tile &tl,
                                          DensityShared &sh, const float4 *band, int lo) {
    for (int j0 = grab_chunk(&sh.next[1]); j0 < tl.len; j0 = grab_chunk(&sh.next[1])) {
        const int j = j0 + lane_id();
        if (j >= tl.len) continue;  // the warp's last chunk: lanes past the tile idle
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
__device__ __forceinline__ bool nh_tile(const Buffers &b, const Params &p, int t,
                                        DensityShared &sh, float4 *band, unsigned &parity) {
    const Tile tl = b.tiles[t];
    const EventDesc ev = b.events[tl.event];
    tile_windows<U>(b, tl, ev, p.rwin_nh, sh);
    if (!tile_sorted(sh, p.band_cap)) {  // per-hit form
        for (int k = threadIdx.x; k < tl.len; k += blockDim.x) {
            const int q = tl.start + k;
            const float4 me = nh_record(b, p, q);
            nh_store(b, p, q, id_of(me), me.z, nh_of_hit(b, p, ev, me.x, me.y, me.z, b.lay_s[q]));
        }
        __syncthreads();
        return true;
    }
    tile_sort(tl, sh);
    const int lo = sh.lo, n_band = sh.hi - sh.lo;
    if (!p.fused) {  // the separate kernels' (x, y, rho, id) records: one copy
        if (!stage_band(b, b.spr + tl.start + lo, n_band, band, sh, parity)) return false;
    } else {
        for (int h = threadIdx.x; h < n_band; h += blockDim.x)
            band[h] = nh_record(b, p, tl.start + lo + h);
        __syncthreads();
    }
    if (sh.rows <= 2)
        nh_sorted<2>(b, p, tl, sh, band, sh.lo);
    else
        nh_sorted<DT_ROWS>(b, p, tl, sh, band, sh.lo);
    __syncthreads();
    return true;
}

// Halo hits of the fused form each thread takes at most (its share of the
// band's hits outside the tile).
constexpr int HALO_PER_THREAD = 4;

// Records a thread restages per round of id loads.
constexpr int RESTAGE_ILP = 4;

// Halo hits per thread whose windows the sizing pass keeps in registers (as
// pack_row words) for the density pass; a fourth one's window is looked up
// again.  At 256 threads a tile of the blob recipe has at most two halo hits
// per thread; denser grid rows have more.
constexpr int HALO_KEPT = 3;

// A halo hit's density window (radius d_c) as up to DT_ROWS runs of sorted
// positions (relative to the tile start): its first and last position and
// its rows (more than DT_ROWS rows: only `rows` is meaningful).
struct HaloWin {
    int a[DT_ROWS], l[DT_ROWS];
    int first, last, rows;
    // from the rows as pack_row keeps them (a and l only)
    __device__ __forceinline__ explicit HaloWin(const unsigned (&pr)[DT_ROWS]) {
#pragma unroll
        for (int r = 0; r < DT_ROWS; ++r) {
            a[r] = row_start(pr[r]);
            l[r] = row_len(pr[r]);
        }
        first = last = rows = 0;
    }
    __device__ __forceinline__ HaloWin(const Buffers &b, const EventDesc &ev, const Params &p,
                                       const float4 &me, int lay, int tstart) {
        const Window w = window_of(me.x, me.y, p.rwin_rho, ev);
        const int32_t *cs = b.cell_start + ev.cell_off;  // the event's cells (32-bit indices)
        const int row0 = lay * (ev.nbx * ev.nby) + w.ly * ev.nbx;
        rows = w.hy - w.ly + 1;
        first = INT_MAX;
        last = INT_MIN;
#pragma unroll
        for (int r = 0; r < DT_ROWS; ++r) {
            const bool in = r < rows;
            const int row = row0 + (in ? r * ev.nbx : 0);
            const int s0 = in ? cs[row + w.lx] : 0, e = in ? cs[row + w.hx + 1] : 0;
            a[r] = s0 - tstart;
            l[r] = e - s0;
            if (in) {
                first = min(first, a[r]);
                last = max(last, e - tstart);
            }
        }
    }
};

// rho of a halo hit (sorted position q) from the staged band (sorted
// position tl.start + lo on): the same arithmetic as rho_sorted, over the
// hit's own d_c window.
template <int CHI>
__device__ __forceinline__ float rho_from_band(const Buffers &b, const Params &p,
                                               const EventDesc &ev, const FixedW &fw,
                                               const float4 *band, const HaloWin &hw, int lo,
                                               const float4 &me, int q) {
    const int T = hw.l[0] + hw.l[1] + hw.l[2];
    const int o1 = hw.l[0], o2 = hw.l[0] + hw.l[1];
    const int b0 = hw.a[0] - lo, b1 = hw.a[1] - lo - o1, b2 = hw.a[2] - lo - o2;
    float r;
    bool ok;
    if (CHI == 0 && fw.on) {
        long long acc = 0;
        for (int c = 0; c < T; ++c) {  // branch-free body
            const float4 h = band[c + (c < o1 ? b0 : (c < o2 ? b1 : b2))];
            acc += sq_dist(me.x, me.y, h.x, h.y) < p.dc2 ? fixed_weight_of(h) : 0ll;
        }
        r = __fmul_rn(__ll2float_rn(acc), fw.unit);
        ok = 32 - __clz(T) <= fw.budget;
    } else {
        TwoSumAcc a;
        for (int c = 0; c < T; ++c) {  // branch-free body
            const float4 h = band[c + (c < o1 ? b0 : (c < o2 ? b1 : b2))];
            const float d2 = sq_dist(me.x, me.y, h.x, h.y);
            const bool near = d2 < p.dc2;
            a.add(near ? term_of<CHI>(d2, h.z, p.chi_inv) : 0.0f, near);
        }
        r = __fadd_rn(a.s, a.c);
        ok = a.exact();
    }
    if (!ok) {
        const Window w = window_of(me.x, me.y, p.rwin_rho, ev);
        const int64_t plane = ev.cell_off + (int64_t)b.lay_s[q] * ev.nbx * ev.nby;
        r = rho_wide<CHI>(b, plane, ev.nbx, w, me.x, me.y, p.dc2, p.chi_inv,
                          CHI == 0 && fw.on ? fw.unit : 0.0f);
    }
    return r;
}

// ---- rho, nh, delta and the decision in one pass (the fused form) ----------
//
// One CTA per tile, with the sorted form's staging done once for both steps:
// the windows of radius max(d_c, d_m) (a superset of both searches' windows;
// the exact d2 tests pick the neighbours), one ordering of the tile's hits by
// window population, one band staged.  Then rho of the tile's hits from the
// band (written to global memory for the intermediates and for other tiles);
// rho of the band's hits outside the tile (the halo, whose densities the
// tile's nh needs), each computed again by every tile whose band holds it
// (identical values): the staging is widened to the halo hits' own d_c
// windows where that fits (their rho then comes from shared memory too), else
// they walk their windows in global memory; the band restaged in place as
// (x, y, rho, id); nh and the decision of the tile's hits.  So rho goes
// straight to nh with no pass over the batch in between.  A tile the sorted
// form does not take (a band beyond the staging capacity, windows of more
// rows) or whose halo holds more hits than the tile itself (dense
// neighbourhoods) gets only its rho here (rho_tile's forms) and joins a list
// that k_nh_rest finishes after every tile's rho is written.
template <int CHI, int U>
__device__ __forceinline__ bool density_tile(const Buffers &b, const Params &p, int t,
                                             DensityShared &sh, float4 *band, unsigned &parity) {
    const Tile tl = b.tiles[t];
    const EventDesc ev = b.events[tl.event];
    const FixedW fw = fixed_weights(b.wexp + 2 * tl.event, CHI);  // uniform per event
    tile_windows<U>(b, tl, ev, fmaxf(p.rwin_rho, p.rwin_nh), sh);
    // fused when the band fits and its halo (whose rho is computed again here)
    // holds at most as many hits as the tile
    const bool fused = tile_sorted(sh, p.band_cap) && sh.hi - sh.lo <= 2 * tl.len;
    if (!fused) {
        __syncthreads();  // every thread has read the shared state rho_tile resets
        if (!rho_tile<CHI, U>(b, p, t, sh, band, parity)) return false;
        if (threadIdx.x == 0) b.rest[atomicAdd(&b.ctrl->nrest, 1)] = t;
        return true;
    }
    tile_sort(tl, sh);
    const int lo = sh.lo, hi = sh.hi, n_band = hi - lo, t0 = -lo;
    const int n_halo = n_band - tl.len;
    // The halo hits' density windows (radius d_c) reach past the band: where
    // every halo hit falls to a thread's HALO_PER_THREAD and the band with
    // those windows fits the staging, all of it is staged and the halo's rho
    // comes from shared memory too; else from global memory (rho_of_hit).
    if (threadIdx.x == 0) {
        sh.lo2 = lo;
        sh.hi2 = hi;
        sh.hrows = 0;
    }
    __syncthreads();
    const bool halo_fits = n_halo <= HALO_PER_THREAD * (int)blockDim.x;
    // the first HALO_KEPT halo hits' windows, relative to the tile start (the
    // wide form's windows lie within the staging, well inside pack_row's range)
    unsigned kept[HALO_KEPT][DT_ROWS];
#pragma unroll
    for (int u = 0; u < HALO_KEPT; ++u)
#pragma unroll
        for (int r = 0; r < DT_ROWS; ++r) kept[u][r] = 0u;
    if (halo_fits) {
        int l2 = lo, h2 = hi, rows = 0;
#pragma unroll
        for (int u = 0; u < HALO_PER_THREAD; ++u) {
            const int i = threadIdx.x + u * (int)blockDim.x;
            if (i >= n_halo) break;
            const int q = tl.start + lo + (i < t0 ? i : i + tl.len);
            const HaloWin hw(b, ev, p, b.sp[q], b.lay_s[q], tl.start);
            if (u < HALO_KEPT)
#pragma unroll
                for (int r = 0; r < DT_ROWS; ++r)
                    kept[u < HALO_KEPT ? u : 0][r] = pack_row(hw.a[r], hw.l[r]);
            l2 = min(l2, hw.first);
            h2 = max(h2, hw.last);
            rows = max(rows, hw.rows);
        }
        l2 = __reduce_min_sync(FULL_MASK, l2);
        h2 = __reduce_max_sync(FULL_MASK, h2);
        rows = __reduce_max_sync(FULL_MASK, rows);
        if (lane_id() == 0) {
            atomicMin(&sh.lo2, l2);
            atomicMax(&sh.hi2, h2);
            atomicMax(&sh.hrows, rows);
        }
    }
    __syncthreads();
    const bool wide = halo_fits && sh.hrows <= DT_ROWS && sh.hi2 - sh.lo2 <= p.band_cap;
    const int base = wide ? sh.lo2 : lo, n_stage = wide ? sh.hi2 - sh.lo2 : n_band;
    if (!stage_band(b, b.sp + tl.start + base, n_stage, band, sh, parity)) return false;
    float hrho[HALO_PER_THREAD];  // the halo's rho, by this thread's halo hits
    if (wide) {
#pragma unroll
        for (int u = 0; u < HALO_PER_THREAD; ++u) {
            const int i = threadIdx.x + u * (int)blockDim.x;
            hrho[u] = 0.0f;
            if (i < n_halo) {
                const int q = tl.start + lo + (i < t0 ? i : i + tl.len);
                const float4 me = band[q - tl.start - base];
                const HaloWin hw = u < HALO_KEPT ? HaloWin(kept[u < HALO_KEPT ? u : 0])
                                                 : HaloWin(b, ev, p, me, b.lay_s[q], tl.start);
                hrho[u] = rho_from_band<CHI>(b, p, ev, fw, band, hw, base, me, q);
            }
        }
    }
    if (sh.rows <= 2)
        rho_sorted<CHI, 2>(b, p, tl, ev, fw, sh, band, base);
    else
        rho_sorted<CHI, DT_ROWS>(b, p, tl, ev, fw, sh, band, base);
    __syncthreads();  // the tile's rho are written; the band's weights are no longer read
    // Restage the band (the nh windows' part of the staging) as (x, y, rho,
    // id): the tile's rho from the windows' slots, the halo's from the
    // threads that computed it (else a walk in global memory); each thread
    // issues its id loads before it writes.
    if (wide) {
        for (int k0 = threadIdx.x; k0 < tl.len; k0 += RESTAGE_ILP * blockDim.x) {
            int id[RESTAGE_ILP];
#pragma unroll
            for (int u = 0; u < RESTAGE_ILP; ++u) {
                const int k = k0 + u * blockDim.x;
                id[u] = k < tl.len ? __ldg(b.sid + tl.start + k) : 0;
            }
#pragma unroll
            for (int u = 0; u < RESTAGE_ILP; ++u) {
                const int k = k0 + u * blockDim.x;
                if (k < tl.len) {
                    const float4 r = band[k - base];
                    band[k - base] = make_float4(r.x, r.y, __uint_as_float(sh.win[k].w),
                                                 __int_as_float(id[u]));
                }
            }
        }
        int hid[HALO_PER_THREAD];
#pragma unroll
        for (int u = 0; u < HALO_PER_THREAD; ++u) {
            const int i = threadIdx.x + u * (int)blockDim.x;
            hid[u] = i < n_halo ? __ldg(b.sid + tl.start + lo + (i < t0 ? i : i + tl.len)) : 0;
        }
#pragma unroll
        for (int u = 0; u < HALO_PER_THREAD; ++u) {
            const int i = threadIdx.x + u * (int)blockDim.x;
            if (i < n_halo) {
                const int h = lo + (i < t0 ? i : i + tl.len) - base;
                const float4 r = band[h];
                band[h] = make_float4(r.x, r.y, hrho[u], __int_as_float(hid[u]));
            }
        }
    } else {
        for (int h = lo - base + threadIdx.x; h < hi - base; h += blockDim.x) {
            const int rel = base + h;  // relative to the tile start
            const bool in_tile = rel >= 0 && rel < tl.len;
            const int u = tl.start + rel;
            const float4 r = band[h];
            const float rh = in_tile ? __uint_as_float(sh.win[rel].w)
                                     : rho_of_hit<CHI>(b, p, ev, fw, r, b.lay_s[u]);
            band[h] = make_float4(r.x, r.y, rh, __int_as_float(__ldg(b.sid + u)));
        }
    }
    __syncthreads();
    if (sh.rows <= 2)
        nh_sorted<2>(b, p, tl, sh, band, base);
    else
        nh_sorted<DT_ROWS>(b, p, tl, sh, band, base);
    __syncthreads();
    return true;
}

}  // namespace clue