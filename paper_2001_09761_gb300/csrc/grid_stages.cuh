// Step S1: the fixed-grid spatial index (Sec. 2.1, Eqs. 1-2): the stage
// bodies, which the kernels in k_grid.cu wrap.
//
// The paper pushes each hit into its bin with an atomic (conflict (i) of
// Sec. 3).  Here the index is a counting sort into one array of hits sorted by
// (event, layer, cell), (x, y, w, id) packed in one float4 per hit, one 16-byte
// load per candidate, which makes every later neighbour scan a walk over
// contiguous memory.  Two forms give the same layout:
//
//  * the two-level sort (every layer of the batch with at most SEG_MAX_CELLS
//    cells, at most SEG_MAX_LAYERS layers): every tile counts its hits per
//    layer in shared memory and writes the counts to a table ordered by
//    (event, layer, tile), whose exclusive prefix sum is each tile's run in
//    the layered order (no global atomic); the records are moved into their
//    runs; then one CTA per (event, layer) segment counts its hits per cell in
//    shared memory, scans the counts and writes the cell offsets and the
//    sorted records.  The atomics that rank hits are shared-memory ones;
//  * the direct sort (any grid): hits are counted per cell with global
//    atomics (each returning the hit's arrival rank), a prefix sum over all
//    cells gives the offsets, hit ids are scattered into their cell's segment
//    and a gather writes the sorted records.
//
// The order of hits inside a cell is the atomics' arrival order in both; no
// result depends on it (the density is an exact sum, the nearest-higher a
// lexicographic minimum).
#pragma once

#include "scan.cuh"

namespace clue {

// --- count: bin of every hit, hits per cell ---------------------------------
__device__ __forceinline__ void fill_count_stage(const Buffers &b, const Params &p) {
    __shared__ unsigned s_w[2];  // the tile's weight range
    for (int t = blockIdx.x; t < b.ntiles; t += gridDim.x) {
        const Tile tl = b.tiles[t];
        const EventDesc ev = b.events[tl.event];
        if (threadIdx.x == 0) s_w[0] = s_w[1] = 0xffffffffu;
        __syncthreads();
        for (int k0 = 0; k0 < tl.len; k0 += blockDim.x) {  // uniform over the warp
            const int k = k0 + threadIdx.x;
            weight_range_add(s_w, b.w[tl.start + (k < tl.len ? k : 0)], k < tl.len);
            if (k >= tl.len) continue;
            const int g = tl.start + k;
            const float x = b.x[g], y = b.y[g], w = b.w[g];
            int l = b.layer[g];
            const bool bad = !isfinite(x) || !isfinite(y) || !isfinite(w) || l < 0 || l >= p.L;
            if (bad) {
                atomicOr(&b.ctrl->err, ERRBIT_INPUT);
                l = min(max(l, 0), p.L - 1);
            }
            const int bx = axis_bin(x, ev.xmin, ev.inv_s, ev.nbx);
            const int by = axis_bin(y, ev.ymin, ev.inv_s, ev.nby);
            const int local = (l * ev.nby + by) * ev.nbx + bx;
            b.key[g] = local;
            b.rank[g] = atomicAdd(&b.count[ev.cell_off + local], 1);
            b.rec[g] = make_float4(x, y, w, __int_as_float(local));  // gathered by the ranking
            if (!p.chase) b.fcount[g] = 0;  // follower counters of the follower lists
        }
        __syncthreads();
        if (threadIdx.x == 0) weight_range_flush(b.wexp + 2 * tl.event, s_w);
    }
}

struct LoadI32 {
    const int32_t *a;
    __device__ __forceinline__ int32_t operator()(int64_t i) const { return a[i]; }
};

// --- scatter: every hit's id into its cell's segment at the rank its count
// returned (order within a cell is not yet fixed); one 4-byte scattered
// store, no atomic. ---------------------------------------------------------
__device__ __forceinline__ void fill_scatter_stage(const Buffers &b) {
    for (int t = blockIdx.x; t < b.ntiles; t += gridDim.x) {
        const Tile tl = b.tiles[t];
        const int64_t coff = b.events[tl.event].cell_off;
        for (int k = threadIdx.x; k < tl.len; k += blockDim.x) {
            const int g = tl.start + k;
            b.perm[b.cell_start[coff + b.key[g]] + b.rank[g]] = g;
        }
    }
}

// --- gather: the sorted copy of every hit, in the order of the segments ---
__device__ __forceinline__ void fill_canon_stage(const Buffers &b, const Params &p) {
    for (int t = blockIdx.x; t < b.ntiles; t += gridDim.x) {
        const Tile tl = b.tiles[t];
        const int ev_nbxy = b.events[tl.event].nbx * b.events[tl.event].nby;
        const FixedW fw = fixed_weights(b.wexp + 2 * tl.event, p.chi);
        for (int k = threadIdx.x; k < tl.len; k += blockDim.x) {
            const int pos = tl.start + k;
            const int g = b.perm[pos];
            const float4 r = b.rec[g];  // x, y, w, cell of hit g: one 16-byte gather
            b.sp[pos] = sorted_record(make_float4(r.x, r.y, r.z, __int_as_float(g)), fw);
            b.sid[pos] = g;
            b.lay_s[pos] = __float_as_int(r.w) / ev_nbxy;
        }
    }
}

// --- two-level sort -----------------------------------------------------------

constexpr int FILL_THREADS = 256;      // block of the tile-wise stages (TILE / 4)
constexpr int SEG_THREADS = 512;       // block of the per-segment stage
constexpr int SEG_SMEM_HITS = 16384;   // segments up to this size are permuted in shared memory
// The per-segment stage's small build (events chosen by the host, see
// SMALL_SEG_CELLS; a segment longer than SMALL_SEG_HITS is still sorted
// right, through global memory).
constexpr int SMALL_SEG_THREADS = 128;
constexpr int SMALL_SEG_HITS = 4096;
static_assert(TILE % FILL_THREADS == 0, "tile / block");

// Where the run table holds (event e, layer l, tile t of e).
// Layer l == L addresses the next event's block (the table's end for the
// last event), so that entry l + 1 ends segment l.
__device__ __forceinline__ int64_t run_index(const EventDesc &ev, int L, int l, int t) {
    return (int64_t)ev.tile0 * L + (int64_t)l * ev.ntiles + (t - ev.tile0);
}

// Layer count: the tile's hits per layer in a shared histogram, written to
// the run table (every layer, zeros included), whose exclusive prefix sum is
// the tile's run in each of its (event, layer) segments.  Layers outside
// [0, L) flag the input error and are clamped, as in the direct sort.  All of
// a thread's loads are issued before its atomics, so their latencies overlap.
// As the run's first kernel it also resets what later kernels accumulate
// into: the control words (CTA 0), the event's weight range (its first tile)
// and, in chase mode, the seed-bit words of the tile's hits (and the word
// after them, so that the word past the last hit is clear too).  Needs
// FILL_THREADS threads and L ints of dynamic shared memory.
__device__ __forceinline__ void fill_layers_stage(const Buffers &b, const Params &p) {
    extern __shared__ int s_hist[];
    constexpr int PER = TILE / FILL_THREADS;
    static_assert(FILL_THREADS >= TILE / 32 + 2, "one thread per seed-bit word");
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        b.ctrl->overflow = 0u;
        b.ctrl->fsize[0] = b.ctrl->fsize[1] = b.ctrl->fsize[2] = 0;
        b.ctrl->npend = 0;
        b.ctrl->nrest = 0;
    }
    for (int t = blockIdx.x; t < b.ntiles; t += gridDim.x) {
        const Tile tl = b.tiles[t];
        for (int l = threadIdx.x; l < p.L; l += FILL_THREADS) s_hist[l] = 0;
        if (t == b.events[tl.event].tile0 && threadIdx.x < 2)
            b.wexp[2 * tl.event + threadIdx.x] = 0xffffffffu;
        if (p.chase) {
            const int w0 = tl.start >> 5, w1 = (tl.start + tl.len) >> 5;
            if ((int)threadIdx.x <= w1 - w0) b.sbits[w0 + threadIdx.x] = 0u;
        }
        int lay[PER];
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            const int k = threadIdx.x + u * FILL_THREADS;
            lay[u] = k < tl.len ? b.layer[tl.start + k] : 0;
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            const int k = threadIdx.x + u * FILL_THREADS;
            if (k < tl.len) {
                int l = lay[u];
                if (l < 0 || l >= p.L) {
                    atomicOr(&b.ctrl->err, ERRBIT_INPUT);
                    l = min(max(l, 0), p.L - 1);
                }
                atomicAdd(&s_hist[l], 1);
                if (!p.chase) b.fcount[tl.start + k] = 0;  // follower counters of the lists
            }
        }
        __syncthreads();
        const EventDesc ev = b.events[tl.event];
        for (int l = threadIdx.x; l < p.L; l += FILL_THREADS)
            b.tcount[run_index(ev, p.L, l, t)] = s_hist[l];
        __syncthreads();  // s_hist is reset for the next tile
    }
}

// Exclusive scan, in place, of a[0..4 * n4) in shared memory (16-byte
// aligned) by the whole CTA: each warp takes a contiguous chunk and walks it
// 32 int4 at a time (lane j reads the j-th 16 bytes: no bank conflicts), each
// lane scanning its four entries, with the warps' chunk sums scanned in `ws`
// (>= 32 ints).  Ends with a barrier.
__device__ __forceinline__ void smem_excl_scan4(int *a, int n4, int *ws) {
    int4 *a4 = reinterpret_cast<int4 *>(a);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int per = (((n4 + nw - 1) / nw) + 31) & ~31;
    const int c0 = min(warp * per, n4), c1 = min(c0 + per, n4);
    int sum = 0;
    for (int c = c0 + lane; c < c1; c += 32) {
        const int4 v = a4[c];
        sum += (v.x + v.y) + (v.z + v.w);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(FULL_MASK, sum, o);
    if (lane == 0) ws[warp] = sum;
    __syncthreads();
    if (warp == 0) {
        const int v = lane < nw ? ws[lane] : 0;
        const int incl = warp_incl_scan(v);
        if (lane < nw) ws[lane] = incl - v;
    }
    __syncthreads();
    int run = ws[warp];
    for (int base = c0; base < c1; base += 32) {
        const int c = base + lane;
        const int4 v = c < c1 ? a4[c] : make_int4(0, 0, 0, 0);
        const int t = (v.x + v.y) + (v.z + v.w);
        const int incl = warp_incl_scan(t);
        const int ex = run + incl - t;
        if (c < c1) a4[c] = make_int4(ex, ex + v.x, ex + v.x + v.y, ex + v.x + v.y + v.z);
        run += __shfl_sync(FULL_MASK, incl, 31);
    }
    __syncthreads();
}

// Zero a[0..4 * n4) in shared memory (16-byte aligned), 16 bytes per store.
__device__ __forceinline__ void smem_zero4(int *a, int n4) {
    int4 *a4 = reinterpret_cast<int4 *>(a);
    for (int c = threadIdx.x; c < n4; c += blockDim.x) a4[c] = make_int4(0, 0, 0, 0);
}

// Exclusive scan, in place, of 16-bit counts packed two to a word (cell 2w in
// the low half of word w, 2w + 1 in the high half), a[0..4 * n4) words in
// shared memory (16-byte aligned), by the whole CTA, as smem_excl_scan4 does
// for ints; every prefix must stay below 2^16.  Ends with a barrier.
__device__ __forceinline__ void smem_excl_scan16(unsigned *a, int n4, int *ws) {
    uint4 *a4 = reinterpret_cast<uint4 *>(a);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int per = (((n4 + nw - 1) / nw) + 31) & ~31;
    const int c0 = min(warp * per, n4), c1 = min(c0 + per, n4);
    // the sum of a word's two halves, and of a uint4's eight
    auto hsum = [](unsigned w) { return (int)((w & 0xffffu) + (w >> 16)); };
    int sum = 0;
    for (int c = c0 + lane; c < c1; c += 32) {
        const uint4 v = a4[c];
        sum += (hsum(v.x) + hsum(v.y)) + (hsum(v.z) + hsum(v.w));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(FULL_MASK, sum, o);
    if (lane == 0) ws[warp] = sum;
    __syncthreads();
    if (warp == 0) {
        const int v = lane < nw ? ws[lane] : 0;
        const int incl = warp_incl_scan(v);
        if (lane < nw) ws[lane] = incl - v;
    }
    __syncthreads();
    int run = ws[warp];
    for (int base = c0; base < c1; base += 32) {
        const int c = base + lane;
        const uint4 v = c < c1 ? a4[c] : make_uint4(0u, 0u, 0u, 0u);
        const int t = (hsum(v.x) + hsum(v.y)) + (hsum(v.z) + hsum(v.w));
        const int incl = warp_incl_scan(t);
        unsigned e = (unsigned)(run + incl - t);  // exclusive offset of the uint4's first cell
        unsigned o[4];
        const unsigned w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const unsigned lo = e, hi = e + (w[i] & 0xffffu);
            o[i] = lo | (hi << 16);
            e = hi + (w[i] >> 16);
        }
        if (c < c1) a4[c] = make_uint4(o[0], o[1], o[2], o[3]);
        run += __shfl_sync(FULL_MASK, incl, 31);
    }
    __syncthreads();
}

// A 16-bit counter of the packed array: add one, return its old value.
__device__ __forceinline__ int inc16(unsigned *a, unsigned c) {
    const unsigned sh = (c & 1u) << 4;
    return (int)((atomicAdd(&a[c >> 1], 1u << sh) >> sh) & 0xffffu);
}
__device__ __forceinline__ int get16(const unsigned *a, unsigned c) {
    return (int)((a[c >> 1] >> ((c & 1u) << 4)) & 0xffffu);
}

__device__ __forceinline__ int cell_in_layer(float x, float y, const EventDesc &ev) {
    return axis_bin(y, ev.ymin, ev.inv_s, ev.nby) * ev.nbx + axis_bin(x, ev.xmin, ev.inv_s, ev.nbx);
}

// Layer placement, one tile at a time: the tile's records are first sorted by
// layer in shared memory (ranks from shared atomics), then written out so that
// consecutive threads write consecutive slots of a layer's run, at the run
// the count reserved, each with its cell in the layer (16 bits, in `cell16`).
// The layer is clamped exactly as the count clamped it.  Needs FILL_THREADS
// threads and 2 L ints (L rounded up to a multiple of 4) of dynamic shared
// memory.
__device__ __forceinline__ void fill_place_stage(const Buffers &b, const Params &p) {
    __shared__ float4 s_rec[TILE];
    __shared__ int s_lay[TILE];
    __shared__ int ws[32];
    __shared__ unsigned s_w[2];  // the tile's weight range
    extern __shared__ int4 s_off4[];  // tile offsets by layer; destinations by layer
    int *s_off = reinterpret_cast<int *>(s_off4);
    constexpr int PER = TILE / FILL_THREADS;
    const int L4 = (p.L + 3) / 4;
    for (int t = blockIdx.x; t < b.ntiles; t += gridDim.x) {
        const Tile tl = b.tiles[t];
        smem_zero4(s_off, L4);
        if (threadIdx.x == 0) s_w[0] = s_w[1] = 0xffffffffu;
        // the tile's run start in the segment of layer threadIdx.x, loaded now
        // and used after the ranking (no round trip of its own; layers past
        // the block size load theirs then)
        const EventDesc ev = b.events[tl.event];
        const int tb0 = (int)threadIdx.x < p.L ? b.tbase[run_index(ev, p.L, threadIdx.x, t)] : 0;
        float4 r[PER];
        int lay[PER];
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            const int k = threadIdx.x + u * FILL_THREADS;
            const int g = tl.start + (k < tl.len ? k : 0);
            r[u] = make_float4(b.x[g], b.y[g], b.w[g], __int_as_float(g));
            lay[u] = b.layer[g];
        }
        __syncthreads();
        // the weight range of this thread's hits, then of the warp (one shared
        // atomic per warp)
        {
            unsigned lo = 0xffffffffu, hi = 0xffffffffu;
#pragma unroll
            for (int u = 0; u < PER; ++u) {
                const unsigned bits = __float_as_uint(r[u].z) & 0x7fffffffu;
                const unsigned eb = bits >> 23;
                if ((int)threadIdx.x + u * FILL_THREADS < tl.len && bits != 0u && eb < 255u) {
                    lo = min(lo, max(eb, 1u));
                    hi = min(hi, 255u - eb);
                }
            }
            weight_range_add_bounds(s_w, lo, hi);
        }
        int rk[PER];
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            const int k = threadIdx.x + u * FILL_THREADS;
            if (k < tl.len) {
                if (!isfinite(r[u].x) || !isfinite(r[u].y) || !isfinite(r[u].z))
                    atomicOr(&b.ctrl->err, ERRBIT_INPUT);
                lay[u] = min(max(lay[u], 0), p.L - 1);
                rk[u] = atomicAdd(&s_off[lay[u]], 1);
            }
        }
        __syncthreads();
        smem_excl_scan4(s_off, L4, ws);
        if (threadIdx.x == 0) {  // no read first: the thread does not wait on the atomics
            if (s_w[0] != 0xffffffffu) atomicMin(&b.wexp[2 * tl.event], s_w[0]);
            if (s_w[1] != 0xffffffffu) atomicMin(&b.wexp[2 * tl.event + 1], s_w[1]);
        }
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            const int k = threadIdx.x + u * FILL_THREADS;
            if (k < tl.len) {
                const int slot = s_off[lay[u]] + rk[u];
                s_rec[slot] = r[u];
                s_lay[slot] = lay[u];
            }
        }
        __syncthreads();
        // slot i of layer l goes to dst[l] + i (only the tile's layers are set)
        int *s_dst = s_off + 4 * L4;
        for (int l = threadIdx.x; l < p.L; l += FILL_THREADS) {
            const int end = l + 1 < p.L ? s_off[l + 1] : tl.len;
            if (end > s_off[l])
                s_dst[l] = (l == (int)threadIdx.x ? tb0 : b.tbase[run_index(ev, p.L, l, t)]) -
                           s_off[l];
        }
        __syncthreads();
        for (int i = threadIdx.x; i < tl.len; i += FILL_THREADS) {
            const float4 r = s_rec[i];
            const int dst = s_dst[s_lay[i]] + i;
            b.rec[dst] = r;
            b.cell16[dst] = (unsigned short)cell_in_layer(r.x, r.y, ev);
        }
        __syncthreads();  // the staging arrays are reused by the next tile
    }
}

// L2 prefetch of `bytes` bytes at `p` (both multiples of 16) by the copy
// engine: one instruction, no registers, no wait.
__device__ __forceinline__ void prefetch_l2_bulk(const void *p, unsigned bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// Cell sort of one segment per CTA.  The segment's records are first
// prefetched into L2 (they are read once more, in sorted order, at the end).
// Its hits are counted per cell in shared memory (cells from `cell16`), the
// counts scanned and the layer's cell offsets written.  A segment of at most
// PERM_HITS hits keeps 16-bit counters, two to a word (its offsets stay
// below 2^16), and is then permuted in shared memory: a second pass over its
// cells (just read, so in L2) takes each hit's slot with a shared atomic on
// its cell's running offset and stores the hit's 16-bit index there; the
// records are then written in slot order, a gather from L2 and coalesced
// stores.  A longer segment counts in 32-bit words, keeps the first pass's
// ranks in `perm` and writes each record at its cell's offset plus its rank.
// Loads are issued in batches ahead of the atomics and stores that use them.
// The last segment also writes the end offset cell_start[C].  Two builds: 512
// threads and SEG_SMEM_HITS-hit permutations (42 registers: three CTAs per
// SM, which the shared memory of a 16k-cell layer allows), and 128 threads
// and SMALL_SEG_HITS for the run's events of few hits per layer and few
// cells (a dozen CTAs per SM, so that their many short segments overlap).
// Needs fill_cells_smem<PERM_HITS>(cells_cap) bytes of dynamic shared memory.
template <int PERM_HITS>
__host__ __device__ constexpr int fill_cells_smem(int max_cells) {
    return (max_cells + 3) / 4 * 16 > (max_cells + 7) / 8 * 16 + PERM_HITS * 2
               ? (max_cells + 3) / 4 * 16
               : (max_cells + 7) / 8 * 16 + PERM_HITS * 2;
}

// THREADS per CTA; segments of at most PERM_HITS hits are permuted in shared
// memory; the CTAs take the segments of events seg_ev[ev0 .. ev0 + n_ev)
// (all events in order when the run has no such list), layer by layer, and
// cells_cap bounds their layers' cells (the shared memory's layout).
template <int THREADS, int PERM_HITS>
__device__ __forceinline__ void fill_cells_stage(const Buffers &b, const Params &p, int ev0,
                                                 int n_ev, int cells_cap) {
    static_assert(PERM_HITS <= 65536, "16-bit indices and offsets");
    extern __shared__ int4 s_cell4[];
    __shared__ int ws[32];
    int *s_cell = reinterpret_cast<int *>(s_cell4);             // 32-bit counters (long segments)
    unsigned *s_c16 = reinterpret_cast<unsigned *>(s_cell4);    // 16-bit counters (short ones)
    unsigned short *s_perm = (unsigned short *)(s_cell4 + (cells_cap + 7) / 8);
    constexpr int C = 8;  // cells loaded per batch
    constexpr int G = 2;  // gathers in flight per thread
    const int64_t nseg = (int64_t)n_ev * p.L;
    for (int64_t i = blockIdx.x; i < nseg; i += gridDim.x) {
        const int at = ev0 + (int)(i / p.L);
        const int e = b.seg_ev ? b.seg_ev[at] : at;
        const int l = (int)(i % p.L);
        const int64_t sg = (int64_t)e * p.L + l;  // the segment's place in the run
        const EventDesc ev = b.events[e];
        const int nbxy = ev.nbx * ev.nby;
        const int64_t cbase = ev.cell_off + (int64_t)l * nbxy;
        // the segment runs from its first tile's run to the next segment's
        const int s0 = b.tbase[run_index(ev, p.L, l, ev.tile0)];
        const int n = b.tbase[run_index(ev, p.L, l + 1, ev.tile0)] - s0;
        const bool small = n <= PERM_HITS;  // uniform over the CTA
        const int n4 = small ? (nbxy + 7) / 8 : (nbxy + 3) / 4;
        const FixedW fw = fixed_weights(b.wexp + 2 * e, p.chi);
        if (small && n > 0 && threadIdx.x == 0) prefetch_l2_bulk(b.rec + s0, (unsigned)n * 16u);
        const unsigned short *cell = b.cell16 + s0;
        // zero the wider (32-bit) counters' extent: it covers the 16-bit ones
        // too, and needs only the event's grid, not the segment's size
        smem_zero4(s_cell, (nbxy + 3) / 4);
        __syncthreads();
        for (int k0 = threadIdx.x; k0 < n; k0 += C * THREADS) {
            unsigned c[C];
#pragma unroll
            for (int u = 0; u < C; ++u) {
                const int k = k0 + u * THREADS;
                c[u] = k < n ? cell[k] : 0xffffu;
            }
#pragma unroll
            for (int u = 0; u < C; ++u) {
                if (c[u] == 0xffffu) break;
                if (small) {
                    inc16(s_c16, c[u]);
                } else {
                    const int rk = atomicAdd(&s_cell[c[u]], 1);
                    b.perm[s0 + k0 + u * THREADS] = rk;
                }
            }
        }
        __syncthreads();
        if (small) {
            smem_excl_scan16(s_c16, n4, ws);
            for (int c = threadIdx.x; c < nbxy; c += THREADS)
                b.cell_start[cbase + c] = s0 + get16(s_c16, (unsigned)c);
        } else {
            smem_excl_scan4(s_cell, n4, ws);
            for (int c = threadIdx.x; c < nbxy; c += THREADS)
                b.cell_start[cbase + c] = s0 + s_cell[c];
        }
        if (sg == b.nseg - 1 && threadIdx.x == 0) b.cell_start[b.C] = s0 + n;
        if (small) {
            __syncthreads();  // the offsets are read before they become cursors
            for (int k0 = threadIdx.x; k0 < n; k0 += C * THREADS) {
                unsigned c[C];
#pragma unroll
                for (int u = 0; u < C; ++u) {
                    const int k = k0 + u * THREADS;
                    c[u] = k < n ? cell[k] : 0xffffu;
                }
#pragma unroll
                for (int u = 0; u < C; ++u) {
                    if (c[u] == 0xffffu) break;
                    s_perm[inc16(s_c16, c[u])] = (unsigned short)(k0 + u * THREADS);
                }
            }
            __syncthreads();
            const float4 *rec = b.rec + s0;
            float4 *sp = b.sp + s0;
            int32_t *sid = b.sid + s0;
            int32_t *lay = b.lay_s + s0;
            for (int q0 = threadIdx.x; q0 < n; q0 += G * THREADS) {
                float4 v[G];
#pragma unroll
                for (int u = 0; u < G; ++u)
                    if (q0 + u * THREADS < n) v[u] = rec[s_perm[q0 + u * THREADS]];
#pragma unroll
                for (int u = 0; u < G; ++u) {
                    const int q = q0 + u * THREADS;
                    if (q < n) {
                        sp[q] = sorted_record(v[u], fw);
                        sid[q] = __float_as_int(v[u].w);
                        lay[q] = l;
                    }
                }
            }
        } else {
            for (int k = threadIdx.x; k < n; k += THREADS) {
                const float4 r = b.rec[s0 + k];
                const int q = s0 + s_cell[cell[k]] + b.perm[s0 + k];
                b.sp[q] = sorted_record(r, fw);
                b.sid[q] = __float_as_int(r.w);
            }
            for (int k = threadIdx.x; k < n; k += THREADS) b.lay_s[s0 + k] = l;
        }
        __syncthreads();  // the shared arrays are reset for the next segment
    }
}

}  // namespace clue
