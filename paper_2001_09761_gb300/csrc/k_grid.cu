// Step S1: the fixed-grid spatial index (Sec. 2.1, Eqs. 1-2).
//
// The paper pushes each hit into its bin with an atomic (conflict (i) of
// Sec. 3), which leaves bin contents in a run-dependent order.  Here the index
// is a counting sort with a canonical result: hits are counted per cell (the
// count's atomic hands each hit its arrival rank), cell offsets come from a
// prefix sum, hit ids are scattered into their cell's segment, and every
// segment is then put in ascending hit index.  The sorted
// copy (x, y, w, id packed in one float4 per hit, one 16-byte load per
// candidate) makes every later neighbour scan a walk over contiguous memory,
// and the ascending order inside each cell is what lets the density step sum
// in ascending hit index.
#include "scan.cuh"

namespace clue {

// --- count: bin of every hit, hits per cell ---------------------------------
__global__ void __launch_bounds__(256) k_fill_count(Buffers b, Params p) {
    for (int t = blockIdx.x; t < b.ntiles; t += gridDim.x) {
        const Tile tl = b.tiles[t];
        const EventDesc ev = b.events[tl.event];
        for (int k = threadIdx.x; k < tl.len; k += blockDim.x) {
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
    }
}

cudaError_t launch_fill_count(const Buffers &b, const Params &p, const LaunchCfg &c, cudaStream_t s) {
    const int grid = b.ntiles < c.grid_cap ? b.ntiles : c.grid_cap;
    k_fill_count<<<grid > 0 ? grid : 1, c.block_fill, 0, s>>>(b, p);
    return cudaGetLastError();
}

struct LoadI32 {
    const int32_t *a;
    __device__ __forceinline__ int32_t operator()(int64_t i) const { return a[i]; }
};

cudaError_t launch_scan_cells(const Buffers &b, const LaunchCfg &c, cudaStream_t s, int *launches) {
    return exclusive_scan<int32_t>(LoadI32{b.count}, b.C, b.cell_start,
                                   (int32_t *)b.scan_partials, c.grid_cap, s, launches);
}

// --- scatter: every hit's id into its cell's segment at the rank its count
// returned (order within a cell is not yet fixed); one 4-byte scattered
// store, no atomic. ---------------------------------------------------------
__global__ void __launch_bounds__(256) k_fill_scatter(Buffers b) {
    for (int t = blockIdx.x; t < b.ntiles; t += gridDim.x) {
        const Tile tl = b.tiles[t];
        const int64_t coff = b.events[tl.event].cell_off;
        for (int k = threadIdx.x; k < tl.len; k += blockDim.x) {
            const int g = tl.start + k;
            b.perm[b.cell_start[coff + b.key[g]] + b.rank[g]] = g;
        }
    }
}

cudaError_t launch_fill_scatter(const Buffers &b, const LaunchCfg &c, cudaStream_t s) {
    const int grid = b.ntiles < c.grid_cap ? b.ntiles : c.grid_cap;
    k_fill_scatter<<<grid > 0 ? grid : 1, c.block_fill, 0, s>>>(b);
    return cudaGetLastError();
}

// --- canonicalise: each slot of a short segment finds its rank among the
// segment's hit ids and writes the sorted copies; long segments go to the CTA
// sorter below --------------------------------------------------------------
__global__ void __launch_bounds__(256) k_fill_canon(Buffers b) {
    for (int t = blockIdx.x; t < b.ntiles; t += gridDim.x) {
        const Tile tl = b.tiles[t];
        const EventDesc ev = b.events[tl.event];
        const int64_t coff = ev.cell_off;
        const int ev_nbxy = ev.nbx * ev.nby;
        for (int k = threadIdx.x; k < tl.len; k += blockDim.x) {
            const int pos = tl.start + k;
            const int g = b.perm[pos];
            const float4 r = b.rec[g];  // x, y, w, cell of hit g: one 16-byte gather
            const int local = __float_as_int(r.w);
            const int64_t c = coff + local;
            const int a = b.cell_start[c], e = b.cell_start[c + 1];
            if (e - a <= SMALL_SEGMENT) {
                int rank = 0;
                for (int q = a; q < e; ++q) rank += (b.perm[q] < g);
                const int dst = a + rank;
                b.sp[dst] = make_float4(r.x, r.y, r.z, __int_as_float(g));
                b.lay_s[dst] = local / ev_nbxy;
            } else if (pos == a) {
                const int i = atomicAdd(&b.ctrl->nbig, 1);
                b.big[i] = (int32_t)(c);
            }
        }
    }
}

cudaError_t launch_fill_canon(const Buffers &b, const LaunchCfg &c, cudaStream_t s) {
    const int grid = b.ntiles < c.grid_cap ? b.ntiles : c.grid_cap;
    k_fill_canon<<<grid > 0 ? grid : 1, c.block_fill, 0, s>>>(b);
    return cudaGetLastError();
}

// --- CTA sorter for long segments: a stable least-significant-digit radix
// sort (8-bit digits) of the segment's hit ids, passed between `perm` and
// `tmp` (both hold the segment at the same offsets, so no memory is shared
// between segments).  Stability within a chunk comes from warp match masks,
// across chunks from processing them in order. ---------------------------------
constexpr int BIG_THREADS = 256;
constexpr int BIG_WARPS = BIG_THREADS / 32;

__global__ void __launch_bounds__(BIG_THREADS) k_fill_big(Buffers b) {
    __shared__ int hist[256];
    __shared__ int base[256];
    __shared__ int wcount[BIG_WARPS][256];
    __shared__ int red[2 * BIG_WARPS];
    __shared__ int ws[32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nbig = b.ctrl->nbig;
    for (int sgi = blockIdx.x; sgi < nbig; sgi += gridDim.x) {
        const int64_t c = b.big[sgi];
        const int a = b.cell_start[c], h = b.cell_start[c + 1] - a;
        // layer of the cell: the event is that of any hit in the segment
        int lay;
        {
            const int g0 = b.perm[a];
            int lo = 0, hi = b.nevents - 1;  // event of g0 by bisection on hit_off
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (b.events[mid].hit_off <= g0) lo = mid; else hi = mid - 1;
            }
            const EventDesc ev = b.events[lo];
            lay = (int)((c - ev.cell_off) / ((int64_t)ev.nbx * ev.nby));
        }
        __syncthreads();  // every thread has read perm[a] before it is overwritten
        // range of ids in the segment
        int vmin = 0x7fffffff, vmax = 0;
        for (int i = tid; i < h; i += BIG_THREADS) {
            const int v = b.perm[a + i];
            vmin = min(vmin, v);
            vmax = max(vmax, v);
        }
        for (int o = 16; o > 0; o >>= 1) {
            vmin = min(vmin, __shfl_xor_sync(FULL_MASK, vmin, o));
            vmax = max(vmax, __shfl_xor_sync(FULL_MASK, vmax, o));
        }
        if (lane == 0) {
            red[warp] = vmin;
            red[BIG_WARPS + warp] = vmax;
        }
        __syncthreads();
        vmin = red[0];
        vmax = red[BIG_WARPS];
        for (int w = 1; w < BIG_WARPS; ++w) {
            vmin = min(vmin, red[w]);
            vmax = max(vmax, red[BIG_WARPS + w]);
        }
        const unsigned range = (unsigned)(vmax - vmin);
        const int bits = range ? 32 - __clz(range) : 1;
        const int passes = (bits + 7) / 8;
        // pass 0 reads absolute ids from perm; later passes ping-pong relative
        // ids between tmp and perm (the whole segment is read before the
        // second pass writes perm)
        const int *ids0 = b.perm + a;
        int *src = nullptr, *dst = b.tmp + a, *other = b.perm + a;
        for (int pass = 0; pass < passes; ++pass) {
            const int shift = 8 * pass;
            const int sub = pass == 0 ? vmin : 0;
#define SRC(i) (pass == 0 ? ids0[(i)] : src[(i)])
            hist[tid] = 0;
            for (int w = 0; w < BIG_WARPS; ++w) wcount[w][tid] = 0;
            __syncthreads();
            for (int i = tid; i < h; i += BIG_THREADS)
                atomicAdd(&hist[((unsigned)(SRC(i) - sub) >> shift) & 255], 1);
            __syncthreads();
            {
                int total;
                const int v = hist[tid];
                base[tid] = block_incl_scan(v, ws, &total) - v;  // BIG_THREADS == 256 digits
            }
            __syncthreads();
            for (int c0 = 0; c0 < h; c0 += BIG_THREADS) {
                const int i = c0 + tid;
                const bool valid = i < h;
                const unsigned v = valid ? (unsigned)(SRC(i) - sub) : 0u;
                const int d = valid ? (int)((v >> shift) & 255) : 256;
                const unsigned peers = __match_any_sync(FULL_MASK, d);
                const int lrank = __popc(peers & lanemask_lt());
                if (valid && lrank == 0) wcount[warp][d] = __popc(peers);
                __syncthreads();
                if (valid) {
                    int off = base[d] + lrank;
                    for (int w = 0; w < warp; ++w) off += wcount[w][d];
                    dst[off] = (int)v;
                }
                __syncthreads();
                int add = 0;
                for (int w = 0; w < BIG_WARPS; ++w) {
                    add += wcount[w][tid];
                    wcount[w][tid] = 0;
                }
                base[tid] += add;
                __syncthreads();
            }
#undef SRC
            src = dst;  // this pass's output is the next pass's input
            dst = other;
            other = src;
        }
        // src now holds the sorted ids relative to vmin
        for (int i = tid; i < h; i += BIG_THREADS) {
            const int g = src[i] + vmin;
            const int q = a + i;
            b.sp[q] = make_float4(b.x[g], b.y[g], b.w[g], __int_as_float(g));
            b.lay_s[q] = lay;
        }
        __syncthreads();
    }
}

cudaError_t launch_fill_big(const Buffers &b, const LaunchCfg &c, cudaStream_t s) {
    // The number of long segments is known only on the device; a persistent
    // grid loops over however many there are (usually none).
    k_fill_big<<<c.grid_cap / 4 > 0 ? c.grid_cap / 4 : 1, BIG_THREADS, 0, s>>>(b);
    return cudaGetLastError();
}

}  // namespace clue
