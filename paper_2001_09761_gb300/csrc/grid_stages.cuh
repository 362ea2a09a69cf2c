// Step S1: the fixed-grid spatial index (Sec. 2.1, Eqs. 1-2): the stage
// bodies, which the kernels in k_grid.cu wrap.
//
// The paper pushes each hit into its bin with an atomic (conflict (i) of
// Sec. 3).  Here the index is a counting sort: hits are counted per cell (the
// count's atomic hands each hit its arrival rank), cell offsets come from a
// prefix sum, hit ids are scattered into their cell's segment, and a gather
// writes the sorted copy (x, y, w, id packed in one float4 per hit, one
// 16-byte load per candidate), which makes every later neighbour scan a walk
// over contiguous memory.  The order of hits inside a cell is the atomics'
// arrival order; no result depends on it (the density is an exact sum, the
// nearest-higher a lexicographic minimum).
#pragma once

#include "scan.cuh"

namespace clue {

// --- count: bin of every hit, hits per cell ---------------------------------
__device__ __forceinline__ void fill_count_stage(const Buffers &b, const Params &p) {
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
__device__ __forceinline__ void fill_canon_stage(const Buffers &b) {
    for (int t = blockIdx.x; t < b.ntiles; t += gridDim.x) {
        const Tile tl = b.tiles[t];
        const int ev_nbxy = b.events[tl.event].nbx * b.events[tl.event].nby;
        for (int k = threadIdx.x; k < tl.len; k += blockDim.x) {
            const int pos = tl.start + k;
            const int g = b.perm[pos];
            const float4 r = b.rec[g];  // x, y, w, cell of hit g: one 16-byte gather
            b.sp[pos] = make_float4(r.x, r.y, r.z, __int_as_float(g));
            b.lay_s[pos] = __float_as_int(r.w) / ev_nbxy;
        }
    }
}

}  // namespace clue
