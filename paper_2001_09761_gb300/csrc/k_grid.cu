// Step S1: the fixed-grid spatial index (Sec. 2.1, Eqs. 1-2) as per-stage
// kernels, both sorts; the stage bodies and their description are in
// grid_stages.cuh.
#include "grid_stages.cuh"

namespace clue {

__global__ void __launch_bounds__(256) k_fill_count(Buffers b, Params p) { fill_count_stage(b, p); }

cudaError_t launch_fill_count(const Buffers &b, const Params &p, const LaunchCfg &c, cudaStream_t s) {
    const int grid = b.ntiles < c.grid_cap ? b.ntiles : c.grid_cap;
    k_fill_count<<<grid > 0 ? grid : 1, c.block_fill, 0, s>>>(b, p);
    return cudaGetLastError();
}

cudaError_t launch_scan_cells(const Buffers &b, const LaunchCfg &c, cudaStream_t s, int *launches) {
    return exclusive_scan<int32_t>(LoadI32{b.count}, b.C, b.cell_start,
                                   (int32_t *)b.scan_partials, c.grid_cap, s, launches);
}

__global__ void __launch_bounds__(256) k_fill_scatter(Buffers b) { fill_scatter_stage(b); }

cudaError_t launch_fill_scatter(const Buffers &b, const LaunchCfg &c, cudaStream_t s) {
    const int grid = b.ntiles < c.grid_cap ? b.ntiles : c.grid_cap;
    k_fill_scatter<<<grid > 0 ? grid : 1, c.block_fill, 0, s>>>(b);
    return cudaGetLastError();
}

__global__ void __launch_bounds__(256) k_fill_canon(Buffers b, Params p) { fill_canon_stage(b, p); }

cudaError_t launch_fill_canon(const Buffers &b, const Params &p, const LaunchCfg &c, cudaStream_t s) {
    const int grid = b.ntiles < c.grid_cap ? b.ntiles : c.grid_cap;
    k_fill_canon<<<grid > 0 ? grid : 1, c.block_fill, 0, s>>>(b, p);
    return cudaGetLastError();
}

__global__ void __launch_bounds__(FILL_THREADS) k_fill_layers(Buffers b, Params p) {
    fill_layers_stage(b, p);
}

// A grid of at most grid_cap CTAs (eight per SM), each taking tiles in turn:
// a tile's count is short, and CTAs that stay resident save the launch of one
// CTA per tile.
cudaError_t launch_fill_layers(const Buffers &b, const Params &p, const LaunchCfg &c,
                               cudaStream_t s) {
    if (p.L < 1 || p.L > SEG_MAX_LAYERS) return cudaErrorInvalidValue;
    const int grid = b.ntiles < c.grid_cap ? b.ntiles : c.grid_cap;
    k_fill_layers<<<grid > 0 ? grid : 1, FILL_THREADS, (size_t)p.L * 4, s>>>(b, p);
    return cudaGetLastError();
}

cudaError_t launch_scan_segs(const Buffers &b, const LaunchCfg &c, cudaStream_t s, int *launches) {
    return exclusive_scan<int32_t>(LoadI32{b.tcount}, b.ntb, b.tbase,
                                   (int32_t *)b.scan_partials, c.grid_cap, s, launches);
}

// The placement runs one CTA per tile: a tile's steps are separated by
// barriers, and many resident CTAs hide each other's latencies.
__global__ void __launch_bounds__(FILL_THREADS, 6) k_fill_place(Buffers b, Params p) {
    fill_place_stage(b, p);
}

cudaError_t launch_fill_place(const Buffers &b, const Params &p, const LaunchCfg &, cudaStream_t s) {
    if (p.L < 1 || p.L > SEG_MAX_LAYERS) return cudaErrorInvalidValue;
    const int grid = b.ntiles;
    k_fill_place<<<grid > 0 ? grid : 1, FILL_THREADS, (size_t)(p.L + 3) / 4 * 32, s>>>(b, p);
    return cudaGetLastError();
}

__global__ void __launch_bounds__(SEG_THREADS, 3)
    k_fill_cells(Buffers b, Params p, int ev0, int n_ev, int cells_cap) {
    fill_cells_stage<SEG_THREADS, SEG_SMEM_HITS>(b, p, ev0, n_ev, cells_cap);
}

__global__ void __launch_bounds__(SMALL_SEG_THREADS, 12)
    k_fill_cells_small(Buffers b, Params p, int ev0, int n_ev, int cells_cap) {
    fill_cells_stage<SMALL_SEG_THREADS, SMALL_SEG_HITS>(b, p, ev0, n_ev, cells_cap);
}

cudaError_t fill_prepare() {
    cudaError_t e = cudaFuncSetAttribute(k_fill_cells, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         fill_cells_smem<SEG_SMEM_HITS>(SEG_MAX_CELLS));
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_fill_cells_small, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                fill_cells_smem<SMALL_SEG_HITS>(SMALL_SEG_CELLS));
}

// One CTA per segment (a grid-stride loop past 2^30 segments): the small
// build over the run's first n_small_ev events of seg_ev, the large one over
// the rest (or over all events when the run has no list).
cudaError_t launch_fill_cells(const Buffers &b, const Params &p, int max_cells, cudaStream_t s) {
    if (max_cells < 1 || max_cells > SEG_MAX_CELLS || max_cells != b.max_cells || b.nseg < 1)
        return cudaErrorInvalidValue;
    const int n_small = b.seg_ev ? b.n_small_ev : 0;
    if (n_small < 0 || n_small > b.nevents || b.small_cells > SMALL_SEG_CELLS) return cudaErrorInvalidValue;
    const int64_t cap = 1 << 30;
    if (n_small > 0) {
        const int64_t nseg = (int64_t)n_small * p.L;
        k_fill_cells_small<<<(unsigned)(nseg < cap ? nseg : cap), SMALL_SEG_THREADS,
                             (size_t)fill_cells_smem<SMALL_SEG_HITS>(b.small_cells), s>>>(
            b, p, 0, n_small, b.small_cells);
    }
    if (n_small < b.nevents) {
        const int64_t nseg = (int64_t)(b.nevents - n_small) * p.L;
        k_fill_cells<<<(unsigned)(nseg < cap ? nseg : cap), SEG_THREADS,
                       (size_t)fill_cells_smem<SEG_SMEM_HITS>(max_cells), s>>>(
            b, p, n_small, b.nevents - n_small, max_cells);
    }
    return cudaGetLastError();
}

}  // namespace clue
