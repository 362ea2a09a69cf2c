// Step S1: the fixed-grid spatial index (Sec. 2.1, Eqs. 1-2) as per-stage
// kernels; the stage bodies and their description are in grid_stages.cuh.
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

__global__ void __launch_bounds__(256) k_fill_canon(Buffers b) { fill_canon_stage(b); }

cudaError_t launch_fill_canon(const Buffers &b, const LaunchCfg &c, cudaStream_t s) {
    const int grid = b.ntiles < c.grid_cap ? b.ntiles : c.grid_cap;
    k_fill_canon<<<grid > 0 ? grid : 1, c.block_fill, 0, s>>>(b);
    return cudaGetLastError();
}

}  // namespace clue
