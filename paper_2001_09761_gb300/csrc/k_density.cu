// Steps S2 and S3 as per-stage kernels, one CTA per tile; the tile bodies and
// their description are in density_tile.cuh.
#include "density_tile.cuh"

namespace clue {

// Each density kernel in two builds: CTAs of up to 256 threads (the usual
// case: four per SM, each with ~46 KB of shared memory) and of up to 1024
// (runs with fewer tiles than SMs: one hit per thread).
// The window pass of a thread issues the loads of DT_ILP hits together.
constexpr int DT_ILP = 2;

// The 256-thread build keeps to 64 registers, so that four CTAs share an SM
// (their shared memory allows four).
template <int CHI, int MAXT>
__global__ void __launch_bounds__(MAXT, MAXT <= 256 ? 4 : 1) k_rho(Buffers b, Params p) {
    __shared__ DensityShared sh;
    __shared__ float4 band[BAND_CAP];
    for (int t = blockIdx.x; t < b.ntiles; t += gridDim.x)
        rho_tile<CHI, DT_ILP>(b, p, t, sh, band);
}

template <int CHI>
void launch_rho_k(int grid, int block, cudaStream_t s, const Buffers &b, const Params &p) {
    if (block > 256)
        k_rho<CHI, 1024><<<grid, block, 0, s>>>(b, p);
    else
        k_rho<CHI, 256><<<grid, block, 0, s>>>(b, p);
}

// One CTA per tile: tiles differ widely in work, and the hardware's CTA
// scheduling balances that better than a persistent grid.
cudaError_t launch_rho(const Buffers &b, const Params &p, const LaunchCfg &c, cudaStream_t s) {
    const int grid = b.ntiles;
    const int g = grid > 0 ? grid : 1;
    if (p.chi == 1)
        launch_rho_k<1>(g, c.block_density, s, b, p);
    else if (p.chi == 2)
        launch_rho_k<2>(g, c.block_density, s, b, p);
    else
        launch_rho_k<0>(g, c.block_density, s, b, p);
    return cudaGetLastError();
}

template <int MAXT>
__global__ void __launch_bounds__(MAXT, MAXT <= 256 ? 4 : 1) k_nh(Buffers b, Params p) {
    __shared__ DensityShared sh;
    __shared__ float4 band[BAND_CAP];
    for (int t = blockIdx.x; t < b.ntiles; t += gridDim.x)
        nh_tile<DT_ILP>(b, p, t, sh, band);
}

cudaError_t launch_nh(const Buffers &b, const Params &p, const LaunchCfg &c, cudaStream_t s) {
    const int grid = b.ntiles;
    if (c.block_density > 256)
        k_nh<1024><<<grid > 0 ? grid : 1, c.block_density, 0, s>>>(b, p);
    else
        k_nh<256><<<grid > 0 ? grid : 1, c.block_density, 0, s>>>(b, p);
    return cudaGetLastError();
}

}  // namespace clue
