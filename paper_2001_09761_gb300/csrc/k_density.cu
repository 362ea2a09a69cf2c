// Steps S2 and S3 as per-stage kernels; the stage bodies and their
// description are in density_stages.cuh.
#include "density_stages.cuh"

namespace clue {

// Each density kernel in two builds: CTAs of up to 256 threads (the usual
// case; the compiler's register choice then keeps several CTAs per SM) and of
// up to 1024 (runs with fewer tiles than SMs: one hit per thread).
template <int CHI, int MAXT>
__global__ void __launch_bounds__(MAXT) k_rho(Buffers b, Params p) { rho_stage<CHI>(b, p); }

template <int CHI>
void launch_rho_k(int grid, int block, cudaStream_t s, const Buffers &b, const Params &p) {
    if (block > 256)
        k_rho<CHI, 1024><<<grid, block, 0, s>>>(b, p);
    else
        k_rho<CHI, 256><<<grid, block, 0, s>>>(b, p);
}

// One CTA per tile: hits differ widely in window population, and the
// hardware's CTA scheduling balances that better than a persistent grid.
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
__global__ void __launch_bounds__(MAXT) k_nh(Buffers b, Params p) { nh_stage(b, p); }

cudaError_t launch_nh(const Buffers &b, const Params &p, const LaunchCfg &c, cudaStream_t s) {
    const int grid = b.ntiles;
    if (c.block_density > 256)
        k_nh<1024><<<grid > 0 ? grid : 1, c.block_density, 0, s>>>(b, p);
    else
        k_nh<256><<<grid > 0 ? grid : 1, c.block_density, 0, s>>>(b, p);
    return cudaGetLastError();
}

}  // namespace clue
