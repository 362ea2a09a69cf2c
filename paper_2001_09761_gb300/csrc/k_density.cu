// Steps S2 and S3 as per-stage kernels; the stage bodies and their
// description are in density_stages.cuh.
#include "density_stages.cuh"

namespace clue {

template <int CHI>
__global__ void __launch_bounds__(256) k_rho(Buffers b, Params p) { rho_stage<CHI>(b, p); }

// One CTA per tile: hits differ widely in window population, and the
// hardware's CTA scheduling balances that better than a persistent grid.
cudaError_t launch_rho(const Buffers &b, const Params &p, const LaunchCfg &c, cudaStream_t s) {
    const int grid = b.ntiles;
    const int g = grid > 0 ? grid : 1;
    if (p.chi == 1)
        k_rho<1><<<g, c.block_density, 0, s>>>(b, p);
    else if (p.chi == 2)
        k_rho<2><<<g, c.block_density, 0, s>>>(b, p);
    else
        k_rho<0><<<g, c.block_density, 0, s>>>(b, p);
    return cudaGetLastError();
}

__global__ void __launch_bounds__(256) k_nh(Buffers b, Params p) { nh_stage(b, p); }

cudaError_t launch_nh(const Buffers &b, const Params &p, const LaunchCfg &c, cudaStream_t s) {
    const int grid = b.ntiles;
    k_nh<<<grid > 0 ? grid : 1, c.block_density, 0, s>>>(b, p);
    return cudaGetLastError();
}

}  // namespace clue
