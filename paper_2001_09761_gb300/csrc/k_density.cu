// Steps S2 and S3 as per-stage kernels, one CTA per tile; the tile bodies and
// their description are in density_tile.cuh.
#include <algorithm>

#include "density_tile.cuh"

namespace clue {

static_assert(sizeof(DensityShared) <= DENSITY_SMEM_FIXED, "the host's occupancy estimate");

size_t band_bytes(const Params &p) { return (size_t)p.band_cap * sizeof(float4); }

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
    extern __shared__ float4 band[];  // Params::band_cap records
    stage_init(sh);
    unsigned parity = 0u;
    for (int t = blockIdx.x; t < b.ntiles; t += gridDim.x)
        if (!rho_tile<CHI, DT_ILP>(b, p, t, sh, band, parity)) return;
}

template <int CHI>
void launch_rho_k(int grid, int block, cudaStream_t s, const Buffers &b, const Params &p) {
    if (block > 256)
        k_rho<CHI, 1024><<<grid, block, band_bytes(p), s>>>(b, p);
    else
        k_rho<CHI, 256><<<grid, block, band_bytes(p), s>>>(b, p);
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
    extern __shared__ float4 band[];  // Params::band_cap records
    stage_init(sh);
    unsigned parity = 0u;
    for (int t = blockIdx.x; t < b.ntiles; t += gridDim.x)
        if (!nh_tile<DT_ILP>(b, p, t, sh, band, parity)) return;
}

cudaError_t launch_nh(const Buffers &b, const Params &p, const LaunchCfg &c, cudaStream_t s) {
    const int grid = b.ntiles;
    if (c.block_density > 256)
        k_nh<1024><<<grid > 0 ? grid : 1, c.block_density, band_bytes(p), s>>>(b, p);
    else
        k_nh<256><<<grid > 0 ? grid : 1, c.block_density, band_bytes(p), s>>>(b, p);
    return cudaGetLastError();
}

// The fused form (density_tile): rho, nh and the decision in one kernel, one
// CTA per tile; then k_nh_rest takes the tiles it left (the list in `rest`)
// on a grid of four CTAs per SM, which ends at once when the list is empty.
template <int CHI, int MAXT>
__global__ void __launch_bounds__(MAXT, MAXT <= 256 ? 4 : 1) k_density(Buffers b, Params p) {
    __shared__ DensityShared sh;
    extern __shared__ float4 band[];  // Params::band_cap records
    stage_init(sh);
    unsigned parity = 0u;
    for (int t = blockIdx.x; t < b.ntiles; t += gridDim.x)
        if (!density_tile<CHI, DT_ILP>(b, p, t, sh, band, parity)) return;
}

template <int CHI>
void launch_density_k(int grid, int block, cudaStream_t s, const Buffers &b, const Params &p) {
    if (block > 256)
        k_density<CHI, 1024><<<grid, block, band_bytes(p), s>>>(b, p);
    else
        k_density<CHI, 256><<<grid, block, band_bytes(p), s>>>(b, p);
}

cudaError_t launch_density(const Buffers &b, const Params &p, const LaunchCfg &c,
                           cudaStream_t s) {
    const int g = b.ntiles > 0 ? b.ntiles : 1;
    if (p.chi == 1)
        launch_density_k<1>(g, c.block_density, s, b, p);
    else if (p.chi == 2)
        launch_density_k<2>(g, c.block_density, s, b, p);
    else
        launch_density_k<0>(g, c.block_density, s, b, p);
    return cudaGetLastError();
}

template <int MAXT>
__global__ void __launch_bounds__(MAXT, MAXT <= 256 ? 4 : 1) k_nh_rest(Buffers b, Params p) {
    __shared__ DensityShared sh;
    extern __shared__ float4 band[];  // Params::band_cap records
    stage_init(sh);
    unsigned parity = 0u;
    const int n = b.ctrl->nrest;
    for (int i = blockIdx.x; i < n; i += gridDim.x)
        if (!nh_tile<DT_ILP>(b, p, b.rest[i], sh, band, parity)) return;
}

cudaError_t launch_nh_rest(const Buffers &b, const Params &p, const LaunchCfg &c,
                           cudaStream_t s) {
    const int grid = std::max(1, std::min(b.ntiles, c.grid_cap / 2));
    if (c.block_density > 256)
        k_nh_rest<1024><<<grid, c.block_density, band_bytes(p), s>>>(b, p);
    else
        k_nh_rest<256><<<grid, c.block_density, band_bytes(p), s>>>(b, p);
    return cudaGetLastError();
}

// Every density kernel may take up to BAND_CAP_MAX staged records of dynamic
// shared memory (beyond the default 48 KB per CTA).
cudaError_t density_prepare() {
    const int bytes = BAND_CAP_MAX * (int)sizeof(float4);
    const void *fns[] = {
        (const void *)k_rho<0, 256>, (const void *)k_rho<0, 1024>,
        (const void *)k_rho<1, 256>, (const void *)k_rho<1, 1024>,
        (const void *)k_rho<2, 256>, (const void *)k_rho<2, 1024>,
        (const void *)k_nh<256>, (const void *)k_nh<1024>,
        (const void *)k_density<0, 256>, (const void *)k_density<0, 1024>,
        (const void *)k_density<1, 256>, (const void *)k_density<1, 1024>,
        (const void *)k_density<2, 256>, (const void *)k_density<2, 1024>,
        (const void *)k_nh_rest<256>, (const void *)k_nh_rest<1024>};
    for (const void *f : fns) {
        const cudaError_t e =
            cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace clue
