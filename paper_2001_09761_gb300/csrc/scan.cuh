// Device-wide exclusive prefix sum in three launches (tile reduce, scan of
// the tile sums in one CTA, tile scan plus offset).  No CTA ever waits on
// another, so nothing can spin.  Used for the grid's cell offsets and for the
// seed ranks / follower-list offsets of the decision step.
#pragma once

#include "device_common.cuh"

namespace clue {

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 16;
constexpr int64_t SCAN_TILE = (int64_t)SCAN_THREADS * SCAN_ITEMS;

// Inclusive scan over the CTA (blockDim.x a multiple of 32, <= 1024).
// `ws` is shared scratch of >= 32 elements; *total gets the CTA sum.
template <typename T>
__device__ __forceinline__ T block_incl_scan(T v, T *ws, T *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    T incl = warp_incl_scan(v);
    if (lane == 31) ws[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        T s = lane < nw ? ws[lane] : T(0);
        s = warp_incl_scan(s);
        if (lane < nw) ws[lane] = s;
    }
    __syncthreads();
    const T add = warp > 0 ? ws[warp - 1] : T(0);
    *total = ws[nw - 1];
    __syncthreads();
    return incl + add;
}

// The three stages as device functions, each wrapped by a kernel below.
template <typename T, typename Load>
__device__ __forceinline__ void scan_reduce_stage(const Load &ld, int64_t n, T *partials,
                                                  int64_t ntiles) {
    __shared__ T ws[32];
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int64_t base = t * SCAN_TILE;
        T sum = 0;
#pragma unroll 4
        for (int i = 0; i < SCAN_ITEMS; ++i) {
            const int64_t idx = base + (int64_t)i * SCAN_THREADS + threadIdx.x;
            if (idx < n) sum += ld(idx);
        }
        T total;
        block_incl_scan(sum, ws, &total);
        if (threadIdx.x == 0) partials[t] = total;
    }
}

// One CTA (any multiple of 32 threads) scans the tile sums.
template <typename T>
__device__ __forceinline__ void scan_mid_stage(T *partials, int64_t ntiles, T *out, int64_t n) {
    __shared__ T ws[32];
    T carry = 0;
    for (int64_t base = 0; base < ntiles; base += blockDim.x) {
        const int64_t i = base + threadIdx.x;
        const T v = i < ntiles ? partials[i] : T(0);
        T total;
        const T incl = block_incl_scan(v, ws, &total);
        if (i < ntiles) partials[i] = carry + incl - v;
        carry += total;
    }
    if (threadIdx.x == 0) {
        partials[ntiles] = carry;
        out[n] = carry;
    }
}

// Tile scan plus offset: warp w of the CTA owns the tile's w-th run of
// 32 * SCAN_ITEMS elements, read in coalesced rows of 32 and scanned with
// warp shuffles; one CTA-wide step adds the earlier warps' totals.
template <typename T, typename Load>
__device__ __forceinline__ void scan_down_stage(const Load &ld, int64_t n, const T *partials,
                                                T *out, int64_t ntiles) {
    __shared__ T wsum[SCAN_THREADS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int64_t base = t * SCAN_TILE + (int64_t)warp * 32 * SCAN_ITEMS;
        T ex[SCAN_ITEMS];
        T run = 0;  // the warp's running total
#pragma unroll
        for (int i = 0; i < SCAN_ITEMS; ++i) {
            const int64_t idx = base + (int64_t)i * 32 + lane;
            const T v = idx < n ? ld(idx) : T(0);
            const T incl = warp_incl_scan(v);
            ex[i] = run + incl - v;
            run += __shfl_sync(FULL_MASK, incl, 31);
        }
        if (lane == 0) wsum[warp] = run;
        __syncthreads();
        T off = partials[t];
        for (int w = 0; w < warp; ++w) off += wsum[w];
#pragma unroll
        for (int i = 0; i < SCAN_ITEMS; ++i) {
            const int64_t idx = base + (int64_t)i * 32 + lane;
            if (idx < n) out[idx] = off + ex[i];
        }
        __syncthreads();  // wsum is reused by the next tile
    }
}

template <typename T, typename Load>
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_reduce(Load ld, int64_t n, T *partials,
                                                              int64_t ntiles) {
    scan_reduce_stage<T, Load>(ld, n, partials, ntiles);
}

template <typename T>
__global__ void __launch_bounds__(1024) k_scan_mid(T *partials, int64_t ntiles, T *out, int64_t n) {
    scan_mid_stage<T>(partials, ntiles, out, n);
}

template <typename T, typename Load>
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_down(Load ld, int64_t n, const T *partials,
                                                            T *out, int64_t ntiles) {
    scan_down_stage<T, Load>(ld, n, partials, out, ntiles);
}

// The whole scan in one CTA of SCAN_SINGLE_THREADS, tile after tile of
// SCAN_SINGLE_TILE with a running carry: for small inputs, where three
// launches cost more than the work (one pass up to SCAN_SINGLE_TILE entries).
constexpr int SCAN_SINGLE_THREADS = 1024;
constexpr int64_t SCAN_SINGLE_TILE = (int64_t)SCAN_SINGLE_THREADS * SCAN_ITEMS;

template <typename T, typename Load>
__device__ __forceinline__ void scan_single_stage(const Load &ld, int64_t n, T *out) {
    static_assert(SCAN_SINGLE_THREADS == 32 * 32, "one warp scans the warps' totals");
    __shared__ T wsum[32];
    __shared__ T wtotal;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T carry = 0;  // the same in every thread
    const int64_t ntiles = (n + SCAN_SINGLE_TILE - 1) / SCAN_SINGLE_TILE;
    for (int64_t t = 0; t < ntiles; ++t) {
        const int64_t base = t * SCAN_SINGLE_TILE + (int64_t)warp * 32 * SCAN_ITEMS;
        T ex[SCAN_ITEMS];
        T run = 0;
#pragma unroll
        for (int i = 0; i < SCAN_ITEMS; ++i) {
            const int64_t idx = base + (int64_t)i * 32 + lane;
            const T v = idx < n ? ld(idx) : T(0);
            const T incl = warp_incl_scan(v);
            ex[i] = run + incl - v;
            run += __shfl_sync(FULL_MASK, incl, 31);
        }
        if (lane == 0) wsum[warp] = run;
        __syncthreads();
        if (warp == 0) {  // the warps' totals, scanned by one warp
            const T v = wsum[lane];
            const T incl = warp_incl_scan(v);
            wsum[lane] = incl - v;
            if (lane == 31) wtotal = incl;
        }
        __syncthreads();
        const T off = carry + wsum[warp], total = wtotal;
#pragma unroll
        for (int i = 0; i < SCAN_ITEMS; ++i) {
            const int64_t idx = base + (int64_t)i * 32 + lane;
            if (idx < n) out[idx] = off + ex[i];
        }
        carry += total;
        __syncthreads();  // wsum is reused by the next tile
    }
    if (threadIdx.x == 0) out[n] = carry;
}

template <typename T, typename Load>
__global__ void __launch_bounds__(SCAN_SINGLE_THREADS) k_scan_single(Load ld, int64_t n, T *out) {
    scan_single_stage<T, Load>(ld, n, out);
}

constexpr int64_t SCAN_SINGLE_MAX_TILES = 4;

// Whether a scan of n elements runs in one CTA (k_scan_single).
__host__ __device__ constexpr bool scan_is_single(int64_t n) {
    return (n + SCAN_TILE - 1) / SCAN_TILE <= SCAN_SINGLE_MAX_TILES;
}

// Exclusive scan of ld(0..n-1) into out[0..n-1], out[n] = total.
// `partials` must hold scan_partials_needed(n) elements of T.
template <typename T, typename Load>
cudaError_t exclusive_scan(Load ld, int64_t n, T *out, T *partials, int grid_cap, cudaStream_t s,
                           int *launches) {
    const int64_t ntiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (scan_is_single(n)) {
        k_scan_single<T, Load><<<1, SCAN_SINGLE_THREADS, 0, s>>>(ld, n, out);
        if (launches) *launches += 1;
        return cudaGetLastError();
    }
    const int grid = (int)(ntiles < grid_cap ? (ntiles > 0 ? ntiles : 1) : grid_cap);
    k_scan_reduce<T, Load><<<grid, SCAN_THREADS, 0, s>>>(ld, n, partials, ntiles);
    k_scan_mid<T><<<1, 1024, 0, s>>>(partials, ntiles, out, n);
    k_scan_down<T, Load><<<grid, SCAN_THREADS, 0, s>>>(ld, n, partials, out, ntiles);
    if (launches) *launches += 3;
    return cudaGetLastError();
}

}  // namespace clue
