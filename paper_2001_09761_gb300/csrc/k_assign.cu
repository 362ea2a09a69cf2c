// Steps S4 and S5: seed / outlier decision with follower lists (Sec. 2.2,
// Eq. 5, Algorithm 3) and the expansion of cluster ids down the followers.
//
// The paper appends seeds and followers with atomics (conflicts (ii) and (iii)
// of Sec. 3), so seed numbering depends on thread timing.  Here seed ids are
// ranks from a prefix sum over hit order, giving Algorithm 3's k++ numbering
// (ascending seed index per event), and the follower lists are a CSR built by
// the same prefix sum.  Expansion is k-way parallel as in the paper, one warp
// per seed walking its follower tree breadth-first with a shared-memory queue.
#include <climits>

#include "scan.cuh"

namespace clue {

__global__ void __launch_bounds__(256) k_decide(Buffers b, Params p) {
    for (int t = blockIdx.x; t < b.ntiles; t += gridDim.x) {
        const Tile tl = b.tiles[t];
        for (int k = threadIdx.x; k < tl.len; k += blockDim.x) {
            const int g = tl.start + k;
            const float r = b.rho[g], d2 = b.delta2[g];
            const int j = b.nh[g];
            const bool seed = (r > p.rhoc) && (d2 > p.dcs2);
            const bool outl = (r < p.rhoc) && (d2 > p.dos2);
            const bool fol = !seed && !outl && j >= 0;
            b.flags[g] = (seed ? F_SEED : 0) | (outl ? F_OUTLIER : 0) | (fol ? F_FOLLOWER : 0);
            if (fol) atomicAdd(&b.fcount[j], 1);
        }
    }
}

cudaError_t launch_decide(const Buffers &b, const Params &p, const LaunchCfg &c, cudaStream_t s) {
    const int grid = b.ntiles < c.grid_cap ? b.ntiles : c.grid_cap;
    k_decide<<<grid > 0 ? grid : 1, c.block_fill, 0, s>>>(b, p);
    return cudaGetLastError();
}

// (is_seed << 32 | follower count): one scan gives both the global seed rank
// (high word) and the follower-list offset (low word) of every hit.
struct LoadPacked {
    const uint8_t *flags;
    const int32_t *fcount;
    __device__ __forceinline__ unsigned long long operator()(int64_t i) const {
        return ((unsigned long long)(flags[i] & F_SEED) << 32) | (unsigned)fcount[i];
    }
};

cudaError_t launch_scan_hits(const Buffers &b, const LaunchCfg &c, cudaStream_t s, int *launches) {
    return exclusive_scan<unsigned long long>(LoadPacked{b.flags, b.fcount}, b.N, b.hs,
                                              (unsigned long long *)b.scan_partials, c.grid_cap,
                                              s, launches);
}

// Seeds take their per-event id and enter the seed list; followers enter the
// CSR list of their nearest-higher (order inside a list is irrelevant: each
// follower has exactly one parent); everything else is noise for now.
__global__ void __launch_bounds__(256) k_link(Buffers b) {
    for (int t = blockIdx.x; t < b.ntiles; t += gridDim.x) {
        const Tile tl = b.tiles[t];
        const int64_t hoff = b.events[tl.event].hit_off;
        const unsigned ebase = (unsigned)(b.hs[hoff] >> 32);
        for (int k = threadIdx.x; k < tl.len; k += blockDim.x) {
            const int g = tl.start + k;
            const uint8_t f = b.flags[g];
            if (f & F_SEED) {
                const unsigned srank = (unsigned)(b.hs[g] >> 32);
                b.cid[g] = (int32_t)(srank - ebase);
                b.seed_list[srank] = g;
                b.is_seed[g] = 1;
            } else {
                b.is_seed[g] = 0;
                if (f & F_FOLLOWER) {
                    const int j = b.nh[g];
                    const int slot = (int)(unsigned)b.hs[j] + atomicSub(&b.fcount[j], 1) - 1;
                    b.fol[slot] = g;
                    b.cid[g] = PENDING;
                } else {
                    b.cid[g] = -1;
                }
            }
        }
    }
}

cudaError_t launch_link(const Buffers &b, const LaunchCfg &c, cudaStream_t s) {
    const int grid = b.ntiles < c.grid_cap ? b.ntiles : c.grid_cap;
    k_link<<<grid > 0 ? grid : 1, c.block_fill, 0, s>>>(b);
    return cudaGetLastError();
}

// One warp per seed (grid-stride over the seed list).  The warp dequeues up to
// 32 nodes, scans their follower counts, and hands out the followers across
// its lanes (each lane finds the node owning its follower by bisection over
// the scanned counts), so a node with many followers does not serialise one
// lane.  A tree whose frontier outgrows the queue is left partly pending and
// finished by k_complete.
constexpr int EXPAND_THREADS = 256;
constexpr int EXPAND_WARPS = EXPAND_THREADS / 32;

__global__ void __launch_bounds__(EXPAND_THREADS) k_expand(Buffers b) {
    __shared__ int queue[EXPAND_WARPS][EXPAND_QCAP];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int *q = queue[warp];
    const int nseeds = (int)(b.hs[b.N] >> 32);
    const int nwarps = gridDim.x * EXPAND_WARPS;
    bool ovf = false;
    for (int si = blockIdx.x * EXPAND_WARPS + warp; si < nseeds; si += nwarps) {
        const int root = b.seed_list[si];
        const int id = b.cid[root];
        if (lane == 0) q[0] = root;
        __syncwarp();
        int head = 0, tail = 1;
        int64_t dequeued = 0;  // a tree holds at most N nodes: bounds the walk
        while (head < tail) {
            const int cnt = min(32, tail - head);
            dequeued += cnt;
            if (dequeued > b.N) {
                if (lane == 0) atomicOr(&b.ctrl->err, ERRBIT_TIMEOUT);
                break;
            }
            int a = 0, c = 0;
            if (lane < cnt) {
                const int node = q[(head + lane) & (EXPAND_QCAP - 1)];
                a = (int)(unsigned)b.hs[node];
                c = (int)(unsigned)b.hs[node + 1] - a;
            }
            const int incl = warp_incl_scan(c);
            const int total = __shfl_sync(FULL_MASK, incl, 31);
            const int excl = incl - c;
            head += cnt;
            if (tail - head + total > EXPAND_QCAP) {
                ovf = true;
                break;
            }
            for (int base = 0; base < total; base += 32) {
                const int u = base + lane;
                int lo = 0, hi = 31;
#pragma unroll
                for (int it = 0; it < 5; ++it) {
                    const int mid = (lo + hi) >> 1;
                    if (__shfl_sync(FULL_MASK, incl, mid) > u) hi = mid; else lo = mid + 1;
                }
                const int ao = __shfl_sync(FULL_MASK, a, lo);
                const int eo = __shfl_sync(FULL_MASK, excl, lo);
                if (u < total) {
                    const int child = b.fol[ao + (u - eo)];
                    b.cid[child] = id;
                    q[(tail + u) & (EXPAND_QCAP - 1)] = child;
                }
            }
            tail += total;
            __syncwarp();
        }
        __syncwarp();
    }
    if (ovf && lane == 0) atomicOr(&b.ctrl->overflow, 1u);
}

cudaError_t launch_expand(const Buffers &b, const LaunchCfg &c, cudaStream_t s) {
    k_expand<<<c.grid_cap > 0 ? c.grid_cap : 1, EXPAND_THREADS, 0, s>>>(b);
    return cudaGetLastError();
}

// Pending followers left after the expansion are noise (their chain ends at an
// outlier or at a hit with no nearest-higher) unless a queue overflowed; then
// each pending hit follows its nh chain to the first hit with a final id (a
// seed, an expanded follower, or noise).  The chain is finite because rho
// rises strictly along it; the walk is still bounded by N steps.
__global__ void __launch_bounds__(256) k_complete(Buffers b) {
    const bool ovf = b.ctrl->overflow != 0;
    for (int t = blockIdx.x; t < b.ntiles; t += gridDim.x) {
        const Tile tl = b.tiles[t];
        for (int k = threadIdx.x; k < tl.len; k += blockDim.x) {
            const int g = tl.start + k;
            if (b.cid[g] != PENDING) continue;
            if (!ovf) {
                b.cid[g] = -1;
                continue;
            }
            int v = b.nh[g];
            int cv = b.cid[v];
            int64_t steps = 0;
            while (cv == PENDING && steps < b.N) {
                v = b.nh[v];
                cv = b.cid[v];
                ++steps;
            }
            if (cv == PENDING) {
                atomicOr(&b.ctrl->err, ERRBIT_TIMEOUT);
                cv = -1;
            }
            b.cid[g] = cv;
        }
    }
}

cudaError_t launch_complete(const Buffers &b, const LaunchCfg &c, cudaStream_t s) {
    const int grid = b.ntiles < c.grid_cap ? b.ntiles : c.grid_cap;
    k_complete<<<grid > 0 ? grid : 1, c.block_fill, 0, s>>>(b);
    return cudaGetLastError();
}

__global__ void __launch_bounds__(256) k_export(Buffers b, float *rho, float *delta, int32_t *nh) {
    for (int t = blockIdx.x; t < b.ntiles; t += gridDim.x) {
        const Tile tl = b.tiles[t];
        const int64_t hoff = b.events[tl.event].hit_off;
        for (int k = threadIdx.x; k < tl.len; k += blockDim.x) {
            const int g = tl.start + k;
            if (rho) rho[g] = b.rho[g];
            if (delta) delta[g] = sqrtf(b.delta2[g]);
            if (nh) {
                const int j = b.nh[g];
                nh[g] = j < 0 ? -1 : (int32_t)(j - hoff);
            }
        }
    }
}

cudaError_t launch_export(const Buffers &b, const LaunchCfg &c, float *rho, float *delta,
                          int32_t *nh, cudaStream_t s) {
    const int grid = b.ntiles < c.grid_cap ? b.ntiles : c.grid_cap;
    k_export<<<grid > 0 ? grid : 1, 256, 0, s>>>(b, rho, delta, nh);
    return cudaGetLastError();
}

int64_t scan_partials_needed(int64_t n) { return (n + SCAN_TILE - 1) / SCAN_TILE + 1; }

}  // namespace clue
