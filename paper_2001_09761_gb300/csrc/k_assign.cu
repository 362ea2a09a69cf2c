// Steps S4 and S5 as per-stage kernels (link, chase; the frontier expansion
// and the completion pass); the link and chase bodies and the description of
// the seed numbering are in assign_stages.cuh.
#include "assign_stages.cuh"

namespace clue {

__global__ void __launch_bounds__(256) k_link(Buffers b, Params p) { link_stage(b, p); }

cudaError_t launch_link(const Buffers &b, const Params &p, const LaunchCfg &c, cudaStream_t s) {
    const int grid = b.ntiles < c.grid_cap ? b.ntiles : c.grid_cap;
    k_link<<<grid > 0 ? grid : 1, c.block_fill, 0, s>>>(b, p);
    return cudaGetLastError();
}

// Chase mode, after the seed scan: every seed's code becomes CODE_SEED - R,
// R its rank among the batch's seeds (word prefix + the set bits below it),
// so that every chain's walk ends with its seed's rank in hand instead of
// two more scattered loads (the rank's word and bits) per hit.  A warp loads
// 32 words of the bitmap and their prefixes at once (coalesced), then takes
// its non-empty words one at a time, a lane per bit (coalesced code stores).
__device__ __forceinline__ void seed_codes_pass(const Buffers &b, int64_t warp, int64_t nwarps) {
    const int64_t nw = b.N / 32 + 1;  // the words the seed scan covers
    const unsigned below = lanemask_lt(), me = 1u << lane_id();
    for (int64_t w0 = warp * 32; w0 < nw; w0 += nwarps * 32) {
        const int64_t wl = w0 + lane_id();
        const unsigned mine = wl < nw ? b.sbits[wl] : 0u;
        const int rmine = wl < nw ? b.sword[wl] : 0;
        unsigned todo = __ballot_sync(FULL_MASK, mine != 0u);
        while (todo) {
            const int j = __ffs(todo) - 1;
            todo &= todo - 1u;
            const unsigned bits = __shfl_sync(FULL_MASK, mine, j);
            const int r = __shfl_sync(FULL_MASK, rmine, j);
            if (bits & me) b.code[(w0 + j) * 32 + lane_id()] = CODE_SEED - (r + __popc(bits & below));
        }
    }
}

__global__ void __launch_bounds__(256) k_seed_codes(Buffers b) {
    seed_codes_pass(b, ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5,
                    ((int64_t)gridDim.x * blockDim.x) >> 5);
}

// A seed bitmap short enough for a one-CTA scan: the scan and the seed codes
// in one kernel (one launch less for a small run).
__global__ void __launch_bounds__(SCAN_SINGLE_THREADS) k_seed_scan_single(Buffers b) {
    scan_single_stage<int32_t, LoadSeedWord>(LoadSeedWord{b.sbits}, b.N / 32 + 1, b.sword);
    __syncthreads();  // the CTA's own prefix stores are visible to it
    seed_codes_pass(b, threadIdx.x >> 5, SCAN_SINGLE_THREADS / 32);
}

// Chase mode: the seed-word scan, and with it the seed codes when the scan
// runs in one CTA (seed_codes_separate then says no separate launch is due).
bool seed_codes_separate(const Buffers &b) { return !scan_is_single(b.N / 32 + 1); }

cudaError_t launch_scan_hits(const Buffers &b, const Params &p, const LaunchCfg &c,
                             cudaStream_t s, int *launches) {
    if (p.chase) {
        if (!seed_codes_separate(b)) {
            k_seed_scan_single<<<1, SCAN_SINGLE_THREADS, 0, s>>>(b);
            if (launches) *launches += 1;
            return cudaGetLastError();
        }
        return exclusive_scan<int32_t>(LoadSeedWord{b.sbits}, b.N / 32 + 1, b.sword,
                                       (int32_t *)b.scan_partials, c.grid_cap, s, launches);
    }
    return exclusive_scan<unsigned long long>(LoadPacked{b.code, b.fcount}, b.N, b.hs,
                                              (unsigned long long *)b.scan_partials, c.grid_cap,
                                              s, launches);
}

cudaError_t launch_seed_codes(const Buffers &b, const LaunchCfg &c, cudaStream_t s) {
    const int64_t blocks = (b.N / 32 + 1 + 255) / 256;  // 32 words per warp
    const int grid = (int)(blocks < c.grid_cap ? blocks : c.grid_cap);
    k_seed_codes<<<grid > 0 ? grid : 1, 256, 0, s>>>(b);
    return cudaGetLastError();
}

__global__ void __launch_bounds__(256, 2) k_assign(Buffers b, Params p) { assign_stage(b, p); }

// One CTA per tile (chain lengths vary; see launch_rho).
cudaError_t launch_assign(const Buffers &b, const Params &p, const LaunchCfg &,
                          cudaStream_t s) {
    const int grid = b.ntiles;
    k_assign<<<grid > 0 ? grid : 1, 256, 0, s>>>(b, p);
    return cudaGetLastError();
}

// Frontier expansion down the follower forest, all seeds of the batch at once
// (k-way parallel at the first level, as in the paper).  Level 0 is the list
// of seeds that have followers; each level hands every frontier node's id to
// its followers and puts
// the followers that have followers of their own into the next frontier.  A
// CTA takes 256 frontier nodes, scans their follower counts, and spreads the
// followers over its threads (each finds its owner node by bisection of the
// scanned counts), so a node with many followers is not left to one thread.
// Appends to the next frontier take one atomic per CTA round (block scan).
// Levels past EXPAND_LEVELS are left to the completion pass.
constexpr int EXPAND_THREADS = 256;

__global__ void __launch_bounds__(EXPAND_THREADS) k_expand_level(Buffers b, int level) {
    __shared__ int s_off[EXPAND_THREADS + 1];
    __shared__ int s_a[EXPAND_THREADS];
    __shared__ int s_id[EXPAND_THREADS];
    __shared__ int ws[32];
    __shared__ int s_base;
    const int tid = threadIdx.x;
    const int *in = level == 0 ? b.seed_list : ((level & 1) ? b.front_a : b.front_b);
    int *out = (level & 1) ? b.front_b : b.front_a;
    const int n_in = b.ctrl->fsize[level % 3];
    int *out_size = &b.ctrl->fsize[(level + 1) % 3];
    if (blockIdx.x == 0 && tid == 0) b.ctrl->fsize[(level + 2) % 3] = 0;  // next level's output
    for (int base = blockIdx.x * EXPAND_THREADS; base < n_in; base += gridDim.x * EXPAND_THREADS) {
        const int i = base + tid;
        int a = 0, c = 0, id = 0;
        if (i < n_in) {
            const int node = in[i];
            a = (int)(unsigned)b.hs[node];
            c = (int)(unsigned)b.hs[node + 1] - a;
            id = b.cid[node];
        }
        int total;
        const int incl = block_incl_scan(c, ws, &total);
        s_off[tid] = incl - c;
        s_a[tid] = a;
        s_id[tid] = id;
        if (tid == 0) s_off[EXPAND_THREADS] = total;
        __syncthreads();
        for (int u0 = 0; u0 < total; u0 += EXPAND_THREADS) {
            const int u = u0 + tid;
            int child = 0, inner = 0;
            if (u < total) {
                int lo = 0, hi = EXPAND_THREADS - 1;  // last owner with s_off <= u
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (s_off[mid] <= u) lo = mid; else hi = mid - 1;
                }
                child = b.fol[s_a[lo] + (u - s_off[lo])];
                b.cid[child] = s_id[lo];
                inner = (unsigned)b.hs[child + 1] != (unsigned)b.hs[child];
            }
            // one append per CTA round: scan the inner flags, one atomic
            int n_inner;
            const int rank = block_incl_scan(inner, ws, &n_inner) - inner;
            if (n_inner) {
                if (tid == 0) s_base = atomicAdd(out_size, n_inner);
                __syncthreads();
                if (inner) out[s_base + rank] = child;
                __syncthreads();
            }
        }
        __syncthreads();
    }
}

cudaError_t launch_expand_level(const Buffers &b, const LaunchCfg &c, int level, cudaStream_t s) {
    k_expand_level<<<c.grid_cap > 0 ? c.grid_cap : 1, EXPAND_THREADS, 0, s>>>(b, level);
    return cudaGetLastError();
}

cudaError_t launch_expand(const Buffers &b, const LaunchCfg &c, cudaStream_t s) {
    for (int level = 0; level < EXPAND_LEVELS; ++level) {
        cudaError_t e = launch_expand_level(b, c, level, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Pending followers left after the expansion are noise (their chain ends at an
// outlier or at a hit with no nearest-higher) unless the expansion stopped
// with a non-empty frontier (a tree deeper than EXPAND_LEVELS); then each
// pending hit follows its nh chain, at most min(CHASE_STEPS, walk limit)
// steps, to the first hit with a final id (a seed, an expanded follower, or
// noise); hits of longer chains are finished by pointer jumping (k_jump).
// Ids other threads finalise meanwhile only shorten a walk.
__global__ void __launch_bounds__(256) k_complete(Buffers b, Params p) {
    const bool ovf = b.ctrl->overflow != 0 || b.ctrl->fsize[EXPAND_LEVELS % 3] != 0;
    const int kmax = min(CHASE_STEPS, p.walk_limit);
    for (int t = blockIdx.x; t < b.ntiles; t += gridDim.x) {
        const Tile tl = b.tiles[t];
        for (int k0 = 0; k0 < tl.len; k0 += blockDim.x) {
            const int k = k0 + threadIdx.x;
            const int g = tl.start + k;
            bool pend = false;
            int v = 0;
            if (k < tl.len && b.cid[g] == PENDING) {
                if (!ovf) {
                    b.cid[g] = -1;
                } else {
                    v = b.code[g];
                    int cv = __ldcg(&b.cid[v]);
                    for (int steps = 1; cv == PENDING && steps < kmax; ++steps) {
                        v = b.code[v];
                        cv = __ldcg(&b.cid[v]);
                    }
                    if (cv != PENDING) b.cid[g] = cv;
                    pend = cv == PENDING;  // v: an unresolved ancestor
                }
            }
            pend_hit(b, FULL_MASK, pend, g, v);  // the k0 loop is uniform over the CTA
        }
    }
}

cudaError_t launch_complete(const Buffers &b, const Params &p, const LaunchCfg &c,
                            cudaStream_t s) {
    const int grid = b.ntiles < c.grid_cap ? b.ntiles : c.grid_cap;
    k_complete<<<grid > 0 ? grid : 1, c.block_fill, 0, s>>>(b, p);
    return cudaGetLastError();
}

// The pointer jumping of the hits a bounded walk left pending, by one CTA
// (it returns at once when there are none, the usual case).
__global__ void __launch_bounds__(1024) k_jump(Buffers b, Params p) {
    const int np = b.ctrl->npend;
    if (np > 0) jump_rounds(b, np, p.walk_limit - min(CHASE_STEPS, p.walk_limit));
}

cudaError_t launch_jump(const Buffers &b, const Params &p, cudaStream_t s) {
    k_jump<<<1, 1024, 0, s>>>(b, p);
    return cudaGetLastError();
}

// Intermediates for tests: the nh step's record is in sorted order; each
// sorted position writes its hit's entries.
__global__ void __launch_bounds__(256) k_export(Buffers b, float *rho, float *delta, int32_t *nh) {
    for (int t = blockIdx.x; t < b.ntiles; t += gridDim.x) {
        const Tile tl = b.tiles[t];
        const int64_t hoff = b.events[tl.event].hit_off;
        for (int k = threadIdx.x; k < tl.len; k += blockDim.x) {
            const int q = tl.start + k;
            const int g = b.sid[q];
            const float2 h = b.hr[q];
            if (rho) rho[g] = b.rho_in_spr ? b.spr[q].z : b.rho[q];
            if (delta) delta[g] = sqrtf(h.x);
            if (nh) {
                const int j = __float_as_int(h.y);
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
