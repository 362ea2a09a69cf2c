// Steps S4 and S5: seed ids (Sec. 2.2, Eq. 5, Algorithm 3) and the expansion
// of cluster ids down the followers: the bodies of the link stage (frontier
// mode) and the assign stage (chase mode), which the kernels in k_assign.cu
// wrap.  The seed / outlier decision itself is taken by the nh step, which
// stores one code per hit.
//
// The paper appends seeds and followers with atomics (conflicts (ii) and (iii)
// of Sec. 3), so seed numbering depends on thread timing.  Here seed ids are
// ranks from a prefix sum over hit order, giving Algorithm 3's k++ numbering
// (ascending seed index per event).  Frontier mode builds the follower lists
// as a CSR from the same prefix sum and expands k-way as in the paper, one
// launch per level of the frontier over all seeds' trees at once; chase mode
// needs no lists (assign_stage below).
#pragma once

#include <climits>

#include "scan.cuh"

namespace clue {

// (is_seed << 32 | follower count): one scan gives both the global seed rank
// (high word) and the follower-list offset (low word) of every hit.
struct LoadPacked {
    const int32_t *code;
    const int32_t *fcount;
    __device__ __forceinline__ unsigned long long operator()(int64_t i) const {
        return ((unsigned long long)(code[i] == CODE_SEED) << 32) | (unsigned)fcount[i];
    }
};

// Chase mode needs no follower lists, only seed ranks: the nh step sets one
// bit per seed, and the scan runs over the words' bit counts.
struct LoadSeedWord {
    const uint32_t *bits;
    __device__ __forceinline__ int32_t operator()(int64_t i) const { return __popc(bits[i]); }
};

// Rank of hit g among the batch's seeds (the seeds before it in hit order).
__device__ __forceinline__ int seed_rank(const Buffers &b, int64_t g) {
    const unsigned below = (1u << (g & 31)) - 1u;
    return b.sword[g >> 5] + __popc(b.sbits[g >> 5] & below);
}

// Frontier mode: seeds take their per-event id; seeds with followers enter
// the first frontier of the expansion (one atomic per CTA); followers enter
// the CSR list of their nearest-higher at the rank the decision step's count
// returned (order inside a list is irrelevant: each follower has exactly one
// parent); everything else is noise for now.
__device__ __forceinline__ void link_stage(const Buffers &b, const Params &) {
    __shared__ int ws[32];
    __shared__ int s_base;
    for (int t = blockIdx.x; t < b.ntiles; t += gridDim.x) {
        const Tile tl = b.tiles[t];
        const int64_t hoff = b.events[tl.event].hit_off;
        const unsigned ebase = (unsigned)(b.hs[hoff] >> 32);
        for (int k0 = 0; k0 < tl.len; k0 += blockDim.x) {
            const int k = k0 + threadIdx.x;
            int root = 0;
            if (k < tl.len) {
                const int g = tl.start + k;
                const int code = b.code[g];
                if (code == CODE_SEED) {
                    const unsigned long long hg = b.hs[g];
                    b.cid[g] = (int32_t)((unsigned)(hg >> 32) - ebase);
                    root = (unsigned)b.hs[g + 1] != (unsigned)hg;  // has followers
                    b.is_seed[g] = 1;
                } else {
                    b.is_seed[g] = 0;
                    if (code >= 0) {  // a follower of nh = code
                        b.fol[(int)(unsigned)b.hs[code] + b.frank[g]] = g;
                        b.cid[g] = PENDING;
                    } else {
                        b.cid[g] = -1;
                    }
                }
            }
            int n_root;
            const int r = block_incl_scan(root, ws, &n_root) - root;
            if (n_root) {
                if (threadIdx.x == 0) s_base = atomicAdd(&b.ctrl->fsize[0], n_root);
                __syncthreads();
                if (root) b.seed_list[s_base + r] = tl.start + k;
                __syncthreads();
            }
        }
    }
}

// Pending hits of a bounded id walk (chase mode's first pass, the frontier's
// completion pass): each stores an unresolved ancestor in jlink and joins the
// pending list (one atomic per warp).  `mask` holds the lanes that call.
__device__ __forceinline__ void pend_hit(const Buffers &b, unsigned mask, bool pend, int g,
                                         int anc) {
    const unsigned pm = __ballot_sync(mask, pend);
    if (!pm) return;
    const int leader = __ffs(pm) - 1;
    int base = 0;
    if (lane_id() == leader) base = atomicAdd(&b.ctrl->npend, __popc(pm));
    base = __shfl_sync(mask, base, leader);
    if (pend) {
        b.jlink[g] = anc;
        b.jlist[base + __popc(pm & lanemask_lt())] = g;
    }
}

// Pointer jumping over the pending hits, by one CTA: in every round each
// pending hit g looks at its link j = jlink[g]; if j's id is final, g takes it,
// else g's link moves to j's link, j's ancestor.  Links only move up their
// chain (an ancestor of an ancestor), so updates in place are safe, and every
// round at least doubles the distance each link spans: a chain of depth D
// needs about log2(D / CHASE_STEPS) + 1 rounds, at most JUMP_ROUNDS_MAX.  At
// most `rounds` rounds run; hits still pending then get -1 and raise
// ERRBIT_TIMEOUT.  Run by one CTA (k_jump) after the walk kernel.
__device__ __forceinline__ void jump_rounds(const Buffers &b, int np, int rounds) {
    __shared__ int s_more;
    rounds = min(rounds, JUMP_ROUNDS_MAX);
    for (int r = 0;; ++r) {
        if (threadIdx.x == 0) s_more = 0;
        __syncthreads();
        const bool last = r >= rounds;
        for (int k = threadIdx.x; k < np; k += blockDim.x) {
            const int g = __ldcg(&b.jlist[k]);
            if (__ldcg(&b.cid[g]) != PENDING) continue;
            if (last) {  // out of rounds: the walk gives up on this hit
                b.cid[g] = -1;
                atomicOr(&b.ctrl->err, ERRBIT_TIMEOUT);
                continue;
            }
            const int j = __ldcg(&b.jlink[g]);
            const int cj = __ldcg(&b.cid[j]);
            if (cj != PENDING) {
                b.cid[g] = cj;
            } else {
                b.jlink[g] = __ldcg(&b.jlink[j]);
                s_more = 1;
            }
        }
        __syncthreads();
        if (last || !s_more) break;
    }
}

// Chase mode (CLUE_EXPAND_CHASE): ids with no follower lists.  Every hit walks
// its chain of codes (a follower's code is its nearest-higher) up to the first
// hit that is not a follower, and takes that hit's id: a seed's rank among its
// event's seeds (the seed-word scan, or k_seed_codes after it, has put the
// seed's rank among the batch's seeds in its code), or -1 at an outlier or at
// a hit with no nearest-higher -- the closed form "a follower inherits the id
// of its nearest-higher" of Algorithm 3's expansion.  A seed's chain is the seed
// itself.  Chains are finite because rho rises strictly along them.  The walk
// takes at most min(CHASE_STEPS, walk limit) steps; a hit whose chain is
// longer stays pending and is finished by pointer jumping (jump_rounds, the
// next kernel) with the rest of the limit, so no chain costs more than
// O(log depth) rounds.
__device__ __forceinline__ void assign_stage(const Buffers &b, const Params &p) {
    // hits in flight per thread: their walks overlap, but a warp walks until
    // the longest of its 32 U chains ends (two measured best)
    constexpr int U = 2;
    const int kmax = min(CHASE_STEPS, p.walk_limit);
    for (int t = blockIdx.x; t < b.ntiles; t += gridDim.x) {
        const Tile tl = b.tiles[t];
        const int ebase = seed_rank(b, b.events[tl.event].hit_off);
        // the next group's codes are loaded while this group's chains are walked
        int cn[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int k = (int)threadIdx.x + u * (int)blockDim.x;
            cn[u] = k < tl.len ? b.code[tl.start + k] : CODE_NOISE;
        }
        for (int k0 = threadIdx.x; k0 < tl.len; k0 += U * blockDim.x) {
            int v[U], c[U];
            bool act[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int k = k0 + u * (int)blockDim.x;
                act[u] = k < tl.len;
                v[u] = tl.start + (act[u] ? k : 0);
                c[u] = cn[u];
                const int kn = k + U * (int)blockDim.x;
                cn[u] = kn < tl.len ? b.code[tl.start + kn] : CODE_NOISE;
                if (act[u]) b.is_seed[v[u]] = c[u] <= CODE_SEED;
            }
            bool any = true;
            for (int steps = 0; any && steps < kmax; ++steps) {
                any = false;
#pragma unroll
                for (int u = 0; u < U; ++u)
                    if (c[u] >= 0) {  // v[u] is a follower of c[u]
                        v[u] = c[u];
                        c[u] = b.code[v[u]];
                        any = true;
                    }
            }
            const unsigned mask = __activemask();
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int g = tl.start + k0 + u * (int)blockDim.x;
                const bool pend = act[u] && c[u] >= 0;  // chain longer than the walk
                int id = -1;
                if (c[u] <= CODE_SEED) id = (CODE_SEED - c[u]) - ebase;  // the seed's rank
                if (pend) id = PENDING;
                if (act[u]) b.cid[g] = id;
                pend_hit(b, mask, pend, g, c[u]);
            }
        }
    }
}

}  // namespace clue
