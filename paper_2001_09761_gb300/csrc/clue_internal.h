// Internal declarations shared by the CUDA translation units of libclue.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace clue {

// Hits are processed in tiles of TILE consecutive indices that never straddle
// an event; tile t covers [tiles[t].start, tiles[t].start + tiles[t].len).
constexpr int TILE = 1024;

// Limits of the grid fill's two-level sort (beyond them the direct sort runs):
// layers (a per-tile histogram in shared memory and a table of tiles x layers)
// and cells per layer (counted in one CTA's shared memory).
constexpr int SEG_MAX_LAYERS = 1024;
constexpr int SEG_MAX_CELLS = 16384;
// Events the cell sort's small build (128-thread CTAs) takes: at most
// SMALL_SEG_CELLS cells per layer and SMALL_SEG_MEAN hits per layer on average.
constexpr int SMALL_SEG_CELLS = 4096;
constexpr int SMALL_SEG_MEAN = 1024;

// Candidates the density kernels stage per tile (16 bytes each): a launch's
// capacity (Params::band_cap) lies in [BAND_CAP_MIN, BAND_CAP_MAX], chosen per
// run from the grid's expected hits per row.  BAND_CAP_MIN keeps a CTA's
// shared memory within the default 48 KB.
constexpr int BAND_CAP_MIN = 1792;
constexpr int BAND_CAP_MAX = 6144;
// Static shared memory of a density CTA (its per-tile state), besides the band.
constexpr int DENSITY_SMEM_FIXED = 18736;

// Cluster id of a follower whose id has not been passed down yet (frontier
// expansion).
constexpr int32_t PENDING = -2;

// Outcome of the decision step per hit (Sec. 2.2): a follower stores its
// nearest-higher (>= 0); otherwise one of these codes.
constexpr int32_t CODE_NOISE = -1, CODE_OUTLIER = -2, CODE_SEED = -3;
// In chase mode, once the seed ranks are known, seed g's code becomes
// CODE_SEED - R, R its rank among the batch's seeds (R <= 2^31 - 3, so the
// code stays at or above INT32_MIN): the codes <= CODE_SEED are the seeds.

// Error bits raised on the device (ctrl->err).
constexpr unsigned ERRBIT_INPUT = 1u, ERRBIT_TIMEOUT = 2u;

struct EventDesc {
    int64_t hit_off;   // first hit of the event in the batch
    int64_t cell_off;  // first grid cell of the event in the batch
    int32_t n;         // hits
    int32_t nbx, nby;  // bins per layer along x and y
    float xmin, ymin;  // grid origin
    float inv_s;       // 1 / bin size
    int32_t tile0;     // first tile of the event
    int32_t ntiles;    // its tiles (0 for an empty event)
};
static_assert(sizeof(EventDesc) == 48, "EventDesc layout");

struct Tile {
    int32_t start;  // first hit (batch index)
    int32_t len;    // hits in the tile (1..TILE)
    int32_t event;  // event index
    int32_t pad;
};

// Levels of the frontier expansion run as separate launches; a tree deeper
// than this is finished by the completion pass.
constexpr int EXPAND_LEVELS = 12;

// Steps of the bounded first pass of the id walk (chase mode's k_assign, the
// frontier's completion pass): trees this shallow (the usual case) finish
// there; the hits of deeper chains are finished by pointer jumping.
constexpr int CHASE_STEPS = 64;
// Pointer-jumping rounds: each at least doubles the distance a pending hit's
// link spans, so 40 rounds exceed any chain of at most 2^31 hits.
constexpr int JUMP_ROUNDS_MAX = 40;

// Device control block.  `err` is sticky until clue_sync reads it; the rest
// is zeroed at the start of every run.
struct Ctrl {
    unsigned err;        // ERRBIT_* raised by any kernel
    unsigned overflow;   // the expansion left nodes for the completion pass
    int32_t fsize[3];    // frontier sizes, rotating over the expansion levels
    int32_t npend;       // hits the bounded walk left pending (pointer jumping)
    int32_t nrest;       // tiles the fused density kernel left for k_nh_rest
};

// Runtime parameters of one run (all events share them).
struct Params {
    float dc2;       // d_c^2 (fp32)
    float dm2;       // d_m^2, d_m = max(delta_c, delta_o)
    float dcs2;      // delta_c^2
    float dos2;      // delta_o^2
    float rhoc;
    float rwin_rho;  // d_c * (1 + 2^-12): window half-width before the |v| margin
    float rwin_nh;   // d_m * (1 + 2^-12)
    int32_t L;       // layers per event (grid planes)
    int32_t chase;   // 1: expansion by chasing nh chains (no follower lists)
    int32_t chi;     // density kernel: 0 flat, 1 Gaussian, 2 exponential
    float chi_inv;   // 1 / (2 s^2) (Gaussian) or 1 / s (exponential)
    int32_t walk_limit;  // most steps of a hit's id walk: bounded walk + jump rounds
    int32_t fused;       // 1: rho, nh and the decision in one kernel (k_density)
    int32_t band_cap;    // staged candidates per tile of the density kernels
};

// Device pointers of one run, carved from the scratch arena.
struct Buffers {
    // inputs / outputs (caller-owned)
    const float *x, *y, *w;
    const int32_t *layer;
    int32_t *cid;
    uint8_t *is_seed;
    // plan tables
    const EventDesc *events;
    const Tile *tiles;
    int32_t ntiles;
    int32_t nevents;
    int64_t N;      // total hits
    int64_t C;      // total cells
    // grid
    int32_t *key;        // [N] direct sort: local cell of hit
    int32_t *rank;       // [N] direct sort: arrival rank of the hit in its cell
    int32_t *count;      // [C] direct sort: hits per cell (zeroed per run)
    int32_t *cell_start; // [C + 1]
    float4 *rec;         // [N] direct sort: by hit, x, y, w, local cell (int bits),
                         //     for the gather; two-level sort: by position in the
                         //     layer segments, x, y, w, id (int bits); aliases hr
    int32_t *perm;       // [N] direct sort: hit ids grouped by cell, unordered within
                         //     a cell; two-level sort: ranks in a segment too long to
                         //     be permuted in shared memory
    int32_t *tcount;     // [ntb] two-level sort: hits of each tile in each layer, by
                         //     (event, layer, tile): event e's block starts at
                         //     tile0 * L, layer l's column at + l * ntiles
    int32_t *tbase;      // [ntb + 1] exclusive scan of tcount: each tile's run in
                         //     the layered order; a segment starts at its first
                         //     tile's entry
    int64_t ntb;         // tiles x layers
    uint32_t *wexp;      // [2 * nevents] weight range of each event, from the fill:
                         //     min over its finite nonzero weights of max(biased
                         //     exponent, 1), and min of 255 - biased exponent
                         //     (0xffffffff: none; set to all ones per run)
    unsigned short *cell16;  // [N] cell in the layer by layered position (two-level
                             //     sort; aliases key)
    int64_t nseg;        // events x layers, or 0: the direct sort
    int32_t max_cells;   // most cells in one layer (the cell sort's shared memory)
    const int32_t *seg_ev;  // the cell sort's event order: its small build's events
                            //     first (n_small_ev of them), or null: all, in order
    int32_t n_small_ev;
    int32_t small_cells;    // most cells in one layer of those events
    int32_t *tmp;        // [N] the sorted ids (sid)
    float4 *sp;          // [N] hits sorted by (event, layer, cell): x, y, w, id (int
                         //     bits), or for an event on the flat kernel's fixed point
                         //     x, y and the 64-bit integer weight (two words)
    int32_t *sid;        // [N] hit id by sorted position (aliases tmp; kept for the
                         //     nh step and the intermediates export)
    int32_t *lay_s;      // [N] layer in sorted order
    // density
    float *rho;          // [N] rho by sorted position (fused density kernel)
    float4 *spr;         // [N] x, y, rho, id by sorted position (separate density
                         //     kernels: the rho kernel writes it, the nh kernel reads
                         //     one record per candidate)
    int32_t rho_in_spr;  // 1: this run's rho is in spr (separate kernels), else in rho
    float2 *hr;          // [N] by sorted position: delta^2, nh (int bits: batch index
                         //     or -1), read only by the intermediates export
    // decision / expansion
    int32_t *code;       // [N] by hit: nh for a follower, else CODE_*; aliases key
                         //     (and cell16: dead once the cells are sorted)
    int32_t *fcount;     // [N] followers per hit (zeroed in the fill step)
    int32_t *frank;      // [N] arrival rank of a follower in its nh's list (aliases rank)
    unsigned long long *hs;  // [N + 1] exclusive scan of (seed << 32 | followers)
    uint32_t *sbits;     // [N / 32 + 1] seed flags by hit, one bit each (chase mode;
                         //     aliases hs; zeroed per run)
    int32_t *sword;      // [N / 32 + 2] exclusive scan of the words' seed counts
    int32_t *fol;        // [N] follower lists (CSR by nh)
    int32_t *seed_list;  // [N] seeds by global seed rank
    int32_t *front_a;    // [N] expansion frontiers (front_a aliases perm, free after S1)
    int32_t *front_b;
    int32_t *jlink;      // [N] pointer jumping: an unresolved ancestor of each pending
                         //     hit (aliases fcount: dead once the scan has read it)
    int32_t *jlist;      // [N] the pending hits (aliases seed_list: dead after the
                         //     frontier's levels, unused in chase mode)
    int32_t *rest;       // [ntiles] tiles the fused density kernel leaves for
                         //     k_nh_rest (aliases seed_list, free until the decision)
    // scan scratch
    void *scan_partials; // [nblocks + 1] block sums
    int64_t scan_partials_cap;
    Ctrl *ctrl;
};

// Launch configuration chosen per run.
struct LaunchCfg {
    int block_fill;     // threads per block: grid fill / decide kernels
    int block_density;  // threads per block: rho / nh kernels
    int grid_cap;       // persistent grid size (multiple of the SM count)
};

// ---- launchers (each enqueues its kernel(s) on `s`; return cudaError_t) ----
cudaError_t launch_fill_count(const Buffers &b, const Params &p, const LaunchCfg &c, cudaStream_t s);
cudaError_t launch_scan_cells(const Buffers &b, const LaunchCfg &c, cudaStream_t s, int *launches);
// The two-level sort (b.nseg > 0): layer count, run-table scan, placement, cell
// sort.  fill_prepare raises the cell sort's shared-memory limit on the
// current device; call it once per device before the first launch.
cudaError_t fill_prepare();
// The density kernels' dynamic shared-memory limit; once per device.
cudaError_t density_prepare();
cudaError_t launch_fill_layers(const Buffers &b, const Params &p, const LaunchCfg &c, cudaStream_t s);
cudaError_t launch_scan_segs(const Buffers &b, const LaunchCfg &c, cudaStream_t s, int *launches);
cudaError_t launch_fill_place(const Buffers &b, const Params &p, const LaunchCfg &c, cudaStream_t s);
cudaError_t launch_fill_cells(const Buffers &b, const Params &p, int max_cells, cudaStream_t s);
cudaError_t launch_fill_scatter(const Buffers &b, const LaunchCfg &c, cudaStream_t s);
cudaError_t launch_fill_canon(const Buffers &b, const Params &p, const LaunchCfg &c, cudaStream_t s);
cudaError_t launch_rho(const Buffers &b, const Params &p, const LaunchCfg &c, cudaStream_t s);
cudaError_t launch_nh(const Buffers &b, const Params &p, const LaunchCfg &c, cudaStream_t s);
cudaError_t launch_density(const Buffers &b, const Params &p, const LaunchCfg &c, cudaStream_t s);
cudaError_t launch_nh_rest(const Buffers &b, const Params &p, const LaunchCfg &c, cudaStream_t s);
cudaError_t launch_scan_hits(const Buffers &b, const Params &p, const LaunchCfg &c, cudaStream_t s,
                             int *launches);
cudaError_t launch_link(const Buffers &b, const Params &p, const LaunchCfg &c, cudaStream_t s);
bool seed_codes_separate(const Buffers &b);
cudaError_t launch_seed_codes(const Buffers &b, const LaunchCfg &c, cudaStream_t s);
cudaError_t launch_assign(const Buffers &b, const Params &p, const LaunchCfg &c, cudaStream_t s);
cudaError_t launch_expand(const Buffers &b, const LaunchCfg &c, cudaStream_t s);  // all levels
cudaError_t launch_expand_level(const Buffers &b, const LaunchCfg &c, int level, cudaStream_t s);
cudaError_t launch_complete(const Buffers &b, const Params &p, const LaunchCfg &c, cudaStream_t s);
cudaError_t launch_jump(const Buffers &b, const Params &p, cudaStream_t s);
cudaError_t launch_export(const Buffers &b, const LaunchCfg &c, float *rho, float *delta,
                          int32_t *nh, cudaStream_t s);

// Scan scratch needed for n elements (in elements of 8 bytes).
int64_t scan_partials_needed(int64_t n);

}  // namespace clue

struct clue_ctx;
namespace clue {
// The context's sticky device error word (ERRBIT_*), for the server, which
// reads it back after each batch.
unsigned *ctx_error_word(clue_ctx *ctx);

}  // namespace clue
