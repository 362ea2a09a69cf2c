// Host side of libclue: the C ABI declared in include/clue.h.
//
// A context owns a stream, a grow-only scratch arena (one allocation per size,
// reused by every later call, as the paper allocates once before its event
// loop), pinned staging for the per-call plan tables, a small cache of CUDA
// graphs for calls that repeat, and the tuning table (bin size per event-size
// class and block size of the density kernels).
#include <cuda_runtime.h>

#include <algorithm>
#include <cinttypes>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <unordered_map>
#include <vector>

#include "clue.h"
#include "clue_internal.h"
#include "scan.cuh"

using namespace clue;

namespace {

constexpr int NCLASS = 6;  // event-size classes of the tuning table, half a decade apart
constexpr int64_t CLASS_EDGE[NCLASS + 1] = {0, 32768, 100000, 316228, 1000000, 3162278,
                                            INT64_MAX};
constexpr int NPROF = 40;  // profiling events: one before the first kernel, one after each group
constexpr int NPSETS = 4;  // profiled runs whose times stay readable (a ring of event sets)
constexpr int NSTAGING = 4;
constexpr size_t GRAPH_CACHE_MAX = 32;
constexpr int MAX_CHUNKS = 16;  // chunks of the host-pointer pipeline
constexpr int64_t MAX_HITS = 2147483646LL;

int class_of(int64_t n) {
    for (int k = 0; k < NCLASS; ++k)
        if (n < CLASS_EDGE[k + 1]) return k;
    return NCLASS - 1;
}

struct GraphEntry {
    uint64_t sig = 0;
    std::vector<unsigned char> key;  // the fields `sig` hashes, compared on a hash match
    cudaGraphExec_t exec = nullptr;
    cudaGraph_t graph = nullptr;  // kept while profiled: its event-record nodes
    std::vector<cudaGraphNode_t> evnodes;  // node stamping profiling event k
    std::vector<const char *> prof_names;
    void *dtables = nullptr;
    Buffers buf{};
    LaunchCfg cfg{};
    int launches = 0;
    uint64_t last_use = 0;
};

struct Staging {
    void *host = nullptr;
    size_t cap = 0;
    cudaEvent_t done = nullptr;
};

struct Plan {
    std::vector<EventDesc> ev;
    std::vector<Tile> tiles;
    int64_t N = 0, C = 0;
    int64_t nseg = 0;   // events x layers when the two-level sort applies, else 0
    int64_t ntb = 0;    // tiles x layers (the two-level sort's run table), else 0
    int max_cells = 0;  // most cells in one layer of the batch
    // the cell sort's event order (two-level sort): the events its small
    // build takes first (n_small of them, small_cells the most cells in one
    // of their layers), then the others
    std::vector<int32_t> seg_ev;
    int n_small = 0, small_cells = 0;
};

uint64_t fnv(uint64_t h, const void *p, size_t n) {
    const unsigned char *c = (const unsigned char *)p;
    for (size_t i = 0; i < n; ++i) {
        h ^= c[i];
        h *= 1099511628211ULL;
    }
    return h;
}

size_t align_up(size_t v) { return (v + 255) & ~(size_t)255; }

}  // namespace

struct clue_ctx {
    clue_opts opts{};
    int device = 0;
    int num_sms = 0;
    cudaStream_t own = nullptr;
    cudaStream_t stream = nullptr;
    cudaStream_t h2d = nullptr, d2h = nullptr;  // copy streams of the host-pointer path
    cudaEvent_t chunk_in[MAX_CHUNKS] = {}, chunk_done[MAX_CHUNKS] = {};
    char *arena = nullptr;
    size_t arena_cap = 0;
    void *dtables = nullptr;
    size_t dtables_cap = 0;
    Staging staging[NSTAGING];
    int staging_next = 0;
    Ctrl *d_ctrl = nullptr;
    Ctrl *h_ctrl = nullptr;
    float bin_scale[NCLASS];
    int tile_len[NCLASS];   // hits per tile (one CTA of every per-tile kernel) per class
    int block_density = 0;  // threads per CTA of rho / nh (one CTA per tile); 0: by run size
    int band_cap = 0;       // staged candidates per tile of the density kernels; 0: by run
    bool profiling = false;
    // ring of event sets: profiled run r stamps set r % NPSETS
    cudaEvent_t pev[NPSETS][NPROF] = {};
    std::vector<const char *> prof_names[NPSETS];  // kernel(s) ending at pev[s][i + 1]
    int prof_set = 0;    // the set the next profiled run stamps
    int prof_count = 0;  // profiled runs so far, capped at NPSETS
    Buffers last{};
    LaunchCfg last_cfg{};
    bool have_last = false;
    int last_launches = 0;
    std::vector<GraphEntry> graphs;
    // one executable graph per pipeline shape, updated to each new call's
    // parameters (calls whose exact signature is not cached)
    std::unordered_map<int, cudaGraphExec_t> templates;
    std::unordered_map<uint64_t, int> seen;
    uint64_t tick = 0;
    char *hio = nullptr;
    size_t hio_cap = 0;
    std::string msg;
};

namespace {

int cuda_fail(clue_ctx *c, cudaError_t e, const char *what) {
    if (c) {
        c->msg = std::string(what) + ": " + cudaGetErrorString(e);
    }
    return e == cudaErrorMemoryAllocation ? CLUE_ERR_OOM : CLUE_ERR_CUDA;
}

#define CK(call)                                                    \
    do {                                                            \
        cudaError_t e_ = (call);                                    \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call);    \
    } while (0)

bool param_ok(float d) { return std::isfinite(d) && d >= 0.0f && d <= 1e18f; }

int check_params(float dc, float rhoc, float delta_c, float delta_o) {
    if (!(dc >= 1e-18f) || !param_ok(dc) || !param_ok(delta_c) || !param_ok(delta_o) ||
        !std::isfinite(rhoc))
        return CLUE_ERR_ARG;
    return CLUE_OK;
}

Params make_params(const clue_ctx *ctx, float dc, float rhoc, float delta_c, float delta_o) {
    Params p{};
    const float dm = delta_o > delta_c ? delta_o : delta_c;
    p.dc2 = dc * dc;
    p.dm2 = dm * dm;
    p.dcs2 = delta_c * delta_c;
    p.dos2 = delta_o * delta_o;
    p.rhoc = rhoc;
    const float grow = 1.0f + 0x1p-12f;
    p.rwin_rho = dc * grow;
    p.rwin_nh = dm * grow;
    p.L = ctx->opts.max_layers;
    p.chase = ctx->opts.expand == CLUE_EXPAND_CHASE;
    p.chi = ctx->opts.chi;
    const float sp = ctx->opts.chi_param;
    p.chi_inv = p.chi == CLUE_CHI_GAUSSIAN ? 1.0f / (2.0f * (sp * sp))
              : p.chi == CLUE_CHI_EXPONENTIAL ? 1.0f / sp : 1.0f;
    p.walk_limit = ctx->opts.walk_limit > 0 ? ctx->opts.walk_limit : INT_MAX;

    return p;
}

float bin_for(const clue_ctx *ctx, int64_t n, float dc) {
    float s = ctx->opts.bin_size > 0.0f ? ctx->opts.bin_size
                                        : ctx->bin_scale[class_of(n)] * 2.0f * dc * 1.001f;
    return s < dc ? dc : s;
}

int build_plan(clue_ctx *ctx, const int64_t *offsets, int32_t E, float dc, Plan &plan) {
    const clue_opts &o = ctx->opts;
    const double wx = (double)o.x_max - o.x_min, wy = (double)o.y_max - o.y_min;
    plan.ev.resize(E);
    plan.tiles.clear();
    int64_t C = 0;
    for (int32_t e = 0; e < E; ++e) {
        const int64_t n = offsets[e + 1] - offsets[e];
        double s = bin_for(ctx, n, dc);
        int64_t nbx, nby;
        // Keep the grid O(n): at most 16 cells per hit plus 64 per layer.
        const double cap = 16.0 * (double)n + 64.0 * o.max_layers;
        for (int it = 0;; ++it) {
            nbx = std::max<int64_t>(1, (int64_t)std::ceil(wx / s));
            nby = std::max<int64_t>(1, (int64_t)std::ceil(wy / s));
            const double cells = (double)nbx * nby * o.max_layers;
            if ((cells <= cap && nbx <= (1 << 20) && nby <= (1 << 20)) || it > 60) break;
            s *= std::max(1.05, std::sqrt(cells / cap));
        }
        if (n == 0) nbx = nby = 1;
        EventDesc &d = plan.ev[e];
        std::memset(&d, 0, sizeof(d));
        d.hit_off = offsets[e];
        d.cell_off = C;
        d.n = (int32_t)n;
        d.nbx = (int32_t)nbx;
        d.nby = (int32_t)nby;
        d.xmin = o.x_min;
        d.ymin = o.y_min;
        d.inv_s = (float)(1.0 / s);
        C += (int64_t)o.max_layers * nbx * nby;
        if (C > MAX_HITS) {
            ctx->msg = "grid too large: raise bin_size or shrink the extent";
            return CLUE_ERR_ARG;
        }
        d.tile0 = (int32_t)plan.tiles.size();
        const int64_t tlen = ctx->tile_len[class_of(n)];
        for (int64_t t = 0; t < n; t += tlen)
            plan.tiles.push_back(Tile{(int32_t)(offsets[e] + t),
                                      (int32_t)std::min<int64_t>(tlen, n - t), e, 0});
        d.ntiles = (int32_t)plan.tiles.size() - d.tile0;
    }
    plan.N = offsets[E];
    plan.C = C;
    int64_t most = 0;
    for (const EventDesc &d : plan.ev) most = std::max(most, (int64_t)d.nbx * d.nby);
    plan.max_cells = (int)std::min<int64_t>(most, SEG_MAX_CELLS + 1);
    // The two-level sort needs every layer's cells in one CTA's shared memory
    // and a run table of tiles x layers of at most a few ints per hit.
    const int64_t ntb = (int64_t)plan.tiles.size() * o.max_layers;
    const bool seg = o.max_layers <= SEG_MAX_LAYERS && plan.max_cells <= SEG_MAX_CELLS &&
                     ntb <= 4 * plan.N + (1 << 22);
    plan.nseg = seg ? (int64_t)E * o.max_layers : 0;
    plan.ntb = seg ? ntb : 0;
    plan.seg_ev.clear();
    plan.n_small = plan.small_cells = 0;
    if (seg) {
        auto small = [&](const EventDesc &d) {
            return (int64_t)d.nbx * d.nby <= SMALL_SEG_CELLS &&
                   d.n <= (int64_t)SMALL_SEG_MEAN * o.max_layers;
        };
        for (int32_t e = 0; e < E; ++e)
            if (small(plan.ev[e])) {
                plan.seg_ev.push_back(e);
                plan.small_cells = std::max(plan.small_cells, plan.ev[e].nbx * plan.ev[e].nby);
            }
        plan.n_small = (int)plan.seg_ev.size();
        for (int32_t e = 0; e < E; ++e)
            if (!small(plan.ev[e])) plan.seg_ev.push_back(e);
    }
    return CLUE_OK;
}

// Carve the scratch arrays of a run out of the arena; grows the arena
// (after draining the stream) when it is too small.  With `dry` set only the
// size is computed.
size_t carve(clue_ctx *ctx, Buffers &b, int64_t N, int64_t C, int64_t E, int64_t nseg,
             int64_t ntb, bool dry) {
    size_t off = 0;
    char *base = ctx->arena;
    auto take = [&](size_t bytes) -> void * {
        void *p = dry ? nullptr : (void *)(base + off);
        off += align_up(bytes);
        return p;
    };
    const size_t n = (size_t)N, c = (size_t)C;
    b.key = (int32_t *)take(n * 4);
    b.rank = (int32_t *)take(n * 4);
    b.count = (int32_t *)take(c * 4);
    b.cell_start = (int32_t *)take((c + 1) * 4);
    b.perm = (int32_t *)take(n * 4);
    b.tmp = (int32_t *)take(n * 4);
    b.sp = (float4 *)take(n * 16);
    b.lay_s = (int32_t *)take(n * 4);
    // one 16-byte-per-hit region: the grid fill's slot records, then (after
    // the fill) the per-hit records delta^2, nh of the nh step (8 bytes each)
    b.rec = (float4 *)take(n * 16);
    b.hr = (float2 *)b.rec;
    b.rho = (float *)take(n * 4);
    b.spr = (float4 *)take(n * 16);
    b.front_b = (int32_t *)take(n * 4);  // the second expansion frontier
    b.code = b.key;  // the cell of each hit is dead once the cells are sorted
    b.cell16 = (unsigned short *)b.key;
    b.fcount = (int32_t *)take(n * 4);
    b.hs = (unsigned long long *)take((n + 1) * 8);
    b.sbits = (uint32_t *)b.hs;  // chase mode: the seed bits and their word scan
    b.sword = (int32_t *)(b.sbits + (n / 32 + 8));
    b.fol = (int32_t *)take(n * 4);
    b.seed_list = (int32_t *)take(n * 4);
    b.frank = b.rank;  // the fill's ranks are dead once the cells are sorted
    b.front_a = b.perm;  // the first frontier reuses the grid fill's scratch
    b.jlink = b.fcount;  // pointer jumping: after the scan (frontier) or unused (chase)
    b.jlist = b.seed_list;
    b.rest = b.seed_list;  // the fused density kernel's left tiles, before any expansion
    b.sid = b.tmp;
    const int64_t parts =
        std::max({scan_partials_needed(N), scan_partials_needed(C), scan_partials_needed(ntb)}) + 1;
    b.scan_partials = take((size_t)parts * 8);
    b.scan_partials_cap = parts;
    b.nseg = nseg;
    b.ntb = ntb;
    b.tcount = ntb ? (int32_t *)take((size_t)ntb * 4) : nullptr;
    b.tbase = ntb ? (int32_t *)take((size_t)(ntb + 1) * 4) : nullptr;
    b.wexp = (uint32_t *)take((size_t)E * 8);
    return off;
}

void drop_graphs(clue_ctx *ctx) {
    for (auto &g : ctx->graphs) {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        if (g.graph) cudaGraphDestroy(g.graph);
        if (g.dtables) cudaFree(g.dtables);
    }
    ctx->graphs.clear();
    ctx->seen.clear();
    for (auto &t : ctx->templates)
        if (t.second) cudaGraphExecDestroy(t.second);
    ctx->templates.clear();
}

int ensure_arena(clue_ctx *ctx, size_t need) {
    if (need <= ctx->arena_cap) return CLUE_OK;
    if (ctx->opts.max_scratch_bytes > 0 && (int64_t)need > ctx->opts.max_scratch_bytes) {
        ctx->msg = "scratch limit (max_scratch_bytes) exceeded";
        return CLUE_ERR_OOM;
    }
    CK(cudaStreamSynchronize(ctx->stream));
    drop_graphs(ctx);
    if (ctx->arena) cudaFree(ctx->arena);
    ctx->arena = nullptr;
    ctx->arena_cap = 0;
    const size_t cap = need + need / 8 + (1 << 20);
    CK(cudaMalloc(&ctx->arena, cap));
    ctx->arena_cap = cap;
    return CLUE_OK;
}

// Device tables of a run: the events, the tiles, the cell sort's event order.
size_t tables_bytes(const Plan &plan) {
    return align_up(plan.ev.size() * sizeof(EventDesc)) +
           align_up(plan.tiles.size() * sizeof(Tile)) + plan.seg_ev.size() * sizeof(int32_t);
}

void fill_tables(const Plan &plan, char *dst) {
    const size_t a = align_up(plan.ev.size() * sizeof(EventDesc));
    const size_t t = align_up(plan.tiles.size() * sizeof(Tile));
    std::memcpy(dst, plan.ev.data(), plan.ev.size() * sizeof(EventDesc));
    std::memcpy(dst + a, plan.tiles.data(), plan.tiles.size() * sizeof(Tile));
    std::memcpy(dst + a + t, plan.seg_ev.data(), plan.seg_ev.size() * sizeof(int32_t));
}

void point_tables(Buffers &b, const Plan &plan, void *dtables) {
    const size_t a = align_up(plan.ev.size() * sizeof(EventDesc));
    const size_t t = align_up(plan.tiles.size() * sizeof(Tile));
    b.events = (const EventDesc *)dtables;
    b.tiles = (const Tile *)((char *)dtables + a);
    b.seg_ev = plan.seg_ev.empty() ? nullptr : (const int32_t *)((char *)dtables + a + t);
    b.n_small_ev = plan.n_small;
    b.small_cells = plan.small_cells;
    b.ntiles = (int32_t)plan.tiles.size();
    b.nevents = (int32_t)plan.ev.size();
    b.N = plan.N;
    b.C = plan.C;
    b.max_cells = plan.max_cells;
}

// Upload the plan tables through pinned staging (stream-ordered, so the host
// can build the next plan while this one is still queued).
int upload_tables_async(clue_ctx *ctx, const Plan &plan) {
    const size_t bytes = tables_bytes(plan);
    if (bytes > ctx->dtables_cap) {
        CK(cudaStreamSynchronize(ctx->stream));
        if (ctx->dtables) cudaFree(ctx->dtables);
        ctx->dtables = nullptr;
        ctx->dtables_cap = 0;
        const size_t cap = bytes + bytes / 4 + 4096;
        CK(cudaMalloc(&ctx->dtables, cap));
        ctx->dtables_cap = cap;
    }
    Staging &st = ctx->staging[ctx->staging_next];
    ctx->staging_next = (ctx->staging_next + 1) % NSTAGING;
    CK(cudaEventSynchronize(st.done));
    if (bytes > st.cap) {
        if (st.host) cudaFreeHost(st.host);
        st.host = nullptr;
        st.cap = 0;
        const size_t cap = bytes + bytes / 4 + 4096;
        CK(cudaMallocHost(&st.host, cap));
        st.cap = cap;
    }
    fill_tables(plan, (char *)st.host);
    CK(cudaMemcpyAsync(ctx->dtables, st.host, bytes, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaEventRecord(st.done, ctx->stream));
    return CLUE_OK;
}

// The density kernels' staging capacity for a run: a tile's band holds its
// own hits and about a window's height of grid rows around them, so the
// expected band of an event is its tile length plus (window rows) x (hits per
// grid row, from the event's mean over max_layers layers).  The capacity is
// the largest over the run's events with a quarter in reserve, within
// [BAND_CAP_MIN, BAND_CAP_MAX] (tiles whose band is larger take the per-hit
// form); *mean_band is the hit-weighted mean of the expected bands.
int band_cap_for(const clue_ctx *ctx, const Plan &plan, const Params &p, double *mean_band) {
    const double r = std::max(p.rwin_rho, p.rwin_nh);
    double most = 0.0, sum = 0.0, hits = 0.0;
    for (const EventDesc &d : plan.ev) {
        if (d.n <= 0) continue;
        const double s = 1.0 / d.inv_s;
        const double rows = std::ceil(2.0 * r / s) + 1.0;
        const double per_row = (double)d.n / ((double)ctx->opts.max_layers * d.nby);
        const double tlen = std::min<double>(d.n, ctx->tile_len[class_of(d.n)]);
        const double band = tlen + rows * per_row;
        most = std::max(most, 1.25 * band);
        sum += band * d.n;
        hits += d.n;
    }
    *mean_band = hits > 0.0 ? sum / hits : 0.0;
    const int cap = ctx->band_cap > 0 ? ctx->band_cap : (int)std::ceil(most / 256.0) * 256;
    return std::min(BAND_CAP_MAX, std::max(BAND_CAP_MIN, cap));
}

// Shared memory of one density CTA: the per-tile state and the staged band.
int density_smem(int band_cap) { return DENSITY_SMEM_FIXED + band_cap * 16; }

// The density kernels run one CTA per tile.  Unless the options or the
// tuning table fix their block size, a run with at least a tile per SM uses
// 256 threads (four CTAs per SM while their shared memory lets four share
// an SM, 57 KB each; else CTAs of 512 threads, two per SM), a smaller one
// 1024 (one hit per thread: its few tiles' hits all in flight at once).
LaunchCfg make_cfg(const clue_ctx *ctx, int64_t ntiles, int band_cap) {
    LaunchCfg c;
    c.block_fill = 256;
    const bool wide = density_smem(band_cap) > 57 * 1024;
    const int automatic = ntiles < ctx->num_sms ? 1024 : wide ? 512 : 256;
    c.block_density = ctx->opts.block_size > 0 ? ctx->opts.block_size
                    : ctx->block_density > 0   ? ctx->block_density
                                               : automatic;
    // a tuned block below 512 threads would leave a run with wide staging (two
    // CTAs per SM) at half occupancy: such runs keep at least 512
    if (ctx->opts.block_size == 0 && wide && ntiles >= ctx->num_sms)
        c.block_density = std::max(c.block_density, 512);
    c.grid_cap = ctx->num_sms * 8;
    return c;
}

// Queue the whole pipeline (S1 grid fill .. S5 expansion) on ctx->stream.
// With profiling on, an event of the current set is recorded before the first
// kernel and after each launch group, named in ctx->prof_names.
int enqueue(clue_ctx *ctx, const Buffers &b, const Params &p, const LaunchCfg &cfg,
            int *launches) {
    const int set = ctx->prof_set;
    cudaStream_t s = ctx->stream;
    int nl = 0;
    const bool prof = ctx->profiling;
    // Inside a stream capture a plain event record is only a dependency edge;
    // an external record becomes a graph node that stamps the event on replay.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    CK(cudaStreamIsCapturing(s, &cap));
    const unsigned rec_flags =
        cap == cudaStreamCaptureStatusActive ? cudaEventRecordExternal : cudaEventRecordDefault;
    int ev = 0;
    ctx->prof_names[set].clear();
    auto rec = [&](const char *name) -> cudaError_t {
        if (!prof) return cudaSuccess;
        if (name) ctx->prof_names[set].push_back(name);
        return cudaEventRecordWithFlags(ctx->pev[set][ev++], s, rec_flags);
    };
    // The two-level sort's first kernel resets the run's control words, weight
    // ranges and seed bits itself (memset nodes cost a run of a small event
    // several microseconds); the direct sort needs them, and its cell
    // counters, set beforehand.
    if (!b.nseg) {
        CK(cudaMemsetAsync(&b.ctrl->overflow, 0, sizeof(Ctrl) - sizeof(unsigned), s));
        CK(cudaMemsetAsync(b.count, 0, (size_t)b.C * 4, s));
        if (p.chase) CK(cudaMemsetAsync(b.sbits, 0, (size_t)(b.N / 32 + 1) * 4, s));
        CK(cudaMemsetAsync(b.wexp, 0xff, (size_t)b.nevents * 8, s));
    }
    CK(rec(nullptr));
    if (b.nseg) {  // two-level sort: layer segments, then cells
        CK(launch_fill_layers(b, p, cfg, s));
        CK(rec("fill_layers"));
        CK(launch_scan_segs(b, cfg, s, &nl));
        CK(rec("scan_segs"));
        CK(launch_fill_place(b, p, cfg, s));
        CK(rec("fill_place"));
        CK(launch_fill_cells(b, p, b.max_cells, s));
        CK(rec("fill_cells"));
        if (b.seg_ev && b.n_small_ev > 0 && b.n_small_ev < b.nevents) ++nl;  // both builds
    } else {  // direct sort over all cells
        CK(launch_fill_count(b, p, cfg, s));
        CK(rec("fill_count"));
        CK(launch_scan_cells(b, cfg, s, &nl));
        CK(rec("scan_cells"));
        CK(launch_fill_scatter(b, cfg, s));
        CK(rec("fill_scatter"));
        CK(launch_fill_canon(b, p, cfg, s));
        CK(rec("fill_canon"));
    }
    nl += 3;
    if (p.fused) {
        CK(launch_density(b, p, cfg, s));
        CK(rec("density"));
        CK(launch_nh_rest(b, p, cfg, s));
        CK(rec("nh_rest"));
    } else {
        CK(launch_rho(b, p, cfg, s));
        CK(rec("rho"));
        CK(launch_nh(b, p, cfg, s));
        CK(rec("nh_delta"));
    }
    CK(launch_scan_hits(b, p, cfg, s, &nl));
    CK(rec("scan_hits"));
    if (p.chase) {
        if (seed_codes_separate(b)) {  // else the one-CTA seed scan wrote them
            CK(launch_seed_codes(b, cfg, s));
            CK(rec("seed_codes"));
            ++nl;
        }
        CK(launch_assign(b, p, cfg, s));
        CK(rec("assign"));
        CK(launch_jump(b, p, s));
        CK(rec("jump"));
        nl += 4;  // rho, nh (with the decision), assign, jump
    } else {
        CK(launch_link(b, p, cfg, s));
        CK(rec("link"));
        for (int level = 0; level < EXPAND_LEVELS; ++level) {
            CK(launch_expand_level(b, cfg, level, s));
            CK(rec("expand_level"));
        }
        CK(launch_complete(b, p, cfg, s));
        CK(rec("complete"));
        CK(launch_jump(b, p, s));
        CK(rec("jump"));
        nl += 5 + EXPAND_LEVELS;  // rho, nh, link, complete, jump, levels
    }
    *launches = nl;
    return CLUE_OK;
}

// A run was queued: with profiling on, its event set becomes the newest one.
void prof_advance(clue_ctx *ctx) {
    if (!ctx->profiling) return;
    ctx->prof_set = (ctx->prof_set + 1) % NPSETS;
    ctx->prof_count = std::min(ctx->prof_count + 1, NPSETS);
}

// Point a captured graph's event-record nodes at the current event set (an
// update of the executable graph; launches already queued keep their events).
int graph_use_set(clue_ctx *ctx, GraphEntry &g) {
    const int set = ctx->prof_set;
    for (size_t k = 0; k < g.evnodes.size(); ++k)
        CK(cudaGraphExecEventRecordNodeSetEvent(g.exec, g.evnodes[k], ctx->pev[set][k]));
    ctx->prof_names[set] = g.prof_names;
    return CLUE_OK;
}

// After capture: the node that stamps each profiling event of the set used.
int find_event_nodes(clue_ctx *ctx, GraphEntry &g, int nev) {
    size_t nn = 0;
    CK(cudaGraphGetNodes(g.graph, nullptr, &nn));
    std::vector<cudaGraphNode_t> nodes(nn);
    CK(cudaGraphGetNodes(g.graph, nodes.data(), &nn));
    g.evnodes.assign(nev, nullptr);
    const int set = ctx->prof_set;
    for (auto n : nodes) {
        cudaGraphNodeType t;
        CK(cudaGraphNodeGetType(n, &t));
        if (t != cudaGraphNodeTypeEventRecord) continue;
        cudaEvent_t ev = nullptr;
        CK(cudaGraphEventRecordNodeGetEvent(n, &ev));
        for (int k = 0; k < nev; ++k)
            if (ctx->pev[set][k] == ev) g.evnodes[k] = n;
    }
    for (auto n : g.evnodes)
        if (!n) {
            ctx->msg = "profiling event missing from the captured graph";
            return CLUE_ERR_CUDA;
        }
    return CLUE_OK;
}

// What identifies a run's launch sequence: the event table (sizes, grids,
// offsets), the caller's pointers, the parameters, the launch configuration,
// profiling and the arena.  Serialised into `key`; returns its hash.
uint64_t signature(const clue_ctx *ctx, const Plan &plan, const Buffers &b, const Params &p,
                   const LaunchCfg &cfg, std::vector<unsigned char> &key) {
    key.clear();
    auto put = [&](const void *d, size_t n) {
        const unsigned char *c = (const unsigned char *)d;
        key.insert(key.end(), c, c + n);
    };
    put(plan.ev.data(), plan.ev.size() * sizeof(EventDesc));
    const void *ptrs[6] = {b.x, b.y, b.layer, b.w, b.cid, b.is_seed};
    put(ptrs, sizeof(ptrs));
    put(&p, sizeof(p));
    put(&cfg, sizeof(cfg));
    const int prof = ctx->profiling;
    put(&prof, sizeof(prof));
    put(&ctx->arena, sizeof(ctx->arena));
    return fnv(1469598103934665603ULL, key.data(), key.size());
}

// The shape of a run's launch sequence: expansion mode, form of the grid
// fill, the density kernels' build (CTAs above 256 threads use another
// kernel, which an executable graph's update cannot swap in), which builds
// of the cell sort run and, for each prefix sum, whether it runs in one CTA
// (at most SCAN_SINGLE_MAX_TILES tiles).
int pipeline_shape(const Buffers &b, const Params &p, const LaunchCfg &cfg) {
    auto one = [](int64_t n) { return (n + SCAN_TILE - 1) / SCAN_TILE <= SCAN_SINGLE_MAX_TILES; };
    const int64_t first = b.nseg ? b.ntb : b.C;           // run table / cells
    const int64_t second = p.chase ? b.N / 32 + 1 : b.N;  // seed words / packed scan
    const bool small = b.seg_ev && b.n_small_ev > 0, large = !b.seg_ev || b.n_small_ev < b.nevents;
    return (p.chase ? 1 : 0) | (one(first) ? 2 : 0) | (one(second) ? 4 : 0) | (b.nseg ? 8 : 0) |
           (cfg.block_density > 256 ? 16 : 0) | (small ? 32 : 0) | (large ? 64 : 0);
}

// Queue a run whose exact signature has no cached graph: capture it, and
// launch it through the executable graph of its shape, updated to this run's
// parameters (one graph launch instead of a dozen API calls per run).
int enqueue_via_template(clue_ctx *ctx, const Buffers &b, const Params &p, const LaunchCfg &cfg,
                         int *launches) {
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal);
    int erc = CLUE_OK;
    if (e == cudaSuccess) {
        erc = enqueue(ctx, b, p, cfg, launches);
        e = cudaStreamEndCapture(ctx->stream, &graph);
        if (erc != CLUE_OK && e == cudaSuccess) e = cudaErrorUnknown;
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (graph) cudaGraphDestroy(graph);
        return cuda_fail(ctx, e, "graph capture");
    }
    cudaGraphExec_t &ex = ctx->templates[pipeline_shape(b, p, cfg)];
    bool updated = false;
    if (ex) {
        cudaGraphExecUpdateResultInfo info;
        updated = cudaGraphExecUpdate(ex, graph, &info) == cudaSuccess;
        if (!updated) {
            cudaGetLastError();
            cudaGraphExecDestroy(ex);
            ex = nullptr;
        }
    }
    if (!updated) e = cudaGraphInstantiate(&ex, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        cudaGetLastError();
        ex = nullptr;
        return cuda_fail(ctx, e, "graph instantiate");
    }
    CK(cudaGraphLaunch(ex, ctx->stream));
    return CLUE_OK;
}

int run_batch(clue_ctx *ctx, const float *x, const float *y, const int32_t *layer,
              const float *energy, const int64_t *offsets, int32_t E, float dc, float rhoc,
              float delta_c, float delta_o, int32_t *cid, uint8_t *is_seed, bool allow_graph) {
    if (!ctx || E < 0 || (E > 0 && !offsets)) return CLUE_ERR_ARG;
    int rc = check_params(dc, rhoc, delta_c, delta_o);
    if (rc) return rc;
    if (E == 0) return CLUE_OK;
    if (offsets[0] != 0) return CLUE_ERR_ARG;
    for (int32_t e = 0; e < E; ++e)
        if (offsets[e + 1] < offsets[e]) return CLUE_ERR_ARG;
    const int64_t N = offsets[E];
    if (N > MAX_HITS) return CLUE_ERR_ARG;
    if (N == 0) return CLUE_OK;
    if (!x || !y || !layer || !energy || !cid || !is_seed) return CLUE_ERR_ARG;
    CK(cudaSetDevice(ctx->device));
    // A caller's own stream capture would record the tables' copy from a
    // reused staging buffer, which a later replay would read stale.
    cudaStreamCaptureStatus outer = cudaStreamCaptureStatusNone;
    if (ctx->stream) CK(cudaStreamIsCapturing(ctx->stream, &outer));
    if (outer != cudaStreamCaptureStatusNone) {
        ctx->msg = "the context's stream is being captured; run outside stream capture "
                   "(repeated calls are captured and replayed by the library itself)";
        return CLUE_ERR_STATE;
    }

    Plan plan;
    rc = build_plan(ctx, offsets, E, dc, plan);
    if (rc) return rc;
    Buffers b{};
    const int64_t E64 = (int64_t)plan.ev.size();
    const size_t need = carve(ctx, b, plan.N, plan.C, E64, plan.nseg, plan.ntb, true);
    rc = ensure_arena(ctx, need);
    if (rc) return rc;
    carve(ctx, b, plan.N, plan.C, E64, plan.nseg, plan.ntb, false);
    b.x = x;
    b.y = y;
    b.w = energy;
    b.layer = layer;
    b.cid = cid;
    b.is_seed = is_seed;
    b.ctrl = ctx->d_ctrl;
    Params p = make_params(ctx, dc, rhoc, delta_c, delta_o);
    double mean_band = 0.0;
    p.band_cap = band_cap_for(ctx, plan, p, &mean_band);
    // the fused density kernel where the run's bands, on the hit-weighted mean,
    // fit the smallest staging (sparse grid rows: its halo recomputation is
    // cheap there), else the separate kernels
    p.fused = ctx->opts.density == CLUE_DENSITY_FUSED ||
              (ctx->opts.density == CLUE_DENSITY_AUTO && mean_band <= BAND_CAP_MIN);
    b.rho_in_spr = p.fused ? 0 : 1;
    const LaunchCfg cfg = make_cfg(ctx, (int64_t)plan.tiles.size(), p.band_cap);

    const bool graphs = allow_graph && ctx->opts.use_graphs && ctx->stream != nullptr;
    if (graphs) {
        std::vector<unsigned char> key;
        const uint64_t sig = signature(ctx, plan, b, p, cfg, key);
        for (auto &g : ctx->graphs)
            if (g.sig == sig && g.key == key) {
                if (ctx->profiling) {
                    rc = graph_use_set(ctx, g);
                    if (rc) return rc;
                }
                CK(cudaGraphLaunch(g.exec, ctx->stream));
                g.last_use = ++ctx->tick;
                ctx->last = g.buf;
                ctx->last_cfg = g.cfg;
                ctx->have_last = true;
                ctx->last_launches = g.launches;
                prof_advance(ctx);
                return CLUE_OK;
            }
        if (ctx->seen.size() > 4096) ctx->seen.clear();  // one-off batches never repeat
        if (ctx->seen[sig]++ >= 1) {  // second sighting: capture
            if (ctx->graphs.size() >= GRAPH_CACHE_MAX) {
                CK(cudaStreamSynchronize(ctx->stream));
                auto it = std::min_element(ctx->graphs.begin(), ctx->graphs.end(),
                                           [](const GraphEntry &a, const GraphEntry &c) {
                                               return a.last_use < c.last_use;
                                           });
                cudaGraphExecDestroy(it->exec);
                if (it->graph) cudaGraphDestroy(it->graph);
                cudaFree(it->dtables);
                ctx->graphs.erase(it);
            }
            GraphEntry g;
            g.sig = sig;
            g.key = std::move(key);
            const size_t tb = tables_bytes(plan);
            std::vector<char> host(tb);
            fill_tables(plan, host.data());
            CK(cudaMalloc(&g.dtables, tb));
            cudaError_t e = cudaMemcpy(g.dtables, host.data(), tb, cudaMemcpyHostToDevice);
            if (e != cudaSuccess) {
                cudaFree(g.dtables);
                return cuda_fail(ctx, e, "cudaMemcpy(tables)");
            }
            g.buf = b;
            point_tables(g.buf, plan, g.dtables);
            g.cfg = cfg;
            cudaGraph_t graph = nullptr;
            e = cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                int launches = 0;
                const int erc = enqueue(ctx, g.buf, p, cfg, &launches);
                g.launches = launches;
                e = cudaStreamEndCapture(ctx->stream, &graph);
                if (erc != CLUE_OK && e == cudaSuccess) e = cudaErrorUnknown;
            }
            if (e == cudaSuccess) e = cudaGraphInstantiate(&g.exec, graph, 0);
            if (e != cudaSuccess) {
                cudaGetLastError();
                if (graph) cudaGraphDestroy(graph);
                cudaFree(g.dtables);
                return cuda_fail(ctx, e, "graph capture");
            }
            if (ctx->profiling) {
                g.graph = graph;
                g.prof_names = ctx->prof_names[ctx->prof_set];
                rc = find_event_nodes(ctx, g, (int)g.prof_names.size() + 1);
                if (rc) {
                    cudaGraphExecDestroy(g.exec);
                    cudaGraphDestroy(graph);
                    cudaFree(g.dtables);
                    return rc;
                }
            } else {
                cudaGraphDestroy(graph);
            }
            CK(cudaGraphLaunch(g.exec, ctx->stream));
            g.last_use = ++ctx->tick;
            ctx->graphs.push_back(g);
            ctx->last = g.buf;
            ctx->last_cfg = cfg;
            ctx->have_last = true;
            ctx->last_launches = g.launches;
            prof_advance(ctx);
            return CLUE_OK;
        }
    }
    rc = upload_tables_async(ctx, plan);
    if (rc) return rc;
    point_tables(b, plan, ctx->dtables);
    int launches = 0;
    rc = graphs && !ctx->profiling ? enqueue_via_template(ctx, b, p, cfg, &launches)
                                   : enqueue(ctx, b, p, cfg, &launches);
    if (rc) return rc;
    ctx->last = b;
    ctx->last_cfg = cfg;
    ctx->have_last = true;
    ctx->last_launches = launches;
    prof_advance(ctx);
    return CLUE_OK;
}

}  // namespace

namespace clue {
unsigned *ctx_error_word(clue_ctx *ctx) { return &ctx->d_ctrl->err; }
}  // namespace clue

extern "C" {

void clue_default_opts(clue_opts *o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->device = 0;
    o->x_min = -250.0f;
    o->x_max = 250.0f;
    o->y_min = -250.0f;
    o->y_max = 250.0f;
    o->max_layers = 128;
    o->bin_size = 0.0f;
    o->block_size = 0;
    o->use_graphs = 1;
    o->stream = nullptr;
    o->expand = CLUE_EXPAND_CHASE;
    o->chi = CLUE_CHI_FLAT;
    o->chi_param = 0.0f;
    o->max_scratch_bytes = 0;
    o->walk_limit = 0;
    o->density = CLUE_DENSITY_AUTO;
}

int clue_create(clue_ctx **out, const clue_opts *opts) {
    if (!out || !opts) return CLUE_ERR_ARG;
    *out = nullptr;
    const clue_opts &o = *opts;
    if (!std::isfinite(o.x_min) || !std::isfinite(o.x_max) || !std::isfinite(o.y_min) ||
        !std::isfinite(o.y_max) || !(o.x_max > o.x_min) || !(o.y_max > o.y_min) ||
        o.max_layers < 1 || !(o.bin_size >= 0.0f) || !std::isfinite(o.bin_size) ||
        o.block_size < 0 || o.block_size > 256 || (o.block_size % 32) != 0 ||
        (o.expand != CLUE_EXPAND_FRONTIER && o.expand != CLUE_EXPAND_CHASE) ||
        o.chi < CLUE_CHI_FLAT || o.chi > CLUE_CHI_EXPONENTIAL || o.max_scratch_bytes < 0 ||
        o.walk_limit < 0 ||
        o.density < CLUE_DENSITY_AUTO || o.density > CLUE_DENSITY_SEPARATE ||
        (o.chi != CLUE_CHI_FLAT && !(o.chi_param > 0.0f && std::isfinite(o.chi_param))))
        return CLUE_ERR_ARG;
    clue_ctx *ctx = new (std::nothrow) clue_ctx();
    if (!ctx) return CLUE_ERR_OOM;
    ctx->opts = o;
    ctx->device = o.device;
    // Bin size in units of 2 d_c per event-size class: about one hit per cell
    // or fewer for events spread over many layers (what the autotuner picks
    // on such events); the smaller the event, the sparser its layers, the
    // larger, the denser (a 5M-hit event of 50 layers picks 0.5).
    const float defaults[NCLASS] = {12.0f, 4.0f, 2.0f, 2.0f, 1.0f, 0.5f};
    for (int k = 0; k < NCLASS; ++k) {
        ctx->bin_scale[k] = defaults[k];
        ctx->tile_len[k] = TILE;
    }
    auto fail = [&](cudaError_t e, const char *what) {
        int rc = cuda_fail(ctx, e, what);
        clue_destroy(ctx);
        return rc;
    };
    cudaError_t e = cudaSetDevice(o.device);
    if (e != cudaSuccess) return fail(e, "cudaSetDevice");
    e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, o.device);
    if (e != cudaSuccess) return fail(e, "cudaDeviceGetAttribute");
    e = fill_prepare();
    if (e == cudaSuccess) e = density_prepare();
    if (e != cudaSuccess) return fail(e, "cudaFuncSetAttribute");
    if (o.stream) {
        ctx->stream = (cudaStream_t)o.stream;
    } else {
        e = cudaStreamCreateWithFlags(&ctx->own, cudaStreamNonBlocking);
        if (e != cudaSuccess) return fail(e, "cudaStreamCreate");
        ctx->stream = ctx->own;
    }
    e = cudaMalloc(&ctx->d_ctrl, sizeof(Ctrl));
    if (e != cudaSuccess) return fail(e, "cudaMalloc(ctrl)");
    e = cudaMemset(ctx->d_ctrl, 0, sizeof(Ctrl));
    if (e != cudaSuccess) return fail(e, "cudaMemset(ctrl)");
    e = cudaMallocHost(&ctx->h_ctrl, sizeof(Ctrl));
    if (e != cudaSuccess) return fail(e, "cudaMallocHost(ctrl)");
    for (int i = 0; i < NSTAGING; ++i) {
        e = cudaEventCreateWithFlags(&ctx->staging[i].done, cudaEventDisableTiming);
        if (e != cudaSuccess) return fail(e, "cudaEventCreate");
    }
    for (auto &set : ctx->pev)
        for (auto &ev : set) {
            e = cudaEventCreate(&ev);
            if (e != cudaSuccess) return fail(e, "cudaEventCreate");
        }
    *out = ctx;
    return CLUE_OK;
}

void clue_destroy(clue_ctx *ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    drop_graphs(ctx);
    if (ctx->arena) cudaFree(ctx->arena);
    if (ctx->dtables) cudaFree(ctx->dtables);
    if (ctx->hio) cudaFree(ctx->hio);
    if (ctx->d_ctrl) cudaFree(ctx->d_ctrl);
    if (ctx->h_ctrl) cudaFreeHost(ctx->h_ctrl);
    for (auto &s : ctx->staging) {
        if (s.host) cudaFreeHost(s.host);
        if (s.done) cudaEventDestroy(s.done);
    }
    for (auto &set : ctx->pev)
        for (auto &ev : set)
            if (ev) cudaEventDestroy(ev);
    if (ctx->h2d) {
        cudaStreamSynchronize(ctx->h2d);
        cudaStreamSynchronize(ctx->d2h);
        cudaStreamDestroy(ctx->h2d);
        cudaStreamDestroy(ctx->d2h);
        for (int i = 0; i < MAX_CHUNKS; ++i) {
            cudaEventDestroy(ctx->chunk_in[i]);
            cudaEventDestroy(ctx->chunk_done[i]);
        }
    }
    if (ctx->own) cudaStreamDestroy(ctx->own);
    delete ctx;
}

int clue_set_stream(clue_ctx *ctx, void *stream) {
    if (!ctx) return CLUE_ERR_ARG;
    cudaStream_t s = stream ? (cudaStream_t)stream : ctx->own;
    if (!s) return CLUE_ERR_ARG;  // context was created on a caller stream and has no own
    if (s == ctx->stream) return CLUE_OK;
    CK(cudaSetDevice(ctx->device));
    CK(cudaStreamSynchronize(ctx->stream));  // keep the shared scratch ordered
    ctx->stream = s;
    drop_graphs(ctx);
    return CLUE_OK;
}

int clue_run(clue_ctx *ctx, const float *x, const float *y, const int32_t *layer,
             const float *energy, int64_t n, float dc, float rhoc, float delta_c,
             float delta_o, int32_t *cluster_id, uint8_t *is_seed) {
    if (!ctx || n < 0 || n > MAX_HITS) return CLUE_ERR_ARG;
    const int64_t offs[2] = {0, n};
    return run_batch(ctx, x, y, layer, energy, offs, 1, dc, rhoc, delta_c, delta_o, cluster_id,
                     is_seed, true);
}

int clue_run_batch(clue_ctx *ctx, const float *x, const float *y, const int32_t *layer,
                   const float *energy, const int64_t *offsets, int32_t n_events, float dc,
                   float rhoc, float delta_c, float delta_o, int32_t *cluster_id,
                   uint8_t *is_seed) {
    return run_batch(ctx, x, y, layer, energy, offsets, n_events, dc, rhoc, delta_c, delta_o,
                     cluster_id, is_seed, true);
}

int clue_sync(clue_ctx *ctx) {
    if (!ctx) return CLUE_ERR_ARG;
    CK(cudaSetDevice(ctx->device));
    CK(cudaMemcpyAsync(ctx->h_ctrl, ctx->d_ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost,
                       ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    const unsigned err = ctx->h_ctrl->err;
    if (err) {
        CK(cudaMemsetAsync(&ctx->d_ctrl->err, 0, sizeof(unsigned), ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        if (err & ERRBIT_INPUT) return CLUE_ERR_INPUT;
        return CLUE_ERR_TIMEOUT;
    }
    return CLUE_OK;
}

namespace {
struct HostIO {
    float *x, *y, *e;
    int32_t *l, *cid;
    uint8_t *seed;
};

// Context-owned device buffers for n hits of inputs and outputs (grow-only).
int ensure_hio(clue_ctx *ctx, int64_t N, HostIO &io) {
    const size_t n = (size_t)N;
    const size_t need = 5 * align_up(n * 4) + align_up(n);
    if (need > ctx->hio_cap) {
        CK(cudaStreamSynchronize(ctx->stream));
        drop_graphs(ctx);
        if (ctx->hio) cudaFree(ctx->hio);
        ctx->hio = nullptr;
        ctx->hio_cap = 0;
        const size_t cap = need + need / 8 + (1 << 20);
        CK(cudaMalloc(&ctx->hio, cap));
        ctx->hio_cap = cap;
    }
    char *p = ctx->hio;
    io.x = (float *)p;
    io.y = (float *)(p + align_up(n * 4));
    io.l = (int32_t *)(p + 2 * align_up(n * 4));
    io.e = (float *)(p + 3 * align_up(n * 4));
    io.cid = (int32_t *)(p + 4 * align_up(n * 4));
    io.seed = (uint8_t *)(p + 5 * align_up(n * 4));
    return CLUE_OK;
}
}  // namespace

int clue_run_batch_host(clue_ctx *ctx, const float *x, const float *y, const int32_t *layer,
                        const float *energy, const int64_t *offsets, int32_t n_events,
                        float dc, float rhoc, float delta_c, float delta_o,
                        int32_t *cluster_id, uint8_t *is_seed) {
    if (!ctx || n_events < 0 || (n_events > 0 && !offsets)) return CLUE_ERR_ARG;
    if (n_events == 0) return CLUE_OK;
    const int64_t N = offsets[n_events];
    if (N < 0 || N > MAX_HITS || offsets[0] != 0) return CLUE_ERR_ARG;
    for (int32_t e = 0; e < n_events; ++e)
        if (offsets[e + 1] < offsets[e]) return CLUE_ERR_ARG;
    if (N == 0) return check_params(dc, rhoc, delta_c, delta_o);
    if (!x || !y || !layer || !energy || !cluster_id || !is_seed) return CLUE_ERR_ARG;
    int rc = check_params(dc, rhoc, delta_c, delta_o);
    if (rc) return rc;
    CK(cudaSetDevice(ctx->device));
    HostIO io;
    rc = ensure_hio(ctx, N, io);
    if (rc) return rc;
    if (!ctx->h2d) {
        CK(cudaStreamCreateWithFlags(&ctx->h2d, cudaStreamNonBlocking));
        CK(cudaStreamCreateWithFlags(&ctx->d2h, cudaStreamNonBlocking));
        for (int i = 0; i < MAX_CHUNKS; ++i) {
            CK(cudaEventCreateWithFlags(&ctx->chunk_in[i], cudaEventDisableTiming));
            CK(cudaEventCreateWithFlags(&ctx->chunk_done[i], cudaEventDisableTiming));
        }
    }
    // Split the batch at event boundaries into chunks, so that the copy of
    // chunk c+1 in and the copy of chunk c-1 out overlap the clustering of
    // chunk c.  Chunks of about N/8: a run of several million hits clusters
    // near the full batch's rate and spreads its fixed cost (a run of 1M hits
    // reaches only about two thirds of it), at the price of the first chunk's
    // copy in being exposed.  The last N/32 is a chunk of its own, so little
    // copy out is left after the clustering.  Batches below 8M hits are one
    // chunk.
    std::vector<int32_t> cuts{0};
    if (N >= (int64_t)(8 << 20)) {
        const int64_t step = N / 8, tail = N / 32;
        int64_t at = 0;
        while ((int)cuts.size() < MAX_CHUNKS - 1) {
            const int64_t target = std::min(at + step, N - tail);
            if (target <= at) break;
            int32_t e = cuts.back() + 1;
            while (e < n_events && offsets[e] < target) ++e;
            if (e >= n_events) break;
            cuts.push_back(e);
            at = offsets[e];
            if (at >= N - tail) break;
        }
    }
    cuts.push_back(n_events);
    // the previous call's output copies must be done before the buffers are reused
    CK(cudaStreamSynchronize(ctx->d2h));
    std::vector<int64_t> sub;
    for (size_t c = 0; c + 1 < cuts.size(); ++c) {
        const int32_t e0 = cuts[c], e1 = cuts[c + 1];
        const int64_t a = offsets[e0], nb = offsets[e1] - a;
        const size_t n4 = (size_t)nb * 4;
        CK(cudaMemcpyAsync(io.x + a, x + a, n4, cudaMemcpyHostToDevice, ctx->h2d));
        CK(cudaMemcpyAsync(io.y + a, y + a, n4, cudaMemcpyHostToDevice, ctx->h2d));
        CK(cudaMemcpyAsync(io.l + a, layer + a, n4, cudaMemcpyHostToDevice, ctx->h2d));
        CK(cudaMemcpyAsync(io.e + a, energy + a, n4, cudaMemcpyHostToDevice, ctx->h2d));
        CK(cudaEventRecord(ctx->chunk_in[c], ctx->h2d));
        CK(cudaStreamWaitEvent(ctx->stream, ctx->chunk_in[c], 0));
        sub.assign(offsets + e0, offsets + e1 + 1);
        for (auto &v : sub) v -= a;
        rc = run_batch(ctx, io.x + a, io.y + a, io.l + a, io.e + a, sub.data(), e1 - e0, dc, rhoc,
                       delta_c, delta_o, io.cid + a, io.seed + a, true);
        if (rc) return rc;
        CK(cudaEventRecord(ctx->chunk_done[c], ctx->stream));
        CK(cudaStreamWaitEvent(ctx->d2h, ctx->chunk_done[c], 0));
        CK(cudaMemcpyAsync(cluster_id + a, io.cid + a, n4, cudaMemcpyDeviceToHost, ctx->d2h));
        CK(cudaMemcpyAsync(is_seed + a, io.seed + a, (size_t)nb, cudaMemcpyDeviceToHost, ctx->d2h));
    }
    CK(cudaStreamSynchronize(ctx->d2h));
    return clue_sync(ctx);
}

int clue_stage_event(const float *x, const float *y, const int32_t *layer,
                     const float *energy, int64_t n, float *dx, float *dy, int32_t *dlayer,
                     float *denergy, int64_t offset, void *stream) {
    if (n < 0 || offset < 0) return CLUE_ERR_ARG;
    if (n == 0) return CLUE_OK;
    if (!x || !y || !layer || !energy || !dx || !dy || !dlayer || !denergy) return CLUE_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t bytes = (size_t)n * 4;
    clue_ctx *ctx = nullptr;  // CK reports without a context
    CK(cudaMemcpyAsync(dx + offset, x, bytes, cudaMemcpyDefault, s));
    CK(cudaMemcpyAsync(dy + offset, y, bytes, cudaMemcpyDefault, s));
    CK(cudaMemcpyAsync(dlayer + offset, layer, bytes, cudaMemcpyDefault, s));
    CK(cudaMemcpyAsync(denergy + offset, energy, bytes, cudaMemcpyDefault, s));
    return CLUE_OK;
}

int clue_get_intermediates(clue_ctx *ctx, float *rho, float *delta, int32_t *nh) {
    if (!ctx) return CLUE_ERR_ARG;
    if (!ctx->have_last) return CLUE_ERR_STATE;
    CK(cudaSetDevice(ctx->device));
    // The last run's tables may live in a graph entry or in the shared table
    // buffer; both stay valid until the next run or arena growth.
    CK(launch_export(ctx->last, ctx->last_cfg, rho, delta, nh, ctx->stream));
    return CLUE_OK;
}

int clue_set_profiling(clue_ctx *ctx, int32_t on) {
    if (!ctx) return CLUE_ERR_ARG;
    ctx->profiling = on != 0;
    return CLUE_OK;
}

int clue_stage_times_back(clue_ctx *ctx, int32_t back, float *ms, int32_t cap, char *names,
                          int64_t names_cap) {
    if (!ctx || (cap > 0 && !ms) || back < 0) return -CLUE_ERR_ARG;
    if (back >= ctx->prof_count) return -CLUE_ERR_STATE;
    const int set = ((ctx->prof_set - 1 - back) % NPSETS + NPSETS) % NPSETS;
    const auto &pn = ctx->prof_names[set];
    if (pn.empty()) return -CLUE_ERR_STATE;
    const int n = (int)pn.size();
    if (names && names_cap > 0) {
        std::string all;
        for (int i = 0; i < n; ++i) {
            if (i) all += ",";
            all += pn[i];
        }
        std::strncpy(names, all.c_str(), (size_t)names_cap - 1);
        names[names_cap - 1] = 0;
    }
    cudaError_t e = cudaEventSynchronize(ctx->pev[set][n]);
    if (e != cudaSuccess) return -cuda_fail(ctx, e, "cudaEventSynchronize");
    for (int i = 0; i < n && i < cap; ++i) {
        e = cudaEventElapsedTime(&ms[i], ctx->pev[set][i], ctx->pev[set][i + 1]);
        if (e != cudaSuccess) return -cuda_fail(ctx, e, "cudaEventElapsedTime");
    }
    return n;
}

int clue_stage_times(clue_ctx *ctx, float *ms, int32_t cap, char *names, int64_t names_cap) {
    return clue_stage_times_back(ctx, 0, ms, cap, names, names_cap);
}

int32_t clue_last_launch_count(clue_ctx *ctx) { return ctx ? ctx->last_launches : 0; }

int64_t clue_scratch_bytes(clue_ctx *ctx) {
    return ctx ? (int64_t)(ctx->arena_cap + ctx->dtables_cap + ctx->hio_cap) : 0;
}

int clue_autotune(clue_ctx *ctx, const float *x, const float *y, const int32_t *layer,
                  const float *energy, const int64_t *offsets, int32_t n_events, float dc,
                  float rhoc, float delta_c, float delta_o, int32_t *cluster_id,
                  uint8_t *is_seed, int32_t reps) {
    if (!ctx || reps < 1 || n_events < 1 || !offsets) return CLUE_ERR_ARG;
    int rc = check_params(dc, rhoc, delta_c, delta_o);
    if (rc) return rc;
    for (int32_t e = 0; e < n_events; ++e)
        if (offsets[e + 1] < offsets[e] || offsets[0] != 0) return CLUE_ERR_ARG;
    if (offsets[n_events] > MAX_HITS) return CLUE_ERR_ARG;
    CK(cudaSetDevice(ctx->device));
    cudaEvent_t t0, t1;
    CK(cudaEventCreate(&t0));
    CK(cudaEventCreate(&t1));
    const bool prof = ctx->profiling;
    ctx->profiling = false;
    // time `reps` runs of a batch after one untimed run (plan, arena growth)
    auto time_run = [&](const float *bx, const float *by, const int32_t *bl, const float *be,
                        const int64_t *offs, int32_t ne, int32_t *bc, uint8_t *bs,
                        float *out_ms) -> int {
        int r = run_batch(ctx, bx, by, bl, be, offs, ne, dc, rhoc, delta_c, delta_o, bc, bs,
                          false);
        if (r) return r;
        cudaError_t e = cudaEventRecord(t0, ctx->stream);
        for (int i = 0; i < reps && r == CLUE_OK && e == cudaSuccess; ++i)
            r = run_batch(ctx, bx, by, bl, be, offs, ne, dc, rhoc, delta_c, delta_o, bc, bs,
                          false);
        if (r) return r;
        if (e == cudaSuccess) e = cudaEventRecord(t1, ctx->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(t1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(out_ms, t0, t1);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "autotune timing");
        return clue_sync(ctx);
    };
    const float scales[] = {0.5f, 0.75f, 1.0f, 1.5f, 2.0f, 3.0f, 4.0f, 6.0f, 8.0f, 12.0f};
    const int tiles[] = {256, 512, 1024};  // hits per tile: 1, 2, 4 per thread at 256 threads
    const int blocks[] = {128, 256, 512};
    const float user_bin = ctx->opts.bin_size;
    const int user_block = ctx->opts.block_size;
    ctx->opts.bin_size = 0.0f;
    ctx->opts.block_size = 0;
    // Each size class is timed on its own events, copied into one contiguous
    // sub-batch, so its choices rest on its own time alone: the bin size at
    // the class's tile length, then the tile length (hits per CTA, so hits
    // per thread) at that bin size, then the bin size again at that length.
    for (int k = 0; k < NCLASS && rc == CLUE_OK; ++k) {
        std::vector<int64_t> sub{0};
        for (int32_t e = 0; e < n_events; ++e) {
            const int64_t n = offsets[e + 1] - offsets[e];
            if (n > 0 && class_of(n) == k) sub.push_back(sub.back() + n);
        }
        if (sub.size() < 2) continue;
        HostIO io;
        rc = ensure_hio(ctx, sub.back(), io);
        if (rc) break;
        int64_t at = 0;
        for (int32_t e = 0; e < n_events && rc == CLUE_OK; ++e) {
            const int64_t n = offsets[e + 1] - offsets[e];
            if (n <= 0 || class_of(n) != k) continue;
            const int64_t o = offsets[e];
            cudaError_t ce = cudaMemcpyAsync(io.x + at, x + o, n * 4, cudaMemcpyDeviceToDevice, ctx->stream);
            if (ce == cudaSuccess) ce = cudaMemcpyAsync(io.y + at, y + o, n * 4, cudaMemcpyDeviceToDevice, ctx->stream);
            if (ce == cudaSuccess) ce = cudaMemcpyAsync(io.l + at, layer + o, n * 4, cudaMemcpyDeviceToDevice, ctx->stream);
            if (ce == cudaSuccess) ce = cudaMemcpyAsync(io.e + at, energy + o, n * 4, cudaMemcpyDeviceToDevice, ctx->stream);
            if (ce != cudaSuccess) rc = cuda_fail(ctx, ce, "autotune gather");
            at += n;
        }
        if (rc) break;
        auto time_class = [&](float *out_ms) {
            return time_run(io.x, io.y, io.l, io.e, sub.data(), (int32_t)sub.size() - 1, io.cid,
                            io.seed, out_ms);
        };
        for (int pass = 0; pass < 3 && rc == CLUE_OK; ++pass) {
            float best = 1e30f;
            if (pass != 1) {
                float best_s = ctx->bin_scale[k];
                for (float sc : scales) {
                    ctx->bin_scale[k] = sc;
                    float ms = 0;
                    rc = time_class(&ms);
                    if (rc) break;
                    if (ms < best) {
                        best = ms;
                        best_s = sc;
                    }
                }
                ctx->bin_scale[k] = best_s;
            } else {
                int best_t = ctx->tile_len[k];
                for (int tl : tiles) {
                    ctx->tile_len[k] = tl;
                    float ms = 0;
                    rc = time_class(&ms);
                    if (rc) break;
                    if (ms < best) {
                        best = ms;
                        best_t = tl;
                    }
                }
                ctx->tile_len[k] = best_t;
            }
        }
    }
    if (rc == CLUE_OK) {  // the density kernels' block size, on the whole batch
        float best = 1e30f;
        int best_b = ctx->block_density;
        for (int bsz : blocks) {
            ctx->block_density = bsz;
            float ms = 0;
            rc = time_run(x, y, layer, energy, offsets, n_events, cluster_id, is_seed, &ms);
            if (rc) break;
            if (ms < best) {
                best = ms;
                best_b = bsz;
            }
        }
        ctx->block_density = best_b;
    }
    ctx->opts.bin_size = user_bin;
    ctx->opts.block_size = user_block;
    ctx->profiling = prof;
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    drop_graphs(ctx);
    return rc;
}

int64_t clue_get_tuning(clue_ctx *ctx, char *buf, int64_t cap) {
    if (!ctx) return -CLUE_ERR_ARG;
    std::string s = "# clue tuning v3: class <lo> <hi> <bin_scale> <tile_hits>; block <threads>; "
                    "band <staged records>\n";
    char line[160];
    for (int k = 0; k < NCLASS; ++k) {
        std::snprintf(line, sizeof(line), "class %" PRId64 " %" PRId64 " %.4f %d\n", CLASS_EDGE[k],
                      CLASS_EDGE[k + 1], (double)ctx->bin_scale[k], ctx->tile_len[k]);
        s += line;
    }
    std::snprintf(line, sizeof(line), "block %d\n", ctx->block_density);
    s += line;
    std::snprintf(line, sizeof(line), "band %d\n", ctx->band_cap);
    s += line;
    if (buf && cap > 0) {
        std::strncpy(buf, s.c_str(), (size_t)cap - 1);
        buf[cap - 1] = 0;
    }
    return (int64_t)s.size() + 1;
}

int clue_set_tuning(clue_ctx *ctx, const char *text) {
    if (!ctx || !text) return CLUE_ERR_ARG;
    float scale[NCLASS];
    int tlen[NCLASS];
    for (int k = 0; k < NCLASS; ++k) {
        scale[k] = ctx->bin_scale[k];
        tlen[k] = ctx->tile_len[k];
    }
    int block = ctx->block_density, band = ctx->band_cap;
    const char *p = text;
    while (*p) {
        const char *eol = std::strchr(p, '\n');
        std::string line(p, eol ? (size_t)(eol - p) : std::strlen(p));
        p = eol ? eol + 1 : p + line.size();
        if (line.empty() || line[0] == '#') continue;
        long long lo, hi;
        float sc;
        int bl, tl = TILE;
        char tail;
        // "class lo hi scale [tile_hits]" (the tile length is optional: v1 text)
        const int nf = std::sscanf(line.c_str(), "class %lld %lld %f %d %c", &lo, &hi, &sc, &tl,
                                   &tail);
        if (nf == 3 || nf == 4) {
            int k = -1;
            for (int i = 0; i < NCLASS; ++i)
                if (CLASS_EDGE[i] == lo && CLASS_EDGE[i + 1] == hi) k = i;
            if (k < 0 || !(sc >= 0.25f && sc <= 64.0f) || tl < 32 || tl > TILE || tl % 32)
                return CLUE_ERR_ARG;
            scale[k] = sc;
            tlen[k] = tl;
        } else if (std::sscanf(line.c_str(), "block %d %c", &bl, &tail) == 1) {
            if (bl != 0 && (bl < 32 || bl > 1024 || bl % 32)) return CLUE_ERR_ARG;  // 0: by run size
            block = bl;
        } else if (std::sscanf(line.c_str(), "band %d %c", &bl, &tail) == 1) {
            if (bl != 0 && (bl < BAND_CAP_MIN || bl > BAND_CAP_MAX)) return CLUE_ERR_ARG;
            band = bl;  // 0: by run
        } else {
            return CLUE_ERR_ARG;
        }
    }
    for (int k = 0; k < NCLASS; ++k) {
        ctx->bin_scale[k] = scale[k];
        ctx->tile_len[k] = tlen[k];
    }
    ctx->block_density = block;
    ctx->band_cap = band;
    drop_graphs(ctx);
    return CLUE_OK;
}

const char *clue_strerror(int code) {
    switch (code) {
        case CLUE_OK: return "ok";
        case CLUE_ERR_ARG: return "invalid argument";
        case CLUE_ERR_INPUT: return "invalid input values (NaN/Inf coordinate or energy, or layer out of range)";
        case CLUE_ERR_OOM: return "out of memory";
        case CLUE_ERR_CUDA: return "CUDA error";
        case CLUE_ERR_TIMEOUT: return "bounded device wait gave up";
        case CLUE_ERR_STATE: return "invalid state for this call";
        default: return "unknown error";
    }
}

const char *clue_last_message(clue_ctx *ctx) { return ctx ? ctx->msg.c_str() : ""; }

const char *clue_version(void) { return "clue-gb300 0.1 (sm_103a)"; }

}  // extern "C"
