// clue_run_static: single-event clustering with no device allocation at all.
//
// Some callers cannot call cudaMalloc: code that runs inside a framework's
// memory pool or a real-time loop where any allocation may block or fail,
// plugins whose host owns every device allocation, or code that must keep its
// footprint fixed at load time.  For them this entry point runs the same
// pipeline as clue_run (the same kernels, so the same results bit for bit)
// with every scratch array placed in one file-scope __device__ array of fixed
// size, STATIC_BYTES below, which every GPU that loads the library holds until
// the process exits.  No context is needed; the caller passes inputs, outputs
// and a stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <mutex>

#include "clue.h"
#include "clue_internal.h"
#include "scan.cuh"

using namespace clue;

namespace {

constexpr int64_t STATIC_MAX_HITS = CLUE_STATIC_MAX_HITS;
constexpr int64_t STATIC_MAX_CELLS = CLUE_STATIC_MAX_CELLS;
constexpr int64_t STATIC_MAX_TILES = (STATIC_MAX_HITS + TILE - 1) / TILE;
constexpr int64_t STATIC_PARTS =
    (std::max(STATIC_MAX_HITS, STATIC_MAX_CELLS) + SCAN_TILE - 1) / SCAN_TILE + 2;

constexpr size_t al(size_t v) { return (v + 255) & ~(size_t)255; }
constexpr size_t NB = (size_t)STATIC_MAX_HITS, CB = (size_t)STATIC_MAX_CELLS;

// Byte layout of the scratch array (offsets in order of the Buffers fields).
constexpr size_t STATIC_BYTES =
    al(sizeof(Ctrl)) + al(sizeof(EventDesc)) + al(STATIC_MAX_TILES * sizeof(Tile)) +
    al(NB * 4) /*key*/ + al(NB * 4) /*rank*/ + al(CB * 4) /*count*/ + al((CB + 1) * 4) /*cell_start*/ +
    al(NB * 4) /*perm*/ + al(NB * 4) /*tmp*/ +
    al(NB * 16) /*sp*/ + al(NB * 4) /*lay_s*/ +
    al(NB * 16) /*rec = hr*/ + al(NB * 4) /*rho*/ + al(NB * 16) /*spr*/ + al(NB * 4) /*front_b*/ +
    al(NB * 4) /*fcount*/ + al((NB + 1) * 8) /*hs*/ + al(NB * 4) /*fol*/ +
    al(NB * 4) /*seed_list*/ + al((size_t)STATIC_PARTS * 8) /*scan partials*/ + al(8) /*wexp*/;

}  // namespace

// The scratch itself.  Host code must not pass this name to a kernel: on the
// host it is only a stand-in symbol; the device address comes from
// cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_static_scratch[STATIC_BYTES];

namespace {

constexpr int MAX_DEVICES = 64;
std::mutex g_setup_mutex;
void *g_scratch_ptr[MAX_DEVICES] = {};

// Once per device, with that device current: the device address of the array.
int scratch_address(int dev, void **out) {
    if (dev < 0 || dev >= MAX_DEVICES) return CLUE_ERR_ARG;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        // The first use on a device loads the library's device code there and
        // reserves the array; without room for it that fails as an allocation.
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return e == cudaErrorMemoryAllocation ? CLUE_ERR_OOM : CLUE_ERR_CUDA;
        }
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return CLUE_OK;
}

bool finite_nonneg(float d) { return std::isfinite(d) && d >= 0.0f && d <= 1e18f; }

}  // namespace

extern "C" int clue_run_static(const float *x, const float *y, const int32_t *layer,
                               const float *energy, int64_t n, float dc, float rhoc,
                               float delta_c, float delta_o, float x_min, float x_max,
                               float y_min, float y_max, int32_t max_layers,
                               int32_t *cluster_id, uint8_t *is_seed, void *stream) {
    if (n < 0 || n > STATIC_MAX_HITS) return CLUE_ERR_ARG;
    if (!(dc >= 1e-18f) || !finite_nonneg(dc) || !finite_nonneg(delta_c) ||
        !finite_nonneg(delta_o) || !std::isfinite(rhoc))
        return CLUE_ERR_ARG;
    if (!std::isfinite(x_min) || !std::isfinite(x_max) || !std::isfinite(y_min) ||
        !std::isfinite(y_max) || !(x_max > x_min) || !(y_max > y_min) || max_layers < 1 ||
        (int64_t)max_layers > STATIC_MAX_CELLS)
        return CLUE_ERR_ARG;
    if (n == 0) return CLUE_OK;
    if (!x || !y || !layer || !energy || !cluster_id || !is_seed) return CLUE_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CLUE_ERR_CUDA;
    void *base = nullptr;
    int rc = scratch_address(dev, &base);
    if (rc) return rc;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return CLUE_ERR_CUDA;

    // Grid: the bin size only changes speed, never results; widen the bins
    // until the grid fits the static cell budget.  Every size test is done in
    // double precision on the bin counts as reals, so no integer product or
    // int32 store happens before the grid is known to fit.
    const double wx = (double)x_max - x_min, wy = (double)y_max - y_min;
    const double cap = std::min<double>(16.0 * (double)n + 64.0 * max_layers,
                                        (double)STATIC_MAX_CELLS);
    double sbin = std::max((double)dc, 6.0 * dc * 1.001);
    double fx = 1.0, fy = 1.0;  // bins per axis as reals
    bool fits = false;
    for (int it = 0; it < 64 && !fits; ++it) {
        fx = std::max(1.0, std::ceil(wx / sbin));
        fy = std::max(1.0, std::ceil(wy / sbin));
        const double cells = fx * fy * (double)max_layers;
        fits = cells <= cap && fx <= (double)(1 << 20) && fy <= (double)(1 << 20);
        if (!fits) sbin *= std::max(1.05, std::sqrt(cells / cap));
    }
    if (!fits) return CLUE_ERR_ARG;  // no bin size gives a grid within the budget
    const int64_t nbx = (int64_t)fx, nby = (int64_t)fy;
    const int64_t C = (int64_t)max_layers * nbx * nby;
    if (C > STATIC_MAX_CELLS) return CLUE_ERR_ARG;

    // Carve the arrays in the order of STATIC_BYTES.
    char *p = (char *)base;
    auto take = [&](size_t bytes) {
        void *r = p;
        p += al(bytes);
        return r;
    };
    Buffers b{};
    Ctrl *ctrl = (Ctrl *)take(sizeof(Ctrl));
    EventDesc *d_ev = (EventDesc *)take(sizeof(EventDesc));
    Tile *d_tiles = (Tile *)take(STATIC_MAX_TILES * sizeof(Tile));
    b.key = (int32_t *)take(NB * 4);
    b.rank = (int32_t *)take(NB * 4);
    b.count = (int32_t *)take(CB * 4);
    b.cell_start = (int32_t *)take((CB + 1) * 4);
    b.perm = (int32_t *)take(NB * 4);
    b.tmp = (int32_t *)take(NB * 4);
    b.sp = (float4 *)take(NB * 16);
    b.lay_s = (int32_t *)take(NB * 4);
    b.rec = (float4 *)take(NB * 16);
    b.hr = (float2 *)b.rec;
    b.rho = (float *)take(NB * 4);
    b.spr = (float4 *)take(NB * 16);
    b.rho_in_spr = 1;  // the separate density kernels
    b.front_b = (int32_t *)take(NB * 4);
    b.code = b.key;
    b.fcount = (int32_t *)take(NB * 4);
    b.hs = (unsigned long long *)take((NB + 1) * 8);
    b.sbits = (uint32_t *)b.hs;  // chase mode: the seed bits and their word scan
    b.sword = (int32_t *)(b.sbits + (NB / 32 + 8));
    b.fol = (int32_t *)take(NB * 4);
    b.seed_list = (int32_t *)take(NB * 4);
    b.frank = b.rank;  // the fill's ranks are dead once the cells are sorted
    b.front_a = b.perm;
    b.jlink = b.fcount;
    b.jlist = b.seed_list;
    b.sid = b.tmp;
    b.scan_partials = take((size_t)STATIC_PARTS * 8);
    b.scan_partials_cap = STATIC_PARTS;
    b.wexp = (uint32_t *)take(8);
    if ((size_t)(p - (char *)base) > STATIC_BYTES) return CLUE_ERR_STATE;

    // The plan of one event: its descriptor and its tiles.
    struct {
        EventDesc ev;
        Tile tiles[STATIC_MAX_TILES];
    } host;
    std::memset(&host, 0, sizeof(host));
    host.ev.hit_off = 0;
    host.ev.cell_off = 0;
    host.ev.n = (int32_t)n;
    host.ev.nbx = (int32_t)nbx;
    host.ev.nby = (int32_t)nby;
    host.ev.xmin = x_min;
    host.ev.ymin = y_min;
    host.ev.inv_s = (float)(1.0 / sbin);
    int ntiles = 0;
    for (int64_t t = 0; t < n; t += TILE)
        host.tiles[ntiles++] = Tile{(int32_t)t, (int32_t)std::min<int64_t>(TILE, n - t), 0, 0};
    host.ev.tile0 = 0;
    host.ev.ntiles = ntiles;

    b.x = x;
    b.y = y;
    b.w = energy;
    b.layer = layer;
    b.cid = cluster_id;
    b.is_seed = is_seed;
    b.events = d_ev;
    b.tiles = d_tiles;
    b.ntiles = ntiles;
    b.nevents = 1;
    b.N = n;
    b.C = C;
    b.ctrl = ctrl;

    Params prm;
    const float dm = delta_o > delta_c ? delta_o : delta_c;
    prm.dc2 = dc * dc;
    prm.dm2 = dm * dm;
    prm.dcs2 = delta_c * delta_c;
    prm.dos2 = delta_o * delta_o;
    prm.rhoc = rhoc;
    prm.rwin_rho = dc * (1.0f + 0x1p-12f);
    prm.rwin_nh = dm * (1.0f + 0x1p-12f);
    prm.L = max_layers;
    prm.chase = 0;
    prm.chi = 0;
    prm.chi_inv = 1.0f;
    prm.walk_limit = INT_MAX;
    prm.fused = 0;
    prm.band_cap = BAND_CAP_MIN;  // within the default shared memory: no set-up needed
    LaunchCfg cfg;
    cfg.block_fill = 256;
    cfg.block_density = 128;
    cfg.grid_cap = sms * 8;

#define SCK(call)                                            \
    do {                                                     \
        if ((call) != cudaSuccess) {                         \
            cudaGetLastError();                              \
            return CLUE_ERR_CUDA;                            \
        }                                                    \
    } while (0)
    // The array keeps the previous call's contents: reset what must start at
    // zero (control word, per-cell counters); every other array is fully
    // written before it is read.
    SCK(cudaMemcpyAsync(d_ev, &host.ev, sizeof(EventDesc), cudaMemcpyHostToDevice, s));
    SCK(cudaMemcpyAsync(d_tiles, host.tiles, ntiles * sizeof(Tile), cudaMemcpyHostToDevice, s));
    SCK(cudaMemsetAsync(ctrl, 0, sizeof(Ctrl), s));
    SCK(cudaMemsetAsync(b.count, 0, (size_t)C * 4, s));
    SCK(cudaMemsetAsync(b.wexp, 0xff, 8, s));
    int nl = 0;
    SCK(launch_fill_count(b, prm, cfg, s));
    SCK(launch_scan_cells(b, cfg, s, &nl));
    SCK(launch_fill_scatter(b, cfg, s));
    SCK(launch_fill_canon(b, prm, cfg, s));
    SCK(launch_rho(b, prm, cfg, s));
    SCK(launch_nh(b, prm, cfg, s));
    SCK(launch_scan_hits(b, prm, cfg, s, &nl));
    SCK(launch_link(b, prm, cfg, s));
    SCK(launch_expand(b, cfg, s));
    SCK(launch_complete(b, prm, cfg, s));
    SCK(launch_jump(b, prm, s));
    Ctrl h{};
    SCK(cudaMemcpyAsync(&h, ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s));
    SCK(cudaStreamSynchronize(s));
#undef SCK
    if (h.err & ERRBIT_INPUT) return CLUE_ERR_INPUT;
    if (h.err) return CLUE_ERR_TIMEOUT;
    return CLUE_OK;
}
