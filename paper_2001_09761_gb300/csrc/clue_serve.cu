// clue_server: continuous batching on one GPU (include/clue.h), the
// scheduler of serve_core.h over a CUDA backend.
//
// The backend keeps n_regions device regions of region_hits hits (inputs and
// outputs).  An admitted event's inputs are copied from the caller's host
// arrays into the region being filled, on that region's copy stream (so the
// copies of different regions can use different copy engines); a launched region is
// one clue_run_batch on the compute stream (after the region's copies), then
// the batch's device error word is read back and cleared there, and on an
// output stream (so the next batch need not wait for them) each event's
// results are copied into the caller's output arrays and a host callback
// (cudaLaunchHostFunc: no CUDA call inside, it only takes the scheduler's
// lock) reports the batch done.  Nothing polls: the scheduler's worker sleeps
// until a submission or such a callback wakes it.
#include <cuda_runtime.h>

#include <cstring>
#include <new>
#include <vector>

#include "clue.h"
#include "clue_internal.h"
#include "serve_core.h"

namespace {

// Device bytes an admitted hit holds against a server's budget: its inputs
// (16) and outputs (5) in a region and the run's scratch (about 120).
constexpr int64_t SERVER_BYTES_PER_HIT = 16 + 5 + 120;

class CudaBackend : public clue_serve::Backend {
  public:
    struct Callback {
        CudaBackend *be = nullptr;
        int region = 0;
        int64_t batch = 0;
    };
    struct Region {
        float *x = nullptr, *y = nullptr, *e = nullptr;
        int32_t *l = nullptr, *cid = nullptr;
        uint8_t *seed = nullptr;
        cudaStream_t copy = nullptr;  // the region's input copies (regions overlap theirs)
        cudaEvent_t staged = nullptr;
        cudaEvent_t computed = nullptr;  // the batch's kernels and error readback are done
    };

    int device = 0;
    int64_t cap = 0;
    int nreg = 0;
    float prm[4] = {};
    clue_ctx *ctx = nullptr;
    cudaStream_t compute = nullptr;
    cudaStream_t out = nullptr;  // result copies and completion callbacks (off the compute
                                 // stream, so the next batch starts at once)
    std::vector<Region> regs;
    std::vector<Callback> cbs;     // one per region: a region runs one batch at a time
    unsigned *err_host = nullptr;  // pinned, one word per region
    clue_serve::Scheduler *sched = nullptr;

    int64_t region_hits() const override { return cap; }
    int n_regions() const override { return nreg; }

    int stage(int region, int64_t off, const clue_serve::Request &r) override {
        if (cudaSetDevice(device) != cudaSuccess) return CLUE_ERR_CUDA;
        Region &g = regs[region];
        void *dst[4] = {g.x + off, g.y + off, g.l + off, g.e + off};
        for (int k = 0; k < 4; ++k)
            if (cudaMemcpyAsync(dst[k], r.in[k], (size_t)r.n * 4, cudaMemcpyDefault, g.copy) !=
                cudaSuccess)
                return CLUE_ERR_CUDA;
        return CLUE_OK;
    }

    int launch(int region, const std::vector<int64_t> &offs,
               const std::vector<clue_serve::Request> &reqs, int64_t batch) override {
        if (cudaSetDevice(device) != cudaSuccess) return CLUE_ERR_CUDA;
        Region &g = regs[region];
        if (cudaEventRecord(g.staged, g.copy) != cudaSuccess ||
            cudaStreamWaitEvent(compute, g.staged, 0) != cudaSuccess)
            return CLUE_ERR_CUDA;
        const int rc = clue_run_batch(ctx, g.x, g.y, g.l, g.e, offs.data(),
                                      (int32_t)reqs.size(), prm[0], prm[1], prm[2], prm[3],
                                      g.cid, g.seed);
        if (rc != CLUE_OK) return rc;
        // the batch's own device errors: read the sticky word back and clear it
        // before the next batch's kernels, on the compute stream
        unsigned *err = clue::ctx_error_word(ctx);
        if (cudaMemcpyAsync(&err_host[region], err, sizeof(unsigned), cudaMemcpyDeviceToHost,
                            compute) != cudaSuccess ||
            cudaMemsetAsync(err, 0, sizeof(unsigned), compute) != cudaSuccess ||
            cudaEventRecord(g.computed, compute) != cudaSuccess ||
            cudaStreamWaitEvent(out, g.computed, 0) != cudaSuccess)
            return CLUE_ERR_CUDA;
        // each event's results into its own arrays, while the next batch runs
        for (size_t k = 0; k < reqs.size(); ++k) {
            const int64_t a = offs[k], n = offs[k + 1] - a;
            if (n == 0) continue;
            if (cudaMemcpyAsync(reqs[k].out[0], g.cid + a, (size_t)n * 4, cudaMemcpyDefault,
                                out) != cudaSuccess ||
                cudaMemcpyAsync(reqs[k].out[1], g.seed + a, (size_t)n, cudaMemcpyDefault,
                                out) != cudaSuccess)
                return CLUE_ERR_CUDA;
        }
        cbs[region] = Callback{this, region, batch};
        if (cudaLaunchHostFunc(out, &CudaBackend::done, &cbs[region]) != cudaSuccess)
            return CLUE_ERR_CUDA;
        return CLUE_OK;
    }

    // Runs on a CUDA callback thread once the batch and its copies are done.
    static void CUDART_CB done(void *p) {
        const Callback *c = static_cast<const Callback *>(p);
        const unsigned e = c->be->err_host[c->region];
        const int status = (e & clue::ERRBIT_INPUT) ? CLUE_ERR_INPUT
                         : e                        ? CLUE_ERR_TIMEOUT
                                                    : CLUE_OK;
        c->be->sched->batch_done(c->batch, status);
    }

    void release() {
        cudaSetDevice(device);
        if (compute) cudaStreamSynchronize(compute);
        if (out) cudaStreamSynchronize(out);
        for (Region &g : regs) {
            if (g.copy) cudaStreamSynchronize(g.copy);
            if (g.x) cudaFree(g.x);
            if (g.staged) cudaEventDestroy(g.staged);
            if (g.computed) cudaEventDestroy(g.computed);
            if (g.copy) cudaStreamDestroy(g.copy);
        }
        regs.clear();
        if (ctx) clue_destroy(ctx);
        ctx = nullptr;
        if (err_host) cudaFreeHost(err_host);
        err_host = nullptr;
        if (compute) cudaStreamDestroy(compute);
        if (out) cudaStreamDestroy(out);
        compute = out = nullptr;
    }
};

}  // namespace

struct clue_server {
    CudaBackend be;
    clue_serve::Scheduler *sched = nullptr;
};

extern "C" {

void clue_server_default_opts(clue_server_opts *o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->region_hits = 16 << 20;
    o->n_regions = 3;
    o->max_inflight = 2;
    o->max_events_per_batch = 512;
    o->mem_budget_bytes = 0;
}

int clue_server_create(clue_server **out, const clue_opts *opts, const clue_server_opts *so,
                       float dc, float rhoc, float delta_c, float delta_o,
                       const char *tuning) {
    if (!out || !opts || !so) return CLUE_ERR_ARG;
    *out = nullptr;
    if (so->region_hits < 1 || so->region_hits > 2147483646LL || so->n_regions < 2 ||
        so->n_regions > 64 || so->max_inflight < 1 || so->max_events_per_batch < 1 ||
        so->mem_budget_bytes < 0)
        return CLUE_ERR_ARG;
    clue_server *s = new (std::nothrow) clue_server();
    if (!s) return CLUE_ERR_OOM;
    CudaBackend &be = s->be;
    be.device = opts->device;
    be.cap = so->region_hits;
    be.nreg = so->n_regions;
    be.prm[0] = dc;
    be.prm[1] = rhoc;
    be.prm[2] = delta_c;
    be.prm[3] = delta_o;
    auto fail = [&](int rc) {
        be.release();
        delete s;
        return rc;
    };
    if (cudaSetDevice(be.device) != cudaSuccess) return fail(CLUE_ERR_CUDA);
    if (cudaStreamCreateWithFlags(&be.compute, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&be.out, cudaStreamNonBlocking) != cudaSuccess)
        return fail(CLUE_ERR_CUDA);
    clue_opts o = *opts;
    o.stream = be.compute;
    int rc = clue_create(&be.ctx, &o);
    if (rc) return fail(rc);
    if (tuning && tuning[0]) {
        rc = clue_set_tuning(be.ctx, tuning);
        if (rc) return fail(rc);
    }
    if (cudaMallocHost(&be.err_host, sizeof(unsigned) * be.nreg) != cudaSuccess)
        return fail(CLUE_ERR_OOM);
    be.regs.resize(be.nreg);
    be.cbs.resize(be.nreg);
    const size_t n = (size_t)be.cap, a4 = (n * 4 + 255) & ~(size_t)255;
    for (auto &g : be.regs) {
        char *p = nullptr;
        const cudaError_t e = cudaMalloc(&p, 5 * a4 + n);
        if (e != cudaSuccess) return fail(e == cudaErrorMemoryAllocation ? CLUE_ERR_OOM : CLUE_ERR_CUDA);
        g.x = (float *)p;
        g.y = (float *)(p + a4);
        g.l = (int32_t *)(p + 2 * a4);
        g.e = (float *)(p + 3 * a4);
        g.cid = (int32_t *)(p + 4 * a4);
        g.seed = (uint8_t *)(p + 5 * a4);
        if (cudaEventCreateWithFlags(&g.staged, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&g.computed, cudaEventDisableTiming) != cudaSuccess ||
            cudaStreamCreateWithFlags(&g.copy, cudaStreamNonBlocking) != cudaSuccess)
            return fail(CLUE_ERR_CUDA);
    }
    s->sched = new (std::nothrow) clue_serve::Scheduler(
        &be, so->max_events_per_batch, so->max_inflight, so->mem_budget_bytes,
        SERVER_BYTES_PER_HIT);
    if (!s->sched) return fail(CLUE_ERR_OOM);
    be.sched = s->sched;
    *out = s;
    return CLUE_OK;
}

int clue_server_submit(clue_server *s, const float *x, const float *y, const int32_t *layer,
                       const float *energy, int64_t n, int32_t *cluster_id, uint8_t *is_seed,
                       int64_t *ticket) {
    if (!s || !ticket || n < 0) return CLUE_ERR_ARG;
    if (n > 0 && (!x || !y || !layer || !energy || !cluster_id || !is_seed)) return CLUE_ERR_ARG;
    clue_serve::Request r;
    r.n = n;
    r.in[0] = x;
    r.in[1] = y;
    r.in[2] = layer;
    r.in[3] = energy;
    r.out[0] = cluster_id;
    r.out[1] = is_seed;
    return s->sched->submit(r, ticket);
}

int clue_server_wait(clue_server *s, int64_t ticket, double timeout_s, int32_t *status,
                     double *latency_ms) {
    if (!s) return CLUE_ERR_ARG;
    int st = CLUE_OK;
    const int rc = s->sched->wait(ticket, timeout_s, &st, latency_ms);
    if (status) *status = st;
    return rc;
}

int64_t clue_server_stats(clue_server *s, double *out, double *latency_ms, int64_t cap) {
    if (!s) return -CLUE_ERR_ARG;
    const clue_serve::Stats st = s->sched->stats();
    if (out) {
        double mean_ev = 0.0;
        for (int32_t v : st.batch_events) mean_ev += v;
        out[0] = (double)st.events;
        out[1] = (double)st.hits;
        out[2] = (double)st.batches;
        out[3] = (double)st.rejected;
        out[4] = st.last_done > st.first_submit && st.first_submit >= 0
                     ? st.last_done - st.first_submit : 0.0;
        out[5] = st.batch_events.empty() ? 0.0 : mean_ev / st.batch_events.size();
    }
    const int64_t n = (int64_t)st.latency_ms.size();
    if (latency_ms)
        for (int64_t i = 0; i < n && i < cap; ++i) latency_ms[i] = st.latency_ms[i];
    return n;
}

int clue_server_reset_stats(clue_server *s) {
    if (!s) return CLUE_ERR_ARG;
    s->sched->reset_stats();
    return CLUE_OK;
}

void clue_server_destroy(clue_server *s) {
    if (!s) return;
    if (s->sched) {
        s->sched->stop();
        delete s->sched;
    }
    s->be.release();
    delete s;
}

}  // extern "C"
