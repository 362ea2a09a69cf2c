// A fake device for the server's scheduler (paper_2001_09761_gb300/csrc/
// serve_core.cpp), so its scheduling runs and is tested on a machine without
// a GPU.  The fake "clusters" an event by writing cluster_id = int(x) and
// is_seed = (x > 0) for each hit; one thread plays the device stream, taking
// batches in launch order and spending `delay_s` on each.  It records what
// the scheduler did (the staged offsets and the events of every batch).
// Built by tests/test_serve.py with g++ into a test-only shared library.
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <vector>

#include "clue.h"
#include "serve_core.h"

namespace {

class FakeBackend : public clue_serve::Backend {
  public:
    struct Batch {
        int64_t id;
        int region;
        std::vector<int64_t> offs;
        std::vector<clue_serve::Request> reqs;
    };
    int64_t cap;
    int nreg;
    double delay;
    clue_serve::Scheduler *sched = nullptr;
    std::vector<std::vector<float>> x;  // each region's staged x
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Batch> queue;
    bool stop = false;
    std::vector<std::vector<int64_t>> launched;  // offsets of every batch
    int64_t staged_hits = 0, max_staged_hits = 0;
    std::thread dev;

    FakeBackend(int64_t c, int n, double d) : cap(c), nreg(n), delay(d) {
        x.assign(n, std::vector<float>((size_t)c));
        dev = std::thread([this] { run(); });
    }
    ~FakeBackend() override {
        {
            std::lock_guard<std::mutex> lk(mu);
            stop = true;
        }
        cv.notify_one();
        dev.join();
    }
    int64_t region_hits() const override { return cap; }
    int n_regions() const override { return nreg; }
    int stage(int region, int64_t off, const clue_serve::Request &r) override {
        std::memcpy(x[region].data() + off, r.in[0], (size_t)r.n * sizeof(float));
        std::lock_guard<std::mutex> lk(mu);
        staged_hits += r.n;
        if (staged_hits > max_staged_hits) max_staged_hits = staged_hits;
        return CLUE_OK;
    }
    int launch(int region, const std::vector<int64_t> &offs,
               const std::vector<clue_serve::Request> &reqs, int64_t batch) override {
        std::lock_guard<std::mutex> lk(mu);
        launched.push_back(offs);
        queue.push_back(Batch{batch, region, offs, reqs});
        cv.notify_one();
        return CLUE_OK;
    }
    void run() {
        for (;;) {
            Batch b;
            {
                std::unique_lock<std::mutex> lk(mu);
                cv.wait(lk, [&] { return stop || !queue.empty(); });
                if (queue.empty()) return;
                b = queue.front();
                queue.pop_front();
            }
            std::this_thread::sleep_for(std::chrono::duration<double>(delay));
            for (size_t k = 0; k < b.reqs.size(); ++k) {
                const int64_t a = b.offs[k], n = b.offs[k + 1] - a;
                int32_t *cid = (int32_t *)b.reqs[k].out[0];
                uint8_t *seed = (uint8_t *)b.reqs[k].out[1];
                for (int64_t i = 0; i < n; ++i) {
                    const float v = x[b.region][(size_t)(a + i)];
                    cid[i] = (int32_t)v;
                    seed[i] = v > 0.0f;
                }
            }
            {
                std::lock_guard<std::mutex> lk(mu);
                staged_hits -= b.offs.back();
            }
            sched->batch_done(b.id, CLUE_OK);
        }
    }
};

struct Fake {
    FakeBackend *be;
    clue_serve::Scheduler *sched;
};

}  // namespace

extern "C" {

void *fake_server_create(int64_t capacity, int32_t n_regions, double delay_s,
                         int32_t max_events, int32_t max_inflight, int64_t budget,
                         int64_t bytes_per_hit) {
    Fake *f = new Fake;
    f->be = new FakeBackend(capacity, n_regions, delay_s);
    f->sched = new clue_serve::Scheduler(f->be, max_events, max_inflight, budget, bytes_per_hit);
    f->be->sched = f->sched;
    return f;
}

int fake_server_submit(void *p, const float *x, int64_t n, int32_t *cid, uint8_t *seed,
                       int64_t *ticket) {
    clue_serve::Request r;
    r.n = n;
    r.in[0] = x;
    r.out[0] = cid;
    r.out[1] = seed;
    return ((Fake *)p)->sched->submit(r, ticket);
}

int fake_server_wait(void *p, int64_t ticket, double timeout_s, int32_t *status,
                     double *latency_ms) {
    int st = 0;
    const int rc = ((Fake *)p)->sched->wait(ticket, timeout_s, &st, latency_ms);
    *status = st;
    return rc;
}

// Offsets of every launched batch, flattened with a -1 after each batch.
int64_t fake_server_launched(void *p, int64_t *out, int64_t cap) {
    FakeBackend *be = ((Fake *)p)->be;
    std::lock_guard<std::mutex> lk(be->mu);
    int64_t k = 0;
    for (const auto &offs : be->launched) {
        for (int64_t v : offs) {
            if (k < cap) out[k] = v;
            ++k;
        }
        if (k < cap) out[k] = -1;
        ++k;
    }
    return k;
}

int64_t fake_server_max_staged(void *p) {
    FakeBackend *be = ((Fake *)p)->be;
    std::lock_guard<std::mutex> lk(be->mu);
    return be->max_staged_hits;
}

// events, hits, batches, rejected, span (s), mean events per batch
void fake_server_stats(void *p, double *out) {
    const clue_serve::Stats st = ((Fake *)p)->sched->stats();
    double ev = 0.0;
    for (int32_t v : st.batch_events) ev += v;
    out[0] = (double)st.events;
    out[1] = (double)st.hits;
    out[2] = (double)st.batches;
    out[3] = (double)st.rejected;
    out[4] = st.last_done - st.first_submit;
    out[5] = st.batch_events.empty() ? 0.0 : ev / st.batch_events.size();
}

void fake_server_stop(void *p) { ((Fake *)p)->sched->stop(); }

void fake_server_destroy(void *p) {
    Fake *f = (Fake *)p;
    f->sched->stop();
    delete f->sched;
    delete f->be;
    delete f;
}

}  // extern "C"
