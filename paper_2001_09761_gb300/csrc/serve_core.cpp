// The continuous-batching scheduler declared in serve_core.h.
#include "serve_core.h"

#include <algorithm>
#include <chrono>

#include "clue.h"

namespace clue_serve {

namespace {
double clock_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}
}  // namespace

Scheduler::Scheduler(Backend *be, int max_events_per_batch, int max_inflight,
                     int64_t budget_bytes, int64_t bytes_per_hit)
    : be_(be),
      max_events_(std::max(1, max_events_per_batch)),
      max_inflight_(std::max(1, std::min(max_inflight, be->n_regions() - 1))),
      budget_(budget_bytes),
      bytes_per_hit_(bytes_per_hit) {
    regions_.resize(be->n_regions());
    for (int i = 0; i < (int)regions_.size(); ++i) regions_[i].idx = i;
    worker_ = std::thread([this] { loop(); });
}

Scheduler::~Scheduler() { stop(); }

double Scheduler::now() const { return clock_s(); }

int Scheduler::submit(const Request &r0, int64_t *ticket) {
    if (!ticket || r0.n < 0) return CLUE_ERR_ARG;
    Request r = r0;
    r.t_submit = clock_s();
    std::lock_guard<std::mutex> lk(mu_);
    if (stopping_) return CLUE_ERR_STATE;
    if (r.n > be_->region_hits() || (budget_ > 0 && r.n * bytes_per_hit_ > budget_)) {
        ++stats_.rejected;
        return CLUE_ERR_ARG;
    }
    r.ticket = next_ticket_++;
    *ticket = r.ticket;
    tickets_[r.ticket] = Ticket{};
    if (stats_.first_submit < 0) stats_.first_submit = r.t_submit;
    waiting_.push_back(r);
    cv_.notify_one();
    return CLUE_OK;
}

int Scheduler::wait(int64_t ticket, double timeout_s, int *status, double *latency_ms) {
    std::unique_lock<std::mutex> lk(mu_);
    auto it = tickets_.find(ticket);
    if (it == tickets_.end()) return CLUE_ERR_ARG;
    auto ready = [&] { return tickets_[ticket].done; };
    if (timeout_s < 0) {
        done_cv_.wait(lk, ready);
    } else if (!done_cv_.wait_for(lk, std::chrono::duration<double>(timeout_s), ready)) {
        return CLUE_ERR_TIMEOUT;
    }
    const Ticket t = tickets_[ticket];
    tickets_.erase(ticket);
    if (latency_ms) *latency_ms = t.latency_ms;
    if (status) *status = t.status;
    return CLUE_OK;
}

void Scheduler::batch_done(int64_t batch, int status) {
    std::lock_guard<std::mutex> lk(mu_);
    batch_done_locked(batch, status);
}

void Scheduler::batch_done_locked(int64_t batch, int status) {
    Done &d = batches_[batch];
    d.done = true;
    d.status = status;
    d.t = clock_s();
    cv_.notify_one();
}

void Scheduler::stop() {
    {
        std::lock_guard<std::mutex> lk(mu_);
        if (stopped_) return;
        stopping_ = true;
        cv_.notify_one();
    }
    if (worker_.joinable()) worker_.join();
    std::lock_guard<std::mutex> lk(mu_);
    stopped_ = true;
}

Stats Scheduler::stats() {
    std::lock_guard<std::mutex> lk(mu_);
    return stats_;
}

void Scheduler::reset_stats() {
    std::lock_guard<std::mutex> lk(mu_);
    stats_ = Stats{};
}

Scheduler::Region *Scheduler::filling_locked() {
    for (auto &r : regions_)
        if (r.state == 1) return &r;
    for (auto &r : regions_)
        if (r.state == 0) {
            r.state = 1;
            r.reqs.clear();
            r.offsets.assign(1, 0);
            r.hits = 0;
            return &r;
        }
    return nullptr;
}

// Resolve the oldest running batches that are done, in launch order (batches
// run in order on the device, so a later one is never done first).
bool Scheduler::complete_locked() {
    bool any = false;
    while (!running_.empty()) {
        Region &r = regions_[running_.front()];
        auto it = batches_.find(r.batch);
        if (it == batches_.end() || !it->second.done) break;
        const Done d = it->second;
        batches_.erase(it);
        for (const Request &q : r.reqs) {
            Ticket &t = tickets_[q.ticket];
            t.done = true;
            t.status = d.status;
            t.latency_ms = (d.t - q.t_submit) * 1e3;
            stats_.latency_ms.push_back(t.latency_ms);
            ++stats_.events;
            stats_.hits += q.n;
            used_ -= q.n * bytes_per_hit_;
        }
        stats_.last_done = d.t;
        r.state = 0;
        r.reqs.clear();
        running_.pop_front();
        any = true;
    }
    if (any) done_cv_.notify_all();
    return any;
}

// A filling region whose staging failed: its requests fail now.
void Scheduler::fail_locked(Region &r, int status) {
    const double t = clock_s();
    for (const Request &q : r.reqs) {
        Ticket &tk = tickets_[q.ticket];
        tk.done = true;
        tk.status = status;
        tk.latency_ms = (t - q.t_submit) * 1e3;
        used_ -= q.n * bytes_per_hit_;
    }
    r.state = 0;
    r.reqs.clear();
    done_cv_.notify_all();
}

// Admission and launch decide under the lock, then call the backend with the
// lock released (a backend call may wait on the device, whose completion
// callbacks take the lock); only the worker changes regions, so its decisions
// stay valid meanwhile.
bool Scheduler::admit_locked(std::unique_lock<std::mutex> &lk) {
    bool any = false;
    while (!waiting_.empty()) {
        Region *r = filling_locked();
        if (!r) break;
        const Request q = waiting_.front();
        if (r->hits + q.n > be_->region_hits() || (int)r->reqs.size() >= max_events_) break;
        if (budget_ > 0 && used_ + q.n * bytes_per_hit_ > budget_) break;  // wait for completions
        waiting_.pop_front();
        used_ += q.n * bytes_per_hit_;
        const int64_t at = r->hits;
        r->reqs.push_back(q);
        r->hits += q.n;
        r->offsets.push_back(r->hits);
        any = true;
        if (q.n > 0) {
            lk.unlock();
            const int rc = be_->stage(r->idx, at, q);
            lk.lock();
            if (rc != CLUE_OK) {  // a failed copy fails the region's batch
                fail_locked(*r, rc);
                break;
            }
        }
    }
    return any;
}

bool Scheduler::launch_locked(std::unique_lock<std::mutex> &lk) {
    Region *r = nullptr;
    for (auto &g : regions_)
        if (g.state == 1 && !g.reqs.empty()) r = &g;
    if (!r || (int)running_.size() >= max_inflight_) return false;
    const int64_t batch = next_batch_++;
    r->batch = batch;
    r->state = 2;
    batches_[batch] = Done{};
    running_.push_back(r->idx);
    ++stats_.batches;
    stats_.batch_events.push_back((int32_t)r->reqs.size());
    lk.unlock();
    const int rc = be_->launch(r->idx, r->offsets, r->reqs, batch);
    lk.lock();
    if (rc != CLUE_OK) batch_done_locked(batch, rc);  // completes, failed, in launch order
    return true;
}

void Scheduler::loop() {
    std::unique_lock<std::mutex> lk(mu_);
    for (;;) {
        bool busy = complete_locked();
        busy |= admit_locked(lk);
        busy |= launch_locked(lk);
        const bool idle = waiting_.empty() && running_.empty() &&
                          std::none_of(regions_.begin(), regions_.end(),
                                       [](const Region &r) { return !r.reqs.empty(); });
        if (stopping_ && idle) break;
        if (!busy) cv_.wait(lk);
    }
}

}  // namespace clue_serve
