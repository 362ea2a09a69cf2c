// Continuous-batching scheduler for CLUE events (host code, no CUDA).
//
// Requests (one event each: host input arrays and host output arrays) arrive
// from any thread.  One worker thread:
//
//  * admits waiting requests, oldest first, into the region being filled while
//    the region has room (hits and events) and the memory budget covers the
//    request; otherwise the request waits (back-pressure).  An admitted
//    request's inputs are staged into the region at once (the backend queues
//    the copies), so copies overlap the batches running on the device;
//  * launches the filled region as one batch as soon as fewer than
//    max_inflight batches are queued on the device (all sizes mixed in one
//    batch), then fills the next free region;
//  * completes batches in launch order when the backend reports them done
//    (Scheduler::batch_done, callable from any thread, e.g. a device-stream
//    callback): each request of the batch is resolved, its budget released
//    and its waiters woken.
//
// The worker sleeps on a condition variable between these events: it is
// woken by a submission, a completion or a stop, never by a timer.  Each
// event's result is the event's alone (the backend clusters every event of a
// batch independently), so batching changes when a result arrives, never
// what it is.  The device work goes through a Backend, so the scheduling can
// run against a fake backend on a machine without a GPU.
#pragma once

#include <condition_variable>
#include <cstdint>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

namespace clue_serve {

struct Request {
    int64_t ticket = 0;
    int64_t n = 0;              // hits
    const void *in[4] = {};     // x, y, layer, energy (host)
    void *out[2] = {};          // cluster_id, is_seed (host)
    double t_submit = 0.0;      // seconds on the scheduler's clock
};

// What the device side does.  stage() and launch() are called by the
// scheduler's worker thread only, in the order regions are filled and
// launched.  launch() queues the batch and its results' copies back into the
// requests' output arrays, and arranges for Scheduler::batch_done(batch,
// status) to be called once those copies are complete.
class Backend {
  public:
    virtual ~Backend() = default;
    virtual int64_t region_hits() const = 0;
    virtual int n_regions() const = 0;
    // queue the copy of r's inputs into `region` at hit offset `offset`
    virtual int stage(int region, int64_t offset, const Request &r) = 0;
    // queue the batch of `reqs` (offsets[k], offsets[k + 1]) in `region`
    virtual int launch(int region, const std::vector<int64_t> &offsets,
                       const std::vector<Request> &reqs, int64_t batch) = 0;
};

struct Stats {
    int64_t events = 0, hits = 0, batches = 0, rejected = 0;
    double first_submit = -1.0, last_done = -1.0;  // seconds, scheduler's clock
    std::vector<double> latency_ms;                // per completed event
    std::vector<int32_t> batch_events;             // events per launched batch
};

class Scheduler {
  public:
    // bytes_per_hit: device bytes an admitted hit holds against the budget
    // (budget_bytes <= 0: no budget).  max_inflight: batches queued on the
    // device at once, at most n_regions - 1 (one region keeps filling).
    Scheduler(Backend *be, int max_events_per_batch, int max_inflight, int64_t budget_bytes,
              int64_t bytes_per_hit);
    ~Scheduler();  // stop(): every admitted and waiting request is completed first

    // Queue a request; CLUE_OK with *ticket set, CLUE_ERR_ARG for an event
    // larger than a region or the budget (nothing queued), CLUE_ERR_STATE
    // after stop().
    int submit(const Request &r, int64_t *ticket);
    // Wait until the ticket's event is done (timeout_s < 0: no limit): then
    // CLUE_OK, with the event's outcome (CLUE_OK or its batch's error) in
    // *status and its latency, and the ticket is released.  CLUE_ERR_TIMEOUT
    // if not done in time (the ticket stays), CLUE_ERR_ARG for an unknown
    // ticket.
    int wait(int64_t ticket, double timeout_s, int *status, double *latency_ms);
    // The backend's report that batch `batch` (and its result copies) ended.
    void batch_done(int64_t batch, int status);
    // Finish everything queued and stop the worker (idempotent).
    void stop();
    Stats stats();
    void reset_stats();  // counters and latencies start again from zero
    double now() const;

  private:
    struct Region {
        int idx = 0;
        int state = 0;  // 0 free, 1 filling, 2 running
        std::vector<Request> reqs;
        std::vector<int64_t> offsets{0};
        int64_t hits = 0, batch = -1;
    };
    struct Ticket {
        bool done = false;
        int status = 0;
        double latency_ms = 0.0;
    };
    struct Done {
        bool done = false;
        int status = 0;
        double t = 0.0;
    };
    void loop();
    bool complete_locked();
    bool admit_locked(std::unique_lock<std::mutex> &lk);
    bool launch_locked(std::unique_lock<std::mutex> &lk);
    void batch_done_locked(int64_t batch, int status);
    void fail_locked(Region &r, int status);
    Region *filling_locked();

    Backend *be_;
    int max_events_, max_inflight_;
    int64_t budget_, bytes_per_hit_, used_ = 0;
    std::mutex mu_;
    std::condition_variable cv_, done_cv_;
    std::deque<Request> waiting_;
    std::vector<Region> regions_;
    std::unordered_map<int64_t, Ticket> tickets_;
    std::unordered_map<int64_t, Done> batches_;  // launched, not yet completed
    std::deque<int> running_;                    // regions in launch order
    int64_t next_ticket_ = 1, next_batch_ = 0;
    bool stopping_ = false, stopped_ = false;
    Stats stats_;
    std::thread worker_;
};

}  // namespace clue_serve
