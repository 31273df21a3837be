// Serving loop over several pipelines on one GPU with admission by device
// memory (Sec. 5.1: a query starts only when the memory it needs is free; the
// queries of different services share the GPU, Sec. 4.2).
//
// Callers queue queries per pipeline into pinned host queues (camelot_server_submit);
// one server thread admits them in FIFO order per pipeline, round robin over
// pipelines, as long as the query bytes in flight on the device stay within the
// budget and the pipeline's rings have room (camelot_submit copies them into the
// pipeline's device data ring), and moves completions into per-pipeline output
// queues (camelot_server_poll).  Batching stays on the device: each pipeline's
// trigger batches whatever has been admitted.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <vector>

#include "../../include/camelot.h"

camelot_status camelot_internal_fail(camelot_status st, const char* msg);
size_t camelot_internal_query_bytes(const camelot_pipeline* p);

namespace {

struct Lane {
    camelot_pipeline* p = nullptr;
    size_t row = 0;                 // query bytes
    uint32_t cap = 0;               // host queue capacity (queries)
    char* data = nullptr;           // pinned [cap][row]
    std::vector<int64_t> arrival;   // [cap]
    std::vector<uint32_t> stream;   // [cap]
    std::mutex mu;                  // producers, and head/tail updates
    uint64_t head = 0, tail = 0;    // queue positions: [head, tail) waiting
    std::mutex out_mu;
    std::condition_variable out_cv;
    std::deque<camelot_completion> done;
    // statistics (server thread writes, readers take out_mu)
    uint64_t submitted = 0, admitted = 0, completed = 0, deferred = 0;
    uint64_t inflight_bytes = 0, peak_inflight_bytes = 0;
    camelot_status failed = CAMELOT_OK;
};

}  // namespace

struct camelot_server {
    std::vector<Lane*> lanes;
    uint64_t budget = 0;            // bytes; 0 = no limit
    uint32_t max_admit = 64;        // queries per pipeline per round
    std::thread thr;
    std::atomic<bool> stop{false};
    std::atomic<uint64_t> inflight{0};
};

static void server_free(camelot_server* s) {
    for (Lane* l : s->lanes) {
        if (l->data) cudaFreeHost(l->data);
        delete l;
    }
    delete s;
}

// One admission pass over lane l: the waiting queries at the head, in runs of
// one stream id that do not wrap the host queue, while the budget allows.
static bool admit(camelot_server* s, Lane& l) {
    uint64_t head, tail;
    {
        std::lock_guard<std::mutex> g(l.mu);
        head = l.head;
        tail = l.tail;
    }
    if (head == tail || l.failed != CAMELOT_OK) return false;
    uint32_t k = (uint32_t)std::min<uint64_t>(tail - head, s->max_admit);
    k = (uint32_t)std::min<uint64_t>(k, l.cap - head % l.cap);              // no wrap in one call
    const uint32_t sid = l.stream[head % l.cap];
    uint32_t run = 1;
    while (run < k && l.stream[(head + run) % l.cap] == sid) ++run;
    k = run;
    if (s->budget) {
        const uint64_t room = s->budget > s->inflight.load() ? s->budget - s->inflight.load() : 0;
        const uint64_t fit = room / l.row;
        if (fit == 0) {
            ++l.deferred;
            return false;
        }
        k = (uint32_t)std::min<uint64_t>(k, fit);
    }
    const uint64_t pos = head % l.cap;
    uint64_t first = 0;
    const camelot_status st = camelot_submit(l.p, sid, l.data + pos * l.row, k, l.arrival.data() + pos, &first);
    if (st == CAMELOT_EAGAIN) {     // the pipeline's rings are full: poll first
        ++l.deferred;
        return false;
    }
    if (st != CAMELOT_OK) {
        std::lock_guard<std::mutex> g(l.out_mu);
        l.failed = st;
        l.out_cv.notify_all();
        return false;
    }
    {
        std::lock_guard<std::mutex> g(l.mu);
        l.head = head + k;
    }
    const uint64_t bytes = (uint64_t)k * l.row;
    const uint64_t now = s->inflight.fetch_add(bytes) + bytes;
    std::lock_guard<std::mutex> g(l.out_mu);
    l.admitted += k;
    l.inflight_bytes += bytes;
    l.peak_inflight_bytes = std::max(l.peak_inflight_bytes, l.inflight_bytes);
    (void)now;
    return true;
}

static bool collect(camelot_server* s, Lane& l) {
    camelot_completion buf[256];
    uint32_t n = 0;
    const camelot_status st = camelot_poll(l.p, buf, 256, &n, 0);
    if (st != CAMELOT_OK && st != CAMELOT_ETIMEDOUT) {
        std::lock_guard<std::mutex> g(l.out_mu);
        l.failed = st;
        l.out_cv.notify_all();
        return false;
    }
    if (n == 0) return false;
    const uint64_t bytes = (uint64_t)n * l.row;
    s->inflight.fetch_sub(bytes);
    std::lock_guard<std::mutex> g(l.out_mu);
    l.done.insert(l.done.end(), buf, buf + n);
    l.completed += n;
    l.inflight_bytes -= bytes;
    l.out_cv.notify_all();
    return true;
}

static void server_main(camelot_server* s) {
    int idle = 0;
    while (!s->stop.load(std::memory_order_acquire)) {
        bool work = false;
        for (Lane* l : s->lanes) work |= collect(s, *l);
        for (Lane* l : s->lanes) work |= admit(s, *l);
        if (work) {
            idle = 0;
        } else if (++idle > 2000) {
            std::this_thread::sleep_for(std::chrono::microseconds(20));
        } else {
            std::this_thread::yield();
        }
    }
}

extern "C" void camelot_server_options_default(camelot_server_options* o) {
    if (!o) return;
    o->device_bytes_budget = 0;
    o->host_queue_queries = 4096;
    o->max_admit = 64;
}

extern "C" camelot_status camelot_server_create(camelot_pipeline* const* pipelines, int n,
                                                const camelot_server_options* opts, camelot_server** out) {
    if (!pipelines || !out || n < 1 || n > CAMELOT_MAX_SERVER_PIPELINES)
        return camelot_internal_fail(CAMELOT_EINVAL, "need 1..16 pipelines and an output pointer");
    camelot_server_options o;
    camelot_server_options_default(&o);
    if (opts) o = *opts;
    if (o.host_queue_queries < 1 || o.max_admit < 1)
        return camelot_internal_fail(CAMELOT_EINVAL, "host_queue_queries and max_admit must be >= 1");
    auto* s = new camelot_server();
    s->budget = o.device_bytes_budget;
    s->max_admit = o.max_admit;
    for (int i = 0; i < n; ++i) {
        if (!pipelines[i]) {
            server_free(s);
            return camelot_internal_fail(CAMELOT_EINVAL, "null pipeline");
        }
        auto* l = new Lane();
        s->lanes.push_back(l);
        l->p = pipelines[i];
        l->row = camelot_internal_query_bytes(pipelines[i]);
        l->cap = o.host_queue_queries;
        if (s->budget && s->budget < l->row) {
            server_free(s);
            return camelot_internal_fail(CAMELOT_EINVAL, "the budget is smaller than one query");
        }
        if (cudaHostAlloc((void**)&l->data, (size_t)l->cap * l->row, cudaHostAllocPortable) != cudaSuccess) {
            server_free(s);
            return camelot_internal_fail(CAMELOT_ENOMEM, "host queue allocation failed");
        }
        l->arrival.resize(l->cap);
        l->stream.resize(l->cap);
    }
    s->thr = std::thread(server_main, s);
    *out = s;
    return CAMELOT_OK;
}

extern "C" camelot_status camelot_server_submit(camelot_server* s, int pipeline, uint32_t stream_id,
                                                const void* queries, uint32_t n, const int64_t* arrival_ns) {
    if (!s || pipeline < 0 || pipeline >= (int)s->lanes.size() || (n && !queries))
        return camelot_internal_fail(CAMELOT_EINVAL, "bad argument");
    Lane& l = *s->lanes[pipeline];
    if (l.failed != CAMELOT_OK) return camelot_internal_fail(CAMELOT_ESTATE, "the pipeline failed");
    std::lock_guard<std::mutex> g(l.mu);
    if (l.tail + n - l.head > l.cap) return camelot_internal_fail(CAMELOT_EAGAIN, "host queue full");
    struct timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    const int64_t now = (int64_t)ts.tv_sec * 1000000000ll + ts.tv_nsec;
    for (uint32_t i = 0; i < n; ++i) {
        const uint64_t pos = (l.tail + i) % l.cap;
        memcpy(l.data + pos * l.row, (const char*)queries + (size_t)i * l.row, l.row);
        l.arrival[pos] = arrival_ns ? arrival_ns[i] : now;
        l.stream[pos] = stream_id;
    }
    l.tail += n;
    l.submitted += n;
    return CAMELOT_OK;
}

extern "C" camelot_status camelot_server_poll(camelot_server* s, int pipeline, camelot_completion* out,
                                              uint32_t max, uint32_t* n_out, int64_t timeout_us) {
    if (!s || pipeline < 0 || pipeline >= (int)s->lanes.size() || !n_out || (max && !out))
        return camelot_internal_fail(CAMELOT_EINVAL, "bad argument");
    Lane& l = *s->lanes[pipeline];
    *n_out = 0;
    std::unique_lock<std::mutex> g(l.out_mu);
    if (l.done.empty() && timeout_us != 0 && l.failed == CAMELOT_OK) {
        auto ready = [&] { return !l.done.empty() || l.failed != CAMELOT_OK; };
        if (timeout_us < 0) l.out_cv.wait(g, ready);
        else l.out_cv.wait_for(g, std::chrono::microseconds(timeout_us), ready);
    }
    const uint32_t k = (uint32_t)std::min<size_t>(max, l.done.size());
    for (uint32_t i = 0; i < k; ++i) {
        out[i] = l.done.front();
        l.done.pop_front();
    }
    *n_out = k;
    if (k == 0 && l.failed != CAMELOT_OK) return camelot_internal_fail(CAMELOT_ESTATE, "the pipeline failed");
    if (k == 0 && timeout_us > 0) return camelot_internal_fail(CAMELOT_ETIMEDOUT, "no completion in time");
    return CAMELOT_OK;
}

extern "C" camelot_status camelot_server_stats(camelot_server* s, int pipeline, camelot_lane_stats* out) {
    if (!s || pipeline < 0 || pipeline >= (int)s->lanes.size() || !out)
        return camelot_internal_fail(CAMELOT_EINVAL, "bad argument");
    Lane& l = *s->lanes[pipeline];
    uint64_t waiting;
    {
        std::lock_guard<std::mutex> g(l.mu);
        waiting = l.tail - l.head;
        out->submitted = l.submitted;
    }
    std::lock_guard<std::mutex> g(l.out_mu);
    out->admitted = l.admitted;
    out->completed = l.completed;
    out->waiting = waiting;
    out->deferred = l.deferred;
    out->inflight_bytes = l.inflight_bytes;
    out->peak_inflight_bytes = l.peak_inflight_bytes;
    out->total_inflight_bytes = s->inflight.load();
    out->status = l.failed;
    return CAMELOT_OK;
}

extern "C" camelot_status camelot_server_destroy(camelot_server* s) {
    if (!s) return camelot_internal_fail(CAMELOT_EINVAL, "null server");
    s->stop.store(true, std::memory_order_release);
    if (s->thr.joinable()) s->thr.join();
    server_free(s);
    return CAMELOT_OK;
}
