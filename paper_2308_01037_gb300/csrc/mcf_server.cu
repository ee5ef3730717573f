// Request serving with continuous batching.
//
// A scheduler thread keeps a FIFO of submitted requests.  Whenever a worker
// stream is free it forms a batch from the head of the queue, admitting
// requests while the device footprint of everything in flight stays within
// the configured budget, and hands the batch to that worker.  Each worker
// plans and runs its batch (mcf_batch_create / mcf_batch_run) on its own
// stream, so batches formed from later arrivals execute on the device while
// earlier ones are still running; when a batch completes its memory is
// released and its requests' tickets are signalled.  Graphs stay resident in
// the library's graph objects between requests.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "mcf_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t ticket = 0;
    mcf_query q{};
    std::vector<double> coeffs;
    int64_t bytes = 0;
    Clock::time_point t_submit, t_done;
    int state = 0;  // 0 queued, 1 running, 2 done
    mcf_status status = MCF_OK;
};

struct Worker {
    cudaStream_t stream = nullptr;
    std::vector<Request*> job;
    bool busy = false;
    std::condition_variable cv;
    std::thread thread;
};

// Device memory a request's batch may take (mcf_query_footprint); -1 for a
// query the batch planner would refuse.
int64_t footprint(const mcf_query& q) {
    size_t b = 0;
    return mcf_query_footprint(&q, &b) == MCF_OK ? (int64_t)b : -1;
}

}  // namespace

struct mcf_server {
    mcf_server_config cfg{};
    int device = 0;
    std::mutex mu;
    std::condition_variable cv_sched, cv_done;
    std::deque<Request*> queue;
    std::unordered_map<uint64_t, Request*> all;
    uint64_t next_ticket = 1;
    int64_t inflight_bytes = 0;
    bool stopping = false;
    std::thread scheduler;
    std::vector<Worker*> workers;
    std::vector<double> latencies;
    // global-timer windows (ns) of the completed batches' device work
    std::vector<std::pair<uint64_t, uint64_t>> windows;
    int64_t submitted = 0, completed = 0, rejected = 0, batches = 0, steps = 0, cancelled = 0;
    double plan_s = 0.0, run_s = 0.0;
    // the walk kernels' L2 fetch granularity, held for the server's life so
    // that concurrent batches do not switch the context-wide setting back and forth
    mcf::ScopedL2Fetch* fetch = nullptr;
    bool any_submit = false;
    Clock::time_point t_first, t_last;
};

using mcf::fail;
using mcf::set_error;

static void worker_loop(mcf_server* s, Worker* w) {
    cudaSetDevice(s->device);
    for (;;) {
        std::vector<Request*> job;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            w->cv.wait(lk, [&] { return !w->job.empty() || (s->stopping && !w->busy); });
            if (w->job.empty()) return;
            job = w->job;
        }
        std::vector<mcf_query> qs;
        qs.reserve(job.size());
        for (Request* r : job) qs.push_back(r->q);
        mcf_batch_t b = nullptr;
        mcf_stats st{};
        const auto t_plan = Clock::now();
        mcf_status rc = mcf_batch_create(qs.data(), (int32_t)qs.size(), 0, w->stream, &b);
        const auto t_run = Clock::now();
        if (rc == MCF_OK) rc = mcf_batch_run(b, w->stream, &st);
        const auto t_end = Clock::now();
        uint64_t t0 = 0, t1 = 0;
        std::vector<mcf_status> qs_status(job.size(), rc);
        if (rc == MCF_OK || rc == MCF_ERR_ACCURACY_BUDGET) {
            mcf::batch_window(b, &t0, &t1);
            for (size_t i = 0; i < job.size(); ++i) qs_status[i] = mcf::batch_query_status(b, (int)i);
        }
        mcf_batch_destroy(b);
        const auto now = Clock::now();
        {
            std::lock_guard<std::mutex> lk(s->mu);
            for (size_t i = 0; i < job.size(); ++i) {
                Request* r = job[i];
                r->state = 2;
                r->status = qs_status[i];
                r->t_done = now;
                s->inflight_bytes -= r->bytes;
                s->latencies.push_back(std::chrono::duration<double, std::milli>(now - r->t_submit).count());
                ++s->completed;
            }
            s->steps += st.walk_steps;
            s->plan_s += std::chrono::duration<double>(t_run - t_plan).count();
            s->run_s += std::chrono::duration<double>(t_end - t_run).count();
            if (t1 > t0) s->windows.push_back({t0, t1});
            ++s->batches;
            s->t_last = now;
            w->job.clear();
            w->busy = false;
        }
        s->cv_done.notify_all();
        s->cv_sched.notify_all();
    }
}

static void scheduler_loop(mcf_server* s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        s->cv_sched.wait(lk, [&] {
            if (s->stopping && s->queue.empty()) return true;
            if (s->queue.empty()) return false;
            for (Worker* w : s->workers)
                if (!w->busy) return true;
            return false;
        });
        if (s->queue.empty() && s->stopping) break;
        if (s->cfg.batch_window_ms > 0 && (int)s->queue.size() < s->cfg.max_batch && !s->stopping) {
            const auto until = Clock::now() + std::chrono::microseconds((int64_t)(s->cfg.batch_window_ms * 1000));
            s->cv_sched.wait_until(lk, until, [&] { return (int)s->queue.size() >= s->cfg.max_batch || s->stopping; });
        }
        Worker* free_w = nullptr;
        for (Worker* w : s->workers)
            if (!w->busy) {
                free_w = w;
                break;
            }
        if (!free_w || s->queue.empty()) continue;
        std::vector<Request*> job;
        while (!s->queue.empty() && (int)job.size() < s->cfg.max_batch) {
            Request* r = s->queue.front();
            if (s->inflight_bytes + r->bytes > (int64_t)s->cfg.hbm_budget_bytes && !(job.empty() && s->inflight_bytes == 0))
                break;   // admitted once memory frees up (a lone request always fits: its size was checked)
            s->queue.pop_front();
            s->inflight_bytes += r->bytes;
            r->state = 1;
            job.push_back(r);
        }
        if (job.empty()) {
            // the head does not fit beside the running batches: wait for a completion
            s->cv_done.wait(lk);
            continue;
        }
        free_w->job = job;
        free_w->busy = true;
        free_w->cv.notify_one();
    }
}

extern "C" {

mcf_status mcf_server_create(const mcf_server_config* config, mcf_server_t* out) {
    set_error("");
    if (!config || !out) return fail(MCF_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    if (config->hbm_budget_bytes == 0 || config->max_inflight < 1 || config->max_batch < 1)
        return fail(MCF_ERR_INVALID_ARG, "hbm_budget_bytes must be > 0, max_inflight and max_batch >= 1");
    mcf_server* s = new (std::nothrow) mcf_server();
    if (!s) return fail(MCF_ERR_OOM, "host allocation failed");
    s->cfg = *config;
    cudaGetDevice(&s->device);
    s->fetch = new mcf::ScopedL2Fetch(mcf::L2_FETCH_BYTES);
    for (int i = 0; i < config->max_inflight; ++i) {
        Worker* w = new Worker();
        if (cudaStreamCreateWithFlags(&w->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete w;
            mcf_server_destroy(s);
            return fail(MCF_ERR_CUDA, "stream creation failed");
        }
        s->workers.push_back(w);
    }
    for (Worker* w : s->workers) w->thread = std::thread(worker_loop, s, w);
    s->scheduler = std::thread(scheduler_loop, s);
    *out = s;
    return MCF_OK;
}

mcf_status mcf_server_submit(mcf_server_t s, const mcf_query* query, uint64_t* ticket) {
    set_error("");
    if (!s || !query || !ticket) return fail(MCF_ERR_INVALID_ARG, "NULL argument");
    if (!query->graph || !query->out) return fail(MCF_ERR_INVALID_ARG, "query graph or out is NULL");
    Request* r = new (std::nothrow) Request();
    if (!r) return fail(MCF_ERR_OOM, "host allocation failed");
    r->q = *query;
    if (query->kind != MCF_QUERY_KATZ) {
        if (!query->params.coeffs || query->params.n_coeffs < 1 || query->params.n_coeffs > MCF_MAX_COEFFS) {
            delete r;
            return fail(MCF_ERR_INVALID_ARG, "coeffs must hold 1.." + std::to_string(MCF_MAX_COEFFS) + " values");
        }
        r->coeffs.assign(query->params.coeffs, query->params.coeffs + query->params.n_coeffs);
        r->q.params.coeffs = r->coeffs.data();
    }
    r->bytes = footprint(r->q);
    if (r->bytes < 0) {
        const std::string why = mcf_last_error();
        delete r;
        return fail(MCF_ERR_INVALID_ARG, "request refused: " + why);
    }
    r->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        r->ticket = s->next_ticket++;
        s->all[r->ticket] = r;
        ++s->submitted;
        if (!s->any_submit) {
            s->any_submit = true;
            s->t_first = r->t_submit;
        }
        if (r->bytes > (int64_t)s->cfg.hbm_budget_bytes) {
            r->state = 2;
            r->status = MCF_ERR_ADMISSION;
            r->t_done = r->t_submit;
            ++s->rejected;
        } else {
            s->queue.push_back(r);
        }
        *ticket = r->ticket;
    }
    s->cv_sched.notify_all();
    s->cv_done.notify_all();
    return MCF_OK;
}

mcf_status mcf_server_poll(mcf_server_t s, uint64_t ticket, int32_t* done, mcf_status* result) {
    if (!s || !done) return fail(MCF_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) return fail(MCF_ERR_INVALID_ARG, "unknown ticket");
    *done = it->second->state == 2;
    if (result) *result = it->second->status;
    return MCF_OK;
}

mcf_status mcf_server_wait(mcf_server_t s, uint64_t ticket, double timeout_s, mcf_status* result,
                           double* latency_ms) {
    if (!s) return fail(MCF_ERR_INVALID_ARG, "server is NULL");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) return fail(MCF_ERR_INVALID_ARG, "unknown ticket");
    Request* r = it->second;
    auto ready = [&] { return r->state == 2; };
    if (timeout_s < 0) s->cv_done.wait(lk, ready);
    else if (!s->cv_done.wait_for(lk, std::chrono::microseconds((int64_t)(timeout_s * 1e6)), ready))
        return fail(MCF_ERR_TIMEOUT, "request still running");
    if (result) *result = r->status;
    if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
    return MCF_OK;
}

mcf_status mcf_server_get_stats(mcf_server_t s, mcf_server_stats* out) {
    if (!s || !out) return fail(MCF_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    *out = mcf_server_stats{};
    out->submitted = s->submitted;
    out->completed = s->completed;
    out->cancelled = s->cancelled;
    out->rejected = s->rejected;
    out->batches = s->batches;
    out->walk_steps = s->steps;
    std::vector<double> l = s->latencies;
    if (!l.empty()) {
        std::sort(l.begin(), l.end());
        auto pct = [&](double p) {
            const double x = p * (double)(l.size() - 1);
            const size_t i = (size_t)x;
            const double f = x - (double)i;
            return i + 1 < l.size() ? l[i] * (1 - f) + l[i + 1] * f : l[i];
        };
        out->p50_ms = pct(0.50);
        out->p99_ms = pct(0.99);
        out->max_ms = l.back();
        double sum = 0;
        for (double x : l) sum += x;
        out->mean_ms = sum / (double)l.size();
    }
    if (s->any_submit && s->completed > 0) out->busy_s = std::chrono::duration<double>(s->t_last - s->t_first).count();
    // sweep over the batches' device windows: time with two or more batches'
    // work on the device, and the largest number at once
    std::vector<std::pair<uint64_t, int>> ev;
    ev.reserve(2 * s->windows.size());
    for (const auto& w : s->windows) {
        ev.push_back({w.first, 1});
        ev.push_back({w.second, -1});
    }
    std::sort(ev.begin(), ev.end(), [](const std::pair<uint64_t, int>& a, const std::pair<uint64_t, int>& b) {
        return a.first != b.first ? a.first < b.first : a.second < b.second;   // ends before starts at a tie
    });
    int live = 0, most = 0;
    uint64_t prev = 0, overlap_ns = 0;
    for (const auto& e : ev) {
        if (live >= 2) overlap_ns += e.first - prev;
        live += e.second;
        most = std::max(most, live);
        prev = e.first;
    }
    out->device_overlap_ms = (double)overlap_ns * 1e-6;
    out->max_concurrent_batches = most;
    out->plan_s = s->plan_s;
    out->run_s = s->run_s;
    return MCF_OK;
}

mcf_status mcf_server_cancel(mcf_server_t s, uint64_t ticket) {
    set_error("");
    if (!s) return fail(MCF_ERR_INVALID_ARG, "server is NULL");
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->all.find(ticket);
        if (it == s->all.end()) return fail(MCF_ERR_INVALID_ARG, "unknown ticket");
        Request* r = it->second;
        if (r->state != 0) return fail(MCF_ERR_INVALID_ARG, "the request is not queued (running or done)");
        auto q = std::find(s->queue.begin(), s->queue.end(), r);
        if (q == s->queue.end()) return fail(MCF_ERR_INVALID_ARG, "the request is not queued");
        s->queue.erase(q);
        r->state = 2;
        r->status = MCF_ERR_CANCELLED;
        r->t_done = Clock::now();
        ++s->cancelled;
        ++s->completed;
    }
    s->cv_done.notify_all();
    s->cv_sched.notify_all();
    return MCF_OK;
}

mcf_status mcf_server_release(mcf_server_t s, uint64_t ticket) {
    set_error("");
    if (!s) return fail(MCF_ERR_INVALID_ARG, "server is NULL");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) return fail(MCF_ERR_INVALID_ARG, "unknown ticket");
    if (it->second->state != 2) return fail(MCF_ERR_INVALID_ARG, "the request has not completed");
    delete it->second;
    s->all.erase(it);
    return MCF_OK;
}

mcf_status mcf_server_destroy(mcf_server_t s) {
    if (!s) return MCF_OK;
    {
        std::unique_lock<std::mutex> lk(s->mu);
        s->stopping = true;
    }
    s->cv_sched.notify_all();
    if (s->scheduler.joinable()) s->scheduler.join();
    {
        // let the workers finish their jobs, then stop them
        std::unique_lock<std::mutex> lk(s->mu);
        s->cv_done.wait(lk, [&] {
            for (Worker* w : s->workers)
                if (w->busy) return false;
            return true;
        });
    }
    for (Worker* w : s->workers) w->cv.notify_all();
    for (Worker* w : s->workers) {
        if (w->thread.joinable()) w->thread.join();
        if (w->stream) cudaStreamDestroy(w->stream);
        delete w;
    }
    for (auto& kv : s->all) delete kv.second;
    delete s->fetch;
    delete s;
    return MCF_OK;
}

}  // extern "C"
