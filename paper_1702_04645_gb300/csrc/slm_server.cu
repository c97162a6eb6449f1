// slm_server.cu -- request server around slm_run (slm_server.h).
//
// Slots are host threads, each with its own non-blocking CUDA stream.  A
// slot takes the oldest queued request once its footprint fits in what is
// left of the HBM budget, runs it to completion on its stream (create, run,
// final partition and modularity copied to host memory, destroy) and gives
// the footprint back.  The device work of the slots overlaps: while one slot
// waits for the few counters its host driver reads each sweep, the others
// keep the GPU busy.  The device memory each run really holds is measured by
// an accountant that counts the library's buffers allocated on that thread.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "slm_internal.cuh"
#include "slm_server.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t ticket = 0;
    int32_t n = 0;
    long long nnz = 0;
    std::vector<int32_t> rp, col, w;  // host copies; w empty = unit weights
    bool directed = false;            // W as out-arcs (slm_create_graph_directed)
    slm_options opt{};
    uint64_t footprint = 0;
    int32_t state = SLM_REQ_QUEUED;
    slm_status status = SLM_OK;
    std::string err;
    int32_t slot = -1;
    double t_submit = 0, t_admit = 0, t_done = 0;
    std::vector<int32_t> labels;
    int32_t K = 0, levels = 0;
    double q = 0;
    long long edges = 0;
    uint64_t peak = 0;
    double deadline = 0;         // steady_seconds() by which the request must end; 0: none
    std::atomic<int> cancel{0};  // set by slm_server_cancel while the request runs
};

}  // namespace

struct slm_server {
    int dev = 0;
    uint64_t budget = 0;
    int32_t nslots = 0;
    Clock::time_point t0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    // threads inside slm_server_wait; destroy waits on cv_idle until none is left
    int32_t waiters = 0;
    std::condition_variable cv_idle;
    std::deque<Request *> queue;
    int32_t queued_deadlines = 0;  // queued requests that carry a deadline
    std::unordered_map<uint64_t, std::unique_ptr<Request>> reqs;
    uint64_t next_ticket = 1;
    uint64_t reserved = 0, max_reserved = 0;
    int32_t running = 0, max_running = 0;
    long long submitted = 0, completed = 0, failed = 0, rejected = 0;
    bool stop = false;
    std::vector<std::thread> workers;
    std::string err;

    double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
};

namespace {

thread_local std::string g_server_create_error;

// One request, start to end, on the slot's stream.  Returns the status of
// the first call that failed.
slm_status run_request(Request &r, cudaStream_t st) {
    slm_graph *g = nullptr;
    const int32_t *w = r.w.empty() ? nullptr : r.w.data();
    slm_status s = r.directed
                       ? slm_create_graph_directed(r.n, r.rp.data(), r.col.data(), w, SLM_HOST, st, &g)
                       : slm_create_graph(r.n, r.rp.data(), r.col.data(), w, SLM_HOST, st, &g);
    if (s != SLM_OK) {
        r.err = slm_last_error(nullptr);
        return s;
    }
    auto done = [&](slm_status e) {
        if (e != SLM_OK) r.err = slm_last_error(g);
        slm_destroy_graph(g);
        return e;
    };
    if ((s = slm_run(g, &r.opt, st)) != SLM_OK) return done(s);
    r.labels.assign((size_t)r.n, 0);
    if ((s = slm_get_partition(g, -1, r.labels.data(), SLM_HOST, &r.K)) != SLM_OK) return done(s);
    if ((s = slm_modularity(g, -1, &r.q)) != SLM_OK) return done(s);
    if ((s = slm_num_levels(g, &r.levels)) != SLM_OK) return done(s);
    r.edges = 0;
    for (int32_t l = -1; l < r.levels; l++) {
        slm_level_stats ls{};
        if ((s = slm_get_stats(g, l, &ls)) != SLM_OK) return done(s);
        r.edges += ls.edges_scanned;
    }
    return done(SLM_OK);
}

// End `r` (queued or just refused) as FAILED with status `st`; mu held.
void end_unrun(slm_server *sv, Request *r, slm_status st, const char *why) {
    r->state = SLM_REQ_FAILED;
    r->status = st;
    r->err = why;
    r->t_done = sv->now();
    sv->failed++;
}

// Queued requests past their deadline end FAILED (SLM_ERR_DEADLINE); mu held.
void drop_expired(slm_server *sv) {
    if (sv->queued_deadlines == 0) return;
    const double now = slm::steady_seconds();
    bool any = false;
    for (auto it = sv->queue.begin(); it != sv->queue.end();) {
        Request *r = *it;
        if (r->deadline > 0 && now > r->deadline) {
            end_unrun(sv, r, SLM_ERR_DEADLINE, "the request passed its deadline while queued");
            sv->queued_deadlines--;
            it = sv->queue.erase(it);
            any = true;
        } else {
            ++it;
        }
    }
    if (any) sv->cv_done.notify_all();
}

void worker(slm_server *sv, int32_t slot) {
    // slots wait for the device by sleeping, so that many of them can share
    // the host's cores
    slm::set_thread_blocking_sync(true);
    cudaStream_t st = nullptr;
    bool ok = cudaSetDevice(sv->dev) == cudaSuccess &&
              cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess;
    std::unique_lock<std::mutex> lk(sv->mu);
    for (;;) {
        drop_expired(sv);
        if (sv->stop) break;
        if (sv->queue.empty() || sv->queue.front()->footprint > sv->budget - sv->reserved) {
            // queued deadlines are checked at least every 10 ms
            if (sv->queued_deadlines > 0) sv->cv_work.wait_for(lk, std::chrono::milliseconds(10));
            else sv->cv_work.wait(lk);
            continue;
        }
        Request *r = sv->queue.front();
        sv->queue.pop_front();
        if (r->deadline > 0) sv->queued_deadlines--;
        sv->reserved += r->footprint;
        sv->max_reserved = std::max(sv->max_reserved, sv->reserved);
        sv->running++;
        sv->max_running = std::max(sv->max_running, sv->running);
        r->state = SLM_REQ_RUNNING;
        r->slot = slot;
        r->t_admit = sv->now();
        lk.unlock();

        slm_status s = SLM_ERR_CUDA;
        slm::MemAcct acct;
        if (ok) {
            slm::MemAcct *prev = slm::set_thread_acct(&acct);
            slm::RunControl rc;
            rc.cancel = &r->cancel;
            rc.deadline = r->deadline;
            slm::RunControl *prev_rc = slm::set_thread_run_control(&rc);
            s = run_request(*r, st);
            slm::set_thread_run_control(prev_rc);
            slm::set_thread_acct(prev);
        } else {
            r->err = "slot could not select the device or create its stream";
        }
        // the inputs are no longer needed once the run has ended
        std::vector<int32_t>().swap(r->rp);
        std::vector<int32_t>().swap(r->col);
        std::vector<int32_t>().swap(r->w);

        lk.lock();
        r->peak = (uint64_t)acct.peak;
        r->status = s;
        r->state = s == SLM_OK ? SLM_REQ_DONE : SLM_REQ_FAILED;
        r->t_done = sv->now();
        sv->reserved -= r->footprint;
        sv->running--;
        if (s == SLM_OK) sv->completed++;
        else sv->failed++;
        sv->cv_done.notify_all();
        sv->cv_work.notify_all();
    }
    lk.unlock();
    if (st) cudaStreamDestroy(st);
}

Request *find(slm_server *sv, uint64_t ticket) {
    auto it = sv->reqs.find(ticket);
    return it == sv->reqs.end() ? nullptr : it->second.get();
}

}  // namespace

extern "C" {

uint64_t slm_server_footprint(int32_t n, int64_t nnz) {
    // input CSR and the aggregated level graph (8 B per entry each), the
    // sort of aggregation (keys, values and their double buffers: 24 B per
    // entry), hub tables (at most 16 B per entry), POSITIVE's copy of its
    // members' internal entries (room for whole rows: at most 8 B per entry),
    // the scan's bucket-ordered copy of the rows (8 B per entry);
    // per node the level workspace, POSITIVE's scratch and the composed
    // labels of the levels, bounded by 512 B; plus 64 MiB for cycle pools and
    // allocation rounding
    const uint64_t N = n > 0 ? (uint64_t)n : 0, E = nnz > 0 ? (uint64_t)nnz : 0;
    return 72 * E + 512 * N + (64ull << 20);
}

const char *slm_server_last_error(const slm_server *sv) {
    return sv ? sv->err.c_str() : g_server_create_error.c_str();
}

slm_status slm_server_create(uint64_t hbm_budget_bytes, int32_t max_slots, slm_server **out) {
    if (!out) return SLM_ERR_INVALID_ARGUMENT;
    *out = nullptr;
    if (max_slots < 1 || max_slots > 64 || hbm_budget_bytes == 0) {
        g_server_create_error = "max_slots must be in [1, 64] and the budget positive";
        return SLM_ERR_INVALID_ARGUMENT;
    }
    auto sv = std::make_unique<slm_server>();
    cudaError_t e = cudaGetDevice(&sv->dev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        g_server_create_error = std::string("no CUDA device: ") + cudaGetErrorString(e);
        return SLM_ERR_CUDA;
    }
    sv->budget = hbm_budget_bytes;
    sv->nslots = max_slots;
    sv->t0 = Clock::now();
    try {
        for (int32_t k = 0; k < max_slots; k++) sv->workers.emplace_back(worker, sv.get(), k);
    } catch (const std::exception &ex) {
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            sv->stop = true;
        }
        sv->cv_work.notify_all();
        for (auto &t : sv->workers) t.join();
        g_server_create_error = std::string("could not start the slots: ") + ex.what();
        return SLM_ERR_CUDA;
    }
    *out = sv.release();
    return SLM_OK;
}

slm_status slm_server_submit(slm_server *sv, const slm_graph_desc *gd, const slm_options *opt,
                             uint64_t *ticket) {
    return slm_server_submit_deadline(sv, gd, opt, 0.0, ticket);
}

namespace {
slm_status submit_request(slm_server *sv, const slm_graph_desc *gd, const slm_options *opt,
                          double deadline_s, bool directed, uint64_t *ticket) {
    if (!sv || !gd || !ticket) return SLM_ERR_INVALID_ARGUMENT;
    *ticket = 0;
    if (!(deadline_s >= 0.0)) {  // also refuses NaN
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->err = "deadline_s must be >= 0 (0: no deadline)";
        return SLM_ERR_INVALID_ARGUMENT;
    }
    const int32_t n = gd->n;
    if (n < 0 || !gd->row_ptr) {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->err = "bad n or row_ptr";
        return SLM_ERR_INVALID_ARGUMENT;
    }
    // the shape of the CSR is checked here; everything else at admission
    const long long nnz = gd->row_ptr[n];
    if (gd->row_ptr[0] != 0 || nnz < 0 || nnz >= (1LL << 31) || (nnz > 0 && !gd->col_idx)) {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->err = "row_ptr must start at 0 and end at the entry count; col_idx must be given";
        return SLM_ERR_INVALID_ARGUMENT;
    }
    auto r = std::make_unique<Request>();
    r->n = n;
    r->nnz = nnz;
    r->directed = directed;
    // a directed graph runs on U = W + W^T (at most twice the entries) and
    // keeps its packed (out, in) strengths
    r->footprint = directed ? slm_server_footprint(n, 2 * nnz) + 8 * ((uint64_t)n + 1)
                            : slm_server_footprint(n, nnz);
    if (opt) r->opt = *opt;
    else slm_default_options(&r->opt);
    if (r->footprint > sv->budget) {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->rejected++;
        sv->err = "the request's footprint exceeds the whole budget";
        return SLM_ERR_BUDGET;
    }
    r->rp.assign(gd->row_ptr, gd->row_ptr + (size_t)n + 1);
    if (nnz > 0) {
        r->col.assign(gd->col_idx, gd->col_idx + nnz);
        if (gd->weights) r->w.assign(gd->weights, gd->weights + nnz);
    }
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->stop) {
        sv->err = "the server is shutting down";
        return SLM_ERR_INVALID_ARGUMENT;
    }
    r->ticket = sv->next_ticket++;
    r->t_submit = sv->now();
    if (deadline_s > 0) {
        r->deadline = slm::steady_seconds() + deadline_s;
        sv->queued_deadlines++;
    }
    *ticket = r->ticket;
    sv->queue.push_back(r.get());
    sv->reqs.emplace(r->ticket, std::move(r));
    sv->submitted++;
    sv->cv_work.notify_all();
    return SLM_OK;
}
}  // namespace

slm_status slm_server_submit_deadline(slm_server *sv, const slm_graph_desc *gd,
                                      const slm_options *opt, double deadline_s, uint64_t *ticket) {
    return submit_request(sv, gd, opt, deadline_s, false, ticket);
}

slm_status slm_server_submit_directed(slm_server *sv, const slm_graph_desc *gd,
                                      const slm_options *opt, double deadline_s, uint64_t *ticket) {
    return submit_request(sv, gd, opt, deadline_s, true, ticket);
}

slm_status slm_server_poll(slm_server *sv, uint64_t ticket, int32_t *state) {
    if (!sv || !state) return SLM_ERR_INVALID_ARGUMENT;
    std::lock_guard<std::mutex> lk(sv->mu);
    Request *r = find(sv, ticket);
    if (!r) return SLM_ERR_INVALID_ARGUMENT;
    *state = r->state;
    return SLM_OK;
}

slm_status slm_server_cancel(slm_server *sv, uint64_t ticket) {
    if (!sv) return SLM_ERR_INVALID_ARGUMENT;
    std::lock_guard<std::mutex> lk(sv->mu);
    Request *r = find(sv, ticket);
    if (!r) {
        sv->err = "slm_server_cancel: unknown or released ticket";
        return SLM_ERR_INVALID_ARGUMENT;
    }
    if (r->state == SLM_REQ_QUEUED) {
        auto it = std::find(sv->queue.begin(), sv->queue.end(), r);
        if (it != sv->queue.end()) sv->queue.erase(it);
        if (r->deadline > 0) sv->queued_deadlines--;
        end_unrun(sv, r, SLM_ERR_CANCELLED, "the request was cancelled while queued");
        sv->cv_done.notify_all();
        sv->cv_work.notify_all();  // the head of the queue may have changed
    } else if (r->state == SLM_REQ_RUNNING) {
        r->cancel.store(1);  // the run stops before its next level or sweep
    }
    return SLM_OK;
}

slm_status slm_server_wait(slm_server *sv, uint64_t ticket, double timeout_s) {
    if (!sv) return SLM_ERR_INVALID_ARGUMENT;
    std::unique_lock<std::mutex> lk(sv->mu);
    if (!find(sv, ticket)) return SLM_ERR_INVALID_ARGUMENT;
    // counted while inside, so that destroy frees nothing a waiter still uses
    struct Inside {
        slm_server *sv;
        explicit Inside(slm_server *s) : sv(s) { sv->waiters++; }
        ~Inside() {  // runs with mu held
            if (--sv->waiters == 0) sv->cv_idle.notify_all();
        }
    } inside(sv);
    // looked up at every wake-up: another thread may take the result with
    // release while this one sleeps, and a released request has ended
    auto ended = [&] {
        const Request *r = find(sv, ticket);
        return !r || r->state == SLM_REQ_DONE || r->state == SLM_REQ_FAILED;
    };
    if (timeout_s < 0) {
        sv->cv_done.wait(lk, ended);
        return SLM_OK;
    }
    const auto limit = std::chrono::duration<double>(timeout_s);
    return sv->cv_done.wait_for(lk, limit, ended) ? SLM_OK : SLM_ERR_TIMEOUT;
}

slm_status slm_server_request_info(slm_server *sv, uint64_t ticket, slm_request_info *info) {
    if (!sv || !info) return SLM_ERR_INVALID_ARGUMENT;
    std::lock_guard<std::mutex> lk(sv->mu);
    Request *r = find(sv, ticket);
    if (!r) return SLM_ERR_INVALID_ARGUMENT;
    slm_request_info o{};
    o.state = r->state;
    o.status = r->status;
    o.n = r->n;
    o.n_communities = r->K;
    o.nnz = r->nnz;
    o.levels = r->levels;
    o.slot = r->slot;
    o.t_submit = r->t_submit;
    o.t_admit = r->t_admit;
    o.t_done = r->t_done;
    o.modularity = r->q;
    o.footprint = r->footprint;
    o.peak_bytes = r->peak;
    o.edges_scanned = r->edges;
    *info = o;
    return SLM_OK;
}

slm_status slm_server_result(slm_server *sv, uint64_t ticket, int32_t *labels,
                             int32_t *n_communities, double *q, int32_t release) {
    if (!sv) return SLM_ERR_INVALID_ARGUMENT;
    std::lock_guard<std::mutex> lk(sv->mu);
    Request *r = find(sv, ticket);
    if (!r) return SLM_ERR_INVALID_ARGUMENT;
    if (r->state == SLM_REQ_QUEUED || r->state == SLM_REQ_RUNNING) return SLM_ERR_NOT_RUN;
    const slm_status s = r->status;
    if (s == SLM_OK) {
        if (labels && r->n > 0) std::memcpy(labels, r->labels.data(), sizeof(int32_t) * (size_t)r->n);
        if (n_communities) *n_communities = r->K;
        if (q) *q = r->q;
    } else {
        sv->err = r->err;
    }
    if (release) sv->reqs.erase(ticket);
    return s;
}

slm_status slm_server_get_stats(slm_server *sv, slm_server_stats *st) {
    if (!sv || !st) return SLM_ERR_INVALID_ARGUMENT;
    std::lock_guard<std::mutex> lk(sv->mu);
    slm_server_stats o{};
    o.submitted = sv->submitted;
    o.completed = sv->completed;
    o.failed = sv->failed;
    o.rejected = sv->rejected;
    o.queued = (int32_t)sv->queue.size();
    o.running = sv->running;
    o.max_running = sv->max_running;
    o.budget_bytes = sv->budget;
    o.reserved_bytes = sv->reserved;
    o.max_reserved_bytes = sv->max_reserved;
    *st = o;
    return SLM_OK;
}

void slm_server_destroy(slm_server *sv) {
    if (!sv) return;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
        for (Request *r : sv->queue)
            end_unrun(sv, r, SLM_ERR_NOT_RUN, "the server was destroyed before the request was admitted");
        sv->queue.clear();
        sv->queued_deadlines = 0;
    }
    sv->cv_work.notify_all();
    sv->cv_done.notify_all();
    for (auto &t : sv->workers) t.join();
    {
        // every request has now ended, so every waiter's condition holds:
        // wake them and let them leave before the mutex and the condition
        // variables are freed
        std::unique_lock<std::mutex> lk(sv->mu);
        sv->cv_done.notify_all();
        sv->cv_idle.wait(lk, [&] { return sv->waiters == 0; });
    }
    delete sv;
    slm::trim_pool();
}

}  // extern "C"
