// Serving: a request loop that takes two-level clustering jobs of mixed shapes as they
// arrive and keeps several of them on the device at once (continuous batching).
//
// A scheduler thread owns `slots` execution slots, each with its own context and CUDA
// stream.  A queued job is admitted when a slot is free and its device footprint (the
// exact byte count of its allocations) fits the budget left; jobs are taken in arrival
// order, and a later job that fits may start ahead of an earlier one that does not
// (backfill), unless the earlier one has been passed over 32 times.  An admitted job's
// whole pipeline (scale, peel, local and final Lloyd, SSE) is queued on its slot's stream
// at once, so the kernels of different jobs overlap on the device; the peel, a
// cooperative launch that needs every SM, goes through one stream shared by all slots so
// that no two peels wait on each other.  Device memory is stream-ordered, so a finishing
// job frees its memory without stalling the others.  When a job's last kernel has run,
// its results are copied to host memory, its device memory is released and its latency
// (submission to completion, host clock) is recorded.
#include <chrono>
#include <cstring>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "pscl_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

double ms_between(Clock::time_point a, Clock::time_point b)
{
    return std::chrono::duration<double, std::milli>(b - a).count();
}

struct Ticket {
    uint64_t id = 0;
    pscl_job_desc desc{};
    int state = PSCL_JOB_QUEUED;
    int err = PSCL_OK;
    std::string msg;
    size_t footprint = 0;
    int passed_over = 0;
    pscl_job *job = nullptr;
    cudaEvent_t done = nullptr;
    std::vector<float> centers;
    std::vector<int32_t> labels;
    double sse = 0.0;
    Clock::time_point t_submit, t_start, t_done;
};

struct Slot {
    pscl_ctx *ctx = nullptr;
    Ticket *cur = nullptr;
};

}  // namespace

struct pscl_server {
    int device = 0;
    int sm_count = 0;
    size_t budget = 0, in_use = 0, peak = 0;
    std::vector<Slot> slots;
    cudaStream_t coop = nullptr;
    std::deque<Ticket *> queue;
    std::map<uint64_t, Ticket *> tickets;
    std::mutex mu;
    std::condition_variable cv;      // worker: new work; clients: a job finished
    std::thread worker;
    bool stop = false;
    uint64_t next_id = 1;
    int64_t completed = 0, failed = 0, max_running = 0;
    pscl_ctx *probe = nullptr;       // footprint queries
};

namespace {

constexpr size_t kMaxQueued = 1 << 20;

void fail_ticket(Ticket *t, int code, const char *msg)
{
    t->err = code;
    t->msg = msg ? msg : "";
    t->state = PSCL_JOB_FAILED;
    t->t_done = Clock::now();
}

// Admit t onto slot sl: create the job (points copied on the slot's stream if on the
// host) and queue its whole pipeline.  Called by the worker with the lock held.
void start(pscl_server *s, Slot &sl, Ticket *t)
{
    const pscl_job_desc &d = t->desc;
    t->t_start = Clock::now();
    int rc = pscl_job_create(sl.ctx, d.points, d.dtype, d.n, d.d, d.on_device, &t->job);
    if (!rc) rc = pscl::job_set_coop_stream(t->job, s->coop);
    if (!rc) rc = pscl_run(t->job, d.N, d.local_k, d.final_k, d.iters, d.seed, d.prec);
    if (!rc && cudaEventRecord(t->done, pscl::ctx_stream(sl.ctx)) != cudaSuccess) {
        cudaGetLastError();
        rc = PSCL_ECUDA;
    }
    if (rc) {
        fail_ticket(t, rc, pscl_last_error());
        if (t->job) {
            pscl_job_destroy(t->job);
            t->job = nullptr;
        }
        s->failed++;
        return;
    }
    t->state = PSCL_JOB_RUNNING;
    sl.cur = t;
    s->in_use += t->footprint;
    if (s->in_use > s->peak) s->peak = s->in_use;
}

// A finished job's results copied to host memory and its device memory released.  Called
// by the worker WITHOUT the lock (the copies block), on a ticket already taken off its
// slot; the ticket stays RUNNING and its bytes counted until settle().
void collect(Ticket *t)
{
    const pscl_job_desc &d = t->desc;
    t->centers.resize((size_t)d.final_k * d.d);
    if (d.want_labels) t->labels.resize((size_t)d.n);
    t->err = pscl_get_result(t->job, t->centers.data(), d.want_labels ? t->labels.data() : nullptr, &t->sse);
    if (t->err) t->msg = pscl_last_error();
    pscl_job_destroy(t->job);
    t->job = nullptr;
}

// The collected job's state, the counters and the bytes in use; with the lock held.
void settle(pscl_server *s, Ticket *t)
{
    if (t->err) {
        fail_ticket(t, t->err, t->msg.c_str());
        s->failed++;
    } else {
        t->state = PSCL_JOB_DONE;
        t->t_done = Clock::now();
        s->completed++;
    }
    s->in_use -= t->footprint;
}

// A job waiting for memory is passed over when a job behind it starts; after this many
// times, no later job starts ahead of it.
constexpr int kMaxPassedOver = 32;

void admit(pscl_server *s)
{
    std::vector<Ticket *> waiting;        // earlier jobs of this pass that did not fit
    for (auto it = s->queue.begin(); it != s->queue.end();) {
        Slot *free_slot = nullptr;
        for (auto &sl : s->slots)
            if (!sl.cur) {
                free_slot = &sl;
                break;
            }
        if (!free_slot) return;
        Ticket *t = *it;
        if (s->in_use + t->footprint <= s->budget) {
            it = s->queue.erase(it);
            start(s, *free_slot, t);
            if (t->state == PSCL_JOB_FAILED) s->cv.notify_all();
            else
                for (Ticket *w : waiting) w->passed_over++;     // t went ahead of each of them
            continue;
        }
        // does not fit yet: later jobs may go ahead, unless this one has been passed over
        // enough times already
        if (t->passed_over >= kMaxPassedOver) return;
        waiting.push_back(t);
        ++it;
    }
}

void loop(pscl_server *s)
{
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    std::vector<Ticket *> done;
    for (;;) {
        bool progress = false;
        int64_t running = 0;
        done.clear();
        for (auto &sl : s->slots) {
            if (!sl.cur) continue;
            const cudaError_t q = cudaEventQuery(sl.cur->done);
            if (q == cudaErrorNotReady) {
                running++;
                continue;
            }
            if (q != cudaSuccess) cudaGetLastError();      // the job's own sync reports it
            done.push_back(sl.cur);
            sl.cur = nullptr;
        }
        if (!done.empty()) {
            // results are copied without the lock: submit, poll and wait go on meanwhile
            lk.unlock();
            for (Ticket *t : done) collect(t);
            lk.lock();
            for (Ticket *t : done) settle(s, t);
            s->cv.notify_all();
            progress = true;
        }
        if (s->stop && running == 0) break;
        if (!s->stop) {
            const size_t before = s->queue.size();
            admit(s);
            progress |= s->queue.size() != before;
        }
        running = 0;
        for (auto &sl : s->slots) running += sl.cur != nullptr;
        if (running > s->max_running) s->max_running = running;
        if (!progress) s->cv.wait_for(lk, std::chrono::microseconds(running ? 50 : 2000));
    }
}

int set_err(int code, const char *msg)
{
    pscl::set_last_error(msg);
    return code;
}

}  // namespace

extern "C" int pscl_server_create(pscl_ctx *ctx, int32_t slots, size_t hbm_budget_bytes, pscl_server **out)
{
    if (!ctx || !out) return set_err(PSCL_EINVAL, "ctx or out is NULL");
    if (slots < 1 || slots > 64) return set_err(PSCL_EINVAL, "slots outside 1..64");
    pscl_server *s = new pscl_server();
    s->device = pscl::ctx_device(ctx);
    s->budget = hbm_budget_bytes;
    // the peel stream gets the highest priority: when SMs free up, the CTAs of a waiting
    // cooperative launch are placed before new CTAs of other jobs
    int lo_prio = 0, hi_prio = 0;
    cudaDeviceGetStreamPriorityRange(&lo_prio, &hi_prio);
    if (cudaSetDevice(s->device) != cudaSuccess ||
        cudaStreamCreateWithPriority(&s->coop, cudaStreamNonBlocking, hi_prio) != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return set_err(PSCL_ECUDA, "could not create the server's streams");
    }
    if (s->budget == 0) {
        size_t free_b = 0, total = 0;
        cudaMemGetInfo(&free_b, &total);
        s->budget = free_b / 10 * 9;
    }
    s->slots.resize(slots);
    int rc = PSCL_OK;
    for (auto &sl : s->slots)
        if (!rc) rc = pscl_ctx_create(&sl.ctx, s->device, 0, nullptr);
    if (!rc) rc = pscl_ctx_create(&s->probe, s->device, 0, nullptr);
    if (rc) {
        for (auto &sl : s->slots)
            if (sl.ctx) pscl_ctx_destroy(sl.ctx);
        if (s->probe) pscl_ctx_destroy(s->probe);
        cudaStreamDestroy(s->coop);
        delete s;
        return rc;
    }
    s->worker = std::thread(loop, s);
    *out = s;
    return PSCL_OK;
}

extern "C" int pscl_submit(pscl_server *s, const pscl_job_desc *d, uint64_t *ticket)
{
    if (!s || !d || !ticket) return set_err(PSCL_EINVAL, "server, desc or ticket is NULL");
    if (!d->points) return set_err(PSCL_EINVAL, "desc.points is NULL");
    if (d->n < 1 || d->n > (int64_t)INT32_MAX || d->d < 1 || d->d > pscl::kMaxD || d->N < 1 || d->local_k < 1 ||
        d->local_k > pscl::kMaxK || d->final_k < 1 || d->final_k > pscl::kMaxK || d->iters < 0)
        return set_err(PSCL_EINVAL, "job shape out of range");
    size_t fp = 0;
    int rc = pscl_job_footprint(s->probe, d->n, d->d, d->N, d->local_k, d->final_k, d->iters, d->dtype, d->on_device,
                                0, &fp);
    if (rc) return rc;
    Ticket *t = new Ticket();
    t->desc = *d;
    t->footprint = fp;
    t->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (fp > s->budget) {
            delete t;
            return set_err(PSCL_ENOMEM, "the job's device footprint exceeds the server's whole budget");
        }
        if (s->queue.size() >= kMaxQueued) {
            delete t;
            return set_err(PSCL_EBUSY, "the queue is full");
        }
        if (cudaSetDevice(s->device) != cudaSuccess ||
            cudaEventCreateWithFlags(&t->done, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            delete t;
            return set_err(PSCL_ECUDA, "cudaEventCreate failed");
        }
        t->id = s->next_id++;
        s->tickets[t->id] = t;
        s->queue.push_back(t);
        *ticket = t->id;
    }
    s->cv.notify_all();
    return PSCL_OK;
}

extern "C" int pscl_poll(pscl_server *s, uint64_t ticket, int32_t *state)
{
    if (!s || !state) return set_err(PSCL_EINVAL, "server or state is NULL");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) return set_err(PSCL_EINVAL, "unknown ticket");
    *state = it->second->state;
    return PSCL_OK;
}

extern "C" int pscl_wait(pscl_server *s, uint64_t ticket, int64_t timeout_us)
{
    if (!s) return set_err(PSCL_EINVAL, "server is NULL");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) return set_err(PSCL_EINVAL, "unknown ticket");
    Ticket *t = it->second;
    auto done = [t] { return t->state == PSCL_JOB_DONE || t->state == PSCL_JOB_FAILED; };
    if (timeout_us < 0) {
        s->cv.wait(lk, done);
    } else if (!s->cv.wait_for(lk, std::chrono::microseconds(timeout_us), done)) {
        return set_err(PSCL_ETIMEOUT, "the job has not finished within the timeout");
    }
    return PSCL_OK;
}

extern "C" int pscl_fetch(pscl_server *s, uint64_t ticket, float *centers, int32_t *labels, double *sse,
                          double *times_ms)
{
    if (!s) return set_err(PSCL_EINVAL, "server is NULL");
    Ticket *t = nullptr;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->tickets.find(ticket);
        if (it == s->tickets.end()) return set_err(PSCL_EINVAL, "unknown ticket");
        t = it->second;
        if (t->state != PSCL_JOB_DONE && t->state != PSCL_JOB_FAILED)
            return set_err(PSCL_ESTATE, "the job has not finished (pscl_wait first)");
        s->tickets.erase(it);
    }
    int rc = t->err;
    if (rc) {
        pscl::set_last_error(t->msg.c_str());
    } else {
        if (centers) memcpy(centers, t->centers.data(), t->centers.size() * sizeof(float));
        if (labels) {
            if (t->labels.empty()) rc = set_err(PSCL_ESTATE, "the job was submitted without want_labels");
            else memcpy(labels, t->labels.data(), t->labels.size() * sizeof(int32_t));
        }
        if (sse) *sse = t->sse;
    }
    if (times_ms) {
        times_ms[0] = ms_between(t->t_submit, t->t_start);    // queued
        times_ms[1] = ms_between(t->t_start, t->t_done);      // admitted to done
        times_ms[2] = ms_between(t->t_submit, t->t_done);     // latency
    }
    if (t->done) cudaEventDestroy(t->done);
    delete t;
    return rc;
}

extern "C" int pscl_server_stats(pscl_server *s, int64_t *out)
{
    if (!s || !out) return set_err(PSCL_EINVAL, "server or out is NULL");
    std::lock_guard<std::mutex> lk(s->mu);
    int64_t running = 0;
    for (auto &sl : s->slots) running += sl.cur != nullptr;
    out[0] = s->completed;
    out[1] = s->failed;
    out[2] = (int64_t)s->queue.size();
    out[3] = running;
    out[4] = (int64_t)s->in_use;
    out[5] = (int64_t)s->peak;
    out[6] = s->max_running;
    out[7] = (int64_t)s->budget;
    return PSCL_OK;
}

extern "C" int pscl_server_destroy(pscl_server *s)
{
    if (!s) return set_err(PSCL_EINVAL, "server is NULL");
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        for (Ticket *t : s->queue) fail_ticket(t, PSCL_ESTATE, "the server was destroyed before the job started");
        s->queue.clear();
    }
    s->cv.notify_all();
    if (s->worker.joinable()) s->worker.join();      // running jobs finish first
    for (auto &kv : s->tickets) {
        if (kv.second->done) cudaEventDestroy(kv.second->done);
        delete kv.second;
    }
    for (auto &sl : s->slots) pscl_ctx_destroy(sl.ctx);
    pscl_ctx_destroy(s->probe);
    cudaStreamDestroy(s->coop);
    delete s;
    return PSCL_OK;
}
