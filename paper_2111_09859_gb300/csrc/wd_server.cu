// wd_server.cu -- request loop: continuous batching of independent wall-distance solves.
//
// One scheduler thread per server.  Requests are admitted in arrival order while the sum of
// their device footprints fits the cap and a slot is free.  Each admitted request is a
// SolveTask (the solve of wd_solve cut into slices that end at a convergence check) on its
// grid's own stream; the scheduler keeps one slice of every running request queued on the
// GPU, so slices of different requests overlap, and it reacts to each slice's completion
// event: evaluate the change norms, queue the next slice or the copy-out, retire.  Grids the
// server creates go back to a per-shape pool when their request is done and are re-used
// through the geometry reset, so neither admission nor retirement calls cudaFree (which
// would wait for every stream on the device).
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "wd_api_internal.h"

using namespace wd;

#define ST(...)                                \
    do {                                       \
        wd_status _s = (__VA_ARGS__);          \
        if (_s != WD_OK) return _s;            \
    } while (0)

namespace {

using Clock = std::chrono::steady_clock;

enum JobState { J_QUEUED, J_RUNNING, J_FINISHING, J_DONE };

// descriptor fields that decide a grid's allocations (pool key)
struct ShapeKey {
    std::vector<double> v;
    explicit ShapeKey(const wd_grid_desc& d)
    {
        v = {(double)d.ndim, (double)d.n[0], (double)d.n[1], (double)d.n[2], (double)d.precision,
             (double)d.scheme, d.L_ref};
        for (int k = 0; k < 3; k++) {
            v.push_back(d.bc_lo[k]);
            v.push_back(d.bc_hi[k]);
            for (int m = 0; m < 3; m++) v.push_back(d.period[k][m]);
        }
    }
    bool operator<(const ShapeKey& o) const { return v < o.v; }
};

struct Job {
    long long id = 0;
    JobState state = J_QUEUED;
    bool owned = true;                 // grid created (or pooled) by the server
    wd_grid_desc desc;
    std::vector<double> xyz, dval;
    std::vector<uint8_t> mask;
    bool has_mask = false, has_dval = false;
    wd_grid grid = nullptr;
    const uint8_t* mask_dev = nullptr; // caller grids: Dirichlet update
    const void* dval_dev = nullptr;
    int warm = 0;
    wd_solve_params p;
    void* phi = nullptr;
    size_t fp = 0;
    SolveTask* task = nullptr;
    cudaEvent_t ev = nullptr;          // end of the work queued last
    cudaEvent_t ev_ready = nullptr;    // caller grids: work queued before the submission
    Clock::time_point t_submit, t_done;
    wd_stats stats;
    wd_status rc = WD_OK;
    std::string err;
};

}  // namespace

struct wd_server_s {
    wd_server_config cfg;
    int device = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Job*> queue;                       // guarded by mu
    std::unordered_map<long long, Job*> jobs;     // guarded: every job not yet waited for
    long long next_id = 1, n_done = 0, n_running = 0, peak = 0;   // guarded
    size_t admitted = 0;                          // guarded
    bool stop = false;                            // guarded
    std::thread th;
    // scheduler thread only
    std::vector<Job*> active;
    std::map<ShapeKey, std::vector<wd_grid>> pool;
    size_t pool_bytes = 0;
};

namespace {

void destroy_job(Job* j)
{
    if (j->task) delete j->task;
    if (j->ev) cudaEventDestroy(j->ev);
    if (j->ev_ready) cudaEventDestroy(j->ev_ready);
    delete j;
}

// frees pooled grids until admitted + pooled bytes fit the cap (cudaFree waits for the
// device, so this only runs when the pool stands in the way of an admission)
void evict(wd_server s, size_t admitted_now)
{
    for (auto it = s->pool.begin(); it != s->pool.end() && admitted_now + s->pool_bytes > s->cfg.max_device_bytes;) {
        while (!it->second.empty() && admitted_now + s->pool_bytes > s->cfg.max_device_bytes) {
            wd_grid g = it->second.back();
            it->second.pop_back();
            s->pool_bytes -= grid_bytes(g);
            wd_destroy_grid(g);
        }
        it = it->second.empty() ? s->pool.erase(it) : std::next(it);
    }
}

void retire(wd_server s, Job* j)
{
    j->t_done = Clock::now();
    if (j->task) {
        delete j->task;
        j->task = nullptr;
    }
    if (j->owned && j->grid) {
        auto& v = s->pool[ShapeKey(j->desc)];
        if (j->rc != WD_ERR_CUDA && (int)v.size() < s->cfg.pool_per_shape) {
            v.push_back(j->grid);
            s->pool_bytes += grid_bytes(j->grid);
        } else {
            wd_destroy_grid(j->grid);
        }
        j->grid = nullptr;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    j->state = J_DONE;
    s->n_done++;
    s->n_running--;
    s->admitted -= j->fp;
    s->cv_done.notify_all();
}

void fail(wd_server s, Job* j, wd_status rc)
{
    j->rc = rc;
    j->err = wd_last_error();
    retire(s, j);
}

// queues slices until one ends at a convergence check whose norms the host must read, or
// the task has finished (then the copy-out is queued); records the job's event after it
wd_status advance(Job* j)
{
    for (;;) {
        if (j->task->finished()) {
            j->rc = j->task->finish(j->phi, &j->stats);
            if (j->rc != WD_OK) j->err = wd_last_error();
            if (j->rc == WD_ERR_CUDA) return j->rc;
            j->state = J_FINISHING;
            break;
        }
        wd_status r = j->task->enqueue();
        if (r != WD_OK) return r;
        if (j->task->check()) break;
        r = j->task->complete();
        if (r != WD_OK) return r;
    }
    if (cudaEventRecord(j->ev, grid_stream(j->grid)) != cudaSuccess)
        return cuda_error(cudaGetLastError(), "slice event");
    return WD_OK;
}

wd_status start(wd_server s, Job* j)
{
    if (j->owned) {
        auto it = s->pool.find(ShapeKey(j->desc));
        if (it != s->pool.end() && !it->second.empty()) {
            j->grid = it->second.back();
            it->second.pop_back();
            s->pool_bytes -= grid_bytes(j->grid);
            ST(wd_reset_geometry(j->grid, j->xyz.data(), j->has_mask ? j->mask.data() : nullptr,
                                 j->has_dval ? j->dval.data() : nullptr));
        } else {
            size_t adm;
            {
                std::lock_guard<std::mutex> lk(s->mu);
                adm = s->admitted;
            }
            evict(s, adm);
            ST(wd_create_grid(&j->desc, j->xyz.data(), j->has_mask ? j->mask.data() : nullptr,
                              j->has_dval ? j->dval.data() : nullptr, nullptr, &j->grid));
        }
        std::vector<double>().swap(j->xyz);
        std::vector<uint8_t>().swap(j->mask);
        std::vector<double>().swap(j->dval);
    } else {
        if (cudaStreamWaitEvent(grid_stream(j->grid), j->ev_ready, 0) != cudaSuccess)
            return cuda_error(cudaGetLastError(), "request ordering");
        if (j->mask_dev) ST(update_dirichlet(j->grid, j->mask_dev, j->dval_dev));
    }
    j->task = make_solve_task(j->grid, &j->p);
    if (!j->task) return set_error(WD_ERR_INVALID_ARG, "bad grid precision");
    ST(j->task->begin(j->phi, j->warm != 0 || j->p.init == WD_INIT_GIVEN));
    j->state = J_RUNNING;
    return advance(j);
}

void scheduler(wd_server s)
{
    cudaSetDevice(s->device);
    for (;;) {
        std::vector<Job*> admit;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            if (s->active.empty())
                s->cv_work.wait(lk, [&] { return s->stop || !s->queue.empty(); });
            if (s->stop && s->queue.empty() && s->active.empty()) break;
            while (!s->queue.empty()) {
                Job* j = s->queue.front();
                if ((int)(s->active.size() + admit.size()) >= s->cfg.max_active) break;
                if (s->admitted + j->fp > s->cfg.max_device_bytes) break;
                s->queue.pop_front();
                s->admitted += j->fp;
                s->n_running++;
                s->peak = std::max(s->peak, s->n_running);
                admit.push_back(j);
            }
        }
        bool progress = !admit.empty();
        for (Job* j : admit) {
            wd_status r = start(s, j);
            if (r != WD_OK) fail(s, j, r);
            else s->active.push_back(j);
        }
        for (size_t k = 0; k < s->active.size();) {
            Job* j = s->active[k];
            cudaError_t e = cudaEventQuery(j->ev);
            if (e == cudaErrorNotReady) {
                k++;
                continue;
            }
            progress = true;
            bool gone = false;
            if (e != cudaSuccess) {
                fail(s, j, cuda_error(e, "request slice"));
                gone = true;
            } else if (j->state == J_RUNNING) {
                wd_status r = j->task->complete();
                if (r == WD_OK) r = advance(j);
                if (r != WD_OK) {
                    fail(s, j, r);
                    gone = true;
                }
            } else {
                retire(s, j);
                gone = true;
            }
            if (gone) {
                s->active[k] = s->active.back();
                s->active.pop_back();
            } else {
                k++;
            }
        }
        if (!progress) {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_work.wait_for(lk, std::chrono::microseconds(40), [&] {
                return s->stop || (!s->queue.empty() && (int)s->active.size() < s->cfg.max_active &&
                                   s->admitted + s->queue.front()->fp <= s->cfg.max_device_bytes);
            });
        }
    }
}

wd_status enqueue_job(wd_server s, Job* j, long long* ticket)
{
    if (cudaEventCreateWithFlags(&j->ev, cudaEventDisableTiming) != cudaSuccess) {
        cudaError_t e = cudaGetLastError();
        destroy_job(j);
        return cuda_error(e, "request event");
    }
    j->t_submit = Clock::now();
    std::lock_guard<std::mutex> lk(s->mu);
    j->id = s->next_id++;
    s->jobs[j->id] = j;
    s->queue.push_back(j);
    *ticket = j->id;
    s->cv_work.notify_all();
    return WD_OK;
}

}  // namespace

extern "C" {

wd_status wd_server_create(const wd_server_config* cfg, wd_server* out)
{
    if (!out) return set_error(WD_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    wd_server_config c;
    std::memset(&c, 0, sizeof(c));
    if (cfg) c = *cfg;
    if (c.max_active < 0) return set_error(WD_ERR_INVALID_ARG, "negative max_active");
    if (c.max_active == 0) c.max_active = 32;
    if (c.pool_per_shape == 0) c.pool_per_shape = 2;
    if (c.pool_per_shape < 0) c.pool_per_shape = 0;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return cuda_error(cudaGetLastError(), "cudaGetDevice");
    if (c.max_device_bytes == 0) {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return cuda_error(cudaGetLastError(), "cudaMemGetInfo");
        c.max_device_bytes = fr / 10 * 8;
    }
    wd_server s = new wd_server_s();
    s->cfg = c;
    s->device = dev;
    s->th = std::thread(scheduler, s);
    *out = s;
    return WD_OK;
}

wd_status wd_server_submit(wd_server s, const wd_grid_desc* desc, const double* xyz_host,
                           const uint8_t* mask_host, const double* dval_host,
                           const wd_solve_params* p, void* phi, long long* ticket)
{
    if (!s || !desc || !xyz_host || !p || !phi || !ticket)
        return set_error(WD_ERR_INVALID_ARG, "NULL argument");
    ST(check_solve_params(p));
    const size_t fp = wd_query_footprint(desc, p);
    if (fp == 0) return WD_ERR_INVALID_ARG;     // the message was set by the descriptor check
    if (fp > s->cfg.max_device_bytes)
        return set_error(WD_ERR_OOM, "request footprint exceeds the server's device-memory cap");
    Job* j = new Job();
    j->owned = true;
    j->desc = *desc;
    const size_t N = (size_t)desc->n[0] * desc->n[1] * desc->n[2];
    j->xyz.assign(xyz_host, xyz_host + (size_t)desc->ndim * N);
    if (mask_host) {
        j->mask.assign(mask_host, mask_host + N);
        j->has_mask = true;
        if (dval_host) {
            j->dval.assign(dval_host, dval_host + N);
            j->has_dval = true;
        }
    }
    j->p = *p;
    j->phi = phi;
    j->fp = fp;
    return enqueue_job(s, j, ticket);
}

wd_status wd_server_submit_grid(wd_server s, wd_grid g, const uint8_t* mask_dev,
                                const void* dval_dev, int warm, const wd_solve_params* p,
                                void* phi, long long* ticket)
{
    if (!s || !g || !p || !phi || !ticket) return set_error(WD_ERR_INVALID_ARG, "NULL argument");
    ST(check_solve_params(p));
    const size_t fp = grid_bytes(g);
    if (fp > s->cfg.max_device_bytes)
        return set_error(WD_ERR_OOM, "grid footprint exceeds the server's device-memory cap");
    Job* j = new Job();
    j->owned = false;
    j->grid = g;
    j->mask_dev = mask_dev;
    j->dval_dev = dval_dev;
    j->warm = warm;
    j->p = *p;
    j->phi = phi;
    j->fp = fp;
    // order the request after the caller's work on the grid's stream (e.g. writes of phi)
    if (cudaEventCreateWithFlags(&j->ev_ready, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventRecord(j->ev_ready, grid_user_stream(g)) != cudaSuccess) {
        cudaError_t e = cudaGetLastError();
        destroy_job(j);
        return cuda_error(e, "request ordering event");
    }
    return enqueue_job(s, j, ticket);
}

wd_status wd_server_wait(wd_server s, long long ticket, double timeout_s, wd_stats* stats,
                         double* latency_s)
{
    if (!s) return set_error(WD_ERR_INVALID_ARG, "server is NULL");
    Job* j = nullptr;
    {
        std::unique_lock<std::mutex> lk(s->mu);
        auto it = s->jobs.find(ticket);
        if (it == s->jobs.end()) return set_error(WD_ERR_INVALID_ARG, "unknown ticket");
        j = it->second;
        auto done = [&] { return j->state == J_DONE; };
        if (timeout_s < 0) {
            s->cv_done.wait(lk, done);
        } else if (!s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), done)) {
            return set_error(WD_ERR_TIMEOUT, "request still queued or running");
        }
        s->jobs.erase(it);
    }
    if (stats) *stats = j->stats;
    if (stats) stats->seconds = std::chrono::duration<double>(j->t_done - j->t_submit).count();
    if (latency_s) *latency_s = std::chrono::duration<double>(j->t_done - j->t_submit).count();
    wd_status rc = j->rc;
    if (rc != WD_OK) set_error(rc, j->err.c_str());
    destroy_job(j);
    return rc;
}

wd_status wd_server_info(wd_server s, long long* queued, long long* running, long long* done,
                         size_t* admitted_bytes, long long* peak_running)
{
    if (!s) return set_error(WD_ERR_INVALID_ARG, "server is NULL");
    std::lock_guard<std::mutex> lk(s->mu);
    if (queued) *queued = (long long)s->queue.size();
    if (running) *running = s->n_running;
    if (done) *done = s->n_done;
    if (admitted_bytes) *admitted_bytes = s->admitted;
    if (peak_running) *peak_running = s->peak;
    return WD_OK;
}

void wd_server_destroy(wd_server s)
{
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->cv_work.notify_all();
    }
    if (s->th.joinable()) s->th.join();
    for (auto& kv : s->pool)
        for (wd_grid g : kv.second) wd_destroy_grid(g);
    for (auto& kv : s->jobs) destroy_job(kv.second);
    delete s;
}

}  // extern "C"
