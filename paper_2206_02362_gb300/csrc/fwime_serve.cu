// Request server: continuous batching of FWIME shot requests on one GPU (Barnier et al.,
// Computational aspects: shots are independent modelling tasks dispatched to the GPU by a host
// layer; here forward-modelling requests f(m), Eq. 1, and gradient requests Phi and B* r + T* r,
// Eqs. 1, 7-9, each on its own grid).
//
// fwime_submit queues a request and returns a ticket at once.  A dispatcher thread admits queued
// requests in arrival order as soon as their device memory (the operator's workspace from the same
// planner as fwime_workspace_bytes, plus staging when the request's buffers are in host memory)
// fits the server's budget and an in-flight slot is free -- while earlier requests are still on the
// GPU.  Admitted requests are handed to enqueue workers: each request gets its own context on a
// stream of its own, so the work of all admitted requests overlaps on the device; forward requests
// admitted in the same round share one grouped launch per time step (fwime_forward_group), whatever
// their grid sizes and record lengths.  Completion is detected with one CUDA event per launch
// group, without synchronising any other stream; the request's memory then returns to the budget
// and the next requests are admitted.  fwime_poll / fwime_wait collect a result once.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "../../include/fwime.h"
#include "fwime_internal.h"

namespace fwk {

namespace {

using Clock = std::chrono::steady_clock;

struct Job {
    uint64_t ticket = 0;
    fwime_request req{};
    std::vector<int> siz, six, riz, rix;    // geometry, copied at submit
    size_t ws = 0, need = 0;                // workspace cap of its context; bytes admitted
    Clock::time_point t_submit, t_admit, t_done;
    double enqueue_s = 0.0;                 // host time spent enqueuing its launch group's work
    fwime_ctx *ctx = nullptr;
    float *stage = nullptr;                 // device staging of host buffers
    double J = 0.0;
    int status = FWIME_OK;
    bool done = false;
};

struct Group {
    std::vector<Job *> jobs;
    int stream = -1;
    cudaEvent_t ev = nullptr;
    bool enqueued = false;                  // set by the worker once the group's work is on its stream
};

size_t al(size_t n) { return (n + 63) & ~(size_t)63; }

size_t nm_of(const fwime_request &r) { return (size_t)r.grid.nz * r.grid.nx; }
size_t nd_of(const fwime_request &r) { return (size_t)r.geom.nshot * r.grid.nt * r.geom.nrec; }
size_t nw_of(const fwime_request &r) { return (size_t)r.geom.nshot * r.grid.nt; }

// floats of device staging a host-memory request needs: v, w, data in/out, p~, gradient
size_t stage_floats(const fwime_request &r)
{
    if (!r.host_io) return 0;
    size_t f = al(nm_of(r)) + al(nw_of(r)) + al(nd_of(r));
    if (r.kind == FWIME_REQ_GRADIENT) f += al((size_t)r.grid.nh * nm_of(r)) + al(nm_of(r));
    return f;
}

}  // namespace

struct Server {
    int device = 0;
    size_t budget = 0, used = 0;
    int max_active = 1, active = 0, options = 0, nworkers = 1;
    std::mutex mu;
    std::condition_variable cv_disp, cv_done, cv_work;
    std::deque<Job *> queue;
    std::map<uint64_t, Job *> jobs;         // submitted and not yet collected
    std::vector<Group *> running;
    std::deque<Group *> work;
    uint64_t next_ticket = 1;
    int pending = 0;                        // submitted and not yet finished
    bool stop = false;
    bool cuda_ready = false;
    int cuda_error = FWIME_OK;
    std::vector<cudaStream_t> streams;
    std::vector<char> stream_busy;
    std::thread dispatcher;
    std::vector<std::thread> workers;
};

namespace {

// Runs on an enqueue worker: creates the group's contexts on its stream, stages host inputs, enqueues
// the operators and the event that completes the group.
void enqueue_group(Server *s, Group *g)
{
    const auto t0 = Clock::now();
    cudaSetDevice(s->device);
    cudaStream_t st = s->streams[g->stream];
    auto fail_all = [&](int code) {
        for (Job *j : g->jobs)
            if (j->status == FWIME_OK) j->status = code;
    };
    std::vector<fwime_ctx *> fctx;
    std::vector<const float *> fv, fw;
    std::vector<float *> fd;
    for (Job *j : g->jobs) {
        fwime_request &r = j->req;
        fwime_geom geo{r.geom.nshot, j->siz.data(), j->six.data(), r.geom.nrec, j->riz.data(), j->rix.data()};
        int rc = fwime_create(&j->ctx, &r.grid, &geo, j->ws, st);
        if (rc == FWIME_OK) rc = fwime_set_option(j->ctx, FWIME_OPT_SHOTS_PER_BATCH, r.geom.nshot);
        if (rc == FWIME_OK && (s->options & FWIME_SERVE_PLAIN)) rc = fwime_set_option(j->ctx, FWIME_OPT_PLAIN, 1);
        const float *v = r.v, *w = r.w, *pt = r.pt, *dobs = r.dobs;
        float *out = r.kind == FWIME_REQ_FORWARD ? r.d : r.grad;
        if (rc == FWIME_OK && r.host_io) {
            const size_t nf = stage_floats(r);
            if (cudaMallocAsync(reinterpret_cast<void **>(&j->stage), nf * sizeof(float), st) != cudaSuccess) {
                cudaGetLastError();
                j->stage = nullptr;
                rc = FWIME_ENOMEM;
            } else {
                float *p = j->stage;
                auto put = [&](const float *src, size_t n) -> float * {
                    float *dst = p;
                    p += al(n);
                    if (src && cudaMemcpyAsync(dst, src, n * sizeof(float), cudaMemcpyHostToDevice, st) != cudaSuccess)
                        rc = FWIME_ECUDA;
                    return dst;
                };
                v = put(r.v, nm_of(r));
                w = put(r.w, nw_of(r));
                if (r.kind == FWIME_REQ_FORWARD) {
                    out = put(nullptr, nd_of(r));
                } else {
                    dobs = put(r.dobs, nd_of(r));
                    pt = put(r.pt, (size_t)r.grid.nh * nm_of(r));
                    out = put(nullptr, nm_of(r));
                }
            }
        }
        if (rc != FWIME_OK) {
            j->status = rc;
            continue;
        }
        if (r.kind == FWIME_REQ_FORWARD && g->jobs.size() > 1) {
            fctx.push_back(j->ctx); fv.push_back(v); fw.push_back(w); fd.push_back(out);
            continue;
        }
        rc = r.kind == FWIME_REQ_FORWARD ? fwime_forward(j->ctx, v, w, out)
                                         : fwime_gradient(j->ctx, v, w, pt, dobs, r.eps, out, &j->J);
        if (rc == FWIME_OK && r.host_io) {
            const size_t n = r.kind == FWIME_REQ_FORWARD ? nd_of(r) : nm_of(r);
            float *dst = r.kind == FWIME_REQ_FORWARD ? r.d : r.grad;
            if (cudaMemcpyAsync(dst, out, n * sizeof(float), cudaMemcpyDeviceToHost, st) != cudaSuccess) rc = FWIME_ECUDA;
        }
        j->status = rc;
    }
    if (!fctx.empty()) {
        const int rc = fwime_forward_group(fctx.data(), (int)fctx.size(), fv.data(), fw.data(), fd.data());
        size_t k = 0;
        for (Job *j : g->jobs) {
            if (j->status != FWIME_OK || j->req.kind != FWIME_REQ_FORWARD) continue;
            j->status = rc;
            if (rc == FWIME_OK && j->req.host_io &&
                cudaMemcpyAsync(j->req.d, fd[k], nd_of(j->req) * sizeof(float), cudaMemcpyDeviceToHost, st) !=
                    cudaSuccess)
                j->status = FWIME_ECUDA;
            ++k;
        }
    }
    if (cudaEventCreateWithFlags(&g->ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventRecord(g->ev, st) != cudaSuccess) {
        cudaGetLastError();
        if (g->ev) cudaEventDestroy(g->ev);
        g->ev = nullptr;
        cudaStreamSynchronize(st);          // no event: complete the group the blocking way
        fail_all(FWIME_ECUDA);
    }
    const double dt = std::chrono::duration<double>(Clock::now() - t0).count();
    for (Job *j : g->jobs) j->enqueue_s = dt;
    std::lock_guard<std::mutex> lk(s->mu);
    g->enqueued = true;
    s->cv_disp.notify_all();
}

void worker_loop(Server *s)
{
    for (;;) {
        Group *g = nullptr;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_work.wait(lk, [&] { return s->stop || !s->work.empty(); });
            if (s->work.empty()) return;   // stop with nothing left to enqueue
            g = s->work.front();
            s->work.pop_front();
        }
        enqueue_group(s, g);
    }
}

// On the dispatcher: the group's work has completed (or failed to enqueue); read statuses and
// objectives, release contexts, staging, stream and memory, and wake the waiters.
void finish_group(Server *s, Group *g)
{
    for (Job *j : g->jobs) {
        if (j->ctx) {
            const int rc = fwime_sync(j->ctx);       // the stream is idle: reads the status word and Phi
            if (j->status == FWIME_OK) j->status = rc;
            if (j->stage) cudaFreeAsync(j->stage, s->streams[g->stream]);
            fwime_destroy(j->ctx);
            j->ctx = nullptr;
        }
        j->stage = nullptr;
    }
    if (g->ev) cudaEventDestroy(g->ev);
    const auto now = Clock::now();
    std::lock_guard<std::mutex> lk(s->mu);
    for (Job *j : g->jobs) {
        j->t_done = now;
        j->done = true;
        s->used -= j->need;
        s->active -= 1;
        s->pending -= 1;
    }
    s->stream_busy[g->stream] = 0;
    delete g;
    s->cv_done.notify_all();
}

int cuda_setup(Server *s)
{
    if (s->cuda_ready) return s->cuda_error;
    s->cuda_ready = true;
    if (cudaSetDevice(s->device) != cudaSuccess) {
        cudaGetLastError();
        return s->cuda_error = FWIME_ECUDA;
    }
    s->streams.assign(s->max_active, nullptr);
    s->stream_busy.assign(s->max_active, 0);
    for (auto &st : s->streams)
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            return s->cuda_error = FWIME_ECUDA;
        }
    return FWIME_OK;
}

void dispatch_loop(Server *s)
{
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        // admission: arrival order, while memory and slots allow
        std::vector<Job *> admitted;
        while (!s->queue.empty() && s->active < s->max_active && s->used + s->queue.front()->need <= s->budget) {
            Job *j = s->queue.front();
            s->queue.pop_front();
            s->used += j->need;
            s->active += 1;
            j->t_admit = Clock::now();
            admitted.push_back(j);
        }
        std::vector<Group *> check;
        for (Group *g : s->running)
            if (g->enqueued) check.push_back(g);
        if (s->stop && s->pending == 0) break;
        lk.unlock();
        if (!admitted.empty()) {
            const int rc = cuda_setup(s);
            std::vector<Group *> groups;
            Group *fwd = nullptr;
            for (Job *j : admitted) {
                if (rc != FWIME_OK) {
                    j->status = rc;
                } else if (j->req.kind == FWIME_REQ_FORWARD && !(s->options & FWIME_SERVE_PLAIN)) {
                    if (!fwd) groups.push_back(fwd = new Group());
                    fwd->jobs.push_back(j);
                    continue;
                }
                Group *g = new Group();
                g->jobs.push_back(j);
                groups.push_back(g);
            }
            lk.lock();
            for (Group *g : groups) {
                if (g->jobs[0]->status != FWIME_OK) {   // CUDA unusable: complete at once
                    for (Job *j : g->jobs) {
                        j->t_done = Clock::now();
                        j->done = true;
                        s->used -= j->need;
                        s->active -= 1;
                        s->pending -= 1;
                    }
                    delete g;
                    s->cv_done.notify_all();
                    continue;
                }
                for (int k = 0; k < (int)s->stream_busy.size(); ++k)
                    if (!s->stream_busy[k]) {
                        s->stream_busy[k] = 1;
                        g->stream = k;
                        break;
                    }
                s->running.push_back(g);
                s->work.push_back(g);
            }
            s->cv_work.notify_all();
            lk.unlock();
        }
        std::vector<Group *> finished;
        for (Group *g : check) {
            const cudaError_t e = g->ev ? cudaEventQuery(g->ev) : cudaSuccess;
            if (e == cudaErrorNotReady) continue;
            if (e != cudaSuccess) {
                cudaGetLastError();
                for (Job *j : g->jobs)
                    if (j->status == FWIME_OK) j->status = FWIME_ECUDA;
            }
            finished.push_back(g);
        }
        for (Group *g : finished) {
            {
                std::lock_guard<std::mutex> l2(s->mu);
                s->running.erase(std::find(s->running.begin(), s->running.end(), g));
            }
            finish_group(s, g);
        }
        lk.lock();
        if (admitted.empty() && finished.empty())
            s->cv_disp.wait_for(lk, std::chrono::microseconds(s->running.empty() ? 20000 : 100));
    }
}

int fail_srv(char *err, size_t n, int code, const char *msg)
{
    if (err) snprintf(err, n, "%s", msg);
    return code;
}

}  // namespace

void server_destroy(Server *s)
{
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->cv_disp.notify_all();
        s->cv_work.notify_all();
    }
    if (s->dispatcher.joinable()) s->dispatcher.join();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->cv_work.notify_all();
    }
    for (auto &t : s->workers)
        if (t.joinable()) t.join();
    for (auto st : s->streams)
        if (st) cudaStreamDestroy(st);
    for (auto &kv : s->jobs) delete kv.second;
    delete s;
}

int server_sync(Server *s)
{
    std::unique_lock<std::mutex> lk(s->mu);
    s->cv_done.wait(lk, [&] { return s->pending == 0; });
    return FWIME_OK;
}

}  // namespace fwk

using namespace fwk;

namespace {
thread_local char g_serr[256] = {0};

int fill(const Job *j, fwime_result *res)
{
    if (!res) return FWIME_OK;
    res->done = j->done ? 1 : 0;
    res->status = j->status;
    res->objective = j->J;
    res->enqueue_s = j->enqueue_s;
    if (j->done) {
        res->queued_s = std::chrono::duration<double>(j->t_admit - j->t_submit).count();
        res->latency_s = std::chrono::duration<double>(j->t_done - j->t_submit).count();
    } else {
        res->queued_s = res->latency_s = 0.0;
    }
    return FWIME_OK;
}
}  // namespace

extern "C" {

int fwime_server_create(fwime_ctx **out, size_t memory_budget, int max_active, int options)
{
    if (!out || max_active < 1 || max_active > 1024 || (options & ~FWIME_SERVE_PLAIN)) return FWIME_EINVAL;
    *out = nullptr;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        dev = 0;
    }
    if (memory_budget == 0) {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
            cudaGetLastError();
            return FWIME_ECUDA;
        }
        memory_budget = fr / 10 * 8;
    }
    Server *s = new Server();
    s->device = dev;
    s->budget = memory_budget;
    s->options = options;
    s->max_active = (options & FWIME_SERVE_PLAIN) ? 1 : max_active;
    s->nworkers = std::min(12, s->max_active);
    s->dispatcher = std::thread(dispatch_loop, s);
    for (int i = 0; i < s->nworkers; ++i) s->workers.emplace_back(worker_loop, s);
    *out = ctx_for_server(s);
    return FWIME_OK;
}

int fwime_request_bytes(const fwime_request *r, size_t *bytes)
{
    if (!r || !bytes) return FWIME_EINVAL;
    if (r->kind != FWIME_REQ_FORWARD && r->kind != FWIME_REQ_GRADIENT) return FWIME_EINVAL;
    const int op = r->kind == FWIME_REQ_FORWARD ? FWIME_OP_FORWARD : FWIME_OP_GRADIENT;
    size_t ws = 0;
    const int rc = fwime_workspace_bytes(&r->grid, &r->geom, op, r->geom.nshot, 0, &ws);
    if (rc != FWIME_OK) return rc;
    // workspace + the context's own small block + staging of host buffers
    *bytes = ws + ((size_t)1 << 20) + stage_floats(*r) * sizeof(float);
    return FWIME_OK;
}

int fwime_submit(fwime_ctx *srv, const fwime_request *req, uint64_t *ticket)
{
    Server *s = ctx_server(srv);
    if (!s || !req || !ticket) return FWIME_EINVAL;
    g_serr[0] = 0;
    size_t need = 0;
    int rc = fwime_request_bytes(req, &need);
    if (rc != FWIME_OK) return fail_srv(g_serr, sizeof(g_serr), rc, "fwime_submit: invalid kind, grid or geometry");
    const bool fwd = req->kind == FWIME_REQ_FORWARD;
    if (!req->v || !req->w || (fwd && !req->d) || (!fwd && (!req->pt || !req->dobs || !req->grad)) ||
        !(req->eps >= 0.f))
        return fail_srv(g_serr, sizeof(g_serr), FWIME_EINVAL, "fwime_submit: missing buffer or eps < 0");
    if (need > s->budget) {
        snprintf(g_serr, sizeof(g_serr), "fwime_submit: the request needs %zu bytes, the server's budget is %zu", need,
                 s->budget);
        return FWIME_ENOMEM;
    }
    Job *j = new Job();
    j->req = *req;
    j->siz.assign(req->geom.src_iz, req->geom.src_iz + req->geom.nshot);
    j->six.assign(req->geom.src_ix, req->geom.src_ix + req->geom.nshot);
    j->riz.assign(req->geom.rec_iz, req->geom.rec_iz + req->geom.nrec);
    j->rix.assign(req->geom.rec_ix, req->geom.rec_ix + req->geom.nrec);
    j->req.geom.src_iz = j->siz.data(); j->req.geom.src_ix = j->six.data();
    j->req.geom.rec_iz = j->riz.data(); j->req.geom.rec_ix = j->rix.data();
    j->need = need;
    fwime_workspace_bytes(&req->grid, &req->geom, fwd ? FWIME_OP_FORWARD : FWIME_OP_GRADIENT, req->geom.nshot, 0,
                          &j->ws);
    j->t_submit = Clock::now();
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) {
        delete j;
        return FWIME_EBUSY;
    }
    j->ticket = s->next_ticket++;
    s->jobs[j->ticket] = j;
    s->queue.push_back(j);
    s->pending += 1;
    *ticket = j->ticket;
    s->cv_disp.notify_all();
    return FWIME_OK;
}

int fwime_poll(fwime_ctx *srv, uint64_t ticket, fwime_result *res)
{
    Server *s = ctx_server(srv);
    if (!s) return FWIME_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->jobs.find(ticket);
    if (it == s->jobs.end()) return FWIME_EINVAL;
    Job *j = it->second;
    fill(j, res);
    if (j->done) {
        s->jobs.erase(it);
        delete j;
        s->cv_done.notify_all();
    }
    return FWIME_OK;
}

int fwime_wait(fwime_ctx *srv, uint64_t ticket, fwime_result *res)
{
    Server *s = ctx_server(srv);
    if (!s) return FWIME_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    if (s->jobs.find(ticket) == s->jobs.end()) return FWIME_EINVAL;
    // re-looked up on every wake: another thread may collect the same ticket first
    s->cv_done.wait(lk, [&] {
        auto it = s->jobs.find(ticket);
        return it == s->jobs.end() || it->second->done;
    });
    auto it = s->jobs.find(ticket);
    if (it == s->jobs.end()) return FWIME_EINVAL;
    Job *j = it->second;
    fill(j, res);
    s->jobs.erase(it);
    delete j;
    return FWIME_OK;
}

int fwime_server_last_error(char *buf, size_t n)
{
    if (!buf || n == 0) return FWIME_EINVAL;
    snprintf(buf, n, "%s", g_serr);
    return FWIME_OK;
}

}  // extern "C"
