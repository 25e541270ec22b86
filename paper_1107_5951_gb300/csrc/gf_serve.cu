// gf_serve.cu -- continuous batching of forward solves (gf_server_* in gf.h).
//
// A scheduler thread takes queued requests in arrival order.  A request is
// admitted as soon as a slot (a non-blocking CUDA stream) is free and its
// plan is resident or fits in the memory budget; idle cached plans are
// evicted least-recently-used first to make room.  On its slot the request
// copies its densities into the plan's resident input buffer, replays the
// plan's forward (captured once as a CUDA graph), copies the result out,
// and a host callback stamps the completion time and frees the slot and
// the plan.  Requests on different slots run concurrently on the device.
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <list>
#include <mutex>
#include <new>
#include <system_error>
#include <thread>
#include <unordered_map>
#include <vector>

#include "gf_internal.cuh"

namespace gf {
namespace {

using Clock = std::chrono::steady_clock;

struct Entry {
    uint64_t gid = 0;
    gf_plan_t plan = nullptr;
    size_t bytes = 0;           // admission estimate held against the budget
    bool busy = false;
    uint64_t last_use = 0;
    int rho_dtype = GF_DTYPE_F32;
    int64_t M = 0, nvox = 0;
    void *rho = nullptr;
    double *gz = nullptr, *g = nullptr;
    cudaGraphExec_t exec = nullptr;
    int kernels = 0;            // kernel nodes of the graph
};

struct Ticket {
    int64_t id = 0;
    gf_request req{};
    std::vector<double> xi, w, obs;   // copies of the request's host geometry
    size_t need = 0;                  // device bytes of a plan for it
    Clock::time_point t_submit, t_done;
    bool done = false;
    gf_status status = GF_OK;
    char msg[256] = "";
    Entry *entry = nullptr;
    int slot = -1;
    gf_server_s *srv = nullptr;
};

}  // namespace
}  // namespace gf

struct gf_server_s {
    gf_server_options opt{};
    std::vector<cudaStream_t> streams;
    cudaStream_t house = nullptr;      // stream for releasing evicted plans
    std::vector<int> free_slots;
    std::list<gf::Ticket *> queue;
    std::unordered_map<int64_t, gf::Ticket *> tickets;
    std::vector<gf::Entry *> entries;
    std::vector<double> lat_ms;        // latency of every completed request
    std::mutex mu;
    std::condition_variable cv;
    std::thread worker;
    bool stop = false;
    int64_t next_id = 1;
    uint64_t use_counter = 0;
    size_t resident = 0;
    int64_t submitted = 0, completed = 0, failed = 0, created = 0, evicted = 0, graphs = 0;
    gf::Clock::time_point t_first{}, t_last{};
    bool have_first = false;
};

namespace gf {
namespace {

size_t dtype_size(int dt) { return dt == GF_DTYPE_F64 ? 8 : 4; }

// Host callback enqueued after a request's last copy: stamps completion and
// frees its slot and plan.  Makes no CUDA call.
void CUDART_CB on_done(void *arg) {
    Ticket *t = static_cast<Ticket *>(arg);
    gf_server_s *s = t->srv;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        t->t_done = Clock::now();
        t->done = true;
        t->entry->busy = false;
        t->entry->last_use = ++s->use_counter;
        s->free_slots.push_back(t->slot);
        ++s->completed;
        s->t_last = t->t_done;
        s->lat_ms.push_back(std::chrono::duration<double, std::milli>(t->t_done - t->t_submit).count());
    }
    s->cv.notify_all();
}

void fail_ticket(gf_server_s *s, Ticket *t, gf_status st, const char *why) {
    t->status = st;
    snprintf(t->msg, sizeof(t->msg), "%s", why);
    t->t_done = Clock::now();
    t->done = true;
    ++s->failed;
}

// Release an idle entry (its last request has completed, so nothing on the
// device still uses its memory).  Called without the server lock held.
void release_entry(gf_server_s *s, Entry *e) {
    if (e->exec) cudaGraphExecDestroy(e->exec);
    if (e->rho) cudaFreeAsync(e->rho, s->house);
    if (e->gz) cudaFreeAsync(e->gz, s->house);
    if (e->g) cudaFreeAsync(e->g, s->house);
    if (e->plan) plan_release(e->plan);
    delete e;
}

gf_options plan_options(const gf_server_options &so) {
    gf_options o{};
    o.mode = GF_MODE_FMM;
    o.precision = so.precision;
    o.p = so.p;
    o.leaf_vox = so.leaf_vox;
    o.max_batch = 1;
    o.G = so.G;
    return o;
}

// Build a resident plan, its input/output buffers and (optionally) the CUDA
// graph of its forward, for the ticket's geometry.  Called without the
// server lock held; waits for its own slot stream only.
gf_status build_entry(gf_server_s *s, Ticket *t, cudaStream_t st, Entry **out) {
    const gf_request &r = t->req;
    Entry *e = new (std::nothrow) Entry();
    if (!e) return GF_ERR_OOM;
    e->gid = r.geometry_id;
    e->rho_dtype = r.rho_dtype;
    e->M = r.M;
    e->nvox = r.grid.n[0] * r.grid.n[1] * r.grid.n[2];
    e->bytes = t->need;
    const gf_options o = plan_options(s->opt);
    double *obs_dev = nullptr;
    cudaError_t ce = cudaMallocAsync((void **)&obs_dev, sizeof(double) * 3 * std::max<int64_t>(r.M, 1), st);
    if (ce == cudaSuccess && r.M > 0)
        ce = cudaMemcpyAsync(obs_dev, t->obs.data(), sizeof(double) * 3 * r.M, cudaMemcpyHostToDevice, st);
    if (ce != cudaSuccess) {
        cudaGetLastError();
        set_error("server: observer upload failed: %s", cudaGetErrorString(ce));
        delete e;
        return ce == cudaErrorMemoryAllocation ? GF_ERR_OOM : GF_ERR_CUDA;
    }
    gf_status rc = gf_plan_create(&r.grid, &r.quad, obs_dev, r.M, &o, st, &e->plan);
    cudaFreeAsync(obs_dev, st);
    if (rc != GF_OK) {
        cudaStreamSynchronize(st);
        delete e;
        return rc;
    }
    ce = cudaMallocAsync(&e->rho, dtype_size(e->rho_dtype) * std::max<int64_t>(e->nvox, 1), st);
    if (ce == cudaSuccess) ce = cudaMallocAsync((void **)&e->gz, sizeof(double) * std::max<int64_t>(e->M, 1), st);
    if (ce == cudaSuccess) ce = cudaMallocAsync((void **)&e->g, sizeof(double) * 3 * std::max<int64_t>(e->M, 1), st);
    // the buffers must exist before a graph refers to them
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    if (ce == cudaSuccess && s->opt.use_graphs && e->M > 0) {
        cudaGraph_t graph = nullptr;
        ce = cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed);
        if (ce == cudaSuccess) {
            const gf_status fr = gf_forward(e->plan, e->rho, e->rho_dtype, 1, e->g, e->gz, st);
            ce = cudaStreamEndCapture(st, &graph);
            if (ce == cudaSuccess && fr != GF_OK) ce = cudaErrorStreamCaptureInvalidated;
        }
        if (ce == cudaSuccess) {
            // the capture counted launches that did not run: count the
            // graph's kernels on each replay instead
            size_t nn = 0;
            ce = cudaGraphGetNodes(graph, nullptr, &nn);
            std::vector<cudaGraphNode_t> nodes(nn);
            if (ce == cudaSuccess && nn) ce = cudaGraphGetNodes(graph, nodes.data(), &nn);
            for (size_t i = 0; ce == cudaSuccess && i < nn; ++i) {
                cudaGraphNodeType ty;
                ce = cudaGraphNodeGetType(nodes[i], &ty);
                if (ty == cudaGraphNodeTypeKernel) ++e->kernels;
            }
            count_launch(-e->kernels);
        }
        if (ce == cudaSuccess) ce = cudaGraphInstantiate(&e->exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (ce == cudaSuccess) ce = cudaGraphUpload(e->exec, st);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    }
    if (ce != cudaSuccess) {
        cudaGetLastError();
        cudaStreamSynchronize(st);
        set_error("server: plan buffers or graph failed: %s", cudaGetErrorString(ce));
        release_entry(s, e);
        return ce == cudaErrorMemoryAllocation ? GF_ERR_OOM : GF_ERR_CUDA;
    }
    *out = e;
    return GF_OK;
}

// Continuous batching: repeatedly admit the oldest queued request that can
// run now (its plan resident and idle, or room for a new plan once idle
// plans are evicted), while a slot is free.
void scheduler(gf_server_s *s) {
    cudaSetDevice(s->opt.device);
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        s->cv.wait(lk, [&] { return s->stop || (!s->queue.empty() && !s->free_slots.empty()); });
        if (s->queue.empty()) {
            if (s->stop) break;
            continue;
        }
        Ticket *t = nullptr;
        Entry *e = nullptr;
        size_t idle_bytes = 0;
        for (Entry *x : s->entries)
            if (!x->busy) idle_bytes += x->bytes;
        for (auto it = s->queue.begin(); it != s->queue.end(); ++it) {
            Ticket *c = *it;
            Entry *hit = nullptr;
            bool busy_hit = false;
            for (Entry *x : s->entries)
                if (x->gid == c->req.geometry_id && x->rho_dtype == c->req.rho_dtype) {
                    if (!x->busy) {
                        hit = x;
                        break;
                    }
                    busy_hit = true;
                }
            if (hit || (!busy_hit && s->resident - idle_bytes + c->need <= s->opt.mem_budget)) {
                t = c;
                e = hit;
                s->queue.erase(it);
                break;
            }
        }
        if (!t) {   // nothing admissible until a request completes
            s->cv.wait(lk);
            continue;
        }
        const int slot = s->free_slots.back();
        s->free_slots.pop_back();
        cudaStream_t st = s->streams[slot];
        if (!e) {
            // evict idle plans, least recently used first, until it fits
            std::vector<Entry *> victims;
            while (s->resident + t->need > s->opt.mem_budget) {
                Entry *v = nullptr;
                for (Entry *x : s->entries)
                    if (!x->busy && (!v || x->last_use < v->last_use)) v = x;
                if (!v) break;
                s->entries.erase(std::find(s->entries.begin(), s->entries.end(), v));
                s->resident -= v->bytes;
                ++s->evicted;
                victims.push_back(v);
            }
            s->resident += t->need;   // reserved while the plan is built
            lk.unlock();
            for (Entry *v : victims) release_entry(s, v);
            Entry *ne = nullptr;
            const gf_status rc = build_entry(s, t, st, &ne);
            lk.lock();
            if (rc != GF_OK) {
                s->resident -= t->need;
                s->free_slots.push_back(slot);
                fail_ticket(s, t, rc, get_error());
                s->cv.notify_all();
                continue;
            }
            ++s->created;
            s->entries.push_back(ne);
            e = ne;
        }
        e->busy = true;
        t->entry = e;
        t->slot = slot;
        if (e->exec) ++s->graphs;
        lk.unlock();
        // the request on its slot: input copy, forward, output copies, stamp
        const gf_request &r = t->req;
        const cudaMemcpyKind in = r.on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        const cudaMemcpyKind outk = r.on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        cudaError_t ce = cudaMemcpyAsync(e->rho, r.rho_host, dtype_size(r.rho_dtype) * e->nvox, in, st);
        gf_status fr = GF_OK;
        if (ce == cudaSuccess && e->M > 0) {
            if (e->exec) {
                ce = cudaGraphLaunch(e->exec, st);
                if (ce == cudaSuccess) count_launch(e->kernels);
            }
            else
                fr = gf_forward(e->plan, e->rho, e->rho_dtype, 1, e->g, e->gz, st);
        }
        if (ce == cudaSuccess && fr == GF_OK && r.gz_host && e->M > 0)
            ce = cudaMemcpyAsync(r.gz_host, e->gz, sizeof(double) * e->M, outk, st);
        if (ce == cudaSuccess && fr == GF_OK && r.g_host && e->M > 0)
            ce = cudaMemcpyAsync(r.g_host, e->g, sizeof(double) * 3 * e->M, outk, st);
        if (ce == cudaSuccess && fr == GF_OK) ce = cudaLaunchHostFunc(st, on_done, t);
        if (ce != cudaSuccess || fr != GF_OK) {
            if (ce != cudaSuccess) set_error("server: %s", cudaGetErrorString(ce));
            cudaGetLastError();
            cudaStreamSynchronize(st);
            lk.lock();
            e->busy = false;
            s->free_slots.push_back(slot);
            fail_ticket(s, t, fr != GF_OK ? fr : GF_ERR_CUDA, get_error());
            s->cv.notify_all();
            continue;
        }
        lk.lock();
    }
}

}  // namespace
}  // namespace gf

using namespace gf;

extern "C" {

gf_status gf_server_create(const gf_server_options *opt, gf_server_t *out) {
    if (!opt || !out) {
        set_error("opt and server must be non-NULL");
        return GF_ERR_INVALID_ARG;
    }
    *out = nullptr;
    if (opt->max_slots < 1 || opt->max_slots > 64 || opt->p < 1 || opt->p > kMaxP ||
        (opt->precision != GF_PREC_FP64 && opt->precision != GF_PREC_MIXED)) {
        set_error("server options: need 1 <= max_slots <= 64, 1 <= p <= %d, a valid precision", kMaxP);
        return GF_ERR_INVALID_ARG;
    }
    GF_CUDA(cudaSetDevice(opt->device));
    gf_server_s *s = new (std::nothrow) gf_server_s();
    if (!s) {
        set_error("host allocation failed");
        return GF_ERR_OOM;
    }
    s->opt = *opt;
    if (s->opt.mem_budget == 0) {
        size_t fr = 0, tot = 0;
        cudaMemGetInfo(&fr, &tot);
        s->opt.mem_budget = (size_t)(0.7 * (double)fr);
    }
    for (int i = 0; i < opt->max_slots; ++i) {
        cudaStream_t st;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            set_error("stream creation failed");
            for (cudaStream_t x : s->streams) cudaStreamDestroy(x);
            delete s;
            return GF_ERR_CUDA;
        }
        s->streams.push_back(st);
        s->free_slots.push_back(opt->max_slots - 1 - i);
    }
    if (cudaStreamCreateWithFlags(&s->house, cudaStreamNonBlocking) != cudaSuccess) {
        set_error("stream creation failed");
        for (cudaStream_t x : s->streams) cudaStreamDestroy(x);
        delete s;
        return GF_ERR_CUDA;
    }
    try {
        s->worker = std::thread(scheduler, s);
    } catch (const std::system_error &) {
        set_error("cannot start the scheduler thread");
        for (cudaStream_t x : s->streams) cudaStreamDestroy(x);
        cudaStreamDestroy(s->house);
        delete s;
        return GF_ERR_CUDA;
    }
    *out = s;
    return GF_OK;
}

gf_status gf_server_submit(gf_server_t s, const gf_request *req, int64_t *ticket) {
    if (!s || !req || !ticket) {
        set_error("server, req and ticket must be non-NULL");
        return GF_ERR_INVALID_ARG;
    }
    if (!req->rho_host || (!req->gz_host && !req->g_host) || req->M < 0 || (req->M > 0 && !req->obs_host) ||
        req->quad.nq < 1 || req->quad.nq > kMaxQuad || !req->quad.xi || !req->quad.w ||
        (req->rho_dtype != GF_DTYPE_F32 && req->rho_dtype != GF_DTYPE_F64)) {
        set_error("request: need densities, an output, observers, a quadrature rule and a valid dtype");
        return GF_ERR_INVALID_ARG;
    }
    // footprint for admission: the plan plus its resident input and outputs;
    // gf_plan_bytes also validates the grid, the rule and M before anything
    // is copied
    const gf_options o = plan_options(s->opt);
    size_t b = 0;
    const gf_status rc = gf_plan_bytes(&req->grid, &req->quad, req->M, &o, &b);
    if (rc != GF_OK) return rc;
    const int64_t nvox = req->grid.n[0] * req->grid.n[1] * req->grid.n[2];
    const size_t need = b + dtype_size(req->rho_dtype) * nvox + 4 * sizeof(double) * req->M;
    if (need > s->opt.mem_budget) {
        set_error("request needs %zu device bytes, more than the server's budget of %zu", need,
                  s->opt.mem_budget);
        return GF_ERR_BUSY;
    }
    Ticket *t = new (std::nothrow) Ticket();
    if (!t) {
        set_error("host allocation failed");
        return GF_ERR_OOM;
    }
    try {
        t->xi.assign(req->quad.xi, req->quad.xi + 3 * req->quad.nq);
        t->w.assign(req->quad.w, req->quad.w + req->quad.nq);
        t->obs.assign(req->obs_host, req->obs_host + 3 * req->M);
    } catch (const std::bad_alloc &) {
        delete t;
        set_error("host allocation of the request's copies failed");
        return GF_ERR_OOM;
    }
    t->req = *req;
    t->req.quad.xi = t->xi.data();
    t->req.quad.w = t->w.data();
    t->req.obs_host = t->obs.data();
    t->srv = s;
    t->need = need;
    t->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        t->id = s->next_id++;
        s->tickets[t->id] = t;
        s->queue.push_back(t);
        ++s->submitted;
        if (!s->have_first) {
            s->t_first = t->t_submit;
            s->have_first = true;
        }
    }
    s->cv.notify_all();
    *ticket = t->id;
    return GF_OK;
}

gf_status gf_server_wait(gf_server_t s, int64_t ticket, double timeout_ms, double *latency_ms) {
    if (!s) {
        set_error("server is NULL");
        return GF_ERR_INVALID_ARG;
    }
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) {
        set_error("unknown ticket %lld", (long long)ticket);
        return GF_ERR_INVALID_ARG;
    }
    Ticket *t = it->second;
    auto ready = [&] { return t->done; };
    if (timeout_ms < 0)
        s->cv.wait(lk, ready);
    else if (!s->cv.wait_for(lk, std::chrono::duration<double, std::milli>(timeout_ms), ready)) {
        set_error("request %lld has not completed", (long long)ticket);
        return GF_ERR_TIMEOUT;
    }
    if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(t->t_done - t->t_submit).count();
    const gf_status rc = t->status;
    if (rc != GF_OK) set_error("request %lld failed: %s", (long long)ticket, t->msg);
    s->tickets.erase(it);
    delete t;
    return rc;
}

gf_status gf_server_stats_get(gf_server_t s, gf_server_stats *st) {
    if (!s || !st) {
        set_error("server and stats must be non-NULL");
        return GF_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    memset(st, 0, sizeof(*st));
    st->submitted = s->submitted;
    st->completed = s->completed;
    st->failed = s->failed;
    st->plans_created = s->created;
    st->plans_evicted = s->evicted;
    st->graph_launches = s->graphs;
    st->resident_bytes = s->resident;
    st->mem_budget = s->opt.mem_budget;
    std::vector<double> lat = s->lat_ms;
    if (!lat.empty()) {
        std::sort(lat.begin(), lat.end());
        auto pct = [&](double q) {
            const double pos = q * (lat.size() - 1);
            const size_t i = (size_t)pos;
            const double f = pos - i;
            return i + 1 < lat.size() ? lat[i] * (1 - f) + lat[i + 1] * f : lat[i];
        };
        st->p50_ms = pct(0.5);
        st->p99_ms = pct(0.99);
        double m = 0;
        for (double v : lat) m += v;
        st->mean_ms = m / lat.size();
    }
    if (s->have_first && s->completed > 0)
        st->busy_s = std::chrono::duration<double>(s->t_last - s->t_first).count();
    return GF_OK;
}

gf_status gf_server_destroy(gf_server_t s) {
    if (!s) return GF_OK;
    {
        std::unique_lock<std::mutex> lk(s->mu);
        s->cv.wait(lk, [&] {
            for (auto &kv : s->tickets)
                if (!kv.second->done) return false;
            return true;
        });
        s->stop = true;
    }
    s->cv.notify_all();
    if (s->worker.joinable()) s->worker.join();
    cudaSetDevice(s->opt.device);
    for (cudaStream_t st : s->streams) cudaStreamSynchronize(st);
    for (Entry *e : s->entries) release_entry(s, e);
    cudaStreamSynchronize(s->house);
    for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
    cudaStreamDestroy(s->house);
    for (auto &kv : s->tickets) delete kv.second;
    delete s;
    return GF_OK;
}

}  // extern "C"
