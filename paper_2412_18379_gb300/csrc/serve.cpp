// Serving: continuous batching of tracking requests over device-resident
// meshes, fields and predictor weights.
//
// A worker thread owns S slots (one CUDA stream each) and one device arena.
// Requests queue in arrival order; whenever a slot is free and the arena has
// room for the head request's buffers (its HBM footprint), the request is
// admitted: its inputs are copied in, its start rule and walk run on the
// slot's stream, its outputs are copied back and an event marks the end.
// Requests admitted while others are in flight run concurrently on the GPU
// (different streams). The worker polls the events, releases the memory of
// finished requests and admits the next ones. Latency is submit-to-finish.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "cnn.h"
#include "internal.h"

namespace cs {

using Clock = std::chrono::steady_clock;

// First-fit allocator over one device block (offsets aligned to 256 B).
struct Arena {
    char *base = nullptr;
    size_t size = 0, used = 0, peak = 0;
    std::map<size_t, size_t> free_;   // offset -> bytes
    bool alloc(size_t bytes, size_t &off) {
        bytes = (bytes + 255) / 256 * 256;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                off = it->first;
                const size_t rest = it->second - bytes;
                free_.erase(it);
                if (rest) free_[off + bytes] = rest;
                used += bytes;
                peak = std::max(peak, used);
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes) {
        bytes = (bytes + 255) / 256 * 256;
        used -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
};

struct Request {
    int64_t ticket = 0;
    cs_request r{};
    Mesh *mesh = nullptr;
    const float *grid = nullptr;   // CNN-SNS: the field's grid velocity, or null (resample u)
    Clock::time_point t_submit, t_admit, t_done;
    size_t off = 0, bytes = 0;
    cs_status result = CS_OK;
    bool done = false;
    int used_mode = 0;
    int in_flight = 0;             // requests on the GPU once it was admitted
};

struct Slot {
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    cudaEvent_t stage[5] = {};     // timed: admit, inputs in, predicted, walked, outputs out
    int32_t *counters = nullptr;   // walk cursors, see Scratch
    int parity = 0;
    Request *req = nullptr;
};

struct Server {
    cs_ctx *ctx = nullptr;
    Arena arena;
    std::vector<Slot> slots;
    std::thread worker;
    std::mutex mu;
    std::condition_variable cv, done_cv;
    std::deque<Request *> pending;
    std::map<int64_t, Request *> all;
    int64_t next_ticket = 1;
    bool stop = false;
    // the 3-D CUDA-core tile engine's workspace is shared: each of its
    // predictions waits for the one enqueued before it (worker thread only)
    cudaEvent_t pred3_ev = nullptr;
    bool pred3_any = false;
    // statistics
    std::vector<double> lat_ms;
    std::vector<cs_serve_record> trace;   // finished requests, in finishing order
    int64_t completed = 0, rejected = 0, particles = 0;
    int32_t active = 0, max_active = 0;
    Clock::time_point t_first, t_last;
    bool any = false;
};

namespace {

size_t request_bytes(const cs_request &r, const Mesh &m, bool cnn, bool own_grid) {
    const int d = m.d.dim;
    const size_t n = size_t(r.n);
    size_t b = 0;
    auto add = [&b](size_t x) { b += (x + 255) / 256 * 256; };
    add(n * d * 8);                  // x
    add(n * d * 8);                  // u
    if (r.start) add(n * 4);         // start
    add(n * 4);                      // host
    add(n * 4);                      // path
    add(n);                          // status
    if (cnn) add(size_t(m.d.n_pasg) * d * 4);        // predicted displacement grid
    if (own_grid) add(size_t(m.d.n_pasg) * d * 4);   // grid velocity of the request's u
    return b;
}

// Enqueue one admitted request on its slot's stream.
cs_status start_request(Server &S, Slot &sl, Request &q) {
    cs_ctx *ctx = S.ctx;
    const cs_request &r = q.r;
    Mesh &m = *q.mesh;
    const int d = m.d.dim;
    const size_t n = size_t(r.n);
    char *p = S.arena.base + q.off;
    auto take = [&p](size_t x) {
        char *o = p;
        p += (x + 255) / 256 * 256;
        return o;
    };
    double *x = reinterpret_cast<double *>(take(n * d * 8));
    double *u = reinterpret_cast<double *>(take(n * d * 8));
    int32_t *start = r.start ? reinterpret_cast<int32_t *>(take(n * 4)) : nullptr;
    int32_t *host = reinterpret_cast<int32_t *>(take(n * 4));
    int32_t *path = reinterpret_cast<int32_t *>(take(n * 4));
    uint8_t *status = reinterpret_cast<uint8_t *>(take(n));
    const bool cnn = q.used_mode == CS_CNN_SNS;
    float *dhat = cnn ? reinterpret_cast<float *>(take(size_t(m.d.n_pasg) * d * 4)) : nullptr;
    float *own_grid = cnn && !q.grid ? reinterpret_cast<float *>(take(size_t(m.d.n_pasg) * d * 4))
                                     : nullptr;
    cudaStream_t st = sl.st;
    cudaError_t e = cudaEventRecord(sl.stage[0], st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(x, r.x, n * d * 8, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(u, r.u, n * d * 8, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && start)
        e = cudaMemcpyAsync(start, r.start, n * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaEventRecord(sl.stage[1], st);
    if (e != cudaSuccess) return CS_ECUDA;
    if (cnn) {
        // the start predictor on the request's own field: the field's resident
        // grid velocity, or (particles = the mesh nodes) the request's u
        // resampled to the predictor grid
        const float *grid = q.grid;
        if (!grid) {
            ctx->launches += launch_resample(pred_view(m.d), m.interp_node, m.interp_w, u, own_grid,
                                             ctx->sm_count, st);
            grid = own_grid;
        }
        // the CUDA-core tile engine (3-D, engine 2) shares one workspace
        const bool shared_ws = d == 3 && ctx->engine == 2;
        if (shared_ws && S.pred3_any) cudaStreamWaitEvent(st, S.pred3_ev, 0);
        const cs_status rc = predict_grid(ctx, &m, grid, r.dt, dhat, st);
        if (rc) return rc;
        if (shared_ws) {
            cudaEventRecord(S.pred3_ev, st);
            S.pred3_any = true;
        }
    }
    if (cudaEventRecord(sl.stage[2], st) != cudaSuccess) return CS_ECUDA;
    TrackArgs a{};
    a.n = r.n;
    a.x = x;
    a.u = u;
    a.dt = r.dt;
    a.start_user = start;
    a.mode = q.used_mode;
    a.dhat = dhat;
    a.host = host;
    a.path = path;
    a.status = status;
    a.start_out = nullptr;
    Scratch sc;
    sc.counters = sl.counters;
    sc.parity = sl.parity;
    ctx->launches += launch_track(m.d, a, sc, ctx->sm_count, st, nullptr);
    sl.parity = sc.parity;
    e = cudaEventRecord(sl.stage[3], st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(r.host_out, host, n * 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(r.path_len_out, path, n * 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(r.status_out, status, n, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaEventRecord(sl.stage[4], st);
    if (e == cudaSuccess) e = cudaEventRecord(sl.ev, st);
    return e == cudaSuccess ? CS_OK : CS_ECUDA;
}

void finish(Server &S, Slot &sl, cs_status rc) {
    Request *q = sl.req;
    sl.req = nullptr;
    std::lock_guard<std::mutex> lock(S.mu);
    S.arena.release(q->off, q->bytes);
    q->t_done = Clock::now();
    q->result = rc;
    q->done = true;
    S.active -= 1;
    if (rc == CS_OK) {
        S.completed += 1;
        S.particles += q->r.n;
        S.lat_ms.push_back(std::chrono::duration<double, std::milli>(q->t_done - q->t_submit).count());
        S.t_last = q->t_done;
    }
    auto ms = [&S](Clock::time_point t) {
        return std::chrono::duration<double, std::milli>(t - S.t_first).count();
    };
    cs_serve_record rec{};
    rec.ticket = q->ticket;
    rec.n = q->r.n;
    rec.mesh_id = q->r.mesh_id;
    rec.mode_used = q->used_mode;
    rec.slot = int32_t(&sl - S.slots.data());
    rec.in_flight = q->in_flight;
    rec.result = rc;
    rec.dt = q->r.dt;
    if (rc == CS_OK) {
        double *span[4] = {&rec.h2d_ms, &rec.predict_ms, &rec.walk_ms, &rec.d2h_ms};
        for (int i = 0; i < 4; ++i) {
            float t = 0.f;
            if (cudaEventElapsedTime(&t, sl.stage[i], sl.stage[i + 1]) == cudaSuccess)
                *span[i] = double(t);
        }
        // no predictor ran: the gap between its two events is only the
        // stream's wait behind other slots' work
        if (q->used_mode != CS_CNN_SNS) rec.predict_ms = 0.0;
    }
    rec.submit_ms = ms(q->t_submit);
    rec.admit_ms = ms(q->t_admit);
    rec.done_ms = ms(q->t_done);
    S.trace.push_back(rec);
    S.done_cv.notify_all();
}

void worker_loop(Server *Sp) {
    Server &S = *Sp;
    cudaSetDevice(S.ctx->device);
    for (;;) {
        bool progress = false;
        // completions
        for (Slot &sl : S.slots) {
            if (!sl.req) continue;
            const cudaError_t e = cudaEventQuery(sl.ev);
            if (e == cudaSuccess) {
                finish(S, sl, CS_OK);
                progress = true;
            } else if (e != cudaErrorNotReady) {
                finish(S, sl, CS_ECUDA);
                progress = true;
            }
        }
        // admissions, in arrival order, while a slot and memory are free
        for (Slot &sl : S.slots) {
            if (sl.req) continue;
            Request *q = nullptr;
            {
                std::lock_guard<std::mutex> lock(S.mu);
                if (S.pending.empty()) break;
                Request *h = S.pending.front();
                size_t off = 0;
                if (!S.arena.alloc(h->bytes, off)) break;   // wait for memory
                h->off = off;
                S.pending.pop_front();
                S.active += 1;
                S.max_active = std::max(S.max_active, S.active);
                h->in_flight = S.active;
                q = h;
            }
            q->t_admit = Clock::now();
            sl.req = q;
            const cs_status rc = start_request(S, sl, *q);
            if (rc != CS_OK) finish(S, sl, rc);
            progress = true;
        }
        std::unique_lock<std::mutex> lock(S.mu);
        bool busy = false;
        for (const Slot &sl : S.slots) busy = busy || sl.req;
        if (S.stop && S.pending.empty() && !busy) break;
        if (!progress) {
            if (busy || !S.pending.empty())
                S.cv.wait_for(lock, std::chrono::microseconds(20));
            else
                S.cv.wait_for(lock, std::chrono::milliseconds(5));
        }
    }
}

cs_status sfail(cs_ctx *ctx, cs_status code, const std::string &msg) {
    ctx->err = msg;
    return code;
}

}  // namespace

void serve_release(cs_ctx *ctx) {
    Server *S = ctx->server;
    if (!S) return;
    {
        std::lock_guard<std::mutex> lock(S->mu);
        S->stop = true;
    }
    S->cv.notify_all();
    if (S->worker.joinable()) S->worker.join();
    for (Slot &sl : S->slots) {
        if (sl.st) cudaStreamDestroy(sl.st);
        if (sl.ev) cudaEventDestroy(sl.ev);
        for (cudaEvent_t &t : sl.stage)
            if (t) cudaEventDestroy(t);
        dfree(ctx, sl.counters);
    }
    if (S->pred3_ev) cudaEventDestroy(S->pred3_ev);
    dfree(ctx, S->arena.base);
    for (auto &kv : S->all) delete kv.second;
    delete S;
    ctx->server = nullptr;
}

}  // namespace cs

using namespace cs;

extern "C" {

cs_status cs_serve_start(cs_ctx *ctx, const cs_serve_cfg *cfg) {
    if (!ctx || !cfg || cfg->slots < 1 || cfg->slots > 64 || cfg->arena_bytes < 4096)
        return ctx ? sfail(ctx, CS_EINVAL, "cs_serve_start: bad configuration") : CS_EINVAL;
    if (ctx->server) return sfail(ctx, CS_EBUSY, "cs_serve_start: already serving");
    cudaSetDevice(ctx->device);
    Server *S = new (std::nothrow) Server();
    if (!S) return CS_ENOMEM;
    S->ctx = ctx;
    // the arena counts against the context's HBM budget like every other block
    {
        void *arena = nullptr;
        if (dmalloc(ctx, &arena, cfg->arena_bytes) != CS_OK) {
            delete S;
            return sfail(ctx, CS_ENOMEM, "cs_serve_start: arena of " +
                                             std::to_string(cfg->arena_bytes) +
                                             " bytes: " + ctx->err);
        }
        S->arena.base = static_cast<char *>(arena);
    }
    S->arena.size = cfg->arena_bytes;
    S->arena.free_[0] = cfg->arena_bytes;
    S->slots.resize(size_t(cfg->slots));
    for (Slot &sl : S->slots) {
        if (cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreate(&sl.stage[0]) != cudaSuccess || cudaEventCreate(&sl.stage[1]) != cudaSuccess ||
            cudaEventCreate(&sl.stage[2]) != cudaSuccess || cudaEventCreate(&sl.stage[3]) != cudaSuccess ||
            cudaEventCreate(&sl.stage[4]) != cudaSuccess ||
            dmalloc_n(ctx, &sl.counters, 16) != CS_OK ||
            cudaMemset(sl.counters, 0, 16 * sizeof(int32_t)) != cudaSuccess) {
            ctx->server = S;
            serve_release(ctx);
            return sfail(ctx, CS_ENOMEM, "cs_serve_start: slot resources");
        }
    }
    if (cudaEventCreateWithFlags(&S->pred3_ev, cudaEventDisableTiming) != cudaSuccess) {
        ctx->server = S;
        serve_release(ctx);
        return sfail(ctx, CS_ECUDA, "cs_serve_start: event");
    }
    // everything the requests' start predictors read, resident before any
    // request: packed 2-D weights, the 3-D tile workspace sized for every
    // mesh, the meshes' interpolation tables and the fields' grid velocities
    const cs_status prc = prepare_serving(ctx);
    if (prc != CS_OK) {
        const std::string msg = ctx->err;
        ctx->server = S;
        serve_release(ctx);
        return sfail(ctx, prc, "cs_serve_start: " + msg);
    }
    cudaDeviceSynchronize();
    ctx->server = S;
    S->worker = std::thread(worker_loop, S);
    return CS_OK;
}

cs_status cs_serve_submit(cs_ctx *ctx, const cs_request *req, int64_t *ticket) {
    if (!ctx || !req || !ticket) return CS_EINVAL;
    Server *S = ctx->server;
    if (!S) return sfail(ctx, CS_EINVAL, "cs_serve_submit: not serving");
    auto it = ctx->meshes.find(req->mesh_id);
    if (it == ctx->meshes.end()) return sfail(ctx, CS_ENOMESH, "cs_serve_submit: unknown mesh");
    Mesh *m = it->second;
    if (req->n < 1 || req->n >= (int64_t(1) << 31) - 1 || !req->x || !req->u || !req->host_out ||
        !req->path_len_out || !req->status_out)
        return sfail(ctx, CS_EINVAL, "cs_serve_submit: bad request");
    if (req->mode != CS_SNS && req->mode != CS_ASG_DIRECT && req->mode != CS_CNN_SNS)
        return sfail(ctx, CS_EINVAL, "cs_serve_submit: unknown mode");
    if (!req->start && req->n != m->d.n_v)
        return sfail(ctx, CS_EINVAL, "cs_serve_submit: start == NULL needs n == n_vertices");
    const Field *f = nullptr;
    if (req->field_id != CS_NO_FIELD) {
        auto fi = ctx->fields.find(req->field_id);
        if (fi == ctx->fields.end() || fi->second->mesh_id != req->mesh_id)
            return sfail(ctx, CS_EINVAL, "cs_serve_submit: field id is not a field of this mesh");
        f = fi->second;
    }
    // CNN-SNS where the grid predictor is resident and the request names its
    // field (or its particles are the mesh nodes, whose u is the field);
    // otherwise the request falls back to plain SNS
    int mode = req->mode;
    const bool nodes = !req->start && req->n == m->d.n_v;
    if (mode == CS_CNN_SNS && !(serving_predictor_ready(ctx, m) && (f || nodes)))
        mode = CS_SNS;
    Request *q = new (std::nothrow) Request();
    if (!q) return CS_ENOMEM;
    q->r = *req;
    q->mesh = m;
    q->used_mode = mode;
    q->grid = mode == CS_CNN_SNS && f ? f->grid_u : nullptr;
    q->bytes = request_bytes(*req, *m, mode == CS_CNN_SNS, mode == CS_CNN_SNS && !f);
    std::lock_guard<std::mutex> lock(S->mu);
    if (q->bytes > S->arena.size) {
        const size_t need = q->bytes;
        S->rejected += 1;
        delete q;
        return sfail(ctx, CS_ENOMEM, "cs_serve_submit: request needs " + std::to_string(need) +
                                         " bytes, more than the serving arena holds (" +
                                         std::to_string(S->arena.size) + ")");
    }
    q->ticket = S->next_ticket++;
    q->t_submit = Clock::now();
    if (!S->any) {
        S->t_first = q->t_submit;
        S->any = true;
    }
    S->pending.push_back(q);
    S->all[q->ticket] = q;
    *ticket = q->ticket;
    S->cv.notify_all();
    return CS_OK;
}

cs_status cs_serve_wait(cs_ctx *ctx, int64_t ticket, int32_t timeout_ms, cs_status *result,
                        int32_t *mode_used) {
    if (!ctx) return CS_EINVAL;
    Server *S = ctx->server;
    if (!S) return sfail(ctx, CS_EINVAL, "cs_serve_wait: not serving");
    std::unique_lock<std::mutex> lock(S->mu);
    auto it = S->all.find(ticket);
    if (it == S->all.end()) return sfail(ctx, CS_EINVAL, "cs_serve_wait: unknown ticket");
    Request *q = it->second;
    const bool ok = S->done_cv.wait_for(lock, std::chrono::milliseconds(std::max(0, timeout_ms)),
                                        [q] { return q->done; });
    if (!ok) return CS_EBUSY;   // still running
    if (result) *result = q->result;
    if (mode_used) *mode_used = q->used_mode;
    S->all.erase(it);
    delete q;
    return CS_OK;
}

cs_status cs_serve_report(cs_ctx *ctx, cs_serve_stats *out) {
    if (!ctx || !out) return CS_EINVAL;
    Server *S = ctx->server;
    if (!S) return sfail(ctx, CS_EINVAL, "cs_serve_report: not serving");
    std::lock_guard<std::mutex> lock(S->mu);
    std::memset(out, 0, sizeof(*out));
    out->completed = S->completed;
    out->rejected = S->rejected;
    out->particles = S->particles;
    out->peak_bytes = int64_t(S->arena.peak);
    out->max_concurrent = S->max_active;
    if (!S->lat_ms.empty()) {
        std::vector<double> v = S->lat_ms;
        std::sort(v.begin(), v.end());
        auto pct = [&v](double p) {
            const size_t i = size_t(std::min<double>(double(v.size() - 1),
                                                     std::ceil(p * double(v.size())) - 1));
            return v[i];
        };
        out->p50_ms = pct(0.50);
        out->p99_ms = pct(0.99);
        out->max_ms = v.back();
        double s = 0;
        for (double x : v) s += x;
        out->mean_ms = s / double(v.size());
        const double wall =
            std::chrono::duration<double>(S->t_last - S->t_first).count();
        out->wall_s = wall;
        out->particles_per_s = wall > 0 ? double(S->particles) / wall : 0.0;
    }
    return CS_OK;
}

cs_status cs_serve_trace(cs_ctx *ctx, int64_t cap, cs_serve_record *out, int64_t *count) {
    if (!ctx) return CS_EINVAL;
    Server *S = ctx->server;
    if (!S) return sfail(ctx, CS_EINVAL, "cs_serve_trace: not serving");
    if (!count || cap < 0) return sfail(ctx, CS_EINVAL, "cs_serve_trace: bad arguments");
    std::lock_guard<std::mutex> lock(S->mu);
    const int64_t held = int64_t(S->trace.size());
    if (!out) {
        *count = held;
        return CS_OK;
    }
    const int64_t k = std::min(cap, held);
    if (k > 0) std::memcpy(out, S->trace.data(), size_t(k) * sizeof(cs_serve_record));
    *count = k;
    return CS_OK;
}

cs_status cs_serve_stop(cs_ctx *ctx) {
    if (!ctx) return CS_EINVAL;
    if (!ctx->server) return CS_OK;
    serve_release(ctx);
    return CS_OK;
}

}  // extern "C"
