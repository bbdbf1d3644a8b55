// C ABI of the particle-location library (declared in include/cnnsns.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>

#include "internal.h"

namespace {

cs_status fail(cs_ctx *ctx, cs_status code, const std::string &msg) {
    if (ctx) ctx->err = msg;
    return code;
}

cs_status cuda_fail(cs_ctx *ctx, cudaError_t e, const char *what) {
    return fail(ctx, CS_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CS_CUDA(ctx, call)                                       \
    do {                                                         \
        cudaError_t e_ = (call);                                 \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
    } while (0)

template <class T>
cs_status dev_copy(cs_ctx *ctx, cs::Mesh *m, const T *src, size_t count, T **dst) {
    void *p = nullptr;
    const size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
    cs_status rc = cs::dmalloc(ctx, &p, bytes);
    if (rc) return rc;
    cudaError_t e = cudaSuccess;
    m->allocs.push_back(p);
    m->info.device_bytes += bytes;
    if (count && src) {
        e = cudaMemcpy(p, src, count * sizeof(T), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMemcpy of mesh data");
    } else if (count) {
        e = cudaMemset(p, 0xff, count * sizeof(T));
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMemset of mesh data");
    }
    *dst = static_cast<T *>(p);
    return CS_OK;
}

void free_mesh(cs_ctx *ctx, cs::Mesh *m) {
    for (void *p : m->allocs) cs::dfree(ctx, p);
    delete m;
}

void free_field(cs_ctx *ctx, cs::Field *f) {
    cs::dfree(ctx, f->u_nodal);
    cs::dfree(ctx, f->grid_u);
    delete f;
}

// release the fields of one mesh (mesh_id) or of every mesh (0)
void release_fields(cs_ctx *ctx, int32_t mesh_id) {
    for (auto it = ctx->fields.begin(); it != ctx->fields.end();) {
        if (mesh_id == 0 || it->second->mesh_id == mesh_id) {
            free_field(ctx, it->second);
            it = ctx->fields.erase(it);
        } else {
            ++it;
        }
    }
}

cs::Mesh *find_mesh(cs_ctx *ctx, int32_t id) {
    auto it = ctx->meshes.find(id);
    return it == ctx->meshes.end() ? nullptr : it->second;
}

// the three non-blocking streams and the events of cs_track_host (created once)
cs_status ensure_host_streams(cs_ctx *ctx) {
    if (ctx->hstream[0]) return CS_OK;
    for (auto &st : ctx->hstream)
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess)
            return fail(ctx, CS_ECUDA, "cs_track_host: stream creation failed");
    for (auto &ev : ctx->hevent)
        if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess)
            return fail(ctx, CS_ECUDA, "cs_track_host: event creation failed");
    return CS_OK;
}

cs_status ensure_scratch(cs_ctx *ctx) {
    cs::Scratch &s = ctx->scratch;
    if (!s.counters) {
        cs_status rc = cs::dmalloc_n(ctx, &s.counters, 16);
        if (rc == CS_OK) rc = cs::dmalloc_n(ctx, &s.stats, 16);
        if (rc) return rc;
        // the walk cursors start at zero; each walk then zeroes the other one
        if (cudaMemset(s.counters, 0, 16 * sizeof(int32_t)) != cudaSuccess)
            return fail(ctx, CS_ECUDA, "cudaMemset of scratch counters failed");
    }
    return CS_OK;
}

}  // namespace

cs_status cs::dmalloc(cs_ctx *ctx, void **p, size_t bytes) {
    *p = nullptr;
    {
        std::lock_guard<std::mutex> lock(ctx->hbm_mu);
        if (ctx->hbm_budget && ctx->hbm_used + bytes > ctx->hbm_budget)
            return fail(ctx, CS_ENOMEM, "device allocation of " + std::to_string(bytes) +
                                            " bytes would pass the context's HBM budget (" +
                                            std::to_string(ctx->hbm_used) + " of " +
                                            std::to_string(ctx->hbm_budget) + " bytes in use)");
        ctx->hbm_used += bytes;   // reserved while cudaMalloc runs
    }
    void *q = nullptr;
    if (cudaMalloc(&q, bytes) != cudaSuccess) {
        cudaGetLastError();
        std::lock_guard<std::mutex> lock(ctx->hbm_mu);
        ctx->hbm_used -= bytes;
        return fail(ctx, CS_ENOMEM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed");
    }
    std::lock_guard<std::mutex> lock(ctx->hbm_mu);
    ctx->hbm_blocks[q] = bytes;
    *p = q;
    return CS_OK;
}

void cs::dfree(cs_ctx *ctx, void *p) {
    if (!p) return;
    {
        std::lock_guard<std::mutex> lock(ctx->hbm_mu);
        auto it = ctx->hbm_blocks.find(p);
        if (it != ctx->hbm_blocks.end()) {
            ctx->hbm_used -= it->second;
            ctx->hbm_blocks.erase(it);
        }
    }
    cudaFree(p);
}

extern "C" {

cs_status cs_create(cs_ctx **out, int cuda_device, size_t hbm_budget_bytes) {
    if (!out) return CS_EINVAL;
    *out = nullptr;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || cuda_device < 0 || cuda_device >= count)
        return CS_EINVAL;
    cs_ctx *ctx = new (std::nothrow) cs_ctx();
    if (!ctx) return CS_ENOMEM;
    ctx->device = cuda_device;
    ctx->hbm_budget = hbm_budget_bytes;
    if (cudaSetDevice(cuda_device) != cudaSuccess ||
        cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, cuda_device) !=
            cudaSuccess) {
        delete ctx;
        return CS_ECUDA;
    }
    *out = ctx;
    return CS_OK;
}

void cs_destroy(cs_ctx *ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    cs::serve_release(ctx);
    release_fields(ctx, 0);
    for (auto &kv : ctx->meshes) free_mesh(ctx, kv.second);
    for (auto &p : ctx->pred) cs::predictor_release(ctx, p);
    cs::classifier_release_all(ctx);
    cs::dfree(ctx, ctx->dev_err);
    cs::dfree(ctx, ctx->hold_flag);
    cs::dfree(ctx, ctx->scratch.counters);
    cs::dfree(ctx, ctx->scratch.stats);
    cs::dfree(ctx, ctx->scratch.stage);
    for (const auto &r : ctx->prof.pending) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (cudaEvent_t e : ctx->prof.pool) cudaEventDestroy(e);
    for (cudaStream_t st : ctx->hstream)
        if (st) cudaStreamDestroy(st);
    for (cudaEvent_t e : ctx->hevent)
        if (e) cudaEventDestroy(e);
    delete ctx;
}

const char *cs_last_error(const cs_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int64_t cs_kernel_launches(const cs_ctx *ctx) { return ctx ? ctx->launches.load() : 0; }

cs_status cs_memory_usage(cs_ctx *ctx, size_t *used_bytes, size_t *budget_bytes) {
    if (!ctx) return CS_EINVAL;
    std::lock_guard<std::mutex> lock(ctx->hbm_mu);
    if (used_bytes) *used_bytes = ctx->hbm_used;
    if (budget_bytes) *budget_bytes = ctx->hbm_budget;
    return CS_OK;
}

cs_status cs_profile_enable(cs_ctx *ctx, int on) {
    if (!ctx) return CS_EINVAL;
    ctx->prof.on = on != 0;
    return CS_OK;
}

cs_status cs_profile_read(cs_ctx *ctx, cs_profile *out, int reset) {
    if (!ctx || !out) return CS_EINVAL;
    std::memset(out, 0, sizeof(*out));
    CS_CUDA(ctx, cudaSetDevice(ctx->device));
    for (const auto &r : ctx->prof.pending) {
        CS_CUDA(ctx, cudaEventSynchronize(r.b));
        float ms = 0.f;
        CS_CUDA(ctx, cudaEventElapsedTime(&ms, r.a, r.b));
        if (r.stage >= 0 && r.stage < 8) {
            out->launches[r.stage] += 1;
            out->ms[r.stage] += ms;
        }
    }
    if (reset) {
        for (const auto &r : ctx->prof.pending) {
            ctx->prof.pool.push_back(r.a);
            ctx->prof.pool.push_back(r.b);
        }
        ctx->prof.pending.clear();
    }
    return CS_OK;
}

cs_status cs_mesh_upload(cs_ctx *ctx, int dim, int64_t n_v, const double *xyz, int64_t n_e,
                         const int32_t *conn, const int32_t *asg_grid, int32_t *mesh_id_out) {
    if (!ctx) return CS_EINVAL;
    if ((dim != 2 && dim != 3) || n_v < dim + 1 || n_e < 1 || !xyz || !conn || !mesh_id_out)
        return fail(ctx, CS_EINVAL, "cs_mesh_upload: bad dim, size or null pointer");
    CS_CUDA(ctx, cudaSetDevice(ctx->device));
    cs::HostMesh H;
    std::string msg;
    cs_status rc;
    try {
        rc = cs::build_host_mesh(dim, n_v, xyz, n_e, conn, asg_grid, H, msg);
    } catch (const std::bad_alloc &) {
        return fail(ctx, CS_ENOMEM, "host allocation failed while building the mesh");
    }
    if (rc != CS_OK) return fail(ctx, rc, "cs_mesh_upload: " + msg);

    if (ctx->server) return fail(ctx, CS_EBUSY, "cs_mesh_upload: stop serving first");
    cs::Mesh *m = new (std::nothrow) cs::Mesh();
    if (!m) return fail(ctx, CS_ENOMEM, "host allocation failed");
    cs::DevMesh &d = m->d;
    d.dim = dim;
    d.n_v = n_v;
    d.n_e = n_e;
    const int nv = dim + 1;
    unsigned char *recw = nullptr, *recx = nullptr;
    int32_t *iperm = nullptr, *node = nullptr, *seed = nullptr, *bstart = nullptr,
            *bitems = nullptr, *cn = nullptr;
    double *cent = nullptr, *xyzd = nullptr;
    std::vector<int32_t> node_int(static_cast<size_t>(n_v));
    for (int64_t v = 0; v < n_v; ++v)
        node_int[v] = H.node_elem[v] < 0 ? -1 : H.iperm[H.node_elem[v]];
    if ((rc = dev_copy(ctx, m, H.recw.data(), H.recw.size(), &recw)) ||
        (rc = dev_copy(ctx, m, H.recx.data(), H.recx.size(), &recx)) ||
        (rc = dev_copy(ctx, m, H.iperm.data(), H.iperm.size(), &iperm)) ||
        (rc = dev_copy(ctx, m, node_int.data(), node_int.size(), &node)) ||
        (rc = dev_copy(ctx, m, H.bstart.data(), H.bstart.size(), &bstart)) ||
        (rc = dev_copy(ctx, m, H.bitems.data(), H.bitems.size(), &bitems)) ||
        (rc = dev_copy(ctx, m, H.conn.data(), H.conn.size(), &cn)) ||
        (rc = dev_copy(ctx, m, H.centroid.data(), H.centroid.size(), &cent)) ||
        (rc = dev_copy(ctx, m, xyz, size_t(n_v) * size_t(dim), &xyzd))) {
        free_mesh(ctx, m);
        return rc;
    }
    m->xyz = xyzd;
    int64_t n_asg = 1, n_b = 1;
    for (int k = 0; k < dim; ++k) {
        n_asg *= H.ga[k];
        n_b *= H.gb[k];
    }
    double *pool = nullptr;
    float *pool_f = nullptr;
    if ((rc = dev_copy<int32_t>(ctx, m, nullptr, size_t(n_asg), &seed)) ||
        (rc = dev_copy(ctx, m, H.pool.data(), H.pool.size(), &pool)) ||
        (rc = dev_copy(ctx, m, H.pool_f.data(), H.pool_f.size(), &pool_f))) {
        free_mesh(ctx, m);
        return rc;
    }
    d.recw = recw;
    d.recx = recx;
    d.conn = cn;
    d.centroid = cent;
    d.iperm = iperm;
    d.node_elem = node;
    d.seed = seed;
    d.pool = pool;
    d.pool_f = pool_f;
    d.bstart = bstart;
    d.bitems = bitems;
    for (int k = 0; k < 3; ++k) {
        d.lo[k] = k < dim ? H.lo[k] : 0;
        d.hi[k] = k < dim ? H.hi[k] : 0;
        d.ga[k] = k < dim ? H.ga[k] : 1;
        d.sa[k] = k < dim ? H.sa[k] : 1;
        d.gb[k] = k < dim ? H.gb[k] : 1;
        d.sb[k] = k < dim ? H.sb[k] : 1;
        d.lo_h[k] = static_cast<float>(d.lo[k]);
        d.lo_l[k] = static_cast<float>(d.lo[k] - static_cast<double>(d.lo_h[k]));
        d.inv_sa[k] = static_cast<float>(1.0 / d.sa[k]);
        d.inv_sb[k] = static_cast<float>(1.0 / d.sb[k]);
    }
    d.margin = H.margin;
    for (int k = 0; k < 3; ++k) {
        d.lo_m[k] = d.lo[k] - d.margin;
        d.hi_m[k] = d.hi[k] + d.margin;
    }
    d.tau = H.tau;
    d.cap = H.cap;
    d.n_asg = n_asg;
    d.n_bucket = n_b;
    // predictor grid: the ASG grid itself until cs_predictor_grid changes it
    d.pstride = 1;
    for (int k = 0; k < 3; ++k) {
        d.pga[k] = d.ga[k];
        d.psa[k] = d.sa[k];
        d.pinv_sa[k] = d.inv_sa[k];
        d.psa_f[k] = static_cast<float>(d.psa[k]);
    }
    d.n_pasg = n_asg;
    d.pseed = seed;

    ctx->launches += cs::launch_seed_grid(d, seed, ctx->sm_count, nullptr);
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
        free_mesh(ctx, m);
        return cuda_fail(ctx, e, "seed grid kernel");
    }

    cs_mesh_info &I = m->info;
    I.dim = dim;
    I.n_vertices = n_v;
    I.n_elements = n_e;
    I.pred_stride = 1;
    for (int k = 0; k < 3; ++k) {
        I.asg_grid[k] = d.ga[k];
        I.pred_grid[k] = d.pga[k];
        I.bucket_grid[k] = d.gb[k];
        I.lo[k] = d.lo[k];
        I.hi[k] = d.hi[k];
    }
    I.bucket_items = int64_t(H.bitems.size());
    I.tau = d.tau;
    I.step_cap = d.cap;
    I.record_bytes = dim == 2 ? int32_t(sizeof(cs::WalkRec2)) : int32_t(sizeof(cs::WalkRec3));
    m->node_elem_user = std::move(H.node_elem);
    (void)nv;
    const int32_t id = ctx->next_mesh++;
    ctx->meshes[id] = m;
    *mesh_id_out = id;
    return CS_OK;
}

cs_status cs_mesh_release(cs_ctx *ctx, int32_t mesh_id) {
    if (!ctx) return CS_EINVAL;
    cs::Mesh *m = find_mesh(ctx, mesh_id);
    if (!m) return fail(ctx, CS_ENOMESH, "cs_mesh_release: unknown mesh id");
    if (ctx->server) return fail(ctx, CS_EBUSY, "cs_mesh_release: stop serving first");
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    release_fields(ctx, mesh_id);
    ctx->meshes.erase(mesh_id);
    free_mesh(ctx, m);
    return CS_OK;
}

cs_status cs_field_upload(cs_ctx *ctx, int32_t mesh_id, const double *u_nodal,
                          int32_t *field_id_out) {
    if (!ctx) return CS_EINVAL;
    cs::Mesh *m = find_mesh(ctx, mesh_id);
    if (!m) return fail(ctx, CS_ENOMESH, "cs_field_upload: unknown mesh id");
    if (!u_nodal || !field_id_out) return fail(ctx, CS_EINVAL, "cs_field_upload: null pointer");
    if (ctx->server) return fail(ctx, CS_EBUSY, "cs_field_upload: stop serving first");
    CS_CUDA(ctx, cudaSetDevice(ctx->device));
    cs::Field *f = new (std::nothrow) cs::Field();
    if (!f) return fail(ctx, CS_ENOMEM, "host allocation failed");
    f->mesh_id = mesh_id;
    const size_t bytes = size_t(m->d.n_v) * m->d.dim * sizeof(double);
    cs_status rc = cs::dmalloc_n(ctx, &f->u_nodal, size_t(m->d.n_v) * m->d.dim);
    if (rc) {
        free_field(ctx, f);
        return rc;
    }
    // host or device source (cudaMemcpyDefault: unified addressing tells which)
    cudaError_t e = cudaMemcpy(f->u_nodal, u_nodal, bytes, cudaMemcpyDefault);
    if (e != cudaSuccess) {
        free_field(ctx, f);
        return cuda_fail(ctx, e, "cs_field_upload: copy of the nodal velocity");
    }
    const float *grid = nullptr;
    rc = cs::field_grid(ctx, m, f, nullptr, &grid);
    if (rc == CS_OK) {
        e = cudaDeviceSynchronize();
        if (e != cudaSuccess) rc = cuda_fail(ctx, e, "cs_field_upload: resample");
    }
    if (rc) {
        free_field(ctx, f);
        return rc;
    }
    const int32_t id = ctx->next_field++;
    ctx->fields[id] = f;
    *field_id_out = id;
    return CS_OK;
}

cs_status cs_field_release(cs_ctx *ctx, int32_t field_id) {
    if (!ctx) return CS_EINVAL;
    auto it = ctx->fields.find(field_id);
    if (it == ctx->fields.end()) return fail(ctx, CS_EINVAL, "cs_field_release: unknown field id");
    if (ctx->server) return fail(ctx, CS_EBUSY, "cs_field_release: stop serving first");
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    free_field(ctx, it->second);
    ctx->fields.erase(it);
    return CS_OK;
}

cs_status cs_mesh_query(cs_ctx *ctx, int32_t mesh_id, cs_mesh_info *info) {
    if (!ctx || !info) return CS_EINVAL;
    cs::Mesh *m = find_mesh(ctx, mesh_id);
    if (!m) return fail(ctx, CS_ENOMESH, "cs_mesh_query: unknown mesh id");
    *info = m->info;
    return CS_OK;
}

cs_status cs_node_start_elements(cs_ctx *ctx, int32_t mesh_id, int32_t *out) {
    if (!ctx || !out) return CS_EINVAL;
    cs::Mesh *m = find_mesh(ctx, mesh_id);
    if (!m) return fail(ctx, CS_ENOMESH, "cs_node_start_elements: unknown mesh id");
    std::memcpy(out, m->node_elem_user.data(), m->node_elem_user.size() * sizeof(int32_t));
    return CS_OK;
}

cs_status cs_seed_grid(cs_ctx *ctx, int32_t mesh_id, int32_t *out) {
    if (!ctx || !out) return CS_EINVAL;
    cs::Mesh *m = find_mesh(ctx, mesh_id);
    if (!m) return fail(ctx, CS_ENOMESH, "cs_seed_grid: unknown mesh id");
    CS_CUDA(ctx, cudaSetDevice(ctx->device));
    std::vector<int32_t> seed(static_cast<size_t>(m->d.n_asg)), iperm(static_cast<size_t>(m->d.n_e)),
        order(static_cast<size_t>(m->d.n_e));
    CS_CUDA(ctx, cudaMemcpy(seed.data(), m->d.seed, seed.size() * 4, cudaMemcpyDeviceToHost));
    CS_CUDA(ctx, cudaMemcpy(iperm.data(), m->d.iperm, iperm.size() * 4, cudaMemcpyDeviceToHost));
    for (size_t u = 0; u < iperm.size(); ++u) order[iperm[u]] = int32_t(u);
    for (size_t c = 0; c < seed.size(); ++c) out[c] = seed[c] < 0 ? -1 : order[seed[c]];
    return CS_OK;
}

cs_status cs_track(cs_ctx *ctx, int32_t mesh_id, int32_t field_id, int64_t n, const double *x,
                   const double *u, double dt, const int32_t *start, int mode, int32_t *host_out,
                   int32_t *path_len_out, uint8_t *status_out, int32_t *start_out,
                   void *stream) {
    if (!ctx) return CS_EINVAL;
    cs::Mesh *m = find_mesh(ctx, mesh_id);
    if (!m) return fail(ctx, CS_ENOMESH, "cs_track: unknown mesh id");
    if (mode != CS_SNS && mode != CS_ASG_DIRECT && mode != CS_CNN_SNS)
        return fail(ctx, CS_EINVAL, "cs_track: unknown mode");
    if (n < 0 || n >= (int64_t(1) << 31) - 1)
        return fail(ctx, CS_EINVAL, "cs_track: n is outside [0, 2^31 - 2]");
    const float *dhat = nullptr;
    if (mode == CS_CNN_SNS) {
        if (!ctx->pred[m->d.dim - 2].loaded)
            return fail(ctx, CS_ENOPRED, "cs_track: no predictor loaded");
        cs::Field *f = nullptr;
        if (field_id != CS_NO_FIELD) {
            auto it = ctx->fields.find(field_id);
            if (it == ctx->fields.end() || it->second->mesh_id != mesh_id)
                return fail(ctx, CS_EINVAL, "cs_track: field id is not a field of this mesh");
            f = it->second;
        }
        if (n == 0) return CS_OK;
        if (!x || !u) return fail(ctx, CS_EINVAL, "cs_track: null pointer");
        // without a field, the particles must be the mesh nodes: their
        // velocities are then the nodal field
        const bool nodes = !start && n == m->d.n_v;
        if (!f && !nodes)
            return fail(ctx, CS_EINVAL,
                        "cs_track: CNN-SNS needs a field id (cs_field_upload) unless the "
                        "particles are the mesh nodes");
        CS_CUDA(ctx, cudaSetDevice(ctx->device));
        cudaStream_t st = static_cast<cudaStream_t>(stream);
        const float *grid = nullptr;
        if (f) {
            cs_status rc = cs::field_grid(ctx, m, f, st, &grid);
            if (rc) return rc;
        }
        cs_status rc = cs::cnn_prepare(ctx, m, grid, f ? nullptr : u, dt, st, &dhat);
        if (rc) return rc;
    }
    return cs::cs_track_impl(ctx, m, n, x, u, dt, start, mode, dhat, host_out, path_len_out,
                             status_out, start_out, static_cast<cudaStream_t>(stream));
}

}  // extern "C"

cs_status cs::cs_track_impl(cs_ctx *ctx, cs::Mesh *m, int64_t n, const double *x,
                            const double *u, double dt, const int32_t *start, int mode,
                            const float *dhat, int32_t *host_out, int32_t *path_len_out,
                            uint8_t *status_out, int32_t *start_out, cudaStream_t stream) {
    if (n < 0 || n >= (int64_t(1) << 31) - 1)
        return fail(ctx, CS_EINVAL, "cs_track: n is outside [0, 2^31 - 2]");
    if (n == 0) return CS_OK;
    if (!x || !u || !host_out || !path_len_out || !status_out)
        return fail(ctx, CS_EINVAL, "cs_track: null pointer");
    if (!start && n != m->d.n_v)
        return fail(ctx, CS_EINVAL, "cs_track: start == NULL needs n == n_vertices");
    CS_CUDA(ctx, cudaSetDevice(ctx->device));
    cs_status rc = ensure_scratch(ctx);
    if (rc) return rc;
    cs::TrackArgs a{};
    a.n = n;
    a.x = x;
    a.u = u;
    a.dt = dt;
    a.start_user = start;
    a.mode = mode;
    a.dhat = dhat;
    a.host = host_out;
    a.path = path_len_out;
    a.status = status_out;
    a.start_out = start_out;
    ctx->launches += cs::launch_track(m->d, a, ctx->scratch, ctx->sm_count, stream, &ctx->prof);
    CS_CUDA(ctx, cudaGetLastError());
    return CS_OK;
}

namespace {

// The host-memory tracking call: x either in host memory (copied in by
// chunks) or, with x_dev, already on the device (the mesh's vertices).
cs_status track_host_impl(cs_ctx *ctx, const std::string &name, cs::Mesh *m, int32_t mesh_id,
                          int32_t field_id, int64_t n, const double *x, const double *x_dev,
                          const double *u, double dt, const int32_t *start, int mode,
                          int32_t *host_out, int32_t *path_len_out, uint8_t *status_out,
                          int32_t *start_out) {
    if (n < 0 || n >= (int64_t(1) << 31) - 1)
        return fail(ctx, CS_EINVAL, name + ": n is outside [0, 2^31 - 2]");
    if (mode != CS_SNS && mode != CS_ASG_DIRECT && mode != CS_CNN_SNS)
        return fail(ctx, CS_EINVAL, name + ": bad mode");
    cs::Field *f = nullptr;
    if (mode == CS_CNN_SNS) {
        if (!ctx->pred[m->d.dim - 2].loaded)
            return fail(ctx, CS_ENOPRED, name + ": no predictor loaded");
        if (field_id != CS_NO_FIELD) {
            auto it = ctx->fields.find(field_id);
            if (it == ctx->fields.end() || it->second->mesh_id != mesh_id)
                return fail(ctx, CS_EINVAL, name + ": field id is not a field of this mesh");
            f = it->second;
        }
    }
    if (n == 0) return CS_OK;
    if ((!x && !x_dev) || !u || !host_out || !path_len_out || !status_out)
        return fail(ctx, CS_EINVAL, name + ": null pointer");
    if (!start && n != m->d.n_v)
        return fail(ctx, CS_EINVAL, name + ": start == NULL needs n == n_vertices");
    // CNN-SNS without a field predicts from the call's own nodal velocity:
    // all of u has to be on the device before the predictor runs
    const bool whole_u = mode == CS_CNN_SNS && !f;
    if (whole_u && start)
        return fail(ctx, CS_EINVAL,
                    name + ": CNN-SNS needs a field id (cs_field_upload) unless the "
                           "particles are the mesh nodes");
    CS_CUDA(ctx, cudaSetDevice(ctx->device));
    cs_status rc = ensure_scratch(ctx);
    if (rc) return rc;
    const int dim = m->d.dim;
    const size_t in_b = size_t(n) * dim * sizeof(double);
    const size_t total = 2 * in_b + size_t(n) * (4 + 4 + 4 + 4 + 1) + 256;
    cs::Scratch &S = ctx->scratch;
    if (S.stage_cap < total) {
        cs::dfree(ctx, S.stage);
        S.stage = nullptr;
        S.stage_cap = 0;
        rc = cs::dmalloc_n(ctx, &S.stage, total);
        if (rc) return rc;
        S.stage_cap = total;
    }
    // node particles walk from their node's element, given explicitly per chunk
    if (!start && !m->node_start_user) {
        rc = dev_copy(ctx, m, m->node_elem_user.data(), m->node_elem_user.size(),
                      &m->node_start_user);
        if (rc) return rc;
    }
    if ((rc = ensure_host_streams(ctx))) return rc;
    char *buf = S.stage;
    const double *dx = x_dev ? x_dev : reinterpret_cast<const double *>(buf);
    double *du = reinterpret_cast<double *>(buf + in_b);
    int32_t *ds = reinterpret_cast<int32_t *>(buf + 2 * in_b);
    int32_t *dh = ds + n, *dp = dh + n, *dso = dp + n;
    uint8_t *dst = reinterpret_cast<uint8_t *>(dso + n);
    cudaStream_t s_in = ctx->hstream[0], s_cmp = ctx->hstream[1], s_out = ctx->hstream[2];
    cudaEvent_t *ev = ctx->hevent;
    // Chunks of the particle range, pipelined over three streams: the copies
    // in of chunk i + 1 and the copies out of chunk i - 1 overlap the walk of
    // chunk i (the two copy directions run at once).
    const int K = int(std::min<int64_t>(cs::kHostChunks, std::max<int64_t>(1, n / (int64_t(1) << 18))));
    cudaError_t e = cudaEventRecord(ev[0], nullptr);   // after the caller's earlier work
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s_in, ev[0], 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s_cmp, ev[0], 0);
    // the whole velocity goes on the compute stream itself: the predictor
    // that reads it follows with no hop between streams
    if (e == cudaSuccess && whole_u) e = cudaMemcpyAsync(du, u, in_b, cudaMemcpyHostToDevice, s_cmp);
    for (int i = 0; i < K && e == cudaSuccess; ++i) {
        const int64_t lo = n * i / K, hi = n * (i + 1) / K, c = hi - lo;
        if (!x_dev)
            e = cudaMemcpyAsync(reinterpret_cast<double *>(buf) + lo * dim, x + lo * dim,
                                size_t(c) * dim * 8, cudaMemcpyHostToDevice, s_in);
        if (e == cudaSuccess && !whole_u)
            e = cudaMemcpyAsync(du + lo * dim, u + lo * dim, size_t(c) * dim * 8, cudaMemcpyHostToDevice,
                                s_in);
        if (e == cudaSuccess && start)
            e = cudaMemcpyAsync(ds + lo, start + lo, size_t(c) * 4, cudaMemcpyHostToDevice, s_in);
        if (e == cudaSuccess) e = cudaEventRecord(ev[2 + i], s_in);
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, (name + ": copy in").c_str());
    const float *dhat = nullptr;
    if (mode == CS_CNN_SNS) {
        const float *grid = nullptr;
        if (f && (rc = cs::field_grid(ctx, m, f, s_cmp, &grid))) return rc;
        if ((rc = cs::cnn_prepare(ctx, m, grid, f ? nullptr : du, dt, s_cmp, &dhat))) return rc;
    }
    for (int i = 0; i < K && rc == CS_OK; ++i) {
        const int64_t lo = n * i / K, hi = n * (i + 1) / K, c = hi - lo;
        e = cudaStreamWaitEvent(s_cmp, ev[2 + i], 0);
        if (e != cudaSuccess) {
            rc = cuda_fail(ctx, e, (name + ": event wait").c_str());
            break;
        }
        const int32_t *st0 = start ? ds + lo : m->node_start_user + lo;
        rc = cs::cs_track_impl(ctx, m, c, dx + lo * dim, du + lo * dim, dt, st0, mode, dhat,
                               dh + lo, dp + lo, dst + lo, start_out ? dso + lo : nullptr, s_cmp);
        if (rc == CS_OK) {
            e = cudaEventRecord(ev[2 + K + i], s_cmp);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(s_out, ev[2 + K + i], 0);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(host_out + lo, dh + lo, size_t(c) * 4, cudaMemcpyDeviceToHost, s_out);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(path_len_out + lo, dp + lo, size_t(c) * 4, cudaMemcpyDeviceToHost,
                                    s_out);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(status_out + lo, dst + lo, size_t(c), cudaMemcpyDeviceToHost, s_out);
            if (e == cudaSuccess && start_out)
                e = cudaMemcpyAsync(start_out + lo, dso + lo, size_t(c) * 4, cudaMemcpyDeviceToHost,
                                    s_out);
            if (e != cudaSuccess) rc = cuda_fail(ctx, e, (name + ": copy out").c_str());
        }
    }
    // every stream drained before return (also after a failed launch)
    const cudaError_t e1 = cudaStreamSynchronize(s_in), e2 = cudaStreamSynchronize(s_cmp),
                      e3 = cudaStreamSynchronize(s_out);
    if (rc) return rc;
    e = e1 != cudaSuccess ? e1 : e2 != cudaSuccess ? e2 : e3;
    if (e != cudaSuccess) return cuda_fail(ctx, e, name.c_str());
    return CS_OK;
}

}  // namespace

extern "C" {

cs_status cs_track_host(cs_ctx *ctx, int32_t mesh_id, int32_t field_id, int64_t n,
                        const double *x, const double *u, double dt, const int32_t *start,
                        int mode, int32_t *host_out, int32_t *path_len_out, uint8_t *status_out,
                        int32_t *start_out) {
    if (!ctx) return CS_EINVAL;
    cs::Mesh *m = find_mesh(ctx, mesh_id);
    if (!m) return fail(ctx, CS_ENOMESH, "cs_track_host: unknown mesh id");
    return track_host_impl(ctx, "cs_track_host", m, mesh_id, field_id, n, x, nullptr, u, dt, start,
                           mode, host_out, path_len_out, status_out, start_out);
}

cs_status cs_track_nodes_host(cs_ctx *ctx, int32_t mesh_id, int32_t field_id, const double *u,
                              double dt, int mode, int32_t *host_out, int32_t *path_len_out,
                              uint8_t *status_out, int32_t *start_out) {
    if (!ctx) return CS_EINVAL;
    cs::Mesh *m = find_mesh(ctx, mesh_id);
    if (!m) return fail(ctx, CS_ENOMESH, "cs_track_nodes_host: unknown mesh id");
    return track_host_impl(ctx, "cs_track_nodes_host", m, mesh_id, field_id, m->d.n_v, nullptr,
                           m->xyz, u, dt, nullptr, mode, host_out, path_len_out, status_out,
                           start_out);
}

cs_status cs_track_stats(cs_ctx *ctx, int64_t n, const int32_t *path_len, const uint8_t *status,
                         int64_t out[6], void *stream) {
    if (!ctx || !out || n < 0 || (n > 0 && (!path_len || !status))) return CS_EINVAL;
    CS_CUDA(ctx, cudaSetDevice(ctx->device));
    cs_status rc = ensure_scratch(ctx);
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    ctx->launches += cs::launch_stats(n, path_len, status, ctx->scratch.stats, ctx->sm_count, st);
    CS_CUDA(ctx, cudaMemcpyAsync(out, ctx->scratch.stats, 6 * sizeof(int64_t),
                                 cudaMemcpyDeviceToHost, st));
    CS_CUDA(ctx, cudaStreamSynchronize(st));
    return CS_OK;
}

cs_status cs_track_error(cs_ctx *ctx, int32_t mesh_id, int64_t n, const double *x,
                         const double *u, double dt, const int32_t *start, const int32_t *host,
                         const float *dhat, cs_error_stats *out, void *stream) {
    if (!ctx) return CS_EINVAL;
    cs::Mesh *m = find_mesh(ctx, mesh_id);
    if (!m) return fail(ctx, CS_ENOMESH, "cs_track_error: unknown mesh id");
    if (!out || n < 0 || (n > 0 && (!host || (dhat && (!x || !u)))))
        return fail(ctx, CS_EINVAL, "cs_track_error: bad arguments");
    CS_CUDA(ctx, cudaSetDevice(ctx->device));
    cs_status rc = ensure_scratch(ctx);
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    double *sums = reinterpret_cast<double *>(ctx->scratch.stats + 8);
    unsigned long long *cnt = reinterpret_cast<unsigned long long *>(ctx->scratch.stats + 12);
    ctx->launches += cs::launch_error_stats(m->d, n, start, host, x, u, dt, dhat, sums, cnt,
                                            ctx->sm_count, st);
    double h[4];
    unsigned long long c[2];
    CS_CUDA(ctx, cudaMemcpyAsync(h, sums, sizeof(h), cudaMemcpyDeviceToHost, st));
    CS_CUDA(ctx, cudaMemcpyAsync(c, cnt, sizeof(c), cudaMemcpyDeviceToHost, st));
    CS_CUDA(ctx, cudaStreamSynchronize(st));
    out->n_err = int64_t(c[0]);
    out->err_sum = h[0];
    out->err_max = h[1];
    out->n_disp = int64_t(c[1]);
    out->disp_sum = h[2];
    out->disp_max = h[3];
    return CS_OK;
}

}  // extern "C"
