// Internal types of the particle-location library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <map>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "cnnsns.h"

namespace cs {

struct Server;   // serve.cpp

// Every element has two records.
//
// The walk record (read at every walk step) carries what the FP32 filter
// needs: the origin vertex v0 split into float hi + lo parts, the inverse-
// affine matrix M rounded to float, the neighbour across face i (internal id,
// -1 on the boundary) and the caller's id of the element. 48 bytes (2-D, two
// 32-byte sectors) / 80 bytes (3-D, three sectors).
//
// The exact record holds v0 and M in FP64 (row k of M gives
// lambda_{k+1} = M[k] . (x_p - v0)); it is read only when the FP32 filter
// cannot certify a decision, and by the exact search.
struct alignas(16) WalkRec2 {
    float vh[2], vl[2];
    float m[4];
    int32_t nbr[3];
    int32_t uid;
};
struct alignas(16) WalkRec3 {
    float vh[3], vl[3];
    float m[9];
    int32_t uid;
    int32_t nbr[4];
};
struct alignas(16) ExactRec2 {
    double v0[2];
    double m[4];
};
struct alignas(16) ExactRec3 {
    double v0[3];
    double m[9];
};
static_assert(sizeof(WalkRec2) == 48, "WalkRec2 is 48 bytes");
static_assert(sizeof(WalkRec3) == 80, "WalkRec3 is 80 bytes");
static_assert(sizeof(ExactRec2) == 48, "ExactRec2 is 48 bytes");
static_assert(sizeof(ExactRec3) == 96, "ExactRec3 is 96 bytes");

// Everything a kernel needs to know about a resident mesh (passed by value).
struct DevMesh {
    int32_t dim;
    int64_t n_v, n_e;
    const void *recw;         // WalkRec2 / WalkRec3 [n_e], Hilbert (internal) order
    const void *recx;         // ExactRec2 / ExactRec3 [n_e], same order
    const int32_t *conn;      // [n_e][dim+1] vertex ids, internal order
    const double *centroid;   // [n_e][dim], internal order
    const int32_t *iperm;     // user id -> internal id
    const int32_t *node_elem; // [n_v] internal id of the plain-SNS start
    const int32_t *seed;      // [n_asg] internal id of the host of each cell centre, or -1
    const double *pool;       // [n_asg][dim] mean element centroid per ASG cell, NaN if none
    const float *pool_f;      // [n_asg][dim][2] the same as float hi + lo (NaN hi if none)
    const int32_t *bstart;    // [n_bucket + 1] offsets into bitems
    const int32_t *bitems;    // internal ids listed per bucket cell
    double lo[3], hi[3];
    int32_t ga[3];            // ASG cells per axis
    double sa[3];             // ASG cell size (hi - lo) / ga
    int32_t gb[3];            // bucket cells per axis
    double sb[3];
    float lo_h[3], lo_l[3];   // lo split into float hi + lo (FP32 cell filter)
    float inv_sa[3];          // 1 / sa rounded to float
    float inv_sb[3];          // 1 / sb rounded to float
    double margin;            // bucket boxes are grown by this much
    double lo_m[3], hi_m[3];  // lo - margin, hi + margin: no host beyond these
    double tau;               // canonicalisation threshold
    int32_t cap;              // step cap
    int64_t n_asg, n_bucket;
    // predictor grid: cells of pstride^dim ASG cells (pstride odd), aligned at
    // lo; a point past the last whole cell belongs to the last one
    int32_t pstride;          // 1: the ASG grid itself
    int32_t pga[3];           // ga / pstride (at least 1)
    double psa[3];            // sa * pstride
    float pinv_sa[3];         // 1 / psa rounded to float
    float psa_f[3];           // psa rounded to float
    int64_t n_pasg;
    const int32_t *pseed;     // [n_pasg] host of each cell centre (the seed of its middle ASG cell)
};

// The mesh as the start predictor sees it: the predictor grid in place of the
// ASG grid (cell geometry, cell count and centre hosts); everything else the same.
inline DevMesh pred_view(const DevMesh &d) {
    DevMesh v = d;
    for (int k = 0; k < 3; ++k) {
        v.ga[k] = d.pga[k];
        v.sa[k] = d.psa[k];
        v.inv_sa[k] = d.pinv_sa[k];
    }
    v.n_asg = d.n_pasg;
    v.seed = d.pseed;
    return v;
}

struct Mesh {
    DevMesh d{};
    cs_mesh_info info{};
    std::vector<void *> allocs;
    std::vector<int32_t> node_elem_user;  // host copy, user ids
    float *grid_u = nullptr;              // [n_pasg][dim] stored grid velocity (CNN input)
    float *grid_dhat = nullptr;           // [n_pasg][dim] predicted displacement
    int32_t *interp_node = nullptr;       // [n_pasg][dim+1] P1 interpolation at cell centres:
    float *interp_w = nullptr;            //   host vertices and weights (static per mesh)
    bool grid_u_valid = false;
    int32_t pgrid_version = 0;            // bumped by every cs_predictor_grid
    int32_t *node_start_user = nullptr;   // [n_v] plain starts as user ids (cs_track_host)
    double *xyz = nullptr;                // [n_v][dim] the uploaded vertices, user order
};

// A velocity field of a mesh (cs_field_upload): the nodal velocity, kept for
// re-resampling, and its grid velocity on the mesh's current predictor grid.
struct Field {
    int32_t mesh_id = 0;
    double *u_nodal = nullptr;            // [n_v][dim]
    float *grid_u = nullptr;              // [n_pasg][dim]
    int32_t grid_version = -1;            // Mesh::pgrid_version grid_u was built for
};

// The start predictor of one dimension: FP32 master weights, gradients, Adam
// state, and the activations of the last forward pass (sized for `cap`).
struct Predictor {
    bool loaded = false;
    int dim = 0;
    int64_t n = 0;
    float *w = nullptr;
    float *g = nullptr;
    float *m = nullptr;
    float *v = nullptr;
    float *loss = nullptr;
    int64_t t = 0;
    int64_t cap = 0;
    std::vector<float *> col, z, y;
    float *z5 = nullptr, *a5 = nullptr, *out = nullptr, *gout = nullptr;
    float *dcol = nullptr, *dy0 = nullptr, *dy1 = nullptr, *da5 = nullptr, *win = nullptr,
          *tgt = nullptr;
    int64_t *idx = nullptr;
    float *splitk = nullptr;     // partial products of the GEMMs' K splits
    int64_t splitk_n = 0;
    std::vector<float *> tiles;  // workspace of the tile engine (fully convolutional)
    std::vector<int64_t> tiles_cap;   // floats held by each buffer of `tiles`
    uint8_t *packed = nullptr;   // weights in the tensor-core kernel's layout
    bool packed_dirty = true;
};

// The classifier start predictor of one dimension (classifier.cpp).
struct Classifier;

// chunks of the particle range that cs_track_host pipelines (at most)
constexpr int kHostChunks = 4;

// Device scratch owned by a context.
struct Scratch {
    int32_t *counters = nullptr;   // [0], [1] work cursors of alternate walks (16 reserved)
    int parity = 0;                // cursor of the next walk; that walk zeroes the other
    int64_t *stats = nullptr;      // [8]
    char *stage = nullptr;         // device staging of cs_track_host
    size_t stage_cap = 0;
};

// Per-call arguments of the track kernels.
struct TrackArgs {
    int64_t n;
    const double *x;
    const double *u;
    double dt;
    const int32_t *start_user;   // may be null: node_elem[p]
    int32_t mode;
    const float *dhat;           // CNN-SNS: [n_asg][dim] displacement in ASG cell units
    int32_t *host;
    int32_t *path;
    uint8_t *status;
    int32_t *start_out;          // may be null
};

// host-side preprocessing (mesh_build.cpp); returns CS_OK or an error code and
// fills `msg`.
struct HostMesh {
    int dim = 0;
    int64_t n_v = 0, n_e = 0;
    std::vector<int32_t> order;      // internal -> user
    std::vector<int32_t> iperm;      // user -> internal
    std::vector<unsigned char> recw; // walk records, internal order
    std::vector<unsigned char> recx; // exact records, internal order
    std::vector<int32_t> conn;       // internal order
    std::vector<double> centroid;    // internal order
    std::vector<double> pool;        // [n_asg][dim] mean centroid per ASG cell, NaN if none
    std::vector<float> pool_f;       // [n_asg][dim][2] the same as float hi, lo
    std::vector<int32_t> node_elem;  // user ids
    std::vector<int32_t> bstart, bitems;
    double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    int32_t ga[3] = {1, 1, 1}, gb[3] = {1, 1, 1};
    double sa[3] = {1, 1, 1}, sb[3] = {1, 1, 1};
    double margin = 0, tau = 0;
    int32_t cap = 0;
};
cs_status build_host_mesh(int dim, int64_t n_v, const double *xyz, int64_t n_e,
                          const int32_t *conn, const int32_t *asg_grid, HostMesh &out,
                          std::string &msg);

// Event pairs recorded around kernels when profiling is on.
struct Profiler {
    bool on = false;
    struct Rec { int stage; cudaEvent_t a, b; };
    std::vector<Rec> pending;
    std::vector<cudaEvent_t> pool;
    cudaEvent_t get() {
        if (!pool.empty()) {
            cudaEvent_t e = pool.back();
            pool.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        return e;
    }
    // record a start event for `stage` (returns index) and later its end
    int begin(int stage, cudaStream_t st) {
        if (!on) return -1;
        Rec r{stage, get(), get()};
        cudaEventRecord(r.a, st);
        pending.push_back(r);
        return int(pending.size()) - 1;
    }
    void end(int idx, cudaStream_t st) {
        if (idx >= 0) cudaEventRecord(pending[idx].b, st);
    }
};

// kernel launchers (walk.cu); each returns the number of kernels launched
int launch_track(const DevMesh &m, const TrackArgs &a, Scratch &s, int sm_count,
                 cudaStream_t st, Profiler *prof = nullptr);
int launch_seed_grid(const DevMesh &m, int32_t *seed, int sm_count, cudaStream_t st);
int launch_stats(int64_t n, const int32_t *path, const uint8_t *status, int64_t *out,
                 int sm_count, cudaStream_t st);
int launch_error_stats(const DevMesh &m, int64_t n, const int32_t *start, const int32_t *host,
                       const double *x, const double *u, double dt, const float *dhat,
                       double *out, unsigned long long *cnt, int sm_count, cudaStream_t st);

}  // namespace cs

struct cs_ctx {
    int device = 0;
    int sm_count = 0;
    std::string err;
    std::map<int32_t, cs::Mesh *> meshes;
    int32_t next_mesh = 1;
    std::map<int32_t, cs::Field *> fields;
    int32_t next_field = 1;
    // device memory held by the context: every allocation goes through
    // cs::dmalloc, which refuses one that would pass the budget (0 = none)
    size_t hbm_budget = 0;
    size_t hbm_used = 0;
    std::unordered_map<void *, size_t> hbm_blocks;
    std::mutex hbm_mu;
    cs::Scratch scratch;
    cs::Profiler prof;
    cs::Predictor pred[2];   // dim 2, dim 3
    cs::Classifier *cls[2] = {nullptr, nullptr};   // classifier predictors, dim 2, 3
    int engine = 1;          // grid prediction: 1 tensor cores, 0 window GEMMs, 2 CUDA-core tiles (3-D)
    int tc_tile_rows = 0;    // 2-D tensor-core predictor tile height, 0 = automatic
    int tc3_tile = 0;        // 3-D tensor-core predictor tile side, 0 = automatic
    int *dev_err = nullptr;  // device error flag of bounded waits
    int *hold_flag = nullptr;  // test hook: a device flag nothing sets (cs_debug_hold_predictor)
    cs::Server *server = nullptr;   // serving loop (serve.cpp), if started
    // cs_track_host: copy-in, compute and copy-out streams, and its events
    // ([0] caller, [1] velocity in, [2, 2 + chunks) chunk in, then chunk walked)
    cudaStream_t hstream[3] = {nullptr, nullptr, nullptr};
    cudaEvent_t hevent[2 + 2 * cs::kHostChunks] = {};
    std::atomic<int64_t> launches{0};
};

namespace cs {
// Device memory of a context (api.cpp). dmalloc fails with CS_ENOMEM when
// cudaMalloc fails or the block would take the context past its HBM budget;
// dfree releases a block dmalloc returned (null is ignored).
cs_status dmalloc(cs_ctx *ctx, void **p, size_t bytes);
void dfree(cs_ctx *ctx, void *p);
template <class T>
cs_status dmalloc_n(cs_ctx *ctx, T **p, size_t count) {
    void *q = nullptr;
    const cs_status rc = dmalloc(ctx, &q, (count ? count : 1) * sizeof(T));
    *p = static_cast<T *>(q);
    return rc;
}
// The grid velocity of a field on its mesh's current predictor grid,
// resampled (allocating) if the predictor grid changed since (predictor.cpp).
cs_status field_grid(cs_ctx *ctx, Mesh *m, Field *f, cudaStream_t st, const float **grid_out);
// shared body of cs_track / cs_track_dhat (api.cpp)
cs_status cs_track_impl(cs_ctx *ctx, Mesh *m, int64_t n, const double *x, const double *u,
                        double dt, const int32_t *start, int mode, const float *dhat,
                        int32_t *host_out, int32_t *path_len_out, uint8_t *status_out,
                        int32_t *start_out, cudaStream_t stream);
// predictor.cpp
void predictor_release(cs_ctx *ctx, Predictor &P);
// prediction at every predictor cell of m from the grid velocity `grid`
cs_status predict_grid(cs_ctx *ctx, Mesh *m, const float *grid, double dt, float *dhat,
                       cudaStream_t st);
// grow the 3-D tile engine's workspace for mesh m (no-op in 2-D)
cs_status reserve_tiles(cs_ctx *ctx, Mesh *m);
// make resident what serving's start predictors read (packed 2-D weights,
// 3-D tile workspace for every mesh, interpolation tables, field grids)
cs_status prepare_serving(cs_ctx *ctx);
// true when a CNN-SNS request on mesh m can run its predictor while serving
bool serving_predictor_ready(cs_ctx *ctx, const Mesh *m);
// serve.cpp
void serve_release(cs_ctx *ctx);
// classifier.cpp: free the context's classifiers
void classifier_release_all(cs_ctx *ctx);
// CNN-SNS start predictions of mesh m into m->grid_dhat: from the grid velocity
// `grid` if given, else from the nodal velocity u_nodal, resampled into the
// mesh's stored grid velocity
cs_status cnn_prepare(cs_ctx *ctx, Mesh *m, const float *grid, const double *u_nodal, double dt,
                      cudaStream_t st, const float **dhat_out);
}  // namespace cs
