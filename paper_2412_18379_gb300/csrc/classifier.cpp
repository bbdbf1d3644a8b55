// The classifier start predictor (Sec. 2.3, Eq. 7-8) as a sequence of
// kernels: pooled-centroid inputs, two zero-padded convolutions (im2col and
// BF16-operand GEMMs with FP32 accumulation on the tensor cores), average
// pooling, the offset branch, fusion, logits; the cross-entropy backward,
// Adam on FP32 master parameters, the training loop, the start element of
// the most probable class, and the C ABI entry points of the classifier.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "classifier.h"
#include "cnn.h"

namespace cs {

// Parameter offsets of the classifier of one dimension (layer order conv1,
// conv2, xp1, xp2, fuse, logits; W then b of each)
struct ClsShape {
    int dim, W, P, Pq, taps, n_pool, n_cls, ldc;
    int64_t w_off[6], b_off[6], n_params;
    explicit ClsShape(int d) : dim(d) {
        W = cls_window(d);
        P = cls_cells(d);
        Pq = d == 2 ? (W + 2) * (W + 2) : (W + 2) * (W + 2) * (W + 2);
        taps = d == 2 ? 9 : 27;
        n_pool = cls_pooled(d);
        n_cls = P;
        ldc = n_pool + kClsH1;
        const int64_t rows[6] = {kClsCh, kClsCh, kClsH1, kClsH1, kClsH2, n_cls};
        const int64_t cols[6] = {int64_t(d) * taps, int64_t(kClsCh) * taps, d, kClsH1, ldc, kClsH2};
        int64_t o = 0;
        for (int l = 0; l < 6; ++l) {
            w_off[l] = o;
            o += rows[l] * cols[l];
            b_off[l] = o;
            o += rows[l];
        }
        n_params = o;
    }
};

struct Classifier {
    int dim = 0;
    int64_t n = 0;
    float *w = nullptr, *g = nullptr, *m = nullptr, *v = nullptr, *loss = nullptr;
    int64_t t = 0;
    // workspace: the fully connected layers' buffers for `cap` rows, the
    // unfused module 1's for `cap_conv` rows and the backward pass's for
    // `cap_grad` rows (0 until a path needs them): the fused inference path
    // runs long chunks without growing the training path's im2col buffers
    int64_t cap = 0, cap_conv = 0, cap_grad = 0;
    std::vector<void *> ws;
    float *a0 = nullptr, *off = nullptr, *col1 = nullptr, *z1 = nullptr, *y1 = nullptr,
          *a1 = nullptr, *col2 = nullptr, *z2 = nullptr, *cat = nullptr, *h1 = nullptr,
          *r1 = nullptr, *h2 = nullptr, *u = nullptr, *ru = nullptr, *H = nullptr;
    float *gH = nullptr, *gu = nullptr, *gcat = nullptr, *gh2 = nullptr, *gh1 = nullptr,
          *gz2 = nullptr;
    int64_t *idx = nullptr;
    float *splitk = nullptr;
    int64_t splitk_n = 0;
    // per-call buffers of cs_track_classifier / cs_classifier_pairs
    double *xp = nullptr;
    int32_t *starts = nullptr;
    int64_t xp_cap = 0;
    // conv1 and conv2 in the fused kernel's layout, refreshed after the
    // parameters change
    uint8_t *packed = nullptr;
    bool packed_dirty = true;
};

}  // namespace cs

using namespace cs;

namespace {

cs_status fail(cs_ctx *ctx, cs_status code, const std::string &msg) {
    if (ctx) ctx->err = msg;
    return code;
}

#define CCHK(call)                                                                       \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess)                                                           \
            return fail(ctx, CS_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

cs::Mesh *find_mesh(cs_ctx *ctx, int32_t id) {
    auto it = ctx->meshes.find(id);
    return it == ctx->meshes.end() ? nullptr : it->second;
}

void free_ws(cs_ctx *ctx, Classifier &C) {
    for (void *p : C.ws) dfree(ctx, p);
    C.ws.clear();
    C.a0 = C.off = C.col1 = C.z1 = C.y1 = C.a1 = C.col2 = C.z2 = C.cat = nullptr;
    C.h1 = C.r1 = C.h2 = C.u = C.ru = C.H = nullptr;
    C.gH = C.gu = C.gcat = C.gh2 = C.gh1 = C.gz2 = nullptr;
    C.idx = nullptr;
    C.splitk = nullptr;
    C.splitk_n = 0;
    C.cap = C.cap_conv = C.cap_grad = 0;
}

void release(cs_ctx *ctx, Classifier *C) {
    if (!C) return;
    free_ws(ctx, *C);
    for (void *p : {static_cast<void *>(C->w), static_cast<void *>(C->g),
                    static_cast<void *>(C->m), static_cast<void *>(C->v),
                    static_cast<void *>(C->loss), static_cast<void *>(C->xp),
                    static_cast<void *>(C->starts), static_cast<void *>(C->packed)})
        dfree(ctx, p);
    delete C;
}

template <class T>
cs_status ws_alloc(cs_ctx *ctx, Classifier &C, T **p, int64_t count) {
    cs_status rc = dmalloc_n(ctx, p, size_t(std::max<int64_t>(count, 1)));
    if (rc == CS_OK) C.ws.push_back(*p);
    return rc;
}

// workspace for B rows of the fully connected layers; `conv` adds the
// unfused module 1's buffers, `grad` the backward pass's (which reuses
// module 1's, so it needs `conv` too). Growing any set reallocates all of
// them, each at its own row count.
cs_status ensure_ws(cs_ctx *ctx, Classifier &C, int64_t B, bool conv, bool grad) {
    if (!ctx->dev_err) {
        cs_status rc = dmalloc_n(ctx, &ctx->dev_err, 1);
        if (rc) return rc;
        if (cudaMemset(ctx->dev_err, 0, sizeof(int)) != cudaSuccess)
            return fail(ctx, CS_ECUDA, "cudaMemset of the device error flag failed");
    }
    conv = conv || grad;
    if (C.cap >= B && (!conv || C.cap_conv >= B) && (!grad || C.cap_grad >= B)) return CS_OK;
    const int64_t rows = std::max(B, C.cap);
    const int64_t rows_conv = conv ? std::max(B, C.cap_conv) : C.cap_conv;
    const int64_t rows_grad = grad ? std::max(B, C.cap_grad) : C.cap_grad;
    free_ws(ctx, C);
    const ClsShape S(C.dim);
    const int64_t d = C.dim, K1 = d * S.taps, K2 = int64_t(kClsCh) * S.taps;
    cs_status rc;
    if ((rc = ws_alloc(ctx, C, &C.off, rows * d)) || (rc = ws_alloc(ctx, C, &C.cat, rows * S.ldc)) ||
        (rc = ws_alloc(ctx, C, &C.h1, rows * kClsH1)) ||
        (rc = ws_alloc(ctx, C, &C.r1, rows * kClsH1)) ||
        (rc = ws_alloc(ctx, C, &C.h2, rows * kClsH1)) ||
        (rc = ws_alloc(ctx, C, &C.u, rows * kClsH2)) ||
        (rc = ws_alloc(ctx, C, &C.ru, rows * kClsH2)) ||
        (rc = ws_alloc(ctx, C, &C.H, rows * S.n_cls)) ||
        (rc = ws_alloc(ctx, C, &C.splitk, tc_gemm_work_floats(ctx->sm_count)))) {
        free_ws(ctx, C);
        return rc;
    }
    const int64_t rv = rows_conv;
    if (rv > 0 &&
        ((rc = ws_alloc(ctx, C, &C.a0, rv * d * S.Pq)) ||
         (rc = ws_alloc(ctx, C, &C.col1, rv * S.P * K1)) ||
         (rc = ws_alloc(ctx, C, &C.z1, rv * S.P * kClsCh)) ||
         (rc = ws_alloc(ctx, C, &C.y1, rv * S.P * kClsCh)) ||
         (rc = ws_alloc(ctx, C, &C.a1, rv * S.Pq * kClsCh)) ||
         (rc = ws_alloc(ctx, C, &C.col2, rv * S.P * K2)) ||
         (rc = ws_alloc(ctx, C, &C.z2, rv * S.P * kClsCh)))) {
        free_ws(ctx, C);
        return rc;
    }
    const int64_t rg = rows_grad;
    if (rg > 0 &&
        ((rc = ws_alloc(ctx, C, &C.gH, rg * S.n_cls)) || (rc = ws_alloc(ctx, C, &C.gu, rg * kClsH2)) ||
         (rc = ws_alloc(ctx, C, &C.gcat, rg * S.ldc)) ||
         (rc = ws_alloc(ctx, C, &C.gh2, rg * kClsH1)) ||
         (rc = ws_alloc(ctx, C, &C.gh1, rg * kClsH1)) ||
         (rc = ws_alloc(ctx, C, &C.gz2, rg * S.P * kClsCh)) || (rc = ws_alloc(ctx, C, &C.idx, rg)))) {
        free_ws(ctx, C);
        return rc;
    }
    C.splitk_n = tc_gemm_work_floats(ctx->sm_count);
    C.cap = rows;
    C.cap_conv = rows_conv;
    C.cap_grad = rows_grad;
    return CS_OK;
}

int gemm(cs_ctx *ctx, Classifier &C, const float *A, const float *Bm, float *Cm, const float *bias,
         int64_t M, int64_t N, int64_t K, bool transA, bool transB, cudaStream_t st) {
    return launch_gemm(A, Bm, Cm, bias, M, N, K, transA, transB, false, st, ctx->dev_err,
                       ctx->sm_count, C.splitk, C.splitk_n);
}

int relu(cs_ctx *ctx, const float *z, float *y, int64_t n, cudaStream_t st) {
    return launch_relu(z, y, n, ctx->sm_count, st);
}

// module 2, fusion and logits of B rows whose pooled features (C.cat's
// first n_pool columns) and offsets (C.off) are in place, into C.H
int forward_fc(cs_ctx *ctx, Classifier &C, int64_t B, cudaStream_t st) {
    const ClsShape S(C.dim);
    const int sm = ctx->sm_count, d = C.dim;
    int n = 0;
    // module 2: the offset of x_p through two fully connected layers
    n += gemm(ctx, C, C.off, C.w + S.w_off[2], C.h1, C.w + S.b_off[2], B, kClsH1, d, false, true,
              st);
    n += relu(ctx, C.h1, C.r1, B * kClsH1, st);
    n += gemm(ctx, C, C.r1, C.w + S.w_off[3], C.h2, C.w + S.b_off[3], B, kClsH1, kClsH1, false,
              true, st);
    launch_cls_cat_relu(C.h2, B, kClsH1, C.cat, S.ldc, S.n_pool, sm, st);
    n += 1;
    // fusion and logits
    n += gemm(ctx, C, C.cat, C.w + S.w_off[4], C.u, C.w + S.b_off[4], B, kClsH2, S.ldc, false,
              true, st);
    n += relu(ctx, C.u, C.ru, B * kClsH2, st);
    n += gemm(ctx, C, C.ru, C.w + S.w_off[5], C.H, C.w + S.b_off[5], B, S.n_cls, kClsH2, false,
              true, st);
    return n;
}

// inference of B particles xp[b] into C.H: module 1 fused on the tensor cores
// (BF16 operands), or, with FP32 operands, the training path's kernels
int forward(cs_ctx *ctx, Classifier &C, const DevMesh &m, int64_t B, const double *xp,
            const int64_t *idx, cudaStream_t st);
int infer(cs_ctx *ctx, Classifier &C, const DevMesh &m, int64_t B, const double *xp,
          cudaStream_t st) {
    if (!gemm_bf16()) return forward(ctx, C, m, B, xp, nullptr, st);
    const ClsShape S(C.dim);
    if (C.packed_dirty) {
        launch_cls_pack(C.dim, C.w, S.w_off[0], S.b_off[0], S.w_off[1], S.b_off[1], C.packed, st);
        C.packed_dirty = false;
    }
    launch_cls_conv_tc(m, m.pool_f, B, xp, C.packed, C.cat, S.ldc, C.off, ctx->dev_err,
                       ctx->sm_count, st);
    return 2 + forward_fc(ctx, C, B, st);
}

// forward of B rows (particles xp[idx[b]], or xp[b]) into C.H [B][n_cls],
// keeping every activation the backward pass reads
int forward(cs_ctx *ctx, Classifier &C, const DevMesh &m, int64_t B, const double *xp,
            const int64_t *idx, cudaStream_t st) {
    const ClsShape S(C.dim);
    const int sm = ctx->sm_count, d = C.dim;
    const int64_t BP = B * S.P;
    int n = 0;
    launch_cls_features(m, B, xp, idx, true, C.a0, C.off, sm, st);
    n += 1;
    // module 1: two zero-padded 3^d convolutions with ReLU, pooling
    n += launch_im2col(d, C.a0, B, d, S.W + 2, true, C.col1, sm, st);
    n += gemm(ctx, C, C.col1, C.w + S.w_off[0], C.z1, C.w + S.b_off[0], BP, kClsCh,
              int64_t(d) * S.taps, false, true, st);
    n += relu(ctx, C.z1, C.y1, BP * kClsCh, st);
    launch_cls_pad(d, C.y1, B, kClsCh, C.a1, sm, st);
    n += 1;
    n += launch_im2col(d, C.a1, B, kClsCh, S.W + 2, false, C.col2, sm, st);
    n += gemm(ctx, C, C.col2, C.w + S.w_off[1], C.z2, C.w + S.b_off[1], BP, kClsCh,
              int64_t(kClsCh) * S.taps, false, true, st);
    launch_cls_pool(d, C.z2, B, C.cat, S.ldc, sm, st);
    n += 1;
    return n + forward_fc(ctx, C, B, st);
}

// gradients of the cross-entropy of C.H against labels[idx[b]] into C.g;
// the loss is added to *loss. Buffers no longer needed are reused: col2
// takes the gradient of its columns, a1 that of the padded input, y1 that of
// the first convolution's output.
int backward(cs_ctx *ctx, Classifier &C, int64_t B, const int32_t *labels, const int64_t *idx,
             float *loss, cudaStream_t st) {
    const ClsShape S(C.dim);
    const int sm = ctx->sm_count, d = C.dim;
    const int64_t BP = B * S.P;
    float *g = C.g;
    const float *w = C.w;
    int n = 0;
    launch_softmax_ce(C.H, labels, idx, B, S.n_cls, C.gH, loss, st);
    n += 1;
    // logits and fusion
    n += gemm(ctx, C, C.gH, C.ru, g + S.w_off[5], nullptr, S.n_cls, kClsH2, B, true, false, st);
    n += launch_colsum(C.gH, B, S.n_cls, g + S.b_off[5], st, C.splitk, C.splitk_n, sm);
    n += gemm(ctx, C, C.gH, w + S.w_off[5], C.gu, nullptr, B, kClsH2, S.n_cls, false, false, st);
    n += launch_relu_back(C.u, C.gu, B * kClsH2, sm, st);
    n += gemm(ctx, C, C.gu, C.cat, g + S.w_off[4], nullptr, kClsH2, S.ldc, B, true, false, st);
    n += launch_colsum(C.gu, B, kClsH2, g + S.b_off[4], st, C.splitk, C.splitk_n, sm);
    n += gemm(ctx, C, C.gu, w + S.w_off[4], C.gcat, nullptr, B, S.ldc, kClsH2, false, false, st);
    // module 2
    launch_cls_uncat_relu_back(C.gcat, S.ldc, S.n_pool, C.h2, B, kClsH1, C.gh2, sm, st);
    n += 1;
    n += gemm(ctx, C, C.gh2, C.r1, g + S.w_off[3], nullptr, kClsH1, kClsH1, B, true, false, st);
    n += launch_colsum(C.gh2, B, kClsH1, g + S.b_off[3], st, C.splitk, C.splitk_n, sm);
    n += gemm(ctx, C, C.gh2, w + S.w_off[3], C.gh1, nullptr, B, kClsH1, kClsH1, false, false, st);
    n += launch_relu_back(C.h1, C.gh1, B * kClsH1, sm, st);
    n += gemm(ctx, C, C.gh1, C.off, g + S.w_off[2], nullptr, kClsH1, d, B, true, false, st);
    n += launch_colsum(C.gh1, B, kClsH1, g + S.b_off[2], st, C.splitk, C.splitk_n, sm);
    // module 1: pooling, second and first convolution
    launch_cls_pool_back(d, C.gcat, S.ldc, C.z2, B, C.gz2, sm, st);
    n += 1;
    const int64_t K2 = int64_t(kClsCh) * S.taps;
    n += gemm(ctx, C, C.gz2, C.col2, g + S.w_off[1], nullptr, kClsCh, K2, BP, true, false, st);
    n += launch_colsum(C.gz2, BP, kClsCh, g + S.b_off[1], st, C.splitk, C.splitk_n, sm);
    float *dcol2 = C.col2, *dpad = C.a1, *gz1 = C.y1;
    n += gemm(ctx, C, C.gz2, w + S.w_off[1], dcol2, nullptr, BP, K2, kClsCh, false, false, st);
    n += launch_col2im(d, dcol2, B, kClsCh, S.W + 2, dpad, sm, st);
    launch_cls_crop_relu_back(d, dpad, C.z1, B, kClsCh, gz1, sm, st);
    n += 1;
    n += gemm(ctx, C, gz1, C.col1, g + S.w_off[0], nullptr, kClsCh, int64_t(d) * S.taps, BP, true,
              false, st);
    n += launch_colsum(gz1, BP, kClsCh, g + S.b_off[0], st, C.splitk, C.splitk_n, sm);
    return n;
}

Classifier *get_cls(cs_ctx *ctx, int dim) {
    if (dim != 2 && dim != 3) return nullptr;
    return ctx->cls[dim - 2];
}

uint64_t splitmix(uint64_t &s) {
    uint64_t z = (s += 0x9e3779b97f4a7c15ull);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

// rows per forward chunk. The fused path needs only the fully connected
// layers' buffers (about 10 KB a row in 2-D, 13 KB in 3-D): chunks of this
// size give those GEMMs enough tiles to fill the GPU without splitting K.
// The unfused path's im2col buffers take about 1 GB at its smaller chunks.
int64_t chunk_rows(int dim, bool fused) {
    if (fused) return dim == 2 ? 32768 : 16384;
    return dim == 2 ? 8192 : 1024;
}

cs_status ensure_xp(cs_ctx *ctx, Classifier &C, int64_t n) {
    if (C.xp_cap >= n) return CS_OK;
    dfree(ctx, C.xp);
    dfree(ctx, C.starts);
    C.xp = nullptr;
    C.starts = nullptr;
    C.xp_cap = 0;
    cs_status rc;
    if ((rc = dmalloc_n(ctx, &C.xp, size_t(n) * C.dim)) ||
        (rc = dmalloc_n(ctx, &C.starts, size_t(n))))
        return rc;
    C.xp_cap = n;
    return CS_OK;
}

// logits of n particles, chunk by chunk, through the workspace; each chunk's
// logits are copied out on the stream (or handed to `each` in place)
template <class F>
cs_status forward_chunks(cs_ctx *ctx, Classifier &C, const DevMesh &m, int64_t n, const double *xp,
                         cudaStream_t st, F each) {
    const bool fused = gemm_bf16();
    const int64_t R = std::min<int64_t>(n, chunk_rows(C.dim, fused));
    cs_status rc = ensure_ws(ctx, C, R, !fused, false);
    if (rc) return rc;
    for (int64_t r0 = 0; r0 < n; r0 += R) {
        const int64_t B = std::min(R, n - r0);
        ctx->launches += infer(ctx, C, m, B, xp + r0 * C.dim, st);
        if ((rc = each(r0, B))) return rc;
    }
    return CS_OK;
}

}  // namespace

namespace cs {
void classifier_release_all(cs_ctx *ctx) {
    for (auto &c : ctx->cls) {
        release(ctx, c);
        c = nullptr;
    }
}
}  // namespace cs

extern "C" {

int64_t cs_classifier_size(int dim) {
    if (dim != 2 && dim != 3) return 0;
    return ClsShape(dim).n_params;
}

int32_t cs_classifier_window(int dim) {
    if (dim != 2 && dim != 3) return 0;
    return cls_window(dim);
}

cs_status cs_classifier_load(cs_ctx *ctx, int dim, const float *params, int64_t n) {
    if (!ctx) return CS_EINVAL;
    if ((dim != 2 && dim != 3) || !params || n != cs_classifier_size(dim))
        return fail(ctx, CS_EINVAL, "cs_classifier_load: bad dim or size (expected " +
                                        std::to_string(cs_classifier_size(dim)) + " floats)");
    if (ctx->server) return fail(ctx, CS_EBUSY, "cs_classifier_load: stop serving first");
    CCHK(cudaSetDevice(ctx->device));
    CCHK(cudaDeviceSynchronize());
    release(ctx, ctx->cls[dim - 2]);
    ctx->cls[dim - 2] = nullptr;
    Classifier *C = new (std::nothrow) Classifier();
    if (!C) return fail(ctx, CS_ENOMEM, "host allocation failed");
    C->dim = dim;
    C->n = n;
    cs_status rc;
    if ((rc = dmalloc_n(ctx, &C->w, size_t(n))) || (rc = dmalloc_n(ctx, &C->g, size_t(n))) ||
        (rc = dmalloc_n(ctx, &C->m, size_t(n))) || (rc = dmalloc_n(ctx, &C->v, size_t(n))) ||
        (rc = dmalloc_n(ctx, &C->loss, 1)) ||
        (rc = dmalloc_n(ctx, &C->packed, size_t(cls_packed_bytes(dim))))) {
        release(ctx, C);
        return rc;
    }
    if (cudaMemcpy(C->w, params, size_t(n) * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(C->m, 0, size_t(n) * sizeof(float)) != cudaSuccess ||
        cudaMemset(C->v, 0, size_t(n) * sizeof(float)) != cudaSuccess) {
        release(ctx, C);
        return fail(ctx, CS_ECUDA, "cs_classifier_load: copy of the parameters failed");
    }
    ctx->cls[dim - 2] = C;
    return CS_OK;
}

cs_status cs_classifier_save(cs_ctx *ctx, int dim, float *out, int64_t n) {
    if (!ctx) return CS_EINVAL;
    if ((dim != 2 && dim != 3) || !out || n != cs_classifier_size(dim))
        return fail(ctx, CS_EINVAL, "cs_classifier_save: bad dim or size");
    Classifier *C = get_cls(ctx, dim);
    if (!C) return fail(ctx, CS_ENOPRED, "cs_classifier_save: no classifier loaded");
    CCHK(cudaSetDevice(ctx->device));
    CCHK(cudaDeviceSynchronize());
    CCHK(cudaMemcpy(out, C->w, size_t(n) * sizeof(float), cudaMemcpyDeviceToHost));
    return CS_OK;
}

cs_status cs_departure(cs_ctx *ctx, int32_t mesh_id, int64_t n, const double *x, const double *u,
                       double dt, double *xp_out, void *stream) {
    if (!ctx) return CS_EINVAL;
    cs::Mesh *m = find_mesh(ctx, mesh_id);
    if (!m) return fail(ctx, CS_ENOMESH, "cs_departure: unknown mesh id");
    if (n < 0 || (n > 0 && (!x || !u || !xp_out)))
        return fail(ctx, CS_EINVAL, "cs_departure: bad arguments");
    if (n == 0) return CS_OK;
    CCHK(cudaSetDevice(ctx->device));
    launch_departure(n, m->d.dim, x, u, dt, xp_out, ctx->sm_count,
                     static_cast<cudaStream_t>(stream));
    ctx->launches += 1;
    CCHK(cudaGetLastError());
    return CS_OK;
}

cs_status cs_classifier_features(cs_ctx *ctx, int32_t mesh_id, int64_t n, const double *xp,
                                 float *window_out, float *offset_out, void *stream) {
    if (!ctx) return CS_EINVAL;
    cs::Mesh *m = find_mesh(ctx, mesh_id);
    if (!m) return fail(ctx, CS_ENOMESH, "cs_classifier_features: unknown mesh id");
    if (n < 0 || (n > 0 && (!xp || !window_out || !offset_out)))
        return fail(ctx, CS_EINVAL, "cs_classifier_features: bad arguments");
    if (n == 0) return CS_OK;
    CCHK(cudaSetDevice(ctx->device));
    launch_cls_features(m->d, n, xp, nullptr, false, window_out, offset_out, ctx->sm_count,
                        static_cast<cudaStream_t>(stream));
    ctx->launches += 1;
    CCHK(cudaGetLastError());
    return CS_OK;
}

cs_status cs_classifier_forward(cs_ctx *ctx, int32_t mesh_id, int64_t n, const double *xp,
                                float *logits_out) {
    if (!ctx) return CS_EINVAL;
    cs::Mesh *m = find_mesh(ctx, mesh_id);
    if (!m) return fail(ctx, CS_ENOMESH, "cs_classifier_forward: unknown mesh id");
    if (n < 0 || (n > 0 && (!xp || !logits_out)))
        return fail(ctx, CS_EINVAL, "cs_classifier_forward: bad arguments");
    Classifier *C = get_cls(ctx, m->d.dim);
    if (!C) return fail(ctx, CS_ENOPRED, "cs_classifier_forward: no classifier loaded");
    if (n == 0) return CS_OK;
    CCHK(cudaSetDevice(ctx->device));
    const int ncls = cls_cells(C->dim);
    cs_status rc = forward_chunks(ctx, *C, m->d, n, xp, nullptr, [&](int64_t r0, int64_t B) {
        if (cudaMemcpyAsync(logits_out + r0 * ncls, C->H, size_t(B) * ncls * sizeof(float),
                            cudaMemcpyDeviceToDevice, nullptr) != cudaSuccess)
            return fail(ctx, CS_ECUDA, "cs_classifier_forward: copy of the logits failed");
        return CS_OK;
    });
    if (rc) return rc;
    CCHK(cudaDeviceSynchronize());
    return cs_device_status(ctx);
}

cs_status cs_classifier_labels(cs_ctx *ctx, int32_t mesh_id, int64_t n, const double *xp,
                               const int32_t *host, int32_t *label_out, void *stream) {
    if (!ctx) return CS_EINVAL;
    cs::Mesh *m = find_mesh(ctx, mesh_id);
    if (!m) return fail(ctx, CS_ENOMESH, "cs_classifier_labels: unknown mesh id");
    if (n < 0 || (n > 0 && (!xp || !host || !label_out)))
        return fail(ctx, CS_EINVAL, "cs_classifier_labels: bad arguments");
    if (n == 0) return CS_OK;
    CCHK(cudaSetDevice(ctx->device));
    launch_cls_labels(m->d, n, xp, host, label_out, ctx->sm_count,
                      static_cast<cudaStream_t>(stream));
    ctx->launches += 1;
    CCHK(cudaGetLastError());
    return CS_OK;
}

cs_status cs_classifier_pairs(cs_ctx *ctx, int32_t mesh_id, int64_t n, const double *x,
                              const double *u, double dt, const int32_t *start, double *xp_out,
                              int32_t *label_out, void *stream) {
    if (!ctx) return CS_EINVAL;
    cs::Mesh *m = find_mesh(ctx, mesh_id);
    if (!m) return fail(ctx, CS_ENOMESH, "cs_classifier_pairs: unknown mesh id");
    if (n < 0 || n >= (int64_t(1) << 31) - 1 || (n > 0 && (!x || !u || !xp_out || !label_out)))
        return fail(ctx, CS_EINVAL, "cs_classifier_pairs: bad arguments");
    if (!start && n != m->d.n_v)
        return fail(ctx, CS_EINVAL, "cs_classifier_pairs: start == NULL needs n == n_vertices");
    if (n == 0) return CS_OK;
    CCHK(cudaSetDevice(ctx->device));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // the walk's outputs: host into label_out (overwritten by the labels),
    // path lengths and status into a scratch block
    void *scratch = nullptr;
    cs_status rc = dmalloc(ctx, &scratch, size_t(n) * 5);
    if (rc) return rc;
    int32_t *path = static_cast<int32_t *>(scratch);
    uint8_t *status = reinterpret_cast<uint8_t *>(path + n);
    rc = cs_track_impl(ctx, m, n, x, u, dt, start, CS_SNS, nullptr, label_out, path, status,
                       nullptr, st);
    if (rc == CS_OK) {
        launch_departure(n, m->d.dim, x, u, dt, xp_out, ctx->sm_count, st);
        launch_cls_labels(m->d, n, xp_out, label_out, label_out, ctx->sm_count, st);
        ctx->launches += 2;
        if (cudaStreamSynchronize(st) != cudaSuccess || cudaGetLastError() != cudaSuccess)
            rc = fail(ctx, CS_ECUDA, "cs_classifier_pairs: kernel failed");
    }
    dfree(ctx, scratch);
    return rc;
}

cs_status cs_classifier_grad(cs_ctx *ctx, int32_t mesh_id, int64_t B, const double *xp,
                             const int32_t *labels, float *grad_out, float *loss_out) {
    if (!ctx) return CS_EINVAL;
    cs::Mesh *m = find_mesh(ctx, mesh_id);
    if (!m) return fail(ctx, CS_ENOMESH, "cs_classifier_grad: unknown mesh id");
    if (B < 1 || !xp || !labels || !grad_out)
        return fail(ctx, CS_EINVAL, "cs_classifier_grad: bad arguments");
    Classifier *C = get_cls(ctx, m->d.dim);
    if (!C) return fail(ctx, CS_ENOPRED, "cs_classifier_grad: no classifier loaded");
    CCHK(cudaSetDevice(ctx->device));
    cs_status rc = ensure_ws(ctx, *C, B, true, true);
    if (rc) return rc;
    CCHK(cudaMemset(C->loss, 0, sizeof(float)));
    ctx->launches += forward(ctx, *C, m->d, B, xp, nullptr, nullptr);
    ctx->launches += backward(ctx, *C, B, labels, nullptr, C->loss, nullptr);
    CCHK(cudaDeviceSynchronize());
    if ((rc = cs_device_status(ctx))) return rc;
    CCHK(cudaMemcpy(grad_out, C->g, size_t(C->n) * sizeof(float), cudaMemcpyDeviceToDevice));
    if (loss_out) CCHK(cudaMemcpy(loss_out, C->loss, sizeof(float), cudaMemcpyDeviceToHost));
    return CS_OK;
}

cs_status cs_classifier_train(cs_ctx *ctx, int32_t mesh_id, const double *xp,
                              const int32_t *labels, int64_t N, int64_t batch, int64_t steps,
                              float lr, uint64_t seed, float *loss_out) {
    if (!ctx) return CS_EINVAL;
    cs::Mesh *m = find_mesh(ctx, mesh_id);
    if (!m) return fail(ctx, CS_ENOMESH, "cs_classifier_train: unknown mesh id");
    if (!xp || !labels || N < 1 || batch < 1 || steps < 0 || !(lr > 0.f))
        return fail(ctx, CS_EINVAL, "cs_classifier_train: bad arguments");
    Classifier *C = get_cls(ctx, m->d.dim);
    if (!C) return fail(ctx, CS_ENOPRED, "cs_classifier_train: no classifier loaded");
    CCHK(cudaSetDevice(ctx->device));
    const int64_t B = std::min(batch, N);
    cs_status rc = ensure_ws(ctx, *C, B, true, true);
    if (rc) return rc;
    float *losses = nullptr;
    if ((rc = dmalloc_n(ctx, &losses, size_t(std::max<int64_t>(steps, 1))))) return rc;
    cs_status out = CS_OK;
    if (cudaMemset(losses, 0, size_t(std::max<int64_t>(steps, 1)) * sizeof(float)) != cudaSuccess)
        out = fail(ctx, CS_ECUDA, "cs_classifier_train: memset");
    std::vector<int64_t> perm(static_cast<size_t>(N));
    for (int64_t i = 0; i < N; ++i) perm[i] = i;
    uint64_t rs = seed;
    int64_t pos = N;   // shuffle at the first step
    std::vector<int64_t> idx(static_cast<size_t>(B));
    for (int64_t s = 0; s < steps && out == CS_OK; ++s) {
        for (int64_t b = 0; b < B; ++b) {
            if (pos >= N) {   // new epoch: Fisher-Yates shuffle
                for (int64_t i = N - 1; i > 0; --i) std::swap(perm[i], perm[splitmix(rs) % (i + 1)]);
                pos = 0;
            }
            idx[b] = perm[pos++];
        }
        if (cudaMemcpy(C->idx, idx.data(), size_t(B) * sizeof(int64_t), cudaMemcpyHostToDevice) !=
            cudaSuccess) {
            out = fail(ctx, CS_ECUDA, "cs_classifier_train: index copy");
            break;
        }
        ctx->launches += forward(ctx, *C, m->d, B, xp, C->idx, nullptr);
        ctx->launches += backward(ctx, *C, B, labels, C->idx, losses + s, nullptr);
        C->t += 1;
        ctx->launches += launch_adam(C->w, C->g, C->m, C->v, C->n, lr, C->t, ctx->sm_count, nullptr);
        C->packed_dirty = true;
    }
    if (out == CS_OK) {
        cudaError_t e = cudaDeviceSynchronize();
        if (e == cudaSuccess && loss_out && steps > 0)
            e = cudaMemcpy(loss_out, losses, size_t(steps) * sizeof(float), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess)
            out = fail(ctx, CS_ECUDA, std::string("cs_classifier_train: ") + cudaGetErrorString(e));
        else
            out = cs_device_status(ctx);
    }
    dfree(ctx, losses);
    return out;
}

cs_status cs_classifier_start(cs_ctx *ctx, int32_t mesh_id, int64_t n, const double *xp,
                              const float *logits, const int32_t *fallback, int32_t *start_out,
                              int32_t *class_out, void *stream) {
    if (!ctx) return CS_EINVAL;
    cs::Mesh *m = find_mesh(ctx, mesh_id);
    if (!m) return fail(ctx, CS_ENOMESH, "cs_classifier_start: unknown mesh id");
    if (n < 0 || (n > 0 && (!xp || !logits || !start_out)))
        return fail(ctx, CS_EINVAL, "cs_classifier_start: bad arguments");
    if (!fallback && n != m->d.n_v)
        return fail(ctx, CS_EINVAL, "cs_classifier_start: fallback == NULL needs n == n_vertices");
    if (n == 0) return CS_OK;
    CCHK(cudaSetDevice(ctx->device));
    launch_cls_start(m->d, n, xp, logits, fallback, 0, start_out, class_out, ctx->sm_count,
                     static_cast<cudaStream_t>(stream));
    ctx->launches += 1;
    CCHK(cudaGetLastError());
    return CS_OK;
}

cs_status cs_track_classifier(cs_ctx *ctx, int32_t mesh_id, int64_t n, const double *x,
                              const double *u, double dt, const int32_t *start,
                              int32_t *host_out, int32_t *path_len_out, uint8_t *status_out,
                              int32_t *start_out, void *stream) {
    if (!ctx) return CS_EINVAL;
    cs::Mesh *m = find_mesh(ctx, mesh_id);
    if (!m) return fail(ctx, CS_ENOMESH, "cs_track_classifier: unknown mesh id");
    if (n < 0 || n >= (int64_t(1) << 31) - 1)
        return fail(ctx, CS_EINVAL, "cs_track_classifier: n is outside [0, 2^31 - 2]");
    Classifier *C = get_cls(ctx, m->d.dim);
    if (!C) return fail(ctx, CS_ENOPRED, "cs_track_classifier: no classifier loaded");
    if (n == 0) return CS_OK;
    if (!x || !u || !host_out || !path_len_out || !status_out)
        return fail(ctx, CS_EINVAL, "cs_track_classifier: null pointer");
    if (!start && n != m->d.n_v)
        return fail(ctx, CS_EINVAL, "cs_track_classifier: start == NULL needs n == n_vertices");
    CCHK(cudaSetDevice(ctx->device));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cs_status rc = ensure_xp(ctx, *C, n);
    if (rc) return rc;
    launch_departure(n, C->dim, x, u, dt, C->xp, ctx->sm_count, st);
    ctx->launches += 1;
    const DevMesh &d = m->d;
    rc = forward_chunks(ctx, *C, d, n, C->xp, st, [&](int64_t r0, int64_t B) {
        launch_cls_start(d, B, C->xp + r0 * C->dim, C->H, start ? start + r0 : nullptr, r0,
                         C->starts + r0, nullptr, ctx->sm_count, st);
        ctx->launches += 1;
        return CS_OK;
    });
    if (rc) return rc;
    rc = cs_track_impl(ctx, m, n, x, u, dt, C->starts, CS_SNS, nullptr, host_out, path_len_out,
                       status_out, nullptr, st);
    if (rc) return rc;
    if (start_out &&
        cudaMemcpyAsync(start_out, C->starts, size_t(n) * sizeof(int32_t), cudaMemcpyDeviceToDevice,
                        st) != cudaSuccess)
        return fail(ctx, CS_ECUDA, "cs_track_classifier: copy of the starts failed");
    CCHK(cudaStreamSynchronize(st));
    return cs_device_status(ctx);
}

}  // extern "C"
