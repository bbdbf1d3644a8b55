// Start predictor runtime (Sec. 2.3, Algorithm 2): weights, the forward and
// backward passes of training as sequences of kernels (im2col, BF16-operand
// GEMM with FP32 accumulation, bias, ReLU, col2im), Adam, the training loop,
// grid prediction, and the C ABI entry points of the predictor.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>

#include "cnn.h"

namespace cs {

NetShape::NetShape(int d) : dim(d) {
    cin = d;
    S0 = d == 2 ? 9 : 7;
    n_conv = d == 2 ? 4 : 3;
    ch = 32;
    hidden = 256;
    int64_t o = 0;
    int c = cin;
    for (int l = 0; l < n_conv; ++l) {
        w_off.push_back(o);
        o += int64_t(ch) * c * taps();
        b_off.push_back(o);
        o += ch;
        c = ch;
    }
    w_off.push_back(o);
    o += int64_t(hidden) * ch;
    b_off.push_back(o);
    o += hidden;
    w_off.push_back(o);
    o += int64_t(dim) * hidden;
    b_off.push_back(o);
    o += dim;
    n_params = o;
}

}  // namespace cs

using namespace cs;

namespace {

cs_status fail(cs_ctx *ctx, cs_status code, const std::string &msg) {
    if (ctx) ctx->err = msg;
    return code;
}

#define PCHK(call)                                                                       \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess)                                                           \
            return fail(ctx, CS_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

template <class T>
cs_status dalloc(cs_ctx *ctx, T **p, size_t count) {
    return dmalloc_n(ctx, p, count);
}

void free_workspace(cs_ctx *ctx, Predictor &P) {
    for (float *p : P.col) dfree(ctx, p);
    for (float *p : P.z) dfree(ctx, p);
    for (float *p : P.y) dfree(ctx, p);
    P.col.clear();
    P.z.clear();
    P.y.clear();
    float **fs[] = {&P.z5, &P.a5, &P.out, &P.gout, &P.dcol, &P.dy0, &P.dy1, &P.da5, &P.win, &P.tgt};
    for (float **f : fs) {
        dfree(ctx, *f);
        *f = nullptr;
    }
    dfree(ctx, P.idx);
    P.idx = nullptr;
    dfree(ctx, P.splitk);
    P.splitk = nullptr;
    P.splitk_n = 0;
    P.cap = 0;
    for (float *p : P.tiles) dfree(ctx, p);
    P.tiles.clear();
    P.tiles_cap.clear();
}

cs_status ensure_workspace(cs_ctx *ctx, Predictor &P, int64_t B) {
    // the error flag of the tensor-core GEMMs' bounded waits
    if (!ctx->dev_err) {
        cs_status rc = dalloc(ctx, &ctx->dev_err, 1);
        if (rc) return rc;
        if (cudaMemset(ctx->dev_err, 0, sizeof(int)) != cudaSuccess)
            return fail(ctx, CS_ECUDA, "cudaMemset of the device error flag failed");
    }
    if (P.cap >= B) return CS_OK;
    free_workspace(ctx, P);
    NetShape S(P.dim);
    int Si = S.S0, C = S.cin;
    int64_t max_col = 0, max_dy = 0;
    for (int l = 0; l < S.n_conv; ++l) {
        const int So = Si - 2;
        const int64_t Po = S.positions(So), K = int64_t(C) * S.taps();
        float *col, *z, *y;
        cs_status rc;
        if ((rc = dalloc(ctx, &col, size_t(B * Po * K))) || (rc = dalloc(ctx, &z, size_t(B * Po * S.ch))) ||
            (rc = dalloc(ctx, &y, size_t(B * Po * S.ch))))
            return rc;
        P.col.push_back(col);
        P.z.push_back(z);
        P.y.push_back(y);
        max_col = std::max(max_col, B * Po * K);
        if (l > 0) max_dy = std::max(max_dy, B * S.positions(Si) * S.ch);
        max_dy = std::max(max_dy, B * Po * S.ch);
        Si = So;
        C = S.ch;
    }
    const int64_t win = int64_t(S.cin) * S.positions(S.S0);
    cs_status rc;
    if ((rc = dalloc(ctx, &P.z5, size_t(B * S.hidden))) || (rc = dalloc(ctx, &P.a5, size_t(B * S.hidden))) ||
        (rc = dalloc(ctx, &P.out, size_t(B * S.dim))) || (rc = dalloc(ctx, &P.gout, size_t(B * S.dim))) ||
        (rc = dalloc(ctx, &P.dcol, size_t(max_col))) || (rc = dalloc(ctx, &P.dy0, size_t(max_dy))) ||
        (rc = dalloc(ctx, &P.dy1, size_t(max_dy))) || (rc = dalloc(ctx, &P.da5, size_t(B * S.hidden))) ||
        (rc = dalloc(ctx, &P.win, size_t(B * win))) || (rc = dalloc(ctx, &P.tgt, size_t(B * S.dim))) ||
        (rc = dalloc(ctx, &P.idx, size_t(B))) ||
        (rc = dalloc(ctx, &P.splitk, size_t(tc_gemm_work_floats(ctx->sm_count)))))
        return rc;
    P.splitk_n = tc_gemm_work_floats(ctx->sm_count);
    P.cap = B;
    return CS_OK;
}

// C = op(A) op(B) (+ bias) of the predictor's workspace: BF16 operands on the
// tensor cores where the shape fits, K splits summed in a fixed order
int gemm(cs_ctx *ctx, Predictor &P, const float *A, const float *Bm, float *C, const float *bias,
         int64_t M, int64_t N, int64_t K, bool transA, bool transB, cudaStream_t st) {
    return launch_gemm(A, Bm, C, bias, M, N, K, transA, transB, false, st, ctx->dev_err,
                       ctx->sm_count, P.splitk, P.splitk_n);
}

// forward of B windows (device, [B][cin][S0^dim]) into P.out [B][dim]
int forward(cs_ctx *ctx, Predictor &P, int64_t B, const float *win, cudaStream_t st) {
    NetShape S(P.dim);
    const int sm = ctx->sm_count;
    int launches = 0;
    const float *x = win;
    bool chfirst = true;
    int C = S.cin, Si = S.S0;
    for (int l = 0; l < S.n_conv; ++l) {
        const int So = Si - 2;
        const int64_t Po = S.positions(So), K = int64_t(C) * S.taps();
        launches += launch_im2col(P.dim, x, B, C, Si, chfirst, P.col[l], sm, st);
        launches += gemm(ctx, P, P.col[l], P.w + S.w_off[l], P.z[l], P.w + S.b_off[l],
                         B * Po, S.ch, K, false, true, st);
        launches += launch_relu(P.z[l], P.y[l], B * Po * S.ch, sm, st);
        x = P.y[l];
        chfirst = false;
        C = S.ch;
        Si = So;
    }
    const int f1 = S.n_conv, f2 = S.n_conv + 1;
    launches += gemm(ctx, P, x, P.w + S.w_off[f1], P.z5, P.w + S.b_off[f1],
                     B, S.hidden, S.ch, false, true, st);
    launches += launch_relu(P.z5, P.a5, B * S.hidden, sm, st);
    launches += gemm(ctx, P, P.a5, P.w + S.w_off[f2], P.out, P.w + S.b_off[f2],
                     B, S.dim, S.hidden, false, true, st);
    return launches;
}

// gradients of the MSE of P.out against tgt into P.g; loss added to *loss
int backward(cs_ctx *ctx, Predictor &P, int64_t B, const float *tgt, float *loss,
             cudaStream_t st) {
    NetShape S(P.dim);
    const int sm = ctx->sm_count;
    int n = 0;
    const int f1 = S.n_conv, f2 = S.n_conv + 1;
    n += launch_mse_grad(P.out, tgt, B * S.dim, P.gout, loss, sm, st);
    n += gemm(ctx, P, P.gout, P.a5, P.g + S.w_off[f2], nullptr,
              S.dim, S.hidden, B, true, false, st);
    n += launch_colsum(P.gout, B, S.dim, P.g + S.b_off[f2], st, P.splitk, P.splitk_n, sm);
    n += gemm(ctx, P, P.gout, P.w + S.w_off[f2], P.da5, nullptr,
              B, S.hidden, S.dim, false, false, st);
    n += launch_relu_back(P.z5, P.da5, B * S.hidden, sm, st);
    const float *h4 = P.y[S.n_conv - 1];
    n += gemm(ctx, P, P.da5, h4, P.g + S.w_off[f1], nullptr, S.hidden, S.ch, B, true, false, st);
    n += launch_colsum(P.da5, B, S.hidden, P.g + S.b_off[f1], st, P.splitk, P.splitk_n, sm);
    float *dy = P.dy0, *dnext = P.dy1;
    n += gemm(ctx, P, P.da5, P.w + S.w_off[f1], dy, nullptr, B, S.ch, S.hidden, false, false, st);
    // conv layers, last to first; edge of layer l's input
    std::vector<int> Sin(S.n_conv);
    int Si = S.S0;
    for (int l = 0; l < S.n_conv; ++l) {
        Sin[l] = Si;
        Si -= 2;
    }
    for (int l = S.n_conv - 1; l >= 0; --l) {
        const int So = Sin[l] - 2;
        const int C = l == 0 ? S.cin : S.ch;
        const int64_t Po = S.positions(So), K = int64_t(C) * S.taps();
        n += launch_relu_back(P.z[l], dy, B * Po * S.ch, sm, st);
        n += gemm(ctx, P, dy, P.col[l], P.g + S.w_off[l], nullptr,
                  S.ch, K, B * Po, true, false, st);
        n += launch_colsum(dy, B * Po, S.ch, P.g + S.b_off[l], st, P.splitk, P.splitk_n, sm);
        if (l > 0) {
            n += gemm(ctx, P, dy, P.w + S.w_off[l], P.dcol, nullptr,
                      B * Po, K, S.ch, false, false, st);
            n += launch_col2im(P.dim, P.dcol, B, S.ch, Sin[l], dnext, sm, st);
            std::swap(dy, dnext);
        }
    }
    return n;
}

Predictor *get_pred(cs_ctx *ctx, int dim) {
    if (dim != 2 && dim != 3) return nullptr;
    return &ctx->pred[dim - 2];
}

uint64_t splitmix(uint64_t &s) {
    uint64_t z = (s += 0x9e3779b97f4a7c15ull);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

cs::Mesh *find_mesh(cs_ctx *ctx, int32_t id) {
    auto it = ctx->meshes.find(id);
    return it == ctx->meshes.end() ? nullptr : it->second;
}

// The static P1 interpolation table of the ASG cell centres (built once).
cs_status ensure_interp(cs_ctx *ctx, cs::Mesh *m, cudaStream_t st) {
    if (m->interp_node) return CS_OK;
    const size_t n = size_t(pred_view(m->d).n_asg) * (m->d.dim + 1);
    cs_status rc = dalloc(ctx, &m->interp_node, n);
    if (rc) return rc;
    m->allocs.push_back(m->interp_node);
    rc = dalloc(ctx, &m->interp_w, n);
    if (rc) return rc;
    m->allocs.push_back(m->interp_w);
    ctx->launches += launch_interp_table(pred_view(m->d), m->interp_node, m->interp_w, ctx->sm_count, st);
    return CS_OK;
}

cs_status ensure_mesh_grid(cs_ctx *ctx, cs::Mesh *m) {
    const size_t n = size_t(pred_view(m->d).n_asg) * m->d.dim;
    if (!m->grid_u) {
        cs_status rc = dalloc(ctx, &m->grid_u, n);
        if (rc) return rc;
        m->allocs.push_back(m->grid_u);
    }
    if (!m->grid_dhat) {
        cs_status rc = dalloc(ctx, &m->grid_dhat, n);
        if (rc) return rc;
        m->allocs.push_back(m->grid_dhat);
    }
    return CS_OK;
}

}  // namespace

namespace cs {

void predictor_release(cs_ctx *ctx, Predictor &P) {
    free_workspace(ctx, P);
    float **fs[] = {&P.w, &P.g, &P.m, &P.v, &P.loss};
    for (float **f : fs) {
        dfree(ctx, *f);
        *f = nullptr;
    }
    dfree(ctx, P.packed);
    P.packed = nullptr;
    P.packed_dirty = true;
    P.loaded = false;
}

// Fully convolutional prediction over the predictor grid on CUDA cores: the
// grid is cut into cubic tiles of T^D cells, each evaluated as one window of
// side T + 2 R through the window engine's layers (convolutions as implicit
// GEMMs fused with bias and ReLU), so the convolutions are shared between
// neighbouring cells instead of being recomputed for each cell's own window.
struct TilePlan {
    int T = 1, nt[3] = {1, 1, 1};
    int64_t n_tiles = 1, Bt = 1;
    std::vector<int64_t> per;   // floats per tile of each workspace buffer
};

TilePlan plan_tiles(const DevMesh &pv) {
    const int D = pv.dim;
    NetShape S(D);
    const int R = S.n_conv;
    TilePlan t;
    for (int k = 0; k < D; ++k) {
        const int n = (pv.ga[k] + 23) / 24;            // tiles of at most 24 cells per axis
        t.T = std::max(t.T, (pv.ga[k] + n - 1) / n);
    }
    for (int k = 0; k < D; ++k) t.nt[k] = (pv.ga[k] + t.T - 1) / t.T;
    t.n_tiles = int64_t(t.nt[0]) * t.nt[1] * t.nt[2];
    // buffer sizes per tile: input, then (col, z, y) per conv layer, z5, a5, out
    int Si = t.T + 2 * R, C = S.cin;
    t.per.push_back(int64_t(C) * S.positions(Si));
    for (int l = 0; l < S.n_conv; ++l) {
        // (col, z, y): the fused convolution needs neither an im2col copy nor
        // the pre-activation, so only y has a size
        const int64_t Po = S.positions(Si - 2);
        t.per.push_back(1);
        t.per.push_back(1);
        t.per.push_back(Po * S.ch);
        Si -= 2;
        C = S.ch;
    }
    t.per.push_back(1);                 // z5, a5: the fused head keeps them in registers
    t.per.push_back(1);
    t.per.push_back(S.positions(t.T) * D);
    int64_t tile_floats = 0;
    for (int64_t v : t.per) tile_floats += v;
    t.Bt = std::max<int64_t>(1, std::min<int64_t>(t.n_tiles, (int64_t(1) << 28) / tile_floats));
    return t;
}

// Grow the tile workspace to hold plan t (buffers only grow, so a workspace
// sized for every mesh of a serving run is never reallocated while in use).
cs_status grow_tiles(cs_ctx *ctx, Predictor &P, const TilePlan &t) {
    std::vector<int64_t> need(t.per.size());
    for (size_t i = 0; i < t.per.size(); ++i) need[i] = t.per[i] * t.Bt;
    bool fits = P.tiles.size() == need.size() && int64_t(P.tiles_cap.size()) == int64_t(need.size());
    for (size_t i = 0; fits && i < need.size(); ++i) fits = P.tiles_cap[i] >= need[i];
    if (fits) return CS_OK;
    std::vector<int64_t> cap(need.size());
    for (size_t i = 0; i < need.size(); ++i)
        cap[i] = std::max(need[i], i < P.tiles_cap.size() ? P.tiles_cap[i] : int64_t(0));
    for (float *p : P.tiles) dfree(ctx, p);
    P.tiles.clear();
    P.tiles_cap.clear();
    for (int64_t v : cap) {
        float *b = nullptr;
        cs_status rc = dalloc(ctx, &b, size_t(v));
        if (rc) {
            for (float *p : P.tiles) dfree(ctx, p);
            P.tiles.clear();
            return rc;
        }
        P.tiles.push_back(b);
    }
    P.tiles_cap = cap;
    return CS_OK;
}

cs_status predict_tiles(cs_ctx *ctx, Predictor &P, cs::Mesh *m, const float *grid, double dt,
                        float *dhat, cudaStream_t st) {
    const DevMesh pv = pred_view(m->d);
    const int D = pv.dim;
    NetShape S(D);
    const int R = S.n_conv;
    const TilePlan tp = plan_tiles(pv);
    cs_status rc = grow_tiles(ctx, P, tp);
    if (rc) return rc;
    const int T = tp.T;
    const int64_t n_tiles = tp.n_tiles, Bt = tp.Bt;
    const int64_t P_out = S.positions(T);
    float scale[3] = {0, 0, 0};
    for (int k = 0; k < D; ++k) scale[k] = float(dt / pv.sa[k]);
    const int sm = ctx->sm_count;
    for (int64_t t0 = 0; t0 < n_tiles; t0 += Bt) {
        const int64_t B = std::min(Bt, n_tiles - t0);
        ctx->launches += launch_tile_input(pv, grid, T, R, tp.nt[0], tp.nt[1], t0, B, scale,
                                           P.tiles[0], sm, st);
        const float *x = P.tiles[0];
        bool chfirst = true;
        int Ci = S.cin, Sl = T + 2 * R;
        for (int l = 0; l < S.n_conv; ++l) {
            float *y = P.tiles[3 + 3 * l];
            ctx->launches += launch_conv_relu(D, x, chfirst, B, Ci, Sl, P.w + S.w_off[l],
                                              P.w + S.b_off[l], y, st);
            x = y;
            chfirst = false;
            Ci = S.ch;
            Sl -= 2;
        }
        const int f1 = S.n_conv, f2 = S.n_conv + 1;
        float *out = P.tiles[3 + 3 * S.n_conv];
        const int64_t M = B * P_out;
        ctx->launches += launch_head(D, x, P.w + S.w_off[f1], P.w + S.b_off[f1], P.w + S.w_off[f2],
                                     P.w + S.b_off[f2], M, out, sm, st);
        ctx->launches += launch_tile_scatter(pv, T, tp.nt[0], tp.nt[1], t0, B, out, dhat, sm, st);
    }
    return CS_OK;
}

// prediction at every predictor cell of mesh m from the grid velocity `grid`
// Prediction at every predictor cell from `src`: the grid velocity, or (the
// tensor-core engine only) the nodal velocity, resampled as the kernel loads
// its tiles
cs_status predict_grid_src(cs_ctx *ctx, cs::Mesh *m, const TcSource &src, double dt, float *dhat,
                           cudaStream_t st) {
    Predictor *P = get_pred(ctx, m->d.dim);
    if (!P || !P->loaded) return fail(ctx, CS_ENOPRED, "no predictor loaded for this dimension");
    const float *grid = src.U;
    if (!grid && !(src.node && ctx->engine == 1))
        return fail(ctx, CS_EINVAL, "the mesh has no grid velocity yet");
    if (ctx->engine == 1) {
        // tensor-core grid kernels: weights repacked after every load / training
        const int64_t bytes = m->d.dim == 2 ? tc_packed_bytes() : tc3_packed_bytes();
        if (!P->packed) {
            cs_status rc = dalloc(ctx, &P->packed, size_t(bytes));
            if (rc) return rc;
        }
        if (!ctx->dev_err) {
            cs_status rc = dalloc(ctx, &ctx->dev_err, 1);
            if (rc) return rc;
            PCHK(cudaMemset(ctx->dev_err, 0, sizeof(int)));
        }
        if (P->packed_dirty) {
            ctx->launches += m->d.dim == 2 ? launch_pack_tc(P->w, NetShape(2), P->packed, st)
                                           : launch_pack_tc3(P->w, NetShape(3), P->packed, st);
            P->packed_dirty = false;
        }
        TcHold hold;
        if (ctx->hold_flag) {
            hold.flag = ctx->hold_flag;
            hold.polls = 1u << 16;
        }
        if (m->d.dim == 2)
            ctx->launches += launch_cnn2d_tc(pred_view(m->d), src, dt, P->packed, dhat,
                                             ctx->dev_err, ctx->sm_count, ctx->tc_tile_rows, st,
                                             hold);
        else
            ctx->launches += launch_cnn3d_tc(pred_view(m->d), src, dt, P->packed, dhat,
                                             ctx->dev_err, ctx->sm_count, ctx->tc3_tile, st, hold);
        return CS_OK;
    }
    if (m->d.dim == 3 && ctx->engine == 2) return predict_tiles(ctx, *P, m, grid, dt, dhat, st);
    const int64_t chunk = 8192;
    cs_status rc = ensure_workspace(ctx, *P, chunk);
    if (rc) return rc;
    const int D = m->d.dim;
    float scale[3] = {0, 0, 0};
    for (int k = 0; k < D; ++k) scale[k] = float(dt / pred_view(m->d).sa[k]);
    for (int64_t c0 = 0; c0 < pred_view(m->d).n_asg; c0 += chunk) {
        const int64_t B = std::min(chunk, pred_view(m->d).n_asg - c0);
        ctx->launches += launch_windows(pred_view(m->d), grid, nullptr, c0, B, scale, P->win,
                                        ctx->sm_count, st);
        ctx->launches += forward(ctx, *P, B, P->win, st);
        PCHK(cudaMemcpyAsync(dhat + c0 * D, P->out, size_t(B) * D * sizeof(float),
                             cudaMemcpyDeviceToDevice, st));
    }
    return CS_OK;
}

cs_status predict_grid(cs_ctx *ctx, cs::Mesh *m, const float *grid, double dt, float *dhat,
                       cudaStream_t st) {
    TcSource src;
    src.U = grid;
    return predict_grid_src(ctx, m, src, dt, dhat, st);
}

cs_status reserve_tiles(cs_ctx *ctx, cs::Mesh *m) {
    if (m->d.dim != 3 || ctx->engine != 2) return CS_OK;
    Predictor *P = get_pred(ctx, 3);
    if (!P || !P->loaded) return CS_OK;
    return grow_tiles(ctx, *P, plan_tiles(pred_view(m->d)));
}

bool serving_predictor_ready(cs_ctx *ctx, const cs::Mesh *m) {
    const Predictor &P = ctx->pred[m->d.dim - 2];
    if (!P.loaded || !m->interp_node) return false;
    if (ctx->engine == 1) return P.packed && !P.packed_dirty && ctx->dev_err;
    return ctx->engine == 2 && m->d.dim == 3 && !P.tiles.empty();
}

cs_status prepare_serving(cs_ctx *ctx) {
    for (int dim = 2; dim <= 3; ++dim) {
        Predictor &P = ctx->pred[dim - 2];
        if (!P.loaded || (ctx->engine != 1 && ctx->engine != 2)) continue;
        if (ctx->engine == 1) {
            const int64_t bytes = dim == 2 ? tc_packed_bytes() : tc3_packed_bytes();
            if (!P.packed) {
                cs_status rc = dalloc(ctx, &P.packed, size_t(bytes));
                if (rc) return rc;
            }
            if (!ctx->dev_err) {
                cs_status rc = dalloc(ctx, &ctx->dev_err, 1);
                if (rc) return rc;
                PCHK(cudaMemset(ctx->dev_err, 0, sizeof(int)));
            }
            if (P.packed_dirty) {
                ctx->launches += dim == 2 ? launch_pack_tc(P.w, NetShape(2), P.packed, nullptr)
                                          : launch_pack_tc3(P.w, NetShape(3), P.packed, nullptr);
                P.packed_dirty = false;
            }
        }
        for (auto &kv : ctx->meshes) {
            cs::Mesh *m = kv.second;
            if (m->d.dim != dim) continue;
            cs_status rc = ensure_interp(ctx, m, nullptr);
            if (rc == CS_OK) rc = reserve_tiles(ctx, m);
            if (rc) return rc;
        }
    }
    for (auto &kv : ctx->fields) {
        auto it = ctx->meshes.find(kv.second->mesh_id);
        if (it == ctx->meshes.end()) continue;
        const float *g = nullptr;
        cs_status rc = field_grid(ctx, it->second, kv.second, nullptr, &g);
        if (rc) return rc;
    }
    PCHK(cudaDeviceSynchronize());
    return CS_OK;
}

cs_status field_grid(cs_ctx *ctx, cs::Mesh *m, cs::Field *f, cudaStream_t st,
                     const float **grid_out) {
    if (f->grid_version != m->pgrid_version || !f->grid_u) {
        dfree(ctx, f->grid_u);
        f->grid_u = nullptr;
        f->grid_version = -1;
        cs_status rc = dalloc(ctx, &f->grid_u, size_t(m->d.n_pasg) * m->d.dim);
        if (rc) return rc;
        rc = ensure_interp(ctx, m, st);
        if (rc) return rc;
        ctx->launches += launch_resample(pred_view(m->d), m->interp_node, m->interp_w, f->u_nodal,
                                         f->grid_u, ctx->sm_count, st);
        f->grid_version = m->pgrid_version;
    }
    *grid_out = f->grid_u;
    return CS_OK;
}

cs_status cnn_prepare(cs_ctx *ctx, cs::Mesh *m, const float *grid, const double *u_nodal,
                      double dt, cudaStream_t st, const float **dhat_out) {
    cs_status rc = ensure_mesh_grid(ctx, m);
    if (rc) return rc;
    if (!grid) {
        if (!u_nodal) return fail(ctx, CS_EINVAL, "no velocity for the start predictor");
        rc = ensure_interp(ctx, m, st);
        if (rc) return rc;
        if (ctx->engine == 1 && m->d.dim == 2) {
            // the 2-D tensor-core kernel resamples as it loads its tiles and
            // stores the grid velocity in the mesh (the same bits as the
            // resample kernel). In 3-D a tile's (T + 6)^3 input cells are
            // many times its T^3 own cells, so the separate resample is
            // cheaper there.
            TcSource src;
            src.node = m->interp_node;
            src.w = m->interp_w;
            src.un = u_nodal;
            src.U_out = m->grid_u;
            const int ev = ctx->prof.begin(CS_STAGE_CNN, st);
            rc = predict_grid_src(ctx, m, src, dt, m->grid_dhat, st);
            ctx->prof.end(ev, st);
            if (rc) return rc;
            m->grid_u_valid = true;
            *dhat_out = m->grid_dhat;
            return CS_OK;
        }
        const int ev = ctx->prof.begin(CS_STAGE_RESAMPLE, st);
        ctx->launches += launch_resample(pred_view(m->d), m->interp_node, m->interp_w, u_nodal, m->grid_u,
                                         ctx->sm_count, st);
        ctx->prof.end(ev, st);
        m->grid_u_valid = true;
        grid = m->grid_u;
    }
    const int ev = ctx->prof.begin(CS_STAGE_CNN, st);
    rc = predict_grid(ctx, m, grid, dt, m->grid_dhat, st);
    ctx->prof.end(ev, st);
    if (rc) return rc;
    *dhat_out = m->grid_dhat;
    return CS_OK;
}

}  // namespace cs

extern "C" {

cs_status cs_predictor_engine(cs_ctx *ctx, int engine) {
    if (!ctx || engine < 0 || engine > 2) return CS_EINVAL;
    if (ctx->server) return fail(ctx, CS_EBUSY, "cs_predictor_engine: stop serving first");
    ctx->engine = engine;
    return CS_OK;
}

cs_status cs_debug_hold_predictor(cs_ctx *ctx, int on) {
    if (!ctx) return CS_EINVAL;
    PCHK(cudaSetDevice(ctx->device));
    PCHK(cudaDeviceSynchronize());
    if (!on) {
        dfree(ctx, ctx->hold_flag);
        ctx->hold_flag = nullptr;
        return CS_OK;
    }
    if (!ctx->hold_flag) {
        cs_status rc = dalloc(ctx, &ctx->hold_flag, 1);
        if (rc) return rc;
    }
    PCHK(cudaMemset(ctx->hold_flag, 0, sizeof(int)));
    return CS_OK;
}

cs_status cs_predictor_tile3(cs_ctx *ctx, int side) {
    if (!ctx) return CS_EINVAL;
    if (side != 0 && side != 2 && side != 3 && side != 4)
        return fail(ctx, CS_EINVAL, "cs_predictor_tile3: side must be 0, 2, 3 or 4");
    ctx->tc3_tile = side;
    return CS_OK;
}

cs_status cs_predictor_tile_rows(cs_ctx *ctx, int rows) {
    if (!ctx) return CS_EINVAL;
    if (rows != 0 && rows != 8 && rows != 13 && rows != 24)
        return fail(ctx, CS_EINVAL, "cs_predictor_tile_rows: rows must be 0, 8, 13 or 24");
    ctx->tc_tile_rows = rows;
    return CS_OK;
}

cs_status cs_device_status(cs_ctx *ctx) {
    if (!ctx) return CS_EINVAL;
    PCHK(cudaSetDevice(ctx->device));
    PCHK(cudaDeviceSynchronize());
    if (!ctx->dev_err) return CS_OK;
    int e = 0;
    PCHK(cudaMemcpy(&e, ctx->dev_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (e) {
        PCHK(cudaMemset(ctx->dev_err, 0, sizeof(int)));
        return fail(ctx, CS_EDEVICE, "a bounded device wait gave up (tensor-core kernel)");
    }
    return CS_OK;
}

cs_status cs_predictor_precision(cs_ctx *ctx, int bf16) {
    if (!ctx) return CS_EINVAL;
    set_gemm_bf16(bf16 != 0);
    return CS_OK;
}

int64_t cs_predictor_size(int dim) {
    if (dim != 2 && dim != 3) return 0;
    return NetShape(dim).n_params;
}

cs_status cs_predictor_load(cs_ctx *ctx, int dim, const float *weights, int64_t n) {
    if (!ctx) return CS_EINVAL;
    Predictor *P = get_pred(ctx, dim);
    if (!P || !weights || n != cs_predictor_size(dim))
        return fail(ctx, CS_EINVAL, "cs_predictor_load: bad dim or size (expected " +
                                        std::to_string(cs_predictor_size(dim)) + " floats)");
    PCHK(cudaSetDevice(ctx->device));
    predictor_release(ctx, *P);
    P->dim = dim;
    P->n = n;
    cs_status rc;
    if ((rc = dalloc(ctx, &P->w, size_t(n))) || (rc = dalloc(ctx, &P->g, size_t(n))) ||
        (rc = dalloc(ctx, &P->m, size_t(n))) || (rc = dalloc(ctx, &P->v, size_t(n))) ||
        (rc = dalloc(ctx, &P->loss, 1))) {
        predictor_release(ctx, *P);
        return rc;
    }
    PCHK(cudaMemcpy(P->w, weights, size_t(n) * sizeof(float), cudaMemcpyHostToDevice));
    PCHK(cudaMemset(P->m, 0, size_t(n) * sizeof(float)));
    PCHK(cudaMemset(P->v, 0, size_t(n) * sizeof(float)));
    P->t = 0;
    P->loaded = true;
    return CS_OK;
}

cs_status cs_predictor_save(cs_ctx *ctx, int dim, float *out, int64_t n) {
    if (!ctx) return CS_EINVAL;
    Predictor *P = get_pred(ctx, dim);
    if (!P || !out || n != cs_predictor_size(dim))
        return fail(ctx, CS_EINVAL, "cs_predictor_save: bad dim or size");
    if (!P->loaded) return fail(ctx, CS_ENOPRED, "cs_predictor_save: no predictor loaded");
    PCHK(cudaSetDevice(ctx->device));
    PCHK(cudaDeviceSynchronize());
    PCHK(cudaMemcpy(out, P->w, size_t(n) * sizeof(float), cudaMemcpyDeviceToHost));
    return CS_OK;
}

cs_status cs_predictor_grid(cs_ctx *ctx, int32_t mesh_id, int32_t stride) {
    if (!ctx) return CS_EINVAL;
    cs::Mesh *m = find_mesh(ctx, mesh_id);
    if (!m) return fail(ctx, CS_ENOMESH, "cs_predictor_grid: unknown mesh id");
    if (ctx->server) return fail(ctx, CS_EBUSY, "cs_predictor_grid: stop serving first");
    cs::DevMesh &d = m->d;
    if (stride < 1 || stride % 2 == 0)
        return fail(ctx, CS_EINVAL, "cs_predictor_grid: the stride must be odd and >= 1");
    for (int k = 0; k < d.dim; ++k)
        if (d.ga[k] < stride)
            return fail(ctx, CS_EINVAL, "cs_predictor_grid: stride larger than the ASG grid");
    PCHK(cudaSetDevice(ctx->device));
    PCHK(cudaDeviceSynchronize());
    // drop the buffers of the old predictor grid (its centre hosts, grid
    // velocity, predictions and interpolation table)
    void *old[] = {d.pseed == d.seed ? nullptr : const_cast<int32_t *>(d.pseed), m->grid_u,
                   m->grid_dhat, m->interp_node, m->interp_w};
    for (void *q : old) {
        if (!q) continue;
        auto it = std::find(m->allocs.begin(), m->allocs.end(), q);
        if (it != m->allocs.end()) m->allocs.erase(it);
        dfree(ctx, q);
    }
    m->pgrid_version += 1;   // the fields' grid velocities are resampled at next use
    m->grid_u = m->grid_dhat = nullptr;
    m->interp_node = nullptr;
    m->interp_w = nullptr;
    m->grid_u_valid = false;
    d.pstride = stride;
    int64_t n = 1;
    for (int k = 0; k < 3; ++k) {
        d.pga[k] = k < d.dim ? d.ga[k] / stride : 1;
        d.psa[k] = k < d.dim ? d.sa[k] * double(stride) : 1.0;
        d.pinv_sa[k] = static_cast<float>(1.0 / d.psa[k]);
        d.psa_f[k] = static_cast<float>(d.psa[k]);
        n *= d.pga[k];
        m->info.pred_grid[k] = d.pga[k];
    }
    d.n_pasg = n;
    m->info.pred_stride = stride;
    if (stride == 1) {
        d.pseed = d.seed;
        return CS_OK;
    }
    int32_t *ps = nullptr;
    cs_status rc = dalloc(ctx, &ps, size_t(n));
    if (rc) return rc;
    m->allocs.push_back(ps);
    d.pseed = ps;
    ctx->launches += launch_pred_seed(d, ps, ctx->sm_count, nullptr);
    PCHK(cudaGetLastError());
    return CS_OK;
}

cs_status cs_grid_velocity(cs_ctx *ctx, int32_t mesh_id, const double *u_nodal, float *grid_out,
                           void *stream) {
    if (!ctx) return CS_EINVAL;
    cs::Mesh *m = find_mesh(ctx, mesh_id);
    if (!m) return fail(ctx, CS_ENOMESH, "cs_grid_velocity: unknown mesh id");
    if (!u_nodal) return fail(ctx, CS_EINVAL, "cs_grid_velocity: null velocity");
    PCHK(cudaSetDevice(ctx->device));
    float *dst = grid_out;
    if (!dst) {
        cs_status rc = ensure_mesh_grid(ctx, m);
        if (rc) return rc;
        dst = m->grid_u;
        m->grid_u_valid = true;
    }
    cs_status rc = ensure_interp(ctx, m, static_cast<cudaStream_t>(stream));
    if (rc) return rc;
    ctx->launches += launch_resample(pred_view(m->d), m->interp_node, m->interp_w, u_nodal, dst,
                                     ctx->sm_count, static_cast<cudaStream_t>(stream));
    PCHK(cudaGetLastError());
    return CS_OK;
}

cs_status cs_windows(cs_ctx *ctx, int32_t mesh_id, const float *grid, double dt,
                     const int64_t *cells, int64_t B, float *out, void *stream) {
    if (!ctx) return CS_EINVAL;
    cs::Mesh *m = find_mesh(ctx, mesh_id);
    if (!m) return fail(ctx, CS_ENOMESH, "cs_windows: unknown mesh id");
    if (B < 0 || !out) return fail(ctx, CS_EINVAL, "cs_windows: bad size or null output");
    if (!grid && !m->grid_u_valid) return fail(ctx, CS_EINVAL, "cs_windows: no grid velocity");
    if (B == 0) return CS_OK;
    PCHK(cudaSetDevice(ctx->device));
    float scale[3] = {0, 0, 0};
    for (int k = 0; k < m->d.dim; ++k) scale[k] = float(dt / pred_view(m->d).sa[k]);
    ctx->launches += launch_windows(pred_view(m->d), grid ? grid : m->grid_u, cells, 0, B, scale, out,
                                    ctx->sm_count, static_cast<cudaStream_t>(stream));
    PCHK(cudaGetLastError());
    return CS_OK;
}

cs_status cs_predictor_forward(cs_ctx *ctx, int dim, int64_t B, const float *windows,
                               float *dhat_out) {
    if (!ctx) return CS_EINVAL;
    Predictor *P = get_pred(ctx, dim);
    if (!P || B < 0 || (B > 0 && (!windows || !dhat_out)))
        return fail(ctx, CS_EINVAL, "cs_predictor_forward: bad arguments");
    if (!P->loaded) return fail(ctx, CS_ENOPRED, "cs_predictor_forward: no predictor loaded");
    PCHK(cudaSetDevice(ctx->device));
    const int64_t chunk = 8192;
    cs_status rc = ensure_workspace(ctx, *P, std::min<int64_t>(std::max<int64_t>(B, 1), chunk));
    if (rc) return rc;
    NetShape S(dim);
    const int64_t row = int64_t(S.cin) * S.positions(S.S0);
    for (int64_t b0 = 0; b0 < B; b0 += P->cap) {
        const int64_t nb = std::min(P->cap, B - b0);
        ctx->launches += forward(ctx, *P, nb, windows + b0 * row, nullptr);
        PCHK(cudaMemcpyAsync(dhat_out + b0 * dim, P->out, size_t(nb) * dim * sizeof(float),
                             cudaMemcpyDeviceToDevice, nullptr));
    }
    PCHK(cudaDeviceSynchronize());
    return CS_OK;
}

cs_status cs_predict(cs_ctx *ctx, int32_t mesh_id, double dt, float *dhat_out, void *stream) {
    if (!ctx) return CS_EINVAL;
    cs::Mesh *m = find_mesh(ctx, mesh_id);
    if (!m) return fail(ctx, CS_ENOMESH, "cs_predict: unknown mesh id");
    PCHK(cudaSetDevice(ctx->device));
    cs_status rc = ensure_mesh_grid(ctx, m);
    if (rc) return rc;
    rc = predict_grid(ctx, m, m->grid_u_valid ? m->grid_u : nullptr, dt,
                      dhat_out ? dhat_out : m->grid_dhat, static_cast<cudaStream_t>(stream));
    if (rc) return rc;
    PCHK(cudaGetLastError());
    return CS_OK;
}

cs_status cs_predictor_train(cs_ctx *ctx, int dim, const float *windows, const float *targets,
                             int64_t N, int64_t batch, int64_t steps, float lr, uint64_t seed,
                             float *loss_out) {
    if (!ctx) return CS_EINVAL;
    Predictor *P = get_pred(ctx, dim);
    if (!P || !windows || !targets || N < 1 || batch < 1 || steps < 0 || !(lr > 0.f))
        return fail(ctx, CS_EINVAL, "cs_predictor_train: bad arguments");
    if (!P->loaded) return fail(ctx, CS_ENOPRED, "cs_predictor_train: no predictor loaded");
    PCHK(cudaSetDevice(ctx->device));
    const int64_t B = std::min(batch, N);
    cs_status rc = ensure_workspace(ctx, *P, B);
    if (rc) return rc;
    NetShape S(dim);
    const int64_t row = int64_t(S.cin) * S.positions(S.S0);
    float *losses = nullptr;
    if ((rc = dalloc(ctx, &losses, size_t(std::max<int64_t>(steps, 1))))) return rc;
    PCHK(cudaMemset(losses, 0, size_t(std::max<int64_t>(steps, 1)) * sizeof(float)));
    std::vector<int64_t> perm(static_cast<size_t>(N));
    for (int64_t i = 0; i < N; ++i) perm[i] = i;
    uint64_t rs = seed;
    int64_t pos = N;   // force a shuffle at the first step
    std::vector<int64_t> idx(static_cast<size_t>(B));
    cs_status out = CS_OK;
    for (int64_t s = 0; s < steps; ++s) {
        for (int64_t b = 0; b < B; ++b) {
            if (pos >= N) {   // new epoch: Fisher-Yates shuffle
                for (int64_t i = N - 1; i > 0; --i) std::swap(perm[i], perm[splitmix(rs) % (i + 1)]);
                pos = 0;
            }
            idx[b] = perm[pos++];
        }
        if (cudaMemcpy(P->idx, idx.data(), size_t(B) * sizeof(int64_t), cudaMemcpyHostToDevice) !=
            cudaSuccess) {
            out = fail(ctx, CS_ECUDA, "cs_predictor_train: index copy");
            break;
        }
        ctx->launches += launch_gather_rows(windows, row, P->idx, B, P->win, ctx->sm_count, nullptr);
        ctx->launches += launch_gather_rows(targets, dim, P->idx, B, P->tgt, ctx->sm_count, nullptr);
        ctx->launches += forward(ctx, *P, B, P->win, nullptr);
        ctx->launches += backward(ctx, *P, B, P->tgt, losses + s, nullptr);
        P->t += 1;
        ctx->launches += launch_adam(P->w, P->g, P->m, P->v, P->n, lr, P->t, ctx->sm_count, nullptr);
        P->packed_dirty = true;
    }
    if (out == CS_OK) {
        cudaError_t e = cudaDeviceSynchronize();
        if (e == cudaSuccess && loss_out && steps > 0)
            e = cudaMemcpy(loss_out, losses, size_t(steps) * sizeof(float), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) out = fail(ctx, CS_ECUDA, std::string("cs_predictor_train: ") +
                                                            cudaGetErrorString(e));
    }
    dfree(ctx, losses);
    return out;
}

cs_status cs_training_pairs(cs_ctx *ctx, int32_t mesh_id, int64_t n, const double *x,
                            const double *u, double dt, float *windows_out, float *targets_out,
                            int64_t *cells_out, void *stream) {
    if (!ctx) return CS_EINVAL;
    cs::Mesh *m = find_mesh(ctx, mesh_id);
    if (!m) return fail(ctx, CS_ENOMESH, "cs_training_pairs: unknown mesh id");
    if (n < 0 || (n > 0 && (!x || !u || !windows_out || !targets_out || !cells_out)))
        return fail(ctx, CS_EINVAL, "cs_training_pairs: bad arguments");
    if (!m->grid_u_valid) return fail(ctx, CS_EINVAL, "cs_training_pairs: no grid velocity");
    if (n == 0) return CS_OK;
    PCHK(cudaSetDevice(ctx->device));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    ctx->launches += launch_pairs(pred_view(m->d), n, x, u, dt, cells_out, targets_out, ctx->sm_count, st);
    float scale[3] = {0, 0, 0};
    for (int k = 0; k < m->d.dim; ++k) scale[k] = float(dt / pred_view(m->d).sa[k]);
    ctx->launches += launch_windows(pred_view(m->d), m->grid_u, cells_out, 0, n, scale, windows_out,
                                    ctx->sm_count, st);
    PCHK(cudaGetLastError());
    return CS_OK;
}

cs_status cs_predictor_grad(cs_ctx *ctx, int dim, int64_t B, const float *windows,
                            const float *targets, float *grad_out, float *loss_out) {
    if (!ctx) return CS_EINVAL;
    Predictor *P = get_pred(ctx, dim);
    if (!P || B < 1 || !windows || !targets || !grad_out)
        return fail(ctx, CS_EINVAL, "cs_predictor_grad: bad arguments");
    if (!P->loaded) return fail(ctx, CS_ENOPRED, "cs_predictor_grad: no predictor loaded");
    PCHK(cudaSetDevice(ctx->device));
    cs_status rc = ensure_workspace(ctx, *P, B);
    if (rc) return rc;
    PCHK(cudaMemset(P->loss, 0, sizeof(float)));
    ctx->launches += forward(ctx, *P, B, windows, nullptr);
    ctx->launches += backward(ctx, *P, B, targets, P->loss, nullptr);
    PCHK(cudaDeviceSynchronize());
    PCHK(cudaMemcpy(grad_out, P->g, size_t(P->n) * sizeof(float), cudaMemcpyDeviceToDevice));
    if (loss_out) PCHK(cudaMemcpy(loss_out, P->loss, sizeof(float), cudaMemcpyDeviceToHost));
    return CS_OK;
}

cs_status cs_track_dhat(cs_ctx *ctx, int32_t mesh_id, int64_t n, const double *x, const double *u,
                        double dt, const int32_t *start, const float *dhat, int32_t *host_out,
                        int32_t *path_len_out, uint8_t *status_out, int32_t *start_out,
                        void *stream) {
    if (!ctx) return CS_EINVAL;
    cs::Mesh *m = find_mesh(ctx, mesh_id);
    if (!m) return fail(ctx, CS_ENOMESH, "cs_track_dhat: unknown mesh id");
    if (!dhat && !m->grid_dhat) return fail(ctx, CS_EINVAL, "cs_track_dhat: no displacement grid");
    return cs_track_impl(ctx, m, n, x, u, dt, start, CS_CNN_SNS, dhat ? dhat : m->grid_dhat,
                         host_out, path_len_out, status_out, start_out,
                         static_cast<cudaStream_t>(stream));
}

}  // extern "C"
