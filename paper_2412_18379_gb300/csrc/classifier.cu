// The paper's classifier start predictor (Sec. 2.3, Eq. 7-8): the kernels
// around its GEMMs. Inputs (pooled centroid windows and the offset of x_p),
// the layout changes between layers (zero padding, average pooling,
// concatenation), the softmax with its cross-entropy gradient, the labels
// from plain SNS hosts and the start element K_p of the most probable class.
//
// Every FP64 step of the inputs, labels and starts is written with explicit
// round-to-nearest intrinsics, so the integer decisions (cells, labels,
// starts) and the FP64 feature values are those of a plain evaluation of the
// same formulas; the network itself runs in BF16/FP32 (classifier.cpp).

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>

#include "classifier.h"
#include "walk_common.cuh"

namespace cs {
namespace {

constexpr int kT = 256;

int blocks_for(int64_t n, int sm_count, int per_sm = 16) {
    const int64_t b = (n + kT - 1) / kT;
    return int(std::max<int64_t>(1, std::min<int64_t>(b, int64_t(sm_count) * per_sm)));
}

template <int D>
struct Win {
    static constexpr int W = D == 2 ? 9 : 7;        // window edge
    static constexpr int P = D == 2 ? W * W : W * W * W;
    static constexpr int Wq = W + 2;                 // zero-padded edge
    static constexpr int Pq = D == 2 ? Wq * Wq : Wq * Wq * Wq;
    static constexpr int Wp = W / 2;                 // pooled edge (odd row dropped)
    static constexpr int Pp = D == 2 ? Wp * Wp : Wp * Wp * Wp;
};

// x_p = x - (u * dt) (Eq. 3)
__global__ void departure_kernel(int64_t n, const double *__restrict__ x,
                                 const double *__restrict__ u, double dt,
                                 double *__restrict__ xp) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += int64_t(gridDim.x) * blockDim.x)
        xp[i] = __dsub_rn(x[i], __dmul_rn(u[i], dt));
}

// Inputs of row b (particle idx[b], or b): the window of dim channels at
// every (padded, if pad) window position, channels first, and the offset.
// Window cell o (x fastest) of a particle whose ASG cell is c is cell
// c - W/2 + o; its point is the pooled centroid of that cell if the cell is
// in the grid and holds one, else its centre lo + (cell + 1/2) s.
template <int D>
__global__ void __launch_bounds__(kT) features_kernel(const DevMesh m, int64_t B,
                                                      const double *__restrict__ xp,
                                                      const int64_t *__restrict__ idx, int pad,
                                                      float *__restrict__ win,
                                                      float *__restrict__ offset) {
    using G = Win<D>;
    const int E = G::W + 2 * pad;                    // stored edge
    const int PE = D == 2 ? E * E : E * E * E;
    const int64_t total = B * PE;
    for (int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; q < total;
         q += int64_t(gridDim.x) * blockDim.x) {
        const int64_t b = q / PE;
        const int pe = int(q % PE);
        int e[3] = {pe % E, (pe / E) % E, D == 3 ? pe / (E * E) : 0};
        bool ring = false;
        #pragma unroll
        for (int k = 0; k < D; ++k) {
            e[k] -= pad;
            ring |= e[k] < 0 || e[k] >= G::W;
        }
        float *out = win + b * D * PE + pe;
        if (ring) {
            #pragma unroll
            for (int k = 0; k < D; ++k) out[int64_t(k) * PE] = 0.f;
            continue;
        }
        const int64_t r = idx ? idx[b] : b;
        double x[D];
        int64_t c0[D], cc[D];
        bool inside = true;
        #pragma unroll
        for (int k = 0; k < D; ++k) {
            x[k] = xp[r * D + k];
            c0[k] = cell_axis64(x[k], m.lo[k], m.sa[k], m.ga[k]);
            cc[k] = c0[k] - G::W / 2 + e[k];
            inside &= cc[k] >= 0 && cc[k] < m.ga[k];
        }
        int64_t flat = 0;
        #pragma unroll
        for (int k = D - 1; k >= 0; --k) {
            const int64_t ck = cc[k] < 0 ? 0 : (cc[k] > m.ga[k] - 1 ? m.ga[k] - 1 : cc[k]);
            flat = flat * m.ga[k] + ck;
        }
        const bool has = inside && !isnan(m.pool[flat * D]);
        #pragma unroll
        for (int k = 0; k < D; ++k) {
            const double pt = has ? m.pool[flat * D + k]
                                  : __dadd_rn(m.lo[k], __dmul_rn(double(cc[k]) + 0.5, m.sa[k]));
            out[int64_t(k) * PE] = float(__ddiv_rn(__dsub_rn(pt, x[k]), m.sa[k]));
        }
        if (e[0] == 0 && e[1] == 0 && e[2] == 0) {
            #pragma unroll
            for (int k = 0; k < D; ++k)
                offset[b * D + k] = float(__dsub_rn(__ddiv_rn(__dsub_rn(x[k], m.lo[k]), m.sa[k]),
                                                    double(c0[k]) + 0.5));
        }
    }
}

// a[b][q][c] = y[b][p(q)][c] at the interior of the padded window, 0 on its
// ring (channels last): the zero padding of the second convolution
template <int D>
__global__ void __launch_bounds__(kT) pad_kernel(const float *__restrict__ y, int64_t B, int C,
                                                 float *__restrict__ a) {
    using G = Win<D>;
    const int64_t total = B * G::Pq * C;
    for (int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; q < total;
         q += int64_t(gridDim.x) * blockDim.x) {
        const int c = int(q % C);
        const int64_t bq = q / C;
        const int pq = int(bq % G::Pq);
        const int64_t b = bq / G::Pq;
        const int qx = pq % G::Wq, qy = (pq / G::Wq) % G::Wq, qz = D == 3 ? pq / (G::Wq * G::Wq) : 1;
        const bool ring = qx == 0 || qy == 0 || qx == G::Wq - 1 || qy == G::Wq - 1 ||
                          (D == 3 && (qz == 0 || qz == G::Wq - 1));
        if (ring) {
            a[q] = 0.f;
            continue;
        }
        const int p = D == 2 ? (qy - 1) * G::W + qx - 1 : ((qz - 1) * G::W + qy - 1) * G::W + qx - 1;
        a[q] = y[(b * G::P + p) * C + c];
    }
}

// dz[b][p][c] = dpad[b][q(p)][c] * (z[b][p][c] > 0): the padded gradient of
// the second convolution's input, cropped, through the first ReLU
template <int D>
__global__ void __launch_bounds__(kT) crop_relu_back_kernel(const float *__restrict__ dpad,
                                                            const float *__restrict__ z, int64_t B,
                                                            int C, float *__restrict__ dz) {
    using G = Win<D>;
    const int64_t total = B * G::P * C;
    for (int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; q < total;
         q += int64_t(gridDim.x) * blockDim.x) {
        const int c = int(q % C);
        const int64_t bp = q / C;
        const int p = int(bp % G::P);
        const int64_t b = bp / G::P;
        const int px = p % G::W, py = (p / G::W) % G::W, pz = D == 3 ? p / (G::W * G::W) : -1;
        const int pq = D == 2 ? (py + 1) * G::Wq + px + 1
                              : ((pz + 1) * G::Wq + py + 1) * G::Wq + px + 1;
        dz[q] = z[q] > 0.f ? dpad[(b * G::Pq + pq) * C + c] : 0.f;
    }
}

// Average pooling of ReLU(z) over 2^D blocks (stride 2, the last odd row
// dropped) into the first 32 Pp columns of cat (row stride ldc), in the
// order [channel][z][y][x]
template <int D>
__global__ void __launch_bounds__(kT) pool_relu_kernel(const float *__restrict__ z, int64_t B,
                                                       float *__restrict__ cat, int64_t ldc) {
    using G = Win<D>;
    constexpr int C = kClsCh;
    const int64_t total = B * C * G::Pp;
    for (int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; q < total;
         q += int64_t(gridDim.x) * blockDim.x) {
        const int pp = int(q % G::Pp);
        const int c = int((q / G::Pp) % C);
        const int64_t b = q / (int64_t(C) * G::Pp);
        const int px = pp % G::Wp, py = (pp / G::Wp) % G::Wp, pz = D == 3 ? pp / (G::Wp * G::Wp) : 0;
        float s = 0.f;
        for (int oz = 0; oz < (D == 3 ? 2 : 1); ++oz)
            for (int oy = 0; oy < 2; ++oy)
                for (int ox = 0; ox < 2; ++ox) {
                    const int x = 2 * px + ox, y = 2 * py + oy, zz = 2 * pz + oz;
                    const int p = D == 2 ? y * G::W + x : (zz * G::W + y) * G::W + x;
                    s += fmaxf(z[(b * G::P + p) * C + c], 0.f);
                }
        cat[b * ldc + int64_t(c) * G::Pp + pp] = s / float(1 << D);
    }
}

// dz[b][p][c] = (dcat[b][c Pp + pooled(p)] / 2^D if p lies in a pooled block,
// else 0) * (z > 0): the pooling's gradient through the second ReLU
template <int D>
__global__ void __launch_bounds__(kT) pool_back_kernel(const float *__restrict__ dcat, int64_t ldc,
                                                       const float *__restrict__ z, int64_t B,
                                                       float *__restrict__ dz) {
    using G = Win<D>;
    constexpr int C = kClsCh;
    const int64_t total = B * G::P * C;
    for (int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; q < total;
         q += int64_t(gridDim.x) * blockDim.x) {
        const int c = int(q % C);
        const int64_t bp = q / C;
        const int p = int(bp % G::P);
        const int64_t b = bp / G::P;
        const int px = p % G::W, py = (p / G::W) % G::W, pz = D == 3 ? p / (G::W * G::W) : 0;
        float g = 0.f;
        if (px < 2 * G::Wp && py < 2 * G::Wp && (D == 2 || pz < 2 * G::Wp) && z[q] > 0.f) {
            const int pp = D == 2 ? (py / 2) * G::Wp + px / 2
                                  : ((pz / 2) * G::Wp + py / 2) * G::Wp + px / 2;
            g = dcat[b * ldc + int64_t(c) * G::Pp + pp] / float(1 << D);
        }
        dz[q] = g;
    }
}

// cat[b][off + j] = relu(y[b][j]) (the offset branch's output) and its
// gradient dy[b][j] = dcat[b][off + j] * (y > 0)
__global__ void cat_relu_kernel(const float *__restrict__ y, int64_t B, int n,
                                float *__restrict__ cat, int64_t ldc, int64_t off) {
    const int64_t total = B * n;
    for (int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; q < total;
         q += int64_t(gridDim.x) * blockDim.x)
        cat[(q / n) * ldc + off + q % n] = fmaxf(y[q], 0.f);
}
__global__ void uncat_relu_back_kernel(const float *__restrict__ dcat, int64_t ldc, int64_t off,
                                       const float *__restrict__ y, int64_t B, int n,
                                       float *__restrict__ dy) {
    const int64_t total = B * n;
    for (int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; q < total;
         q += int64_t(gridDim.x) * blockDim.x)
        dy[q] = y[q] > 0.f ? dcat[(q / n) * ldc + off + q % n] : 0.f;
}

__device__ __forceinline__ float warp_sum(float v) {
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}
__device__ __forceinline__ float warp_max(float v) {
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(kFull, v, o));
    return v;
}

// Softmax of every row of H (Eq. 7) and the gradient of the mean
// cross-entropy over the rows with a label in [0, n_cls):
// dH = (softmax - onehot) / n_valid, 0 on the other rows; the loss is added
// to *loss. One block, one warp per row, reductions in a fixed order: the
// same bits on every run.
__global__ void __launch_bounds__(1024) softmax_ce_kernel(const float *__restrict__ H,
                                                          const int32_t *__restrict__ labels,
                                                          const int64_t *__restrict__ idx,
                                                          int64_t B, int n_cls,
                                                          float *__restrict__ dH,
                                                          float *__restrict__ loss) {
    __shared__ float red[32];
    __shared__ int cnt[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int c = 0;
    for (int64_t b = threadIdx.x; b < B; b += blockDim.x) {
        const int32_t l = labels[idx ? idx[b] : b];
        c += l >= 0 && l < n_cls;
    }
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(kFull, c, o);
    if (lane == 0) cnt[warp] = c;
    __syncthreads();
    int n_valid = 0;
    for (int w = 0; w < nw; ++w) n_valid += cnt[w];
    const float inv = n_valid > 0 ? 1.f / float(n_valid) : 0.f;
    float lsum = 0.f;
    for (int64_t b = warp; b < B; b += nw) {
        const int32_t l = labels[idx ? idx[b] : b];
        const bool valid = l >= 0 && l < n_cls;
        const float *h = H + b * n_cls;
        float mx = -INFINITY;
        for (int j = lane; j < n_cls; j += 32) mx = fmaxf(mx, h[j]);
        mx = warp_max(mx);
        float se = 0.f;
        for (int j = lane; j < n_cls; j += 32) se += expf(h[j] - mx);
        se = warp_sum(se);
        const float rse = 1.f / se;
        float *g = dH + b * n_cls;
        for (int j = lane; j < n_cls; j += 32)
            g[j] = valid ? (expf(h[j] - mx) * rse - (j == l ? 1.f : 0.f)) * inv : 0.f;
        if (valid && lane == 0) lsum += logf(se) - (h[l] - mx);
    }
    if (lane == 0) red[warp] = lsum;
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.f;
        for (int w = 0; w < nw; ++w) s += red[w];
        *loss += s * inv;
    }
}

// label = window cell (x fastest) holding the centroid of the host element,
// the cell coordinates clamped into the window around x_p's ASG cell (label
// may be host: each row is read before it is written)
template <int D>
__global__ void __launch_bounds__(kT) labels_kernel(const DevMesh m, int64_t n,
                                                    const double *__restrict__ xp,
                                                    const int32_t *host, int32_t *label) {
    using G = Win<D>;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += int64_t(gridDim.x) * blockDim.x) {
        const int32_t h = host[i];
        if (h < 0 || h >= m.n_e) {
            label[i] = -1;
            continue;
        }
        const int64_t li = m.iperm[h];
        int32_t cls = 0;
        #pragma unroll
        for (int k = D - 1; k >= 0; --k) {
            const int64_t c0 = cell_axis64(xp[i * D + k], m.lo[k], m.sa[k], m.ga[k]);
            const int64_t cc = cell_axis64(m.centroid[li * D + k], m.lo[k], m.sa[k], m.ga[k]);
            int64_t rel = cc - (c0 - G::W / 2);
            rel = rel < 0 ? 0 : (rel > G::W - 1 ? G::W - 1 : rel);
            cls = cls * G::W + int32_t(rel);
        }
        label[i] = cls;
    }
}

template <int D>
__device__ __forceinline__ int32_t rec_uid(const DevMesh &m, int32_t internal) {
    if (D == 2) return static_cast<const WalkRec2 *>(m.recw)[internal].uid;
    return static_cast<const WalkRec3 *>(m.recw)[internal].uid;
}

// K_p (Eq. 8): one warp per particle takes the class of the largest logit
// (the lowest among equal ones; NaN never wins), then the ASG seed of that
// window cell (user id), else the fallback start (fallback[i], or the plain
// start of mesh node row0 + i)
template <int D>
__global__ void __launch_bounds__(kT) start_kernel(const DevMesh m, int64_t n,
                                                   const double *__restrict__ xp,
                                                   const float *__restrict__ logits,
                                                   const int32_t *__restrict__ fallback,
                                                   int64_t row0, int32_t *__restrict__ start,
                                                   int32_t *__restrict__ cls_out) {
    using G = Win<D>;
    const int lane = threadIdx.x & 31;
    const int64_t warps = int64_t(gridDim.x) * (blockDim.x >> 5);
    for (int64_t i = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; i < n; i += warps) {
        const float *h = logits + i * G::P;
        float best = -INFINITY;
        int bj = G::P;
        for (int j = lane; j < G::P; j += 32) {
            const float v = h[j];
            if (v > best) {   // lanes scan increasing j: the first of equal values stays
                best = v;
                bj = j;
            }
        }
        #pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float ov = __shfl_xor_sync(kFull, best, o);
            const int oj = __shfl_xor_sync(kFull, bj, o);
            if (ov > best || (ov == best && oj < bj)) {
                best = ov;
                bj = oj;
            }
        }
        if (lane != 0) continue;
        // no finite maximum: no class
        const bool has_cls = bj < G::P && best > -INFINITY && best < INFINITY;
        int32_t s = -1;
        if (has_cls) {
            int r = bj;
            bool inside = true;
            int64_t cc[D];
            #pragma unroll
            for (int k = 0; k < D; ++k) {
                const int64_t c0 = cell_axis64(xp[i * D + k], m.lo[k], m.sa[k], m.ga[k]);
                cc[k] = c0 - G::W / 2 + r % G::W;
                r /= G::W;
                inside &= cc[k] >= 0 && cc[k] < m.ga[k];
            }
            if (inside) {
                int64_t flat = 0;
                #pragma unroll
                for (int k = D - 1; k >= 0; --k) flat = flat * m.ga[k] + cc[k];
                const int32_t seed = m.seed[flat];
                if (seed >= 0) s = rec_uid<D>(m, seed);
            }
        }
        if (s < 0) {
            if (fallback) {
                s = fallback[i];
            } else {
                const int32_t e = m.node_elem[row0 + i];
                s = e < 0 ? -1 : rec_uid<D>(m, e);
            }
        }
        start[i] = s;
        if (cls_out) cls_out[i] = has_cls ? bj : -1;
    }
}

}  // namespace

void launch_departure(int64_t n, int dim, const double *x, const double *u, double dt,
                      double *xp, int sm_count, cudaStream_t st) {
    const int64_t total = n * dim;
    departure_kernel<<<blocks_for(total, sm_count), kT, 0, st>>>(total, x, u, dt, xp);
}

void launch_cls_features(const DevMesh &m, int64_t B, const double *xp, const int64_t *idx,
                         bool pad, float *win, float *offset, int sm_count, cudaStream_t st) {
    const int E = cls_window(m.dim) + (pad ? 2 : 0);
    const int64_t total = B * (m.dim == 2 ? E * E : E * E * E);
    const int g = blocks_for(total, sm_count);
    if (m.dim == 2)
        features_kernel<2><<<g, kT, 0, st>>>(m, B, xp, idx, pad ? 1 : 0, win, offset);
    else
        features_kernel<3><<<g, kT, 0, st>>>(m, B, xp, idx, pad ? 1 : 0, win, offset);
}

void launch_cls_pad(int dim, const float *y, int64_t B, int C, float *a, int sm_count,
                    cudaStream_t st) {
    const int Wq = cls_window(dim) + 2;
    const int64_t total = B * (dim == 2 ? Wq * Wq : Wq * Wq * Wq) * C;
    if (dim == 2)
        pad_kernel<2><<<blocks_for(total, sm_count), kT, 0, st>>>(y, B, C, a);
    else
        pad_kernel<3><<<blocks_for(total, sm_count), kT, 0, st>>>(y, B, C, a);
}

void launch_cls_crop_relu_back(int dim, const float *dpad, const float *z, int64_t B, int C,
                               float *dz, int sm_count, cudaStream_t st) {
    const int W = cls_window(dim);
    const int64_t total = B * (dim == 2 ? W * W : W * W * W) * C;
    if (dim == 2)
        crop_relu_back_kernel<2><<<blocks_for(total, sm_count), kT, 0, st>>>(dpad, z, B, C, dz);
    else
        crop_relu_back_kernel<3><<<blocks_for(total, sm_count), kT, 0, st>>>(dpad, z, B, C, dz);
}

void launch_cls_pool(int dim, const float *z, int64_t B, float *cat, int64_t ldc, int sm_count,
                     cudaStream_t st) {
    const int64_t total = B * cls_pooled(dim);
    if (dim == 2)
        pool_relu_kernel<2><<<blocks_for(total, sm_count), kT, 0, st>>>(z, B, cat, ldc);
    else
        pool_relu_kernel<3><<<blocks_for(total, sm_count), kT, 0, st>>>(z, B, cat, ldc);
}

void launch_cls_pool_back(int dim, const float *dcat, int64_t ldc, const float *z, int64_t B,
                          float *dz, int sm_count, cudaStream_t st) {
    const int W = cls_window(dim);
    const int64_t total = B * (dim == 2 ? W * W : W * W * W) * kClsCh;
    if (dim == 2)
        pool_back_kernel<2><<<blocks_for(total, sm_count), kT, 0, st>>>(dcat, ldc, z, B, dz);
    else
        pool_back_kernel<3><<<blocks_for(total, sm_count), kT, 0, st>>>(dcat, ldc, z, B, dz);
}

void launch_cls_cat_relu(const float *y, int64_t B, int n, float *cat, int64_t ldc, int64_t off,
                         int sm_count, cudaStream_t st) {
    cat_relu_kernel<<<blocks_for(B * n, sm_count), kT, 0, st>>>(y, B, n, cat, ldc, off);
}

void launch_cls_uncat_relu_back(const float *dcat, int64_t ldc, int64_t off, const float *y,
                                int64_t B, int n, float *dy, int sm_count, cudaStream_t st) {
    uncat_relu_back_kernel<<<blocks_for(B * n, sm_count), kT, 0, st>>>(dcat, ldc, off, y, B, n,
                                                                       dy);
}

void launch_softmax_ce(const float *H, const int32_t *labels, const int64_t *idx, int64_t B,
                       int n_cls, float *dH, float *loss, cudaStream_t st) {
    softmax_ce_kernel<<<1, 1024, 0, st>>>(H, labels, idx, B, n_cls, dH, loss);
}

void launch_cls_labels(const DevMesh &m, int64_t n, const double *xp, const int32_t *host,
                       int32_t *label, int sm_count, cudaStream_t st) {
    if (m.dim == 2)
        labels_kernel<2><<<blocks_for(n, sm_count), kT, 0, st>>>(m, n, xp, host, label);
    else
        labels_kernel<3><<<blocks_for(n, sm_count), kT, 0, st>>>(m, n, xp, host, label);
}

void launch_cls_start(const DevMesh &m, int64_t n, const double *xp, const float *logits,
                      const int32_t *fallback, int64_t row0, int32_t *start, int32_t *cls,
                      int sm_count, cudaStream_t st) {
    const int g = int(std::max<int64_t>(1, std::min<int64_t>((n + 7) / 8, int64_t(sm_count) * 16)));
    if (m.dim == 2)
        start_kernel<2><<<g, kT, 0, st>>>(m, n, xp, logits, fallback, row0, start, cls);
    else
        start_kernel<3><<<g, kT, 0, st>>>(m, n, xp, logits, fallback, row0, start, cls);
}

}  // namespace cs
