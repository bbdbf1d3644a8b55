// The classifier start predictor (Sec. 2.3, Eq. 7-8): shapes and the
// launchers of its non-GEMM kernels (internal).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "internal.h"

namespace cs {

constexpr int kClsCh = 32;     // channels of both convolutions
constexpr int kClsH1 = 256;    // width of the offset branch (h1, Sec. 3.1)
constexpr int kClsH2 = 512;    // width of the fused layer (h2, Sec. 3.1)

inline int cls_window(int dim) { return dim == 2 ? 9 : 7; }
inline int cls_cells(int dim) {           // W^dim: window cells = classes
    const int W = cls_window(dim);
    return dim == 2 ? W * W : W * W * W;
}
inline int cls_pooled(int dim) {          // 32 (W/2)^dim pooled features
    const int p = cls_window(dim) / 2;
    return kClsCh * (dim == 2 ? p * p : p * p * p);
}

void launch_departure(int64_t n, int dim, const double *x, const double *u, double dt,
                      double *xp, int sm_count, cudaStream_t st);
// window [B][dim][E^dim] (E = W, or W + 2 with a zero ring when pad) and
// offset [B][dim] of the particles xp[idx[b]] (idx may be null: b)
void launch_cls_features(const DevMesh &m, int64_t B, const double *xp, const int64_t *idx,
                         bool pad, float *win, float *offset, int sm_count, cudaStream_t st);
void launch_cls_pad(int dim, const float *y, int64_t B, int C, float *a, int sm_count,
                    cudaStream_t st);
void launch_cls_crop_relu_back(int dim, const float *dpad, const float *z, int64_t B, int C,
                               float *dz, int sm_count, cudaStream_t st);
void launch_cls_pool(int dim, const float *z, int64_t B, float *cat, int64_t ldc, int sm_count,
                     cudaStream_t st);
void launch_cls_pool_back(int dim, const float *dcat, int64_t ldc, const float *z, int64_t B,
                          float *dz, int sm_count, cudaStream_t st);
void launch_cls_cat_relu(const float *y, int64_t B, int n, float *cat, int64_t ldc, int64_t off,
                         int sm_count, cudaStream_t st);
void launch_cls_uncat_relu_back(const float *dcat, int64_t ldc, int64_t off, const float *y,
                                int64_t B, int n, float *dy, int sm_count, cudaStream_t st);
void launch_softmax_ce(const float *H, const int32_t *labels, const int64_t *idx, int64_t B,
                       int n_cls, float *dH, float *loss, cudaStream_t st);
void launch_cls_labels(const DevMesh &m, int64_t n, const double *xp, const int32_t *host,
                       int32_t *label, int sm_count, cudaStream_t st);
// start[i] (user ids) and class of rows i < n from their logits; fallback
// null means the plain start of mesh node row0 + i
void launch_cls_start(const DevMesh &m, int64_t n, const double *xp, const float *logits,
                      const int32_t *fallback, int64_t row0, int32_t *start, int32_t *cls,
                      int sm_count, cudaStream_t st);

// module 1 fused on the tensor cores (classifier_tc.cu): conv1 and conv2
// weights packed for the kernel (bytes, and the packing from the FP32
// parameters), then per particle the window inputs, both convolutions and the
// pooling into cat[b][0, 32 (W/2)^dim) (row stride ldc) and the offset into
// off[b][dim]. pool_f: the mesh's pooled centroids as float hi + lo.
int64_t cls_packed_bytes(int dim);
void launch_cls_pack(int dim, const float *w, int64_t off_w1, int64_t off_b1, int64_t off_w2,
                     int64_t off_b2, uint8_t *packed, cudaStream_t st);
void launch_cls_conv_tc(const DevMesh &m, const float *pool_f, int64_t B, const double *xp,
                        const uint8_t *packed, float *cat, int64_t ldc, float *off, int *err,
                        int sm_count, cudaStream_t st);

}  // namespace cs
