// Start predictor: device state and kernel launchers (internal).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "internal.h"

namespace cs {

// Layer geometry of the regressor for dim 2 / 3.
struct NetShape {
    int dim;
    int cin;        // input channels (= dim)
    int S0;         // window edge (9 / 7)
    int n_conv;     // 4 / 3
    int ch;         // 32
    int hidden;     // 256
    int64_t n_params;
    // offsets of W and b of every layer in the flat vector
    std::vector<int64_t> w_off, b_off;
    explicit NetShape(int d);
    int taps() const { return dim == 2 ? 9 : 27; }
    int64_t positions(int S) const { return dim == 2 ? int64_t(S) * S : int64_t(S) * S * S; }
};

int launch_tile_input(const DevMesh &m, const float *U, int T, int R, int tx, int ty, int64_t t0,
                      int64_t B, const float scale[3], float *out, int sm_count, cudaStream_t st);
int launch_tile_scatter(const DevMesh &m, int T, int tx, int ty, int64_t t0, int64_t B,
                        const float *rows, float *dhat, int sm_count, cudaStream_t st);
int launch_pred_seed(const DevMesh &m, int32_t *pseed, int sm_count, cudaStream_t st);
int launch_interp_table(const DevMesh &m, int32_t *node, float *w, int sm_count,
                        cudaStream_t st);
int launch_resample(const DevMesh &m, const int32_t *node, const float *w, const double *u_nodal,
                    float *U, int sm_count, cudaStream_t st);
int launch_windows(const DevMesh &m, const float *U, const int64_t *cells, int64_t cell0,
                   int64_t B, const float scale[3], float *out, int sm_count, cudaStream_t st);
int launch_im2col(int dim, const float *x, int64_t B, int C, int Si, bool chfirst, float *col,
                  int sm_count, cudaStream_t st);
int launch_col2im(int dim, const float *dcol, int64_t B, int C, int Si, float *dx, int sm_count,
                  cudaStream_t st);
// C[M][N] = op(A) op(B) (+ bias[N]), A [M][K] (transA: [K][M]), B [K][N]
// (transB: [N][K]). With BF16 operands the tensor-core GEMM takes every shape
// it fits (tc_gemm_fits); the rest, and FP32 operands, run on CUDA cores.
// err: device flag a bounded wait of the tensor-core GEMM raises. A long K
// is split over CTAs only with a workspace (work, work_floats): the partial
// products are summed in a fixed order, so every run gives the same bits.
int launch_gemm(const float *A, const float *Bm, float *C, const float *bias, int64_t M,
                int64_t N, int64_t K, bool transA, bool transB, bool accumulate,
                cudaStream_t st, int *err, int sm_count, float *work, int64_t work_floats);
// the tensor-core GEMM (tc_gemm.cu)
bool tc_gemm_fits(int64_t M, int64_t N, int64_t K);
int64_t tc_gemm_work_floats(int sm_count);   // workspace that allows every split
// C[M][N] = sum over z, in order, of part[z][M][N] (+ bias[N])
void launch_reduce_splits(const float *part, int64_t splits, int64_t M, int64_t N,
                          const float *bias, float *C, int sm_count, cudaStream_t st);
int launch_tc_gemm(const float *A, const float *Bm, float *C, const float *bias, int64_t M,
                   int64_t N, int64_t K, bool transA, bool transB, int *err, int sm_count,
                   float *work, int64_t work_floats, cudaStream_t st);
void set_gemm_bf16(bool on);
bool gemm_bf16();   // the current operand precision (true: BF16)
int launch_relu(const float *z, float *y, int64_t n, int sm_count, cudaStream_t st);
// ReLU(conv(x) + bias) of one valid 3^D convolution of 32 output channels,
// without an im2col copy (inference). x: [B][C][Si^D] (chfirst) or
// [B][Si^D][C]; y: [B * So^D][32].
// W2 ReLU(W1 y + b1) + b2 per row of y [M][32] (the predictor head, inference)
int launch_head(int dim, const float *y, const float *W1, const float *b1, const float *W2,
                const float *b2, int64_t M, float *out, int sm_count, cudaStream_t st);
int launch_conv_relu(int dim, const float *x, bool chfirst, int64_t B, int C, int Si,
                     const float *W, const float *bias, float *y, cudaStream_t st);
int launch_relu_back(const float *z, float *dy, int64_t n, int sm_count, cudaStream_t st);
// out[n] = sum_m x[m][n] in a fixed order; with a workspace (work,
// work_floats) in two coalesced passes, else one block per column
int launch_colsum(const float *x, int64_t M, int64_t N, float *out, cudaStream_t st,
                  float *work = nullptr, int64_t work_floats = 0, int sm_count = 0);
int launch_mse_grad(const float *out, const float *tgt, int64_t n, float *g, float *loss,
                    int sm_count, cudaStream_t st);
int launch_adam(float *w, const float *g, float *m, float *v, int64_t n, float lr, int64_t t,
                int sm_count, cudaStream_t st);
// Test hook of the tensor-core predictor kernels: when flag is not null, the
// kernel first waits (bounded, `polls` polls) for *flag != 0 before any MMA;
// nothing sets the flag, so the wait runs out and the kernel ends through its
// abort path with the device error flag raised.
struct TcHold {
    const int *flag = nullptr;
    uint32_t polls = 0;
};
// Where a tensor-core grid predictor kernel takes its input velocities: the
// grid velocity U (node null), or the P1 interpolation of the nodal velocity
// un at each predictor cell centre through the mesh's static table (node, w),
// computed as the tile's input is loaded (the resample kernel's arithmetic,
// in its order, so the same bits) and written to U_out for the tile's own
// cells. The 2-D kernel takes either; the 3-D kernel takes the grid
// velocity only (a tile's (T + 6)^3 input cells are many times its T^3 own
// cells, so interpolating them costs more than the separate resample).
struct TcSource {
    const float *U = nullptr;
    const int32_t *node = nullptr;
    const float *w = nullptr;
    const double *un = nullptr;
    float *U_out = nullptr;
};
// tensor-core grid inference of the 2-D predictor (cnn_tc.cu)
int64_t tc_packed_bytes();
int launch_pack_tc(const float *w, const NetShape &S, uint8_t *packed, cudaStream_t st);
// tile_rows: output rows per tile (24, 13 or 8), 0 = tc_pick_tile_rows
int launch_cnn2d_tc(const DevMesh &m, const TcSource &src, double dt, const uint8_t *packed,
                    float *dhat, int *err, int sm_count, int tile_rows, cudaStream_t st,
                    TcHold hold = TcHold());
// the tile height with the least estimated cost on a grid (24, 13 or 8)
int tc_pick_tile_rows(const DevMesh &m, int sm_count);
// tensor-core grid inference of the 3-D predictor (cnn3d_tc.cu); tile: side of
// the cubic output tiles (4, 3 or 2), 0 = tc3_pick_tile
int64_t tc3_packed_bytes();
int launch_pack_tc3(const float *w, const NetShape &S, uint8_t *packed, cudaStream_t st);
int launch_cnn3d_tc(const DevMesh &m, const TcSource &src, double dt, const uint8_t *packed,
                    float *dhat, int *err, int sm_count, int tile, cudaStream_t st,
                    TcHold hold = TcHold());
int tc3_pick_tile(const DevMesh &m, int sm_count);
int launch_pairs(const DevMesh &m, int64_t n, const double *x, const double *u, double dt,
                 int64_t *cells, float *target, int sm_count, cudaStream_t st);
int launch_gather_rows(const float *src, int64_t row, const int64_t *idx, int64_t B, float *dst,
                       int sm_count, cudaStream_t st);

}  // namespace cs
