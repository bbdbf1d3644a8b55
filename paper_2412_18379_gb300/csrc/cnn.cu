// Learned start predictor (Sec. 2.3, Algorithm 2): the velocity field on the
// ASG grid, input windows, and the kernels of training around its GEMMs
// (im2col / col2im, ReLU and its gradient, bias gradients, the loss, Adam on
// the FP32 master weights). The GEMMs run on the tensor cores with BF16
// operands and FP32 accumulation (tc_gemm.cu); the CUDA-core GEMMs here take
// the shapes too small for them and the FP32-operand accuracy mode.
//
// Network (regressor form): a window of the grid velocity around the cell of
// the particle, channels u_k * dt / s_k, zero outside the grid, goes through
// valid 3x3 (3x3x3) convolutions of 32 channels with ReLU, then 32 -> 256
// (ReLU) -> dim; the output is the particle's displacement in cell units.
// 2-D: window 9x9, 4 convolutions; 3-D: window 7^3, 3 convolutions.
#include <cuda_bf16.h>

#include <cmath>
#include <cstdint>

#include "cnn.h"
#include "walk_common.cuh"

namespace cs {
namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ float bf16_round(float x) {
    return __bfloat162float(__float2bfloat16_rn(x));
}

int grid_for(int64_t n, int sm_count, int per_sm = 8) {
    const int64_t need = (n + kThreads - 1) / kThreads;
    return int(std::max<int64_t>(1, std::min<int64_t>(need, int64_t(sm_count) * per_sm)));
}

// The P1 interpolation at the ASG cell centres as a static table, built once
// per mesh: node[c][i] = vertex i of the host element seed[c] of the centre of
// cell c, w[c][i] = its barycentric coordinate (FP64 from the exact record,
// rounded to float); node[c][0] = -1 where the centre has no host.
template <int D>
__global__ void __launch_bounds__(kThreads) interp_table_kernel(const DevMesh m,
                                                                int32_t *__restrict__ node,
                                                                float *__restrict__ w) {
    using XR = typename Recs<D>::X;
    const XR *__restrict__ rx = static_cast<const XR *>(m.recx);
    for (int64_t c = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; c < m.n_asg;
         c += int64_t(gridDim.x) * blockDim.x) {
        const int32_t s = m.seed[c];
        if (s < 0) {
            #pragma unroll
            for (int i = 0; i <= D; ++i) {
                node[c * (D + 1) + i] = -1;
                w[c * (D + 1) + i] = 0.f;
            }
            continue;
        }
        double x[D];
        int64_t r = c;
        #pragma unroll
        for (int k = 0; k < D; ++k) {
            const int64_t i = r % m.ga[k];
            r /= m.ga[k];
            x[k] = __dadd_rn(m.lo[k], __dmul_rn(double(i) + 0.5, m.sa[k]));
        }
        double lam[D + 1];
        bary64(rx, s, x, lam);
        #pragma unroll
        for (int i = 0; i <= D; ++i) {
            node[c * (D + 1) + i] = m.conn[int64_t(s) * (D + 1) + i];
            w[c * (D + 1) + i] = float(lam[i]);
        }
    }
}

// pseed[c] = seed of the middle ASG cell of predictor cell c: with an odd
// stride p, predictor cell I spans ASG cells p I .. p I + p - 1 per axis and
// shares its centre with ASG cell p I + (p - 1) / 2.
__global__ void __launch_bounds__(kThreads) pred_seed_kernel(const DevMesh m,
                                                             int32_t *__restrict__ pseed) {
    for (int64_t c = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; c < m.n_pasg;
         c += int64_t(gridDim.x) * blockDim.x) {
        int64_t r = c, fine = 0, mul = 1;
        for (int k = 0; k < m.dim; ++k) {
            const int64_t i = r % m.pga[k];
            r /= m.pga[k];
            fine += (i * m.pstride + (m.pstride - 1) / 2) * mul;
            mul *= m.ga[k];
        }
        pseed[c] = __ldg(m.seed + fine);
    }
}

// U[c] = P1 interpolation of the nodal velocity at the centre of ASG cell c
// through the static table (FP32); 0 where the centre has no host.
template <int D>
__global__ void __launch_bounds__(kThreads) resample_kernel(int64_t n_asg,
                                                            const int32_t *__restrict__ node,
                                                            const float *__restrict__ w,
                                                            const double *__restrict__ un,
                                                            float *__restrict__ U) {
    for (int64_t c = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; c < n_asg;
         c += int64_t(gridDim.x) * blockDim.x) {
        float out[D];
        #pragma unroll
        for (int k = 0; k < D; ++k) out[k] = 0.f;
        if (__ldg(node + c * (D + 1)) >= 0) {
            #pragma unroll
            for (int i = 0; i <= D; ++i) {
                const int32_t v = __ldg(node + c * (D + 1) + i);
                const float wi = __ldg(w + c * (D + 1) + i);
                #pragma unroll
                for (int k = 0; k < D; ++k)
                    out[k] = fmaf(wi, trunc_to_float(__ldg(un + int64_t(v) * D + k)), out[k]);
            }
        }
        #pragma unroll
        for (int k = 0; k < D; ++k) U[c * D + k] = out[k];
    }
}

// windows[b][k][w] = U[cell_b + offset(w)][k] * scale_k, 0 outside the grid;
// w runs over the S^D window positions, x fastest; offsets -S/2..S/2.
template <int D>
__global__ void __launch_bounds__(kThreads) window_kernel(const DevMesh m, const float *__restrict__ U,
                                                          const int64_t *__restrict__ cells,
                                                          int64_t cell0, int64_t B, float s0,
                                                          float s1, float s2,
                                                          float *__restrict__ out) {
    constexpr int S = D == 2 ? 9 : 7;
    constexpr int W = D == 2 ? 81 : 343;
    const float scale[3] = {s0, s1, s2};
    const int64_t total = B * W;
    for (int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; q < total;
         q += int64_t(gridDim.x) * blockDim.x) {
        const int64_t b = q / W;
        int w = int(q % W);
        const int64_t cell = cells ? __ldg(cells + b) : cell0 + b;
        int64_t r = cell;
        int64_t src = 0, mul = 1;
        bool inside = true;
        #pragma unroll
        for (int k = 0; k < D; ++k) {
            const int64_t ic = r % m.ga[k];
            r /= m.ga[k];
            const int64_t j = ic + (w % S) - S / 2;
            w /= S;
            inside = inside && j >= 0 && j < m.ga[k];
            src += j * mul;
            mul *= m.ga[k];
        }
        #pragma unroll
        for (int k = 0; k < D; ++k)
            out[(b * D + k) * W + (q % W)] = inside ? __ldg(U + src * D + k) * scale[k] : 0.f;
    }
}

// Fully convolutional evaluation over the grid (the "tile engine"): the grid
// is cut into cubic tiles of T^D cells; tile b's input is the block of side
// T + 2 R (R = number of 3^D convolutions) around it, channels u_k * scale_k,
// zero outside the grid, in the channel-first window layout [b][k][S^D]. The
// valid convolutions then leave exactly the tile's T^D cells, and cell c's
// value equals that of the window of side 2 R + 1 centred at c.
template <int D>
__global__ void __launch_bounds__(kThreads) tile_input_kernel(const DevMesh m,
                                                              const float *__restrict__ U, int T,
                                                              int R, int tx, int ty, int64_t t0,
                                                              int64_t B, float s0, float s1,
                                                              float s2, float *__restrict__ out) {
    const int S = T + 2 * R;
    const int64_t P = D == 2 ? int64_t(S) * S : int64_t(S) * S * S;
    const float scale[3] = {s0, s1, s2};
    const int64_t total = B * P;
    for (int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; q < total;
         q += int64_t(gridDim.x) * blockDim.x) {
        const int64_t b = q / P;
        const int64_t p = q % P;
        const int64_t tile = t0 + b;
        const int tc[3] = {int(tile % tx), int((tile / tx) % ty), int(tile / (int64_t(tx) * ty))};
        const int pc[3] = {int(p % S), int((p / S) % S), D == 3 ? int(p / (int64_t(S) * S)) : 0};
        bool inside = true;
        int64_t cell = 0, mul = 1;
        #pragma unroll
        for (int k = 0; k < D; ++k) {
            const int j = tc[k] * T + pc[k] - R;
            inside = inside && j >= 0 && j < m.ga[k];
            cell += int64_t(j) * mul;
            mul *= m.ga[k];
        }
        #pragma unroll
        for (int k = 0; k < D; ++k)
            out[(b * D + k) * P + p] = inside ? __ldg(U + cell * D + k) * scale[k] : 0.f;
    }
}

// dhat[cell] = row (b, position) of the tile engine's output, for the cells
// of tile t0 + b that lie inside the grid.
template <int D>
__global__ void __launch_bounds__(kThreads) tile_scatter_kernel(const DevMesh m, int T, int tx,
                                                                int ty, int64_t t0, int64_t B,
                                                                const float *__restrict__ rows,
                                                                float *__restrict__ dhat) {
    const int64_t P = D == 2 ? int64_t(T) * T : int64_t(T) * T * T;
    const int64_t total = B * P;
    for (int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; q < total;
         q += int64_t(gridDim.x) * blockDim.x) {
        const int64_t b = q / P;
        const int64_t p = q % P;
        const int64_t tile = t0 + b;
        const int tc[3] = {int(tile % tx), int((tile / tx) % ty), int(tile / (int64_t(tx) * ty))};
        const int pc[3] = {int(p % T), int((p / T) % T), D == 3 ? int(p / (int64_t(T) * T)) : 0};
        bool inside = true;
        int64_t cell = 0, mul = 1;
        #pragma unroll
        for (int k = 0; k < D; ++k) {
            const int j = tc[k] * T + pc[k];
            inside = inside && j < m.ga[k];
            cell += int64_t(j) * mul;
            mul *= m.ga[k];
        }
        if (inside) {
            #pragma unroll
            for (int k = 0; k < D; ++k) dhat[cell * D + k] = rows[q * D + k];
        }
    }
}

// im2col of one valid 3^D convolution: col[(b*Po + p)][i*taps + t] =
// x(b, i, p + offset(t)); x is channels-first [B][C][Si^D] (first layer) or
// channels-last [B][Si^D][C]. I: the index type (32-bit when the sizes allow:
// its divisions are far cheaper than 64-bit ones).
template <int D, class I>
__global__ void __launch_bounds__(kThreads) im2col_kernel(const float *__restrict__ x, I B,
                                                          int C, int Si, bool chfirst,
                                                          float *__restrict__ col) {
    const int So = Si - 2;
    const int taps = D == 2 ? 9 : 27;
    int Po = So * So, Pi = Si * Si;
    if (D == 3) {
        Po *= So;
        Pi *= Si;
    }
    const I K = I(C) * taps;
    const I total = B * Po * K;
    for (I q = I(blockIdx.x) * blockDim.x + threadIdx.x; q < total; q += I(gridDim.x) * blockDim.x) {
        const I row = q / K;
        const int kk = int(q % K);
        const I b = row / Po;
        const int p = int(row % Po);
        const int i = kk / taps, t = kk % taps;
        int px = p % So, py = (p / So) % So, pz = D == 3 ? p / (So * So) : 0;
        px += t % 3;
        py += (t / 3) % 3;
        pz += D == 3 ? t / 9 : 0;
        const int pin = D == 2 ? py * Si + px : (pz * Si + py) * Si + px;
        col[q] = chfirst ? x[(int64_t(b) * C + i) * Pi + pin] : x[(int64_t(b) * Pi + pin) * C + i];
    }
}

// col2im (gather form): dx[b][pin][i] = sum over taps t with a valid output
// position p = pin - offset(t) of dcol[(b*Po + p)][i*taps + t]. Channels-last.
template <int D, class I>
__global__ void __launch_bounds__(kThreads) col2im_kernel(const float *__restrict__ dcol, I B,
                                                          int C, int Si, float *__restrict__ dx) {
    const int So = Si - 2;
    const int taps = D == 2 ? 9 : 27;
    int Po = So * So, Pi = Si * Si;
    if (D == 3) {
        Po *= So;
        Pi *= Si;
    }
    const I total = B * Pi * C;
    for (I q = I(blockIdx.x) * blockDim.x + threadIdx.x; q < total; q += I(gridDim.x) * blockDim.x) {
        const int i = int(q % C);
        const I bp = q / C;
        const int pin = int(bp % Pi);
        const I b = bp / Pi;
        const int ix = pin % Si, iy = (pin / Si) % Si, iz = D == 3 ? pin / (Si * Si) : 0;
        float s = 0.f;
        for (int t = 0; t < taps; ++t) {
            const int ox = ix - t % 3, oy = iy - (t / 3) % 3, oz = D == 3 ? iz - t / 9 : 0;
            if (ox < 0 || oy < 0 || oz < 0 || ox >= So || oy >= So || (D == 3 && oz >= So))
                continue;
            const int p = D == 2 ? oy * So + ox : (oz * So + oy) * So + ox;
            s += dcol[(int64_t(b) * Po + p) * (int64_t(C) * taps) + int64_t(i) * taps + t];
        }
        dx[q] = s;
    }
}

// C[M][N] = op(A) op(B) (+ bias[N]) with operands rounded to BF16 and FP32
// accumulation. A is [M][K] (transA: [K][M]); B is [K][N] (transB: [N][K]).
// 64x64 output tile, 16-deep K slabs in shared memory, 4x4 per thread.
// Split-K: block z sums K-range [z*kc, (z+1)*kc) into partial product z
// (C + z M N, no bias); launch_reduce_splits sums them in order.
__global__ void __launch_bounds__(kThreads) gemm_kernel(const float *__restrict__ A,
                                                        const float *__restrict__ Bm, float *C,
                                                        const float *__restrict__ bias, int64_t M,
                                                        int64_t N, int64_t K, bool transA,
                                                        bool transB, bool accumulate,
                                                        bool round_bf16, int64_t kc) {
    __shared__ float As[16][64 + 4];
    __shared__ float Bs[16][64 + 4];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int64_t m0 = int64_t(blockIdx.y) * 64, n0 = int64_t(blockIdx.x) * 64;
    const int64_t kbeg = int64_t(blockIdx.z) * kc, kend = min(K, kbeg + kc);
    const bool split = gridDim.z > 1;
    float acc[4][4] = {};
    for (int64_t k0 = kbeg; k0 < kend; k0 += 16) {
        for (int q = threadIdx.x; q < 16 * 64; q += kThreads) {
            // consecutive threads read consecutive addresses of each operand
            const int ka = transA ? q / 64 : q % 16, ma = transA ? q % 64 : q / 16;
            const int64_t gm = m0 + ma, gka = k0 + ka;
            float a = 0.f;
            if (gm < M && gka < kend) a = transA ? A[gka * M + gm] : A[gm * K + gka];
            As[ka][ma] = round_bf16 ? bf16_round(a) : a;
            const int kb = transB ? q % 16 : q / 64, nb = transB ? q / 16 : q % 64;
            const int64_t gn = n0 + nb, gkb = k0 + kb;
            float bv = 0.f;
            if (gn < N && gkb < kend) bv = transB ? Bm[gn * K + gkb] : Bm[gkb * N + gn];
            Bs[kb][nb] = round_bf16 ? bf16_round(bv) : bv;
        }
        __syncthreads();
        #pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            float a[4], b[4];
            #pragma unroll
            for (int r = 0; r < 4; ++r) {
                a[r] = As[kk][ty * 4 + r];
                b[r] = Bs[kk][tx * 4 + r];
            }
            #pragma unroll
            for (int r = 0; r < 4; ++r)
                #pragma unroll
                for (int s = 0; s < 4; ++s) acc[r][s] = fmaf(a[r], b[s], acc[r][s]);
        }
        __syncthreads();
    }
    #pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int64_t gm = m0 + ty * 4 + r;
        if (gm >= M) continue;
        #pragma unroll
        for (int s = 0; s < 4; ++s) {
            const int64_t gn = n0 + tx * 4 + s;
            if (gn >= N) continue;
            float v = acc[r][s] + (bias ? bias[gn] : 0.f);
            if (split) {
                C[(int64_t(blockIdx.z) * M + gm) * N + gn] = v;   // partial product z
            } else {
                if (accumulate) v += C[gm * N + gn];
                C[gm * N + gn] = v;
            }
        }
    }
}

// y = relu(z) (elementwise), and dz = dy * (z > 0)
__global__ void relu_kernel(const float *__restrict__ z, float *__restrict__ y, int64_t n) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += int64_t(gridDim.x) * blockDim.x)
        y[i] = fmaxf(z[i], 0.f);
}
__global__ void relu_back_kernel(const float *__restrict__ z, float *__restrict__ dy, int64_t n) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += int64_t(gridDim.x) * blockDim.x)
        dy[i] = z[i] > 0.f ? dy[i] : 0.f;
}

// Column sums in two passes (bias gradients): block b sums its range of rows
// for every column (consecutive threads on consecutive columns: coalesced)
// into part[b][n]; then out[n] = sum over b, in order, of part[b][n]. The
// order of every sum is fixed, so the result has the same bits on every run.
__global__ void __launch_bounds__(kThreads) colsum_part_kernel(const float *__restrict__ x,
                                                               int64_t M, int64_t N, int64_t rows,
                                                               float *__restrict__ part) {
    const int64_t m0 = int64_t(blockIdx.x) * rows, m1 = min(M, m0 + rows);
    for (int64_t n = threadIdx.x; n < N; n += blockDim.x) {
        float s = 0.f;
        for (int64_t m = m0; m < m1; ++m) s += x[m * N + n];
        part[int64_t(blockIdx.x) * N + n] = s;
    }
}
// Thin products with a long K (weight gradients of narrow layers):
// part[b][i N + j] = sum over k of block b's range of op(A)(i, k) B(k, j),
// A stored [K][M] (op(A) = A^T), B [K][N], operands rounded to BF16 as in the
// other training GEMMs; colsum_final_kernel then sums the blocks in order.
__global__ void __launch_bounds__(kThreads) thin_part_kernel(const float *__restrict__ A,
                                                             const float *__restrict__ B,
                                                             int64_t M, int64_t N, int64_t K,
                                                             int64_t rows, bool round_bf16,
                                                             float *__restrict__ part) {
    const int64_t k0 = int64_t(blockIdx.x) * rows, k1 = min(K, k0 + rows);
    for (int64_t q = threadIdx.x; q < M * N; q += blockDim.x) {
        const int64_t i = q / N, j = q % N;
        float s = 0.f;
        for (int64_t k = k0; k < k1; ++k) {
            float a = A[k * M + i], b = B[k * N + j];
            if (round_bf16) {
                a = __bfloat162float(__float2bfloat16_rn(a));
                b = __bfloat162float(__float2bfloat16_rn(b));
            }
            s = fmaf(a, b, s);
        }
        part[int64_t(blockIdx.x) * M * N + q] = s;
    }
}

// one warp per column: lane l sums partials l, l + 32, ... in order, then a
// butterfly over the lanes (a fixed order as well)
__global__ void __launch_bounds__(kThreads) colsum_final_kernel(const float *__restrict__ part,
                                                                int64_t G, int64_t N,
                                                                float *__restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = int64_t(gridDim.x) * (blockDim.x >> 5);
    for (int64_t n = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; n < N; n += warps) {
        float s = 0.f;
        for (int64_t b = lane; b < G; b += 32) s += part[b * N + n];
        #pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) out[n] = s;
    }
}

// column sums: out[n] = sum_m x[m][n]  (bias gradients); one block per column
__global__ void colsum_kernel(const float *__restrict__ x, int64_t M, int64_t N,
                              float *__restrict__ out) {
    __shared__ float red[kThreads];
    for (int64_t n = blockIdx.x; n < N; n += gridDim.x) {
        float s = 0.f;
        for (int64_t m = threadIdx.x; m < M; m += blockDim.x) s += x[m * N + n];
        red[threadIdx.x] = s;
        __syncthreads();
        for (int o = kThreads / 2; o > 0; o >>= 1) {
            if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) out[n] = red[0];
        __syncthreads();
    }
}

// dL/dout of L = mean over batch and components of (out - target)^2, and L
// added to *loss. One block: its fixed-order reduction gives the same loss
// bits on every run (the outputs are a batch of a few thousand values).
__global__ void mse_grad_kernel(const float *__restrict__ out, const float *__restrict__ tgt,
                                int64_t n, float *__restrict__ g, float *__restrict__ loss) {
    __shared__ float red[kThreads];
    float s = 0.f;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += int64_t(gridDim.x) * blockDim.x) {
        const float d = out[i] - tgt[i];
        g[i] = 2.f * d / float(n);
        s += d * d;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = kThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *loss += red[0] / float(n);
}

// Adam on the FP32 master weights (Sec. 2.3 names Adam; constants are the
// customary ones): m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
// w -= lr * m/(1-b1^t) / (sqrt(v/(1-b2^t)) + eps).
__global__ void adam_kernel(float *__restrict__ w, const float *__restrict__ g,
                            float *__restrict__ mo, float *__restrict__ ve, int64_t n, float lr,
                            float b1, float b2, float eps, float c1, float c2) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += int64_t(gridDim.x) * blockDim.x) {
        const float gi = g[i];
        const float m = b1 * mo[i] + (1.f - b1) * gi;
        const float v = b2 * ve[i] + (1.f - b2) * gi * gi;
        mo[i] = m;
        ve[i] = v;
        w[i] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
    }
}

// Training pairs: the ASG cell of every particle's position x and its true
// displacement in cell units, target_k = (x_p,k - x_k) / s_k with
// x_p = x - (u * dt) (Eq. 3, first order).
template <int D>
__global__ void pairs_kernel(const DevMesh m, int64_t n, const double *__restrict__ x,
                             const double *__restrict__ u, double dt, int64_t *__restrict__ cells,
                             float *__restrict__ target) {
    for (int64_t p = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; p < n;
         p += int64_t(gridDim.x) * blockDim.x) {
        double xv[D];
        #pragma unroll
        for (int k = 0; k < D; ++k) {
            xv[k] = x[p * D + k];
            const double xp = __dsub_rn(xv[k], __dmul_rn(u[p * D + k], dt));
            target[p * D + k] = float(__ddiv_rn(__dsub_rn(xp, xv[k]), m.sa[k]));
        }
        cells[p] = grid_cell<D>(xv, m.lo, m.sa, m.ga);
    }
}

// dst[b][:] = src[idx[b]][:] for rows of `row` floats (batch gather)
__global__ void gather_rows_kernel(const float *__restrict__ src, int64_t row,
                                   const int64_t *__restrict__ idx, int64_t B,
                                   float *__restrict__ dst) {
    const int64_t total = B * row;
    for (int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; q < total;
         q += int64_t(gridDim.x) * blockDim.x)
        dst[q] = src[__ldg(idx + q / row) * row + q % row];
}

}  // namespace

int launch_pairs(const DevMesh &m, int64_t n, const double *x, const double *u, double dt,
                 int64_t *cells, float *target, int sm_count, cudaStream_t st) {
    const int g = grid_for(n, sm_count);
    if (m.dim == 2)
        pairs_kernel<2><<<g, kThreads, 0, st>>>(m, n, x, u, dt, cells, target);
    else
        pairs_kernel<3><<<g, kThreads, 0, st>>>(m, n, x, u, dt, cells, target);
    return 1;
}

int launch_gather_rows(const float *src, int64_t row, const int64_t *idx, int64_t B, float *dst,
                       int sm_count, cudaStream_t st) {
    gather_rows_kernel<<<grid_for(B * row, sm_count, 16), kThreads, 0, st>>>(src, row, idx, B, dst);
    return 1;
}

int launch_tile_input(const DevMesh &m, const float *U, int T, int R, int tx, int ty, int64_t t0,
                      int64_t B, const float scale[3], float *out, int sm_count,
                      cudaStream_t st) {
    const int64_t S = T + 2 * R;
    const int64_t P = m.dim == 2 ? S * S : S * S * S;
    const int g = grid_for(B * P, sm_count, 32);
    if (m.dim == 2)
        tile_input_kernel<2><<<g, kThreads, 0, st>>>(m, U, T, R, tx, ty, t0, B, scale[0],
                                                     scale[1], scale[2], out);
    else
        tile_input_kernel<3><<<g, kThreads, 0, st>>>(m, U, T, R, tx, ty, t0, B, scale[0],
                                                     scale[1], scale[2], out);
    return 1;
}

int launch_tile_scatter(const DevMesh &m, int T, int tx, int ty, int64_t t0, int64_t B,
                        const float *rows, float *dhat, int sm_count, cudaStream_t st) {
    const int64_t P = m.dim == 2 ? int64_t(T) * T : int64_t(T) * T * T;
    const int g = grid_for(B * P, sm_count, 32);
    if (m.dim == 2)
        tile_scatter_kernel<2><<<g, kThreads, 0, st>>>(m, T, tx, ty, t0, B, rows, dhat);
    else
        tile_scatter_kernel<3><<<g, kThreads, 0, st>>>(m, T, tx, ty, t0, B, rows, dhat);
    return 1;
}

int launch_pred_seed(const DevMesh &m, int32_t *pseed, int sm_count, cudaStream_t st) {
    pred_seed_kernel<<<grid_for(m.n_pasg, sm_count), kThreads, 0, st>>>(m, pseed);
    return 1;
}

int launch_interp_table(const DevMesh &m, int32_t *node, float *w, int sm_count,
                        cudaStream_t st) {
    const int g = grid_for(m.n_asg, sm_count);
    if (m.dim == 2)
        interp_table_kernel<2><<<g, kThreads, 0, st>>>(m, node, w);
    else
        interp_table_kernel<3><<<g, kThreads, 0, st>>>(m, node, w);
    return 1;
}

int launch_resample(const DevMesh &m, const int32_t *node, const float *w, const double *u_nodal,
                    float *U, int sm_count, cudaStream_t st) {
    const int g = grid_for(m.n_asg, sm_count);
    if (m.dim == 2)
        resample_kernel<2><<<g, kThreads, 0, st>>>(m.n_asg, node, w, u_nodal, U);
    else
        resample_kernel<3><<<g, kThreads, 0, st>>>(m.n_asg, node, w, u_nodal, U);
    return 1;
}

int launch_windows(const DevMesh &m, const float *U, const int64_t *cells, int64_t cell0,
                   int64_t B, const float scale[3], float *out, int sm_count, cudaStream_t st) {
    const int W = m.dim == 2 ? 81 : 343;
    const int g = grid_for(B * W, sm_count);
    if (m.dim == 2)
        window_kernel<2><<<g, kThreads, 0, st>>>(m, U, cells, cell0, B, scale[0], scale[1], scale[2],
                                                  out);
    else
        window_kernel<3><<<g, kThreads, 0, st>>>(m, U, cells, cell0, B, scale[0], scale[1], scale[2],
                                                  out);
    return 1;
}

int launch_im2col(int dim, const float *x, int64_t B, int C, int Si, bool chfirst, float *col,
                  int sm_count, cudaStream_t st) {
    const int So = Si - 2, taps = dim == 2 ? 9 : 27;
    const int64_t Po = dim == 2 ? So * So : int64_t(So) * So * So;
    const int64_t total = B * Po * C * taps;
    const int g = grid_for(total, sm_count, 32);
    // unsigned 32-bit indices while q + the grid's stride cannot wrap
    if (total < (int64_t(1) << 31)) {
        if (dim == 2)
            im2col_kernel<2, uint32_t><<<g, kThreads, 0, st>>>(x, uint32_t(B), C, Si, chfirst, col);
        else
            im2col_kernel<3, uint32_t><<<g, kThreads, 0, st>>>(x, uint32_t(B), C, Si, chfirst, col);
    } else if (dim == 2) {
        im2col_kernel<2, int64_t><<<g, kThreads, 0, st>>>(x, B, C, Si, chfirst, col);
    } else {
        im2col_kernel<3, int64_t><<<g, kThreads, 0, st>>>(x, B, C, Si, chfirst, col);
    }
    return 1;
}

int launch_col2im(int dim, const float *dcol, int64_t B, int C, int Si, float *dx, int sm_count,
                  cudaStream_t st) {
    const int64_t Pi = dim == 2 ? Si * Si : int64_t(Si) * Si * Si;
    const int64_t total = B * Pi * C;
    const int g = grid_for(total, sm_count, 32);
    if (total < (int64_t(1) << 31)) {
        if (dim == 2)
            col2im_kernel<2, uint32_t><<<g, kThreads, 0, st>>>(dcol, uint32_t(B), C, Si, dx);
        else
            col2im_kernel<3, uint32_t><<<g, kThreads, 0, st>>>(dcol, uint32_t(B), C, Si, dx);
    } else if (dim == 2) {
        col2im_kernel<2, int64_t><<<g, kThreads, 0, st>>>(dcol, B, C, Si, dx);
    } else {
        col2im_kernel<3, int64_t><<<g, kThreads, 0, st>>>(dcol, B, C, Si, dx);
    }
    return 1;
}

// C[M][N] = A B^T (+ bias) for N <= 32 (the convolution layers: A [M][K] the
// im2col rows, B [N][K] the weights): 32 x 32 output tiles of 64 threads, each
// 4 x 4, 32-deep K slabs prefetched into registers while the previous slab is
// multiplied. The same BF16 operand rounding and the same FMA chain over k in
// increasing order as gemm_kernel, so the results are the same bits.
__global__ void __launch_bounds__(64) gemm_nt32_kernel(const float *__restrict__ A,
                                                       const float *__restrict__ Bm,
                                                       float *__restrict__ C,
                                                       const float *__restrict__ bias, int64_t M,
                                                       int N, int64_t K, bool round_bf16) {
    __shared__ float As[32][33];   // [k][m]
    __shared__ float Bs[32][33];   // [k][n]
    const int tid = threadIdx.x, tx = tid & 7, ty = tid >> 3;
    const int64_t m0 = int64_t(blockIdx.x) * 32;
    // element e = tid + 64 i of a slab: row e / 32 (m or n), column e % 32 (k)
    float ra[16], rb[16];
    auto fetch = [&](int64_t k0) {
        #pragma unroll
        for (int i = 0; i < 16; ++i) {
            const int e = tid + 64 * i, r = e >> 5, kk = e & 31;
            const int64_t gk = k0 + kk, gm = m0 + r;
            const float av = (gm < M && gk < K) ? __ldg(A + gm * K + gk) : 0.f;
            const float bv = (r < N && gk < K) ? __ldg(Bm + int64_t(r) * K + gk) : 0.f;
            ra[i] = round_bf16 ? bf16_round(av) : av;
            rb[i] = round_bf16 ? bf16_round(bv) : bv;
        }
    };
    float acc[4][4] = {};
    fetch(0);
    for (int64_t k0 = 0; k0 < K; k0 += 32) {
        #pragma unroll
        for (int i = 0; i < 16; ++i) {
            const int e = tid + 64 * i;
            As[e & 31][e >> 5] = ra[i];
            Bs[e & 31][e >> 5] = rb[i];
        }
        __syncthreads();
        if (k0 + 32 < K) fetch(k0 + 32);
        const int kn = int(min(int64_t(32), K - k0));
        #pragma unroll 8
        for (int kk = 0; kk < kn; ++kk) {
            float a[4], bq[4];
            #pragma unroll
            for (int r = 0; r < 4; ++r) {
                a[r] = As[kk][ty * 4 + r];
                bq[r] = Bs[kk][tx * 4 + r];
            }
            #pragma unroll
            for (int r = 0; r < 4; ++r)
                #pragma unroll
                for (int c = 0; c < 4; ++c) acc[r][c] = fmaf(a[r], bq[c], acc[r][c]);
        }
        __syncthreads();
    }
    #pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int64_t gm = m0 + ty * 4 + r;
        if (gm >= M) continue;
        #pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int gn = tx * 4 + c;
            if (gn < N) C[gm * N + gn] = acc[r][c] + (bias ? bias[gn] : 0.f);
        }
    }
}

// One valid 3^D convolution of 32 output channels as an implicit GEMM, fused
// with its bias and ReLU (inference only): y[b*Po + p][o] = ReLU(bias[o] +
// sum_{i,t} W[o][i*taps + t] x[b][i][p + offset(t)]). The A operand is read
// straight from the input instead of an im2col copy: for row (b, p) and
// column k = (i, t) the input address splits into a row part and a column
// part, so each thread precomputes the row parts of its 16 rows once and adds
// one column part per K slab. A block computes a 32 x 32 output tile with 4
// groups of 64 threads, group g summing the 32-deep K slabs g, g + 4, ...;
// the four partial tiles are added in group order at the end (the grids here
// are small, so the K split is what keeps enough warps in flight).
template <int D>
__global__ void __launch_bounds__(256) conv_nt32_kernel(const float *__restrict__ x, bool chfirst,
                                                        int64_t Bn, int C, int Si,
                                                        const float *__restrict__ Wt,
                                                        const float *__restrict__ bias,
                                                        float *__restrict__ y, bool round_bf16) {
    constexpr int taps = D == 2 ? 9 : 27;
    constexpr int N = 32;
    __shared__ float As[4][32][33];
    __shared__ float Bs[4][32][33];
    const int g = threadIdx.x >> 6, tid = threadIdx.x & 63, tx = tid & 7, ty = tid >> 3;
    const int So = Si - 2;
    const int64_t Po = D == 2 ? int64_t(So) * So : int64_t(So) * So * So;
    const int64_t Pi = D == 2 ? int64_t(Si) * Si : int64_t(Si) * Si * Si;
    const int64_t M = Bn * Po, K = int64_t(C) * taps;
    const int64_t m0 = int64_t(blockIdx.x) * 32;
    // this thread loads column kk = tid & 31 of rows (tid >> 5) + 2 i, i < 16
    const int kk = tid & 31;
    int64_t rowbase[16];
    bool rowok[16];
    // rows and positions fit in 32 bits (a tile-engine batch holds at most
    // 2^23 rows), so the divisions here are 32-bit ones
    #pragma unroll
    for (int i = 0; i < 16; ++i) {
        const uint32_t gm = uint32_t(m0) + uint32_t((tid >> 5) + 2 * i);
        rowok[i] = gm < uint32_t(M);
        const uint32_t b = rowok[i] ? gm / uint32_t(Po) : 0u;
        const uint32_t p = rowok[i] ? gm - b * uint32_t(Po) : 0u;
        const uint32_t q = p / uint32_t(So), px = p - q * uint32_t(So);
        const uint32_t pz = D == 3 ? q / uint32_t(So) : 0u, py = q - pz * uint32_t(So);
        const int64_t pb = D == 2 ? int64_t(py) * Si + px : (int64_t(pz) * Si + py) * Si + px;
        rowbase[i] = chfirst ? int64_t(b) * C * Pi + pb : (int64_t(b) * Pi + pb) * C;
    }
    float ra[16], rb[16];
    // K order: (channel, tap) for a channels-first input, as W is stored;
    // (tap, channel) for a channels-last one, so that the 32 lanes of a warp,
    // which take 32 consecutive k, read 32 consecutive channels of one input
    // position (one 128-byte line) instead of 32 scattered taps
    auto fetch = [&](int64_t k0) {
        const int64_t gk = k0 + kk;
        int64_t koff = 0, wk = 0;
        const bool kok = gk < K;
        if (kok) {
            const int ch = chfirst ? int(gk / taps) : int(gk % C);
            const int t = chfirst ? int(gk % taps) : int(gk / C);
            const int dx = t % 3, dy = (t / 3) % 3, dz = D == 3 ? t / 9 : 0;
            const int64_t toff = D == 2 ? int64_t(dy) * Si + dx : (int64_t(dz) * Si + dy) * Si + dx;
            koff = chfirst ? int64_t(ch) * Pi + toff : toff * C + ch;
            wk = int64_t(ch) * taps + t;
        }
        #pragma unroll
        for (int i = 0; i < 16; ++i) {
            const float av = (rowok[i] && kok) ? __ldg(x + rowbase[i] + koff) : 0.f;
            const int r = (tid >> 5) + 2 * i;   // weight row (output channel)
            const float bv = kok ? __ldg(Wt + int64_t(r) * K + wk) : 0.f;
            ra[i] = round_bf16 ? bf16_round(av) : av;
            rb[i] = round_bf16 ? bf16_round(bv) : bv;
        }
    };
    float acc[4][4] = {};
    const int64_t n_slabs = (K + 31) / 32, rounds = (n_slabs + 3) / 4;
    fetch(32 * int64_t(g));
    for (int64_t j = 0; j < rounds; ++j) {
        const int64_t k0 = 32 * (g + 4 * j);
        #pragma unroll
        for (int i = 0; i < 16; ++i) {
            const int e = tid + 64 * i;
            As[g][e & 31][e >> 5] = ra[i];
            Bs[g][e & 31][e >> 5] = rb[i];
        }
        __syncthreads();
        if (k0 + 128 < K) fetch(k0 + 128);
        const int kn = k0 < K ? int(min(int64_t(32), K - k0)) : 0;
        #pragma unroll 8
        for (int q = 0; q < kn; ++q) {
            float a[4], bq[4];
            #pragma unroll
            for (int r = 0; r < 4; ++r) {
                a[r] = As[g][q][ty * 4 + r];
                bq[r] = Bs[g][q][tx * 4 + r];
            }
            #pragma unroll
            for (int r = 0; r < 4; ++r)
                #pragma unroll
                for (int c = 0; c < 4; ++c) acc[r][c] = fmaf(a[r], bq[c], acc[r][c]);
        }
        __syncthreads();
    }
    // partial tiles of groups 1..3 into shared memory, group 0 adds them in order
    float *red = &As[0][0][0];   // [3][64 threads][16]
    if (g > 0) {
        #pragma unroll
        for (int r = 0; r < 4; ++r)
            #pragma unroll
            for (int c = 0; c < 4; ++c) red[((g - 1) * 64 + tid) * 16 + r * 4 + c] = acc[r][c];
    }
    __syncthreads();
    if (g == 0) {
        #pragma unroll
        for (int h = 0; h < 3; ++h)
            #pragma unroll
            for (int r = 0; r < 4; ++r)
                #pragma unroll
                for (int c = 0; c < 4; ++c) acc[r][c] += red[(h * 64 + tid) * 16 + r * 4 + c];
        #pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int64_t gm = m0 + ty * 4 + r;
            if (gm >= M) continue;
            float4 v;
            v.x = fmaxf(acc[r][0] + bias[tx * 4 + 0], 0.f);
            v.y = fmaxf(acc[r][1] + bias[tx * 4 + 1], 0.f);
            v.z = fmaxf(acc[r][2] + bias[tx * 4 + 2], 0.f);
            v.w = fmaxf(acc[r][3] + bias[tx * 4 + 3], 0.f);
            *reinterpret_cast<float4 *>(y + gm * N + tx * 4) = v;
        }
    }
}

// The predictor's head on rows of conv features (inference): out[r] =
// W2 ReLU(W1 y[r] + b1) + b2 for y [M][32], W1 [256][32], W2 [dim][256]. One
// warp per row: lane l computes features n = l, l + 32, ..., l + 224 (each a
// sum over k in order), the row's 256 features meet in shared memory, and
// lanes d < dim sum W2 over n in order. Same BF16 operand rounding and the
// same summation orders as the two GEMMs plus ReLU it replaces, so the same
// bits. W1 is stored transposed in shared memory ([k][n]) so that the lanes
// read consecutive words.
template <int DIM>
__global__ void __launch_bounds__(256) head_kernel(const float *__restrict__ y,
                                                   const float *__restrict__ W1,
                                                   const float *__restrict__ b1,
                                                   const float *__restrict__ W2,
                                                   const float *__restrict__ b2, int64_t M,
                                                   float *__restrict__ out, bool round_bf16) {
    __shared__ float w1t[32 * 256];
    __shared__ float w2[DIM * 256];
    __shared__ float bb1[256];
    __shared__ float hs[8][256];
    for (int i = threadIdx.x; i < 256 * 32; i += blockDim.x) {
        const float v = W1[i];                        // W1[n][k], i = 32 n + k
        w1t[(i & 31) * 256 + (i >> 5)] = round_bf16 ? bf16_round(v) : v;
    }
    for (int i = threadIdx.x; i < DIM * 256; i += blockDim.x)
        w2[i] = round_bf16 ? bf16_round(W2[i]) : W2[i];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) bb1[i] = b1[i];
    __syncthreads();
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    float *h = hs[wib];
    for (int64_t r = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; r < M;
         r += (int64_t(gridDim.x) * blockDim.x) >> 5) {
        // the row's 32 inputs, in every lane (one broadcast load each)
        float f[32];
        #pragma unroll
        for (int k = 0; k < 32; ++k) {
            const float v = __ldg(y + r * 32 + k);
            f[k] = round_bf16 ? bf16_round(v) : v;
        }
        float hv[8];
        #pragma unroll
        for (int j = 0; j < 8; ++j) hv[j] = 0.f;
        #pragma unroll
        for (int k = 0; k < 32; ++k)
            #pragma unroll
            for (int j = 0; j < 8; ++j) hv[j] = fmaf(f[k], w1t[k * 256 + lane + 32 * j], hv[j]);
        #pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int n = lane + 32 * j;
            float v = fmaxf(hv[j] + bb1[n], 0.f);
            h[n] = round_bf16 ? bf16_round(v) : v;
        }
        __syncwarp();
        if (lane < DIM) {
            float o = 0.f;
            #pragma unroll 8
            for (int n = 0; n < 256; ++n) o = fmaf(h[n], w2[lane * 256 + n], o);
            out[r * DIM + lane] = o + b2[lane];
        }
        __syncwarp();
    }
}

// BF16 operands (the training arithmetic) unless switched off for an
// accuracy check; process-wide.
static bool g_gemm_bf16 = true;
void set_gemm_bf16(bool on) { g_gemm_bf16 = on; }
bool gemm_bf16() { return g_gemm_bf16; }

int launch_gemm(const float *A, const float *Bm, float *C, const float *bias, int64_t M,
                int64_t N, int64_t K, bool transA, bool transB, bool accumulate,
                cudaStream_t st, int *err, int sm_count, float *work, int64_t work_floats) {
    if (g_gemm_bf16 && err && !accumulate && tc_gemm_fits(M, N, K))
        return launch_tc_gemm(A, Bm, C, bias, M, N, K, transA, transB, err, sm_count, work,
                               work_floats, st);
    if (transA && !transB && !accumulate && !bias && work && M * N <= 4096 && K >= 2048) {
        // thin product with a long K: blocks of K rows, then a fixed-order sum
        int64_t G = std::min<int64_t>((K + 63) / 64, int64_t(sm_count) * 4);
        G = std::min<int64_t>(G, work_floats / (M * N));
        if (G >= 2) {
            const int64_t rows = (K + G - 1) / G;
            G = (K + rows - 1) / rows;
            thin_part_kernel<<<unsigned(G), kThreads, 0, st>>>(A, Bm, M, N, K, rows, g_gemm_bf16,
                                                              work);
            const int64_t per_block = kThreads / 32;
            colsum_final_kernel<<<unsigned(std::min<int64_t>((M * N + per_block - 1) / per_block,
                                                             4096)),
                                  kThreads, 0, st>>>(work, G, M * N, C);
            return 2;
        }
    }
    if (!transA && transB && !accumulate && N <= 32) {
        gemm_nt32_kernel<<<unsigned((M + 31) / 32), 64, 0, st>>>(A, Bm, C, bias, M, int(N), K,
                                                                 g_gemm_bf16);
        return 1;
    }
    // split K when the output has few tiles and K is long (weight gradients):
    // the splits write partial products to the workspace, summed in order
    const int64_t tiles = ((N + 63) / 64) * ((M + 63) / 64);
    int64_t splits = 1;
    if (tiles < 512 && K > 2048 && work && !accumulate)
        splits = std::min<int64_t>((K + 1023) / 1024, (1024 + tiles - 1) / tiles);
    splits = std::max<int64_t>(1, std::min<int64_t>(splits, work_floats / std::max<int64_t>(1, M * N)));
    const int64_t kc = ((K + splits - 1) / splits + 15) / 16 * 16;
    splits = (K + kc - 1) / kc;
    const dim3 grid(unsigned((N + 63) / 64), unsigned((M + 63) / 64), unsigned(splits));
    if (splits == 1) {
        gemm_kernel<<<grid, kThreads, 0, st>>>(A, Bm, C, bias, M, N, K, transA, transB, accumulate,
                                               g_gemm_bf16, kc);
        return 1;
    }
    gemm_kernel<<<grid, kThreads, 0, st>>>(A, Bm, work, nullptr, M, N, K, transA, transB, false,
                                           g_gemm_bf16, kc);
    launch_reduce_splits(work, splits, M, N, bias, C, sm_count, st);
    return 2;
}

int launch_conv_relu(int dim, const float *x, bool chfirst, int64_t B, int C, int Si,
                     const float *W, const float *bias, float *y, cudaStream_t st) {
    const int64_t So = Si - 2;
    const int64_t M = B * (dim == 2 ? So * So : So * So * So);
    if (dim == 2)
        conv_nt32_kernel<2><<<unsigned((M + 31) / 32), 256, 0, st>>>(x, chfirst, B, C, Si, W, bias,
                                                                     y, g_gemm_bf16);
    else
        conv_nt32_kernel<3><<<unsigned((M + 31) / 32), 256, 0, st>>>(x, chfirst, B, C, Si, W, bias,
                                                                     y, g_gemm_bf16);
    return 1;
}

int launch_head(int dim, const float *y, const float *W1, const float *b1, const float *W2,
                const float *b2, int64_t M, float *out, int sm_count, cudaStream_t st) {
    // 8 rows in flight per block (one per warp); at most two blocks per SM,
    // since each block first stages the 35 KB of head weights
    const int g = int(std::max<int64_t>(1, std::min<int64_t>((M + 7) / 8, int64_t(sm_count) * 2)));
    if (dim == 2)
        head_kernel<2><<<g, 256, 0, st>>>(y, W1, b1, W2, b2, M, out, g_gemm_bf16);
    else
        head_kernel<3><<<g, 256, 0, st>>>(y, W1, b1, W2, b2, M, out, g_gemm_bf16);
    return 1;
}

int launch_relu(const float *z, float *y, int64_t n, int sm_count, cudaStream_t st) {
    relu_kernel<<<grid_for(n, sm_count, 16), kThreads, 0, st>>>(z, y, n);
    return 1;
}

int launch_relu_back(const float *z, float *dy, int64_t n, int sm_count, cudaStream_t st) {
    relu_back_kernel<<<grid_for(n, sm_count, 16), kThreads, 0, st>>>(z, dy, n);
    return 1;
}

int launch_colsum(const float *x, int64_t M, int64_t N, float *out, cudaStream_t st,
                  float *work, int64_t work_floats, int sm_count) {
    // blocks of at least 64 rows, about 4 per SM, as the workspace allows
    int64_t G = std::min<int64_t>((M + 63) / 64, int64_t(sm_count) * 4);
    if (work && N > 0) G = std::min<int64_t>(G, work_floats / N);
    if (!work || G < 2) {
        colsum_kernel<<<unsigned(std::min<int64_t>(N, 1024)), kThreads, 0, st>>>(x, M, N, out);
        return 1;
    }
    const int64_t rows = (M + G - 1) / G;
    G = (M + rows - 1) / rows;
    colsum_part_kernel<<<unsigned(G), kThreads, 0, st>>>(x, M, N, rows, work);
    const int64_t per_block = kThreads / 32;
    colsum_final_kernel<<<unsigned(std::max<int64_t>(1, std::min<int64_t>((N + per_block - 1) / per_block,
                                                                            4096))),
                          kThreads, 0, st>>>(work, G, N, out);
    return 2;
}

int launch_mse_grad(const float *out, const float *tgt, int64_t n, float *g, float *loss,
                    int sm_count, cudaStream_t st) {
    (void)sm_count;
    mse_grad_kernel<<<1, kThreads, 0, st>>>(out, tgt, n, g, loss);
    return 1;
}

int launch_adam(float *w, const float *g, float *m, float *v, int64_t n, float lr, int64_t t,
                int sm_count, cudaStream_t st) {
    const double b1 = 0.9, b2 = 0.999;
    const float c1 = float(1.0 - std::pow(b1, double(t)));
    const float c2 = float(1.0 - std::pow(b2, double(t)));
    adam_kernel<<<grid_for(n, sm_count, 4), kThreads, 0, st>>>(w, g, m, v, n, lr, float(b1),
                                                                float(b2), 1e-8f, c1, c2);
    return 1;
}

}  // namespace cs
