// General GEMM of the predictor's training on the tensor cores (tcgen05):
// C(i, j) (+)= sum_k A(i, k) B(j, k) (+ bias[j]), with FP32 operands in global
// memory at arbitrary element strides, rounded to BF16 as they are staged
// into shared memory, and FP32 accumulation in TMEM (Sec. 2.3: the network is
// trained on pairs the tracking generates; BF16 operands, FP32 master
// weights). The strides let one kernel serve every product of training: the
// forward convolutions and fully connected layers, the transposed operands
// of the weight gradients (as C^T = B A^T, with the long batch dimension as
// K, split over CTAs into partial products that reduce_splits_kernel sums in
// a fixed order, so every run gives the same bits), and the input gradients.
//
// A CTA computes a 128 x BN tile of C. K runs in chunks of 64: all 256
// threads load a chunk of A (128 x 64) and B (BN x 64), four elements at a
// time where the strides allow, convert to BF16 and store it in the
// canonical no-swizzle K-major layout ([8-element K chunk][rows][8]); one
// thread issues the chunk's K = 16 MMAs (M = 128, N = BN; a short last chunk
// issues only the steps it fills) and commits them to the stage's mbarrier.
// Two stages alternate, so the loads of chunk c + 1 overlap the MMAs of
// chunk c; a stage is refilled once its MMAs have completed. The epilogue
// reads TMEM in 16-column pieces (warp w: rows 32 (w % 4) .., every other
// piece). Waits are bounded: one that gives up sets the device
// error flag and the CTA skips the rest.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>

#include "cnn.h"
#include "tc_common.cuh"

namespace cs {
namespace {

constexpr int kBM = 128, kBK = 64, kThreadsG = 256;

struct TcGemm {
    const float *A;
    int64_t a_i, a_k;          // A(i, k) = A[i a_i + k a_k]
    const float *B;
    int64_t b_j, b_k;          // B(j, k) = B[j b_j + k b_k]
    float *C;
    int64_t c_i, c_j;          // C(i, j) at C[i c_i + j c_j]
    const float *bias;         // [N] or null, added by the first K split
    int64_t M, N, K;
    int64_t kc;                // K per split (gridDim.z), a multiple of kBK
    int split;                 // split z writes its partial tile to part[z][M][N]
    float *part;
    int vec_a, vec_b;          // operand loads in float4 along its contiguous axis
};

template <int BN>
struct GemmGeo {
    static_assert(BN % 16 == 0 && BN >= 16 && BN <= 256, "MMA N");
    static constexpr int kA = kBM * kBK * 2;                // bytes of an A stage
    static constexpr int kB = BN * kBK * 2;
    static constexpr int kStage = kA + kB;
    static constexpr int kSmBar = 2 * kStage;
    static constexpr int kSmSlot = kSmBar + 3 * 8;
    static constexpr int kSmTotal = kSmSlot + 16;
    static_assert(8 * 32 * 17 * 4 <= kSmBar, "the epilogue's per-warp tiles fit the operand stages");
    static constexpr uint32_t kCols = BN <= 32 ? 32 : BN <= 64 ? 64 : BN <= 128 ? 128 : 256;
};

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    #pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Stage rows x kn elements of an operand (element (r, k) at P[r s_r + k s_k],
// rows from r0, K from k0; zero outside [0, nr) x [k0, kend)) as BF16 into
// the K-major layout dst[k / 8][r][k % 8]; kn is the chunk's K span rounded
// up to 16. Consecutive threads take consecutive addresses along whichever
// axis is contiguous, four elements at a time (float4) when `vec` says the
// addresses allow it: s_k == 1 with s_r % 4 == 0, or s_r == 1 with
// s_k % 4 == 0, a 16-byte aligned base, and the contiguous extent a
// multiple of 4.
template <int ROWS>
__device__ __forceinline__ void stage_operand(uint8_t *dst, const float *__restrict__ P,
                                              int64_t s_r, int64_t s_k, int64_t r0, int64_t nr,
                                              int64_t k0, int64_t kend, int kn, bool vec, int tid) {
    // Every path loads a batch of elements per thread before it converts and
    // stores any of them, so a chunk costs a few load latencies instead of
    // one per element.
    constexpr int kB4 = 8, kB1 = 16;
    __nv_bfloat16 *d = reinterpret_cast<__nv_bfloat16 *>(dst);
    const int kv = int(min(kend - k0, int64_t(kn)));            // valid K of the chunk
    const int rv = int(max(min(nr - r0, int64_t(ROWS)), int64_t(0)));   // valid rows
    if (s_k == 1) {
        const float *base = P + r0 * s_r + k0;
        if (vec) {
            // groups of 4 consecutive k; kv is a multiple of 4 (K % 4 == 0)
            const int g4 = kn / 4, total = ROWS * g4;
            for (int e0 = tid; e0 < total; e0 += kThreadsG * kB4) {
                float4 v[kB4];
                #pragma unroll
                for (int u = 0; u < kB4; ++u) {
                    const int e = e0 + u * kThreadsG;
                    const int r = e / g4, k = 4 * (e % g4);
                    v[u] = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (e < total && r < rv && k < kv)
                        v[u] = __ldg(reinterpret_cast<const float4 *>(base + int64_t(r) * s_r + k));
                }
                #pragma unroll
                for (int u = 0; u < kB4; ++u) {
                    const int e = e0 + u * kThreadsG;
                    if (e >= total) break;
                    const int r = e / g4, k = 4 * (e % g4);
                    const __nv_bfloat162 lo = __floats2bfloat162_rn(v[u].x, v[u].y);
                    const __nv_bfloat162 hi = __floats2bfloat162_rn(v[u].z, v[u].w);
                    uint2 w;
                    w.x = *reinterpret_cast<const uint32_t *>(&lo);
                    w.y = *reinterpret_cast<const uint32_t *>(&hi);
                    *reinterpret_cast<uint2 *>(d + ((k >> 3) * ROWS + r) * 8 + (k & 7)) = w;
                }
            }
        } else {
            const int total = ROWS * kn;
            for (int e0 = tid; e0 < total; e0 += kThreadsG * kB1) {
                float v[kB1];
                #pragma unroll
                for (int u = 0; u < kB1; ++u) {
                    const int e = e0 + u * kThreadsG;
                    const int r = e / kn, k = e % kn;
                    v[u] = (e < total && r < rv && k < kv) ? __ldg(base + int64_t(r) * s_r + k) : 0.f;
                }
                #pragma unroll
                for (int u = 0; u < kB1; ++u) {
                    const int e = e0 + u * kThreadsG;
                    if (e >= total) break;
                    const int r = e / kn, k = e % kn;
                    d[((k >> 3) * ROWS + r) * 8 + (k & 7)] = __float2bfloat16_rn(v[u]);
                }
            }
        }
    } else {
        const float *base = P + r0 * s_r + k0 * s_k;
        if (vec && s_r == 1) {
            // groups of 4 consecutive rows; rv is a multiple of 4 or the tail
            constexpr int g4 = ROWS / 4;
            const int total = g4 * kn;
            for (int e0 = tid; e0 < total; e0 += kThreadsG * kB4) {
                float4 v[kB4];
                #pragma unroll
                for (int u = 0; u < kB4; ++u) {
                    const int e = e0 + u * kThreadsG;
                    const int r = 4 * (e % g4), k = e / g4;
                    v[u] = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (e < total && r < rv && k < kv)
                        v[u] = __ldg(reinterpret_cast<const float4 *>(base + int64_t(k) * s_k + r));
                }
                #pragma unroll
                for (int u = 0; u < kB4; ++u) {
                    const int e = e0 + u * kThreadsG;
                    if (e >= total) break;
                    const int r = 4 * (e % g4), k = e / g4;
                    const int o = ((k >> 3) * ROWS + r) * 8 + (k & 7);
                    d[o] = __float2bfloat16_rn(v[u].x);
                    d[o + 8] = __float2bfloat16_rn(v[u].y);
                    d[o + 16] = __float2bfloat16_rn(v[u].z);
                    d[o + 24] = __float2bfloat16_rn(v[u].w);
                }
            }
        } else {
            const int total = ROWS * kn;
            for (int e0 = tid; e0 < total; e0 += kThreadsG * kB1) {
                float v[kB1];
                #pragma unroll
                for (int u = 0; u < kB1; ++u) {
                    const int e = e0 + u * kThreadsG;
                    const int r = e % ROWS, k = e / ROWS;
                    v[u] = (e < total && r < rv && k < kv)
                               ? __ldg(base + int64_t(r) * s_r + int64_t(k) * s_k)
                               : 0.f;
                }
                #pragma unroll
                for (int u = 0; u < kB1; ++u) {
                    const int e = e0 + u * kThreadsG;
                    if (e >= total) break;
                    const int r = e % ROWS, k = e / ROWS;
                    d[((k >> 3) * ROWS + r) * 8 + (k & 7)] = __float2bfloat16_rn(v[u]);
                }
            }
        }
    }
}

template <int BN>
__global__ void __launch_bounds__(kThreadsG, 2) tc_gemm_kernel(const TcGemm g, int *err) {
    using G = GemmGeo<BN>;
    extern __shared__ __align__(1024) uint8_t smem[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + G::kSmBar);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + G::kSmSlot);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + G::kSmSlot + 4);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t i0 = int64_t(blockIdx.x) * kBM, j0 = int64_t(blockIdx.y) * BN;
    const int64_t kbeg = int64_t(blockIdx.z) * g.kc, kend = min(g.K, kbeg + g.kc);
    const int nch = int((kend - kbeg + kBK - 1) / kBK);

    if (tid == 0) {
        for (int i = 0; i < 3; ++i) mbar_init(bars + i, 1u);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_addr(tmem_slot)),
                     "r"(G::kCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_slot;
    constexpr uint32_t id = idesc_bf16(kBM, BN);
    bool ok = true;
    for (int c = 0; c < nch && ok; ++c) {
        const int s = c & 1;
        uint8_t *sa = smem + s * G::kStage, *sb = sa + G::kA;
        // the stage's previous MMAs (chunk c - 2) must be complete
        if (c >= 2) ok = __syncthreads_and(mbar_wait(bars + s, uint32_t((c - 2) >> 1) & 1u, abort_flag, err));
        if (!ok) break;
        const int64_t k0 = kbeg + int64_t(c) * kBK;
        // the chunk's K span, rounded up to the MMA's K = 16
        const int kn = int(min(int64_t(kBK), (kend - k0 + 15) / 16 * 16));
        stage_operand<kBM>(sa, g.A, g.a_i, g.a_k, i0, g.M, k0, kend, kn, g.vec_a != 0, tid);
        stage_operand<BN>(sb, g.B, g.b_j, g.b_k, j0, g.N, k0, kend, kn, g.vec_b != 0, tid);
        fence_async_smem();
        fence_before();
        __syncthreads();
        fence_after();
        if (tid == 0) {
            const uint64_t da = sdesc(smem_addr(sa), kBM * 16, 128);
            const uint64_t db = sdesc(smem_addr(sb), BN * 16, 128);
            for (int q = 0; q < kn / 16; ++q)
                mma_bf16(tmem, da + uint64_t(2 * q * kBM), db + uint64_t(2 * q * BN), id,
                         (c | q) != 0 ? 1u : 0u);
            mma_commit(bars + s);
        }
    }
    // every MMA of the CTA complete (they complete in issue order)
    if (ok && nch > 0) {
        if (tid == 0) mma_commit(bars + 2);
        ok = __syncthreads_and(mbar_wait(bars + 2, 0u, abort_flag, err));
    }
    if (ok && nch > 0) {
        fence_after();
        // warp w reads TMEM lanes 32 (w % 4) ..; warps w and w + 4 take
        // alternate 16-column pieces. A row-major output (a split's partial
        // tile, or C with c_j == 1) goes through a per-warp tile in the now
        // idle operand stages, so that a store instruction writes 16
        // consecutive floats of two rows instead of one float of 32 rows.
        const int64_t i = i0 + 32 * (warp & 3) + lane;
        const uint32_t tq = tmem + (uint32_t(32 * (warp & 3)) << 16);
        if (!(g.split || g.c_j == 1)) {
            // C with c_i == 1 (a swapped product): consecutive lanes write
            // consecutive addresses already
            #pragma unroll 1
            for (int jc = 16 * (warp >> 2); jc < BN; jc += 32) {
                float v[16];
                tmem_ld16(tq + uint32_t(jc), v);
                if (i < g.M) {
                    #pragma unroll
                    for (int e = 0; e < 16; ++e) {
                        const int64_t j = j0 + jc + e;
                        if (j >= g.N) break;
                        float x = v[e];
                        if (g.bias) x += __ldg(g.bias + j);
                        g.C[i * g.c_i + j * g.c_j] = x;
                    }
                }
            }
        } else {
            float *tile = reinterpret_cast<float *>(smem) + warp * (32 * 17);
            float *dst = g.split ? g.part + int64_t(blockIdx.z) * g.M * g.N : g.C;
            const int64_t ld = g.split ? g.N : g.c_i;
            const int e = lane & 15;
            #pragma unroll 1
            for (int jc = 16 * (warp >> 2); jc < BN; jc += 32) {
                float v[16];
                tmem_ld16(tq + uint32_t(jc), v);
                #pragma unroll
                for (int q = 0; q < 16; ++q) tile[lane * 17 + q] = v[q];
                __syncwarp();
                const int64_t j = j0 + jc + e;
                const float bj = (!g.split && g.bias && j < g.N) ? __ldg(g.bias + j) : 0.f;
                #pragma unroll 1
                for (int r = lane >> 4; r < 32; r += 2) {
                    const int64_t ii = i0 + 32 * (warp & 3) + r;
                    if (ii < g.M && j < g.N) dst[ii * ld + j] = tile[r * 17 + e] + bj;
                }
                __syncwarp();
            }
        }
    }
    // release TMEM once no MMA of this CTA can still write it (bounded)
    if (tid == 0 && nch > 0 && !ok) {
        mma_commit(bars + 2);
        for (uint32_t t = 0; t < (1u << 24) && !mbar_try_wait(bars + 2, 0); ++t)
            if (t > 64) __nanosleep(64);
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(G::kCols));
}

// C(i, j) = sum over the splits, in order, of part[z][i][j] (+ bias[j]): the
// split-K sum is the same bits on every run.
__global__ void __launch_bounds__(256) reduce_splits_kernel(const float *__restrict__ part,
                                                            int64_t splits, int64_t M, int64_t N,
                                                            const float *__restrict__ bias,
                                                            float *C, int64_t c_i, int64_t c_j) {
    const int64_t MN = M * N;
    for (int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; q < MN;
         q += int64_t(gridDim.x) * blockDim.x) {
        float x = 0.f;
        for (int64_t z = 0; z < splits; ++z) x += __ldg(part + z * MN + q);
        const int64_t i = q / N, j = q % N;
        if (bias) x += __ldg(bias + j);
        C[i * c_i + j * c_j] = x;
    }
}

template <int BN>
void launch_bn(const TcGemm &g, int64_t splits, int *err, cudaStream_t st) {
    using G = GemmGeo<BN>;
    // at most two CTAs per SM, so their TMEM columns always fit the SM's 512
    constexpr int kSmem = G::kSmTotal < 80 * 1024 && G::kCols > 128 ? 80 * 1024 : G::kSmTotal;
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(tc_gemm_kernel<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
        attr = true;
    }
    const dim3 grid(unsigned((g.M + kBM - 1) / kBM), unsigned((g.N + BN - 1) / BN), unsigned(splits));
    tc_gemm_kernel<BN><<<grid, kThreadsG, kSmem, st>>>(g, err);
}

}  // namespace

bool tc_gemm_fits(int64_t M, int64_t N, int64_t K) {
    return std::min(M, N) >= 16 && K >= 16;
}

int64_t tc_gemm_work_floats(int sm_count) { return int64_t(2) * sm_count * kBM * 256; }

void launch_reduce_splits(const float *part, int64_t splits, int64_t M, int64_t N,
                          const float *bias, float *C, int sm_count, cudaStream_t st) {
    const int grid = int(std::min<int64_t>(int64_t(sm_count) * 4, (M * N + 255) / 256));
    reduce_splits_kernel<<<grid, 256, 0, st>>>(part, splits, M, N, bias, C, N, 1);
}

int launch_tc_gemm(const float *A, const float *Bm, float *C, const float *bias, int64_t M,
                   int64_t N, int64_t K, bool transA, bool transB, int *err, int sm_count,
                   float *work, int64_t work_floats, cudaStream_t st) {
    TcGemm g{};
    // C[M][N] = op(A) op(B): A(i, k) and B(j, k) of C(i, j) = sum_k A(i, k) B(j, k)
    g.A = A;
    g.a_i = transA ? 1 : K;
    g.a_k = transA ? M : 1;
    g.B = Bm;
    g.b_j = transB ? K : 1;
    g.b_k = transB ? 1 : N;
    g.C = C;
    g.c_i = N;
    g.c_j = 1;
    g.bias = bias;
    g.M = M;
    g.N = N;
    g.K = K;
    auto vec_ok = [K](const float *p, int64_t s_r, int64_t s_k, int64_t nr) {
        const bool aligned = (reinterpret_cast<uintptr_t>(p) & 15u) == 0;
        if (s_k == 1) return aligned && s_r % 4 == 0 && K % 4 == 0;
        return aligned && s_r == 1 && s_k % 4 == 0 && nr % 4 == 0;
    };
    // the larger dimension runs along the MMA's 128 rows: C^T = B A^T
    if (M < N && !bias) {
        std::swap(g.A, g.B);
        std::swap(g.a_i, g.b_j);
        std::swap(g.a_k, g.b_k);
        std::swap(g.c_i, g.c_j);
        std::swap(g.M, g.N);
    }
    g.vec_a = vec_ok(g.A, g.a_i, g.a_k, g.M);
    g.vec_b = vec_ok(g.B, g.b_j, g.b_k, g.N);
    const int BN = g.N <= 32 ? 32 : g.N <= 128 ? 128 : g.N <= 144 ? 144 : g.N <= 256 ? 256 : 144;
    const int64_t tiles = ((g.M + kBM - 1) / kBM) * ((g.N + BN - 1) / BN);
    // split a long K when the output has fewer tiles than about two waves;
    // the partial tiles must fit the workspace
    int64_t splits = 1;
    const int64_t chunks = (K + kBK - 1) / kBK;
    if (tiles < 2 * sm_count && chunks > 8 && work)
        splits = std::min<int64_t>(chunks / 4, (2 * sm_count + tiles - 1) / tiles);
    splits = std::max<int64_t>(1, std::min<int64_t>(splits, work_floats / std::max<int64_t>(1, g.M * g.N)));
    g.kc = ((chunks + splits - 1) / splits) * kBK;
    splits = (K + g.kc - 1) / g.kc;
    g.split = splits > 1;
    g.part = work;
    if (BN == 32)
        launch_bn<32>(g, splits, err, st);
    else if (BN == 128)
        launch_bn<128>(g, splits, err, st);
    else if (BN == 144)
        launch_bn<144>(g, splits, err, st);
    else
        launch_bn<256>(g, splits, err, st);
    if (!g.split) return 1;
    const int64_t MN = g.M * g.N;
    const int grid = int(std::min<int64_t>(int64_t(sm_count) * 4, (MN + 255) / 256));
    reduce_splits_kernel<<<grid, 256, 0, st>>>(work, splits, g.M, g.N, g.bias, g.C, g.c_i, g.c_j);
    return 2;
}

}  // namespace cs
