// Grid inference of the 3-D start predictor on the tensor cores (tcgen05).
//
// The 3-D predictor maps the 7x7x7 window of the predictor-grid velocity
// around a cell (channels u_k dt / s_k) through three valid 3x3x3
// convolutions of 32 channels with ReLU, then 32 -> 256 (ReLU) -> 3, to the
// cell's displacement (Sec. 2.3, Algorithm 2). As in 2-D, the windows of
// neighbouring cells overlap and the valid convolutions make the window
// result at cell c equal to a fully convolutional pass over the zero-padded
// grid, read at c: each CTA takes cubic tiles of T^3 output cells and their
// (T + 6)^3 input cells.
//
// Layout. A tile's cells sit on a flat index r = (z D + y) D + x, D = T + 6,
// for the input and for every layer (a layer's output at r reads its input at
// r + shift(tap), shift = (dz D + dy) D + dx): a tap is a row offset of the
// shared-memory operand, so every convolution is an implicit GEMM with no
// im2col copy. Rows past a layer's valid volume hold garbage that only ever
// feeds garbage rows (a valid output at (x, y, z) < T reads positions < D on
// every axis, so nothing wraps into it).
//
//   input  [rows][8] BF16: u_0..u_2 dt / s_k and 5 zero channels
//   conv1  tcgen05.mma kind::f16, M = 128 rows, N = 32, K = 16 = two taps of
//          8 channels each: the A descriptor's leading byte offset is the row
//          distance between the two taps, so one MMA reads both (14 MMAs per
//          M-tile for 27 taps; the 28th tap has zero weights)
//   conv2  implicit GEMM, K = 32 channels of one tap in two K = 16 steps;
//   conv3  27 taps x 2 MMAs per M-tile; conv2 writes its output over conv1's
//          in one activation buffer [4 chunks][rows][8] BF16 (M-tile m's rows
//          are read only by the MMAs of M-tiles m - 2 .. m of the next layer,
//          complete before its epilogue); conv3 writes the T^3 valid rows,
//          compacted, to the fc1 input
//   fc1    one MMA pair, M = 128 (the T^3 <= 64 cells), N = 256, K = 32
//   fc2    CUDA cores in the fc1 epilogue (256 -> 3, FP32 weights)
//   FP32 accumulation in TMEM; bias + ReLU + BF16 in the epilogues.
//
// Warps. Warps 0-3 are the epilogue warps (warp w reads TMEM lanes
// 32 w .. 32 w + 31) and warp 4 issues the MMAs. The items of a tile (conv1,
// conv2 and conv3 M-tiles, then fc1) run in order; the issuing warp runs ahead
// of the epilogues as far as the items' inputs and TMEM columns allow (four
// rotating 32-column accumulators for the convolutions, columns [256, 512)
// for fc1), each item committing to its own mbarrier and each epilogue
// counting itself in a shared-memory counter. Every wait is bounded; a wait
// that gives up raises the CTA's abort flag and the device error flag.
#include <cuda_bf16.h>

#include <cstdint>

#include "cnn.h"
#include "tc_common.cuh"

namespace cs {
namespace {

constexpr int kEpi3 = 4;                 // epilogue warps 0..3
constexpr int kMma3 = 4;                 // the MMA-issuing warp
constexpr int kThreads3 = (kEpi3 + 1) * 32;

// packed weights of the 3-D predictor (bytes); produced by pack3_kernel
struct Tc3Layout {
    static constexpr int w1 = 0;                          // bf16 [14 pairs][2 halves][32][8]
    static constexpr int w1_bytes = 14 * 2 * 32 * 8 * 2;
    static constexpr int b1 = w1 + w1_bytes;              // fp32 [32]
    static constexpr int wc = b1 + 32 * 4;                // 2 x bf16 [27 taps][4][32][8]
    static constexpr int wc_bytes = 27 * 4 * 32 * 8 * 2;
    static constexpr int cb = wc + 2 * wc_bytes;          // fp32 [2][32]
    static constexpr int f1 = cb + 2 * 32 * 4;            // bf16 [4][256][8]
    static constexpr int f1_bytes = 4 * 256 * 8 * 2;
    static constexpr int f1b = f1 + f1_bytes;             // fp32 [256]
    static constexpr int f2w = f1b + 256 * 4;             // fp32 [3][256]
    static constexpr int f2b = f2w + 3 * 256 * 4;         // fp32 [4] (3 used)
    static constexpr int total = (f2b + 16 + 127) / 128 * 128;
};

// Geometry of a tile of T^3 output cells (see the file comment).
template <int T>
struct Geo3 {
    static_assert(T >= 2 && T <= 4, "tile side");
    static constexpr int D = T + 6;                          // input side, flat pitch
    static constexpr int S = (2 * D + 2) * D + 2;            // largest tap shift (rows)
    static constexpr int R3 = (((T - 1) * D + (T - 1)) * D) + T;   // rows up to the last output
    static constexpr int m3 = (R3 + 127) / 128;              // M-tiles per layer
    static constexpr int m2 = (128 * m3 + S + 127) / 128;
    static constexpr int m1 = (128 * m2 + S + 127) / 128;
    static constexpr int kDep = (127 + S) / 128;             // M-tiles read past m
    static constexpr int kItems = m1 + m2 + m3 + 1;
    static constexpr int kCells = T * T * T;
    static constexpr int kInRows = (128 * m1 + S + 8 + 7) / 8 * 8;   // + the zero tap's shift
    static constexpr int kActRows = 128 * m1;

    static constexpr int kSmIn = 0;                          // bf16 [kInRows][8]
    static constexpr int kSmAct = kSmIn + kInRows * 16;      // bf16 [4][kActRows][8]
    static constexpr int kSmFc = kSmAct + 4 * kActRows * 16; // bf16 [4][128][8]
    static constexpr int kSmW = kSmFc + 4 * 128 * 16;        // packed weights
    static constexpr int kSmBar = kSmW + Tc3Layout::total;   // mbarriers [5] (4 conv + fc1) + final
    static constexpr int kSmCnt = kSmBar + 6 * 8;            // u32 epilogue counter
    static constexpr int kSmSlot = kSmCnt + 16;              // TMEM address, abort flag
    static constexpr int kSmTotal = kSmSlot + 16;

    static_assert(kCells <= 128, "fc1 takes the cells of a tile in one M-tile");
    static_assert(kSmTotal <= 232448, "shared memory of one CTA");
    static_assert(kDep == 2, "an M-tile reads the rows of M-tiles m .. m + 2");
    // reads: conv1 up to row 128 m1 - 1 + S; conv2 up to 128 m2 - 1 + S < kActRows;
    // conv3 up to 128 m3 - 1 + S < 128 m2 (conv2's rows, written in place)
    static_assert(128 * m1 - 1 + S < kInRows, "conv1 reads in bounds");
    static_assert(128 * m2 - 1 + S < kActRows, "conv2 reads in bounds");
    static_assert(128 * m3 - 1 + S < 128 * m2, "conv3 reads conv2 rows");
    static_assert(kSmBar % 8 == 0, "mbarrier alignment");

    // layer (0..3, 3 = fc1) and M-tile of item j
    static __device__ __forceinline__ void item(int j, int &l, int &m) {
        l = j < m1 ? 0 : j < m1 + m2 ? 1 : j < m1 + m2 + m3 ? 2 : 3;
        m = j - (l == 0 ? 0 : l == 1 ? m1 : l == 2 ? m1 + m2 : m1 + m2 + m3);
    }
    // items of this tile that must be complete before item j's MMAs: the
    // M-tiles of the previous layer it reads, and the item that last used its
    // TMEM columns (j - 4)
    static __device__ __forceinline__ int need(int j) {
        int l, m;
        item(j, l, m);
        int r = j - 3;
        if (l == 1) r = max(r, min(m + kDep, m1 - 1) + 1);
        if (l == 2) r = max(r, m1 + min(m + kDep, m2 - 1) + 1);
        if (l == 3) r = j;
        return max(r, 0);
    }
};

__device__ __forceinline__ constexpr int tap_shift(int t, int D) {
    return ((t / 9) * D + (t / 3) % 3) * D + t % 3;
}

// Named barrier 1 over the epilogue warps, with an OR over their flags.
__device__ __forceinline__ bool epi3_or(bool flag) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 q, %1, 0;\n\t"
        "bar.red.or.pred p, 1, %2, q;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(r)
        : "r"(uint32_t(flag)), "n"(kEpi3 * 32)
        : "memory");
    return r != 0;
}

template <int T>
__global__ void __launch_bounds__(kThreads3, 1) cnn3d_tc_kernel(
    const DevMesh m, const TcSource src, float s0, float s1, float s2,
    const uint8_t *__restrict__ packed, float *__restrict__ dhat, int *err, TcHold hold) {
    using G = Geo3<T>;
    constexpr int D = G::D;
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t *in = smem + G::kSmIn;
    uint8_t *act = smem + G::kSmAct;
    uint8_t *fcin = smem + G::kSmFc;
    uint8_t *wsm = smem + G::kSmW;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + G::kSmBar);   // [0..3] conv, [4] fc1, [5] final
    uint32_t *epi_done = reinterpret_cast<uint32_t *>(smem + G::kSmCnt);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + G::kSmSlot);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + G::kSmSlot + 4);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int gx = m.ga[0], gy = m.ga[1], gz = m.ga[2];
    const int tx = (gx + T - 1) / T, ty = (gy + T - 1) / T, tz = (gz + T - 1) / T;
    const int n_tiles = tx * ty * tz;

    // set-up that touches no global memory (overlaps the previous kernel under
    // programmatic dependent launch): clear the buffers, barriers, TMEM
    for (int i = tid; i < G::kSmW / 16; i += kThreads3)
        reinterpret_cast<uint4 *>(smem)[i] = make_uint4(0, 0, 0, 0);
    if (tid == 0) {
        for (int i = 0; i < 6; ++i) mbar_init(bars + i, 1u);
        *epi_done = 0;
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_addr(tmem_slot)),
                     "r"(512u));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    pdl_wait();
    for (int i = tid; i < Tc3Layout::total / 16; i += kThreads3)
        cp_async16(wsm + 16 * i, packed + 16 * i);
    cp_async_wait_all();
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_slot;
    const float scale[3] = {s0, s1, s2};

    uint32_t ph = 0;    // epilogue warps: parity of each conv mbarrier's next phase
    for (int k = 0;; ++k) {
        const int tile = blockIdx.x + k * gridDim.x;
        if (tile >= n_tiles) break;
        // the previous tile is finished: every MMA completed (its epilogues
        // waited for them) and every epilogue stored its results
        fence_before();
        __syncthreads();
        fence_after();
        if (*abort_flag) break;
        const int cx0 = (tile % tx) * T, cy0 = ((tile / tx) % ty) * T, cz0 = (tile / (tx * ty)) * T;
        // ---- input: (T + 6)^3 cells around the tile, zero outside the grid;
        //      kB cells per thread at a time, their loads in flight together
        //      (the grid velocity src.U; this kernel does not take the nodal
        //      source: a tile's input cells are many times its own) ----
        constexpr int kB = 3, kCells3 = D * D * D;
        for (int i0 = tid; i0 < kCells3; i0 += kB * kThreads3) {
            int64_t cc[kB];
            #pragma unroll
            for (int j = 0; j < kB; ++j) {
                const int i = i0 + j * kThreads3;
                const int ix = i % D, iy = (i / D) % D, iz = i / (D * D);
                const int cx = cx0 + ix - 3, cy = cy0 + iy - 3, cz = cz0 + iz - 3;
                cc[j] = i < kCells3 && cx >= 0 && cx < gx && cy >= 0 && cy < gy && cz >= 0 && cz < gz
                            ? (int64_t(cz) * gy + cy) * gx + cx
                            : -1;
            }
            float v[kB][3];
            #pragma unroll
            for (int j = 0; j < kB; ++j)
                #pragma unroll
                for (int k2 = 0; k2 < 3; ++k2)
                    v[j][k2] = cc[j] >= 0 ? __ldg(src.U + cc[j] * 3 + k2) : 0.f;
            #pragma unroll
            for (int j = 0; j < kB; ++j) {
                const int i = i0 + j * kThreads3;
                if (i >= kCells3) break;
                *reinterpret_cast<uint4 *>(in + 16 * i) =
                    make_uint4(pack_bf16x2(v[j][0] * scale[0], v[j][1] * scale[1]),
                               pack_bf16x2(v[j][2] * scale[2], 0.f), 0u, 0u);
            }
        }
        fence_async_smem();
        fence_before();
        __syncthreads();
        fence_after();
        const uint32_t base = uint32_t(k) * uint32_t(G::kItems);   // items done before this tile

        if (warp == kMma3) {
            // ---- MMA issue: items in order, as far ahead as inputs and TMEM allow ----
            const bool leader = elect_one();
            const uint64_t d_in = sdesc(smem_addr(in), 16, 128);
            const uint64_t d_act = sdesc(smem_addr(act), G::kActRows * 16, 128);
            const uint64_t d_fc = sdesc(smem_addr(fcin), 128 * 16, 128);
            const uint64_t d_w1 = sdesc(smem_addr(wsm + Tc3Layout::w1), 32 * 16, 128);
            const uint64_t d_wc = sdesc(smem_addr(wsm + Tc3Layout::wc), 32 * 16, 128);
            const uint64_t d_f1 = sdesc(smem_addr(wsm + Tc3Layout::f1), 256 * 16, 128);
            constexpr uint32_t id32 = idesc_bf16(128, 32), id256 = idesc_bf16(128, 256);
            // test hook: a wait for a flag that nothing sets runs out before any MMA
            const bool held = hold.flag && k == 0 &&
                              !__all_sync(kFull, wait_flag(hold.flag, hold.polls, abort_flag, err));
            for (int j = 0; j < G::kItems && !held; ++j) {
                if (!wait_count(epi_done, base + uint32_t(G::need(j)), abort_flag, err)) break;
                fence_after();
                int l, mt;
                G::item(j, l, mt);
                if (leader) {
                    const uint32_t dcol = tmem + uint32_t(l == 3 ? 256 : 32 * (j & 3));
                    const int r0 = 128 * mt;
                    if (l == 0) {
                        // 14 K-steps of two taps: chunk 0 = tap 2i at rows r0 + shift,
                        // chunk 1 = tap 2i + 1 (LBO = the row distance of the two)
                        #pragma unroll
                        for (int i = 0; i < 14; ++i) {
                            const int t0 = 2 * i, t1 = 2 * i + 1 < 27 ? 2 * i + 1 : 2 * i;
                            const int sh0 = tap_shift(t0, D), sh1 = tap_shift(t1, D);
                            const uint64_t a = (d_in & ~(uint64_t(0x3fff) << 16)) +
                                               uint64_t(r0 + sh0) +
                                               (uint64_t((sh1 - sh0 > 0 ? sh1 - sh0 : 1)) << 16);
                            mma_bf16(dcol, a, d_w1 + uint64_t(i * 2 * 32), id32, i > 0 ? 1u : 0u);
                        }
                    } else if (l < 3) {
                        const uint64_t dw = d_wc + uint64_t((l - 1) * (Tc3Layout::wc_bytes / 16));
                        #pragma unroll 3
                        for (int t = 0; t < 27; ++t) {
                            const int sh = tap_shift(t, D);
                            #pragma unroll
                            for (int kk = 0; kk < 2; ++kk) {
                                const uint64_t a = d_act + uint64_t(2 * kk * G::kActRows + r0 + sh);
                                const uint64_t b = dw + uint64_t((t * 4 + 2 * kk) * 32);
                                mma_bf16(dcol, a, b, id32, (t | kk) != 0 ? 1u : 0u);
                            }
                        }
                    } else {
                        #pragma unroll
                        for (int kk = 0; kk < 2; ++kk)
                            mma_bf16(dcol, d_fc + uint64_t(2 * kk * 128), d_f1 + uint64_t(2 * kk * 256),
                                     id256, uint32_t(kk));
                    }
                    mma_commit(bars + (l == 3 ? 4 : (j & 3)));
                }
                __syncwarp();
            }
        } else {
            // ---- epilogues: warp w reads TMEM lanes 32 w .. 32 w + 31 ----
            const float *b1 = reinterpret_cast<const float *>(wsm + Tc3Layout::b1);
            const float *cb = reinterpret_cast<const float *>(wsm + Tc3Layout::cb);
            const float *f1b = reinterpret_cast<const float *>(wsm + Tc3Layout::f1b);
            const float *f2w = reinterpret_cast<const float *>(wsm + Tc3Layout::f2w);
            const float *f2b = reinterpret_cast<const float *>(wsm + Tc3Layout::f2b);
            const uint32_t tq = tmem + (uint32_t(32 * warp) << 16);
            for (int j = 0; j < G::kItems; ++j) {
                int l, mt;
                G::item(j, l, mt);
                const int bi = l == 3 ? 4 : (j & 3);
                const uint32_t par = l == 3 ? uint32_t(k & 1) : (ph >> bi) & 1u;
                const bool ok = __all_sync(kFull, mbar_wait(bars + bi, par, abort_flag, err)) != 0;
                if (epi3_or(!ok)) break;
                if (l < 3) ph ^= 1u << bi;
                fence_after();
                if (l < 3) {
                    float v[32];
                    tmem_ld32(tq + uint32_t(32 * (j & 3)), v);
                    uint32_t hv[16];
                    bias_relu_bf16(v, l == 0 ? b1 : cb + 32 * (l - 1), hv);
                    const int row = 128 * mt + 32 * warp + lane;
                    if (l < 2) {
                        store_act<G::kActRows>(act, row, hv);
                    } else {
                        const int x = row % D, y = (row / D) % D, z = row / (D * D);
                        if (x < T && y < T && z < T) store_act<128>(fcin, (z * T + y) * T + x, hv);
                    }
                } else {
                    // fc1 + ReLU + fc2 of cell ci of the tile
                    const int ci = 32 * warp + lane;
                    float o0 = f2b[0], o1 = f2b[1], o2 = f2b[2];
                    #pragma unroll 1
                    for (int c = 0; c < 8; ++c) {
                        float v[32];
                        tmem_ld32(tq + 256u + uint32_t(32 * c), v);
                        #pragma unroll
                        for (int e = 0; e < 32; ++e) {
                            const int n = 32 * c + e;
                            const float h = fmaxf(v[e] + f1b[n], 0.f);
                            o0 = fmaf(h, f2w[n], o0);
                            o1 = fmaf(h, f2w[256 + n], o1);
                            o2 = fmaf(h, f2w[512 + n], o2);
                        }
                    }
                    const int x = ci % T, y = (ci / T) % T, z = ci / (T * T);
                    const int cx = cx0 + x, cy = cy0 + y, cz = cz0 + z;
                    if (ci < G::kCells && cx < gx && cy < gy && cz < gz) {
                        float *o = dhat + ((int64_t(cz) * gy + cy) * gx + cx) * 3;
                        o[0] = o0;
                        o[1] = o1;
                        o[2] = o2;
                    }
                }
                // the stores are complete and visible to the tensor cores'
                // operand reads before the item counts as done
                fence_before();
                fence_async_smem();
                epi3_or(false);
                if (tid == 0) red_release_add(epi_done, 1u);
            }
        }
    }
    // wait (bounded) for this CTA's MMAs in flight before TMEM is released
    if (warp == kMma3) {
        if (elect_one()) {
            mma_commit(bars + 5);
            for (uint32_t i = 0; i < (1u << 24) && !mbar_try_wait(bars + 5, 0); ++i)
                if (i > 64) __nanosleep(64);
        }
        __syncwarp();
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512u));
}

// Pack the FP32 master weights of the 3-D predictor into the kernel's layout.
__global__ void pack3_kernel(const float *__restrict__ w, uint8_t *__restrict__ out,
                             int64_t off_w1, int64_t off_b1, int64_t off_w2, int64_t off_b2,
                             int64_t off_w3, int64_t off_b3, int64_t off_f1w, int64_t off_f1b,
                             int64_t off_f2w, int64_t off_f2b) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
    // conv1 W[o][i][t] (i < 3) -> [pair p][half h][o][8]: tap 2p + h, channel j (zero for
    // j >= 3 and for tap 27)
    __nv_bfloat16 *w1 = reinterpret_cast<__nv_bfloat16 *>(out + Tc3Layout::w1);
    for (int e = tid; e < 14 * 2 * 32 * 8; e += nth) {
        const int j = e % 8, o = (e / 8) % 32, h = (e / 256) % 2, p = e / 512;
        const int t = 2 * p + h;
        w1[e] = __float2bfloat16_rn(t < 27 && j < 3 ? w[off_w1 + (o * 3 + j) * 27 + t] : 0.f);
    }
    for (int i = tid; i < 32; i += nth) {
        reinterpret_cast<float *>(out + Tc3Layout::b1)[i] = w[off_b1 + i];
        reinterpret_cast<float *>(out + Tc3Layout::cb)[i] = w[off_b2 + i];
        reinterpret_cast<float *>(out + Tc3Layout::cb)[32 + i] = w[off_b3 + i];
    }
    // conv2, conv3 W[o][i][t] -> [t][q][o][8], i = 8 q + j
    const int64_t offs[2] = {off_w2, off_w3};
    for (int l = 0; l < 2; ++l) {
        __nv_bfloat16 *bw = reinterpret_cast<__nv_bfloat16 *>(out + Tc3Layout::wc + l * Tc3Layout::wc_bytes);
        for (int e = tid; e < 27 * 32 * 32; e += nth) {
            const int t = e / 1024, o = (e / 32) % 32, i = e % 32;
            bw[((t * 4 + i / 8) * 32 + o) * 8 + i % 8] =
                __float2bfloat16_rn(w[offs[l] + (o * 32 + i) * 27 + t]);
        }
    }
    // fc1 W[n][k] (256 x 32) -> [q][n][8], k = 8 q + j
    __nv_bfloat16 *f1 = reinterpret_cast<__nv_bfloat16 *>(out + Tc3Layout::f1);
    for (int e = tid; e < 256 * 32; e += nth) {
        const int n = e / 32, kq = e % 32;
        f1[((kq / 8) * 256 + n) * 8 + kq % 8] = __float2bfloat16_rn(w[off_f1w + e]);
    }
    for (int i = tid; i < 256; i += nth) {
        reinterpret_cast<float *>(out + Tc3Layout::f1b)[i] = w[off_f1b + i];
        for (int k = 0; k < 3; ++k)
            reinterpret_cast<float *>(out + Tc3Layout::f2w)[k * 256 + i] = w[off_f2w + k * 256 + i];
    }
    if (tid < 4) reinterpret_cast<float *>(out + Tc3Layout::f2b)[tid] = tid < 3 ? w[off_f2b + tid] : 0.f;
}

template <int T>
int64_t tiles3(const DevMesh &m) {
    return int64_t((m.ga[0] + T - 1) / T) * ((m.ga[1] + T - 1) / T) * ((m.ga[2] + T - 1) / T);
}

// relative cost of a pass with tiles of side T: waves of one tile per SM,
// each worth its MMAs (conv1 14 per M-tile, conv2/conv3 54, fc1 2)
template <int T>
int64_t cost3(const DevMesh &m, int sm_count) {
    using G = Geo3<T>;
    const int64_t waves = (tiles3<T>(m) + sm_count - 1) / sm_count;
    return waves * (14 * G::m1 + 54 * (G::m2 + G::m3) + 2 + 64);
}

template <int T>
int launch3(const DevMesh &m, const TcSource &src, double dt, const uint8_t *packed, float *dhat,
            int *err, int sm_count, cudaStream_t st, TcHold hold) {
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(cnn3d_tc_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             Geo3<T>::kSmTotal);
        attr = true;
    }
    const int grid = int(std::min<int64_t>(tiles3<T>(m), sm_count));
    launch_pdl(cnn3d_tc_kernel<T>, dim3(grid), dim3(kThreads3), size_t(Geo3<T>::kSmTotal), st, m,
               src, float(dt / m.sa[0]), float(dt / m.sa[1]), float(dt / m.sa[2]), packed, dhat, err,
               hold);
    return 1;
}

}  // namespace

int64_t tc3_packed_bytes() { return Tc3Layout::total; }

int launch_pack_tc3(const float *w, const NetShape &S, uint8_t *packed, cudaStream_t st) {
    pack3_kernel<<<64, 256, 0, st>>>(w, packed, S.w_off[0], S.b_off[0], S.w_off[1], S.b_off[1],
                                     S.w_off[2], S.b_off[2], S.w_off[3], S.b_off[3], S.w_off[4],
                                     S.b_off[4]);
    return 1;
}

int tc3_pick_tile(const DevMesh &m, int sm_count) {
    const int64_t c4 = cost3<4>(m, sm_count), c3 = cost3<3>(m, sm_count);
    return c4 <= c3 ? 4 : 3;
}

int launch_cnn3d_tc(const DevMesh &m, const TcSource &src, double dt, const uint8_t *packed,
                    float *dhat, int *err, int sm_count, int tile, cudaStream_t st, TcHold hold) {
    const int t = tile ? tile : tc3_pick_tile(m, sm_count);
    if (t == 4) return launch3<4>(m, src, dt, packed, dhat, err, sm_count, st, hold);
    if (t == 3) return launch3<3>(m, src, dt, packed, dhat, err, sm_count, st, hold);
    return launch3<2>(m, src, dt, packed, dhat, err, sm_count, st, hold);
}

}  // namespace cs
