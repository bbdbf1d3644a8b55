// Grid inference of the 2-D start predictor on the tensor cores (tcgen05).
//
// The predictor maps the 9x9 window of the ASG-grid velocity around a cell to
// the cell's displacement (Sec. 2.3, Algorithm 2). Windows of neighbouring
// cells overlap, so the network is evaluated for all cells at once: with
// valid convolutions, the window result at cell c equals a fully
// convolutional pass over the zero-padded grid, read at c. One persistent CTA
// per SM walks over 24 x 24-cell output tiles:
//
//   input   32 x 32 cells x 2 channels (tile + 4-cell halo), FP32, in smem
//   conv1   CUDA cores, 30 x 30 x 32, ReLU, stored BF16
//   conv2-4 tcgen05.mma kind::f16 (BF16 x BF16 -> FP32 in TMEM), implicit
//           GEMM: M = 128 pixels, N = 32 channels, K = 16 channels of one tap;
//           9 taps x 2 K-steps per M-tile; ReLU + BF16 in the epilogue
//   fc1     tcgen05.mma, M = 128 pixels, N = 256, K = 32
//   fc2     CUDA cores in the fc1 epilogue (256 -> 2)
//
// Activations live in shared memory as [8-channel chunk q][pixel r][8] BF16,
// with pixels on a flat 32-wide row-major index for every layer (columns past
// the valid width hold garbage that only ever feeds garbage outputs). A tap
// (dy, dx) is then a shift of dy*32 + dx pixels, i.e. an offset of the MMA's
// shared-memory descriptor: no im2col copy. The canonical no-swizzle K-major
// layout has 8x16-byte core matrices, SBO = 128 B between 8-pixel groups and
// LBO = 16 KiB between channel chunks.
#include <cuda_bf16.h>

#include <cstdint>

#include "cnn.h"
#include "walk_common.cuh"

namespace cs {
namespace {

constexpr int kTile = 24;            // output cells per tile edge
constexpr int kW = 32;               // flat row width (= tile + 8)
constexpr int kRows = 1024;          // pixel rows of an activation buffer
constexpr int kThreadsTC = 512;      // 16 warps: 4 per TMEM lane quarter
constexpr int kFcTiles = 5;          // 576 compacted pixels -> 5 M-tiles of fc1
constexpr uint32_t kTmemCols = 512;

// packed weights (bytes); produced by pack_weights_kernel
struct TcLayout {
    static constexpr int w1 = 0;                          // bf16 [9][32][8]: W1/2, channels >= 2 zero
    static constexpr int b1 = w1 + 9 * 32 * 8 * 2;        // fp32 [32]
    static constexpr int bconv = b1 + 32 * 4;             // 3 x bf16 [9][4][32][8]
    static constexpr int bconv_bytes = 9 * 4 * 32 * 8 * 2;
    static constexpr int cb = bconv + 3 * bconv_bytes;    // fp32 [3][32] conv biases
    static constexpr int bfc1 = cb + 3 * 32 * 4;          // bf16 [4][256][8]
    static constexpr int bfc1_bytes = 4 * 256 * 8 * 2;
    static constexpr int fc1b = bfc1 + bfc1_bytes;        // fp32 [256]
    static constexpr int fc2w = fc1b + 256 * 4;           // fp32 [2][256]
    static constexpr int fc2b = fc2w + 2 * 256 * 4;       // fp32 [2]
    static constexpr int total = ((fc2b + 2 * 4) + 127) / 128 * 128;
};

// shared memory map (bytes)
constexpr int kRowsX0 = 1152;                               // 32 x 32 input + shifted reads
constexpr int kSmX0 = 0;                                    // bf16 [1152][8] (2 channels used)
constexpr int kSmAct0 = kSmX0 + kRowsX0 * 16;               // bf16 [4][1024][8]
constexpr int kSmAct1 = kSmAct0 + 4 * kRows * 16;
constexpr int kSmW = kSmAct1 + 4 * kRows * 16;              // packed weights
constexpr int kSmRed = kSmW + TcLayout::total;              // float2 [2][128] fc2 partials
constexpr int kSmBar = kSmRed + 2 * 128 * 8;                // mbarrier + tmem slot
constexpr int kSmTotal = kSmBar + 64;
static_assert(kSmTotal <= 232448, "shared memory of one CTA");

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// shared-memory matrix descriptor: no swizzle, K-major core matrices
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return uint64_t((addr >> 4) & 0x3fff) | (uint64_t((lbo >> 4) & 0x3fff) << 16) |
           (uint64_t((sbo >> 4) & 0x3fff) << 32) | (uint64_t(1) << 46);
}

// instruction descriptor, kind::f16: D f32, A and B bf16, both K-major
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(N >> 3) << 17) |
           (uint32_t(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t dt, uint64_t a, uint64_t b, uint32_t id,
                                         uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(dt),
        "l"(a), "l"(b), "r"(id), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait: false (and the error flag set) if the MMAs never complete
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, int *err) {
    for (uint32_t i = 0; i < (1u << 24); ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if (i > 64) __nanosleep(64);
    }
    atomicExch(err, 1);
    return false;
}

__device__ __forceinline__ void fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// 32 lanes x 32 columns of FP32 from TMEM (this warp's lane quarter)
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float *v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
        "%28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    #pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t *>(&h);
}

// Store one pixel's 32 channels (ReLU already applied) into an activation
// buffer in the chunked layout.
__device__ __forceinline__ void store_act(uint8_t *buf, int row, const float *v) {
    #pragma unroll
    for (int q = 0; q < 4; ++q) {
        uint4 w;
        w.x = pack_bf16x2(v[8 * q + 0], v[8 * q + 1]);
        w.y = pack_bf16x2(v[8 * q + 2], v[8 * q + 3]);
        w.z = pack_bf16x2(v[8 * q + 4], v[8 * q + 5]);
        w.w = pack_bf16x2(v[8 * q + 6], v[8 * q + 7]);
        *reinterpret_cast<uint4 *>(buf + (size_t(q) * kRows + row) * 16) = w;
    }
}

// Issue the MMAs of one 3x3 convolution layer (called by one thread):
// n_mt M-tiles of 128 pixels, TMEM columns [32*mt, 32*mt + 32).
__device__ __forceinline__ void issue_conv(uint32_t tmem, const uint8_t *act, const uint8_t *wb,
                                           int n_mt) {
    constexpr uint32_t id = idesc_bf16(128, 32);
    const uint32_t a0 = smem_addr(act), b0 = smem_addr(wb);
    for (int mt = 0; mt < n_mt; ++mt) {
        uint32_t acc = 0;
        for (int t = 0; t < 9; ++t) {
            const int shift = (t / 3) * kW + (t % 3);
            for (int kk = 0; kk < 2; ++kk) {
                const uint64_t a = sdesc(a0 + uint32_t((2 * kk * kRows + 128 * mt + shift) * 16),
                                         kRows * 16, 128);
                const uint64_t b = sdesc(b0 + uint32_t(((t * 4 + 2 * kk) * 32) * 16), 32 * 16, 128);
                mma_bf16(tmem + uint32_t(32 * mt), a, b, id, acc);
                acc = 1;
            }
        }
    }
}

// Issue the MMAs of conv1 (called by one thread): the input has one 8-channel
// chunk (u0, u1, 0 ... 0); a K = 16 step reads that chunk twice (LBO = 0 on
// both operands) against halved weights, so the sum is the 8-channel product.
// 8 M-tiles cover the 30 valid rows (rows past them are garbage).
__device__ __forceinline__ void issue_conv1(uint32_t tmem, const uint8_t *x0, const uint8_t *wb) {
    constexpr uint32_t id = idesc_bf16(128, 32);
    const uint32_t a0 = smem_addr(x0), b0 = smem_addr(wb);
    for (int mt = 0; mt < 8; ++mt)
        for (int t = 0; t < 9; ++t) {
            const int shift = (t / 3) * kW + (t % 3);
            const uint64_t a = sdesc(a0 + uint32_t((128 * mt + shift) * 16), 0, 128);
            const uint64_t b = sdesc(b0 + uint32_t(t * 32 * 16), 0, 128);
            mma_bf16(tmem + uint32_t(32 * mt), a, b, id, t > 0 ? 1u : 0u);
        }
}

// Epilogue of a conv layer: TMEM -> +bias, ReLU -> BF16 activations. Warp w
// reads TMEM lane quarter w % 4 (the only one it may access) of M-tiles
// w / 4, w / 4 + 4, ... With `compact`, pixel (y, x) goes to row y * 24 + x
// and the garbage columns x >= 24 are dropped (input of fc1).
__device__ __forceinline__ void epilogue_conv(uint32_t tmem, uint8_t *out, const float *bias,
                                              int n_mt, bool compact) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = warp & 3, h = warp >> 2;
    for (int mt = h; mt < n_mt; mt += kThreadsTC / 128) {
        float v[32];
        tmem_ld32(tmem + (uint32_t(32 * g) << 16) + uint32_t(32 * mt), v);
        #pragma unroll
        for (int c = 0; c < 32; ++c) v[c] = fmaxf(v[c] + bias[c], 0.f);
        const int row = 128 * mt + 32 * g + lane;
        if (!compact) {
            store_act(out, row, v);
        } else if (row % kW < kTile && row / kW < kTile) {
            store_act(out, (row / kW) * kTile + row % kW, v);
        }
    }
}

__global__ void __launch_bounds__(kThreadsTC, 1) cnn2d_tc_kernel(
    const DevMesh m, const float *__restrict__ U, float scale0, float scale1,
    const uint8_t *__restrict__ packed, float *__restrict__ dhat, int *err) {
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t *x0 = smem + kSmX0;
    uint8_t *act0 = smem + kSmAct0;
    uint8_t *act1 = smem + kSmAct1;
    uint8_t *wsm = smem + kSmW;
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + kSmBar);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + kSmBar + 8);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int gx = m.ga[0], gy = m.ga[1];
    const int tiles_x = (gx + kTile - 1) / kTile, tiles_y = (gy + kTile - 1) / kTile;
    const int n_tiles = tiles_x * tiles_y;

    // weights into shared memory (once per CTA)
    for (int i = tid; i < TcLayout::total / 16; i += kThreadsTC)
        reinterpret_cast<uint4 *>(wsm)[i] = reinterpret_cast<const uint4 *>(packed)[i];
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_addr(tmem_slot)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    // zero the activation rows past the computed pixels (read only by garbage)
    for (int i = tid; i < 4 * kRows; i += kThreadsTC) {
        reinterpret_cast<uint4 *>(act0)[i] = make_uint4(0, 0, 0, 0);
        reinterpret_cast<uint4 *>(act1)[i] = make_uint4(0, 0, 0, 0);
    }
    for (int i = tid; i < kRowsX0; i += kThreadsTC)
        reinterpret_cast<uint4 *>(x0)[i] = make_uint4(0, 0, 0, 0);
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_slot;
    const float *b1 = reinterpret_cast<const float *>(wsm + TcLayout::b1);
    const float *cb = reinterpret_cast<const float *>(wsm + TcLayout::cb);
    const float *fc1b = reinterpret_cast<const float *>(wsm + TcLayout::fc1b);
    const float *fc2w = reinterpret_cast<const float *>(wsm + TcLayout::fc2w);
    const float *fc2b = reinterpret_cast<const float *>(wsm + TcLayout::fc2b);
    uint32_t phase = 0;
    bool ok = true;

    for (int tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x) {
        const int tx = tile % tiles_x, ty = tile / tiles_x;
        const int cx0 = tx * kTile - 4, cy0 = ty * kTile - 4;
        // ---- input: 32 x 32 cells, channels u_k * dt / s_k (BF16), zero outside ----
        for (int i = tid; i < kW * kW; i += kThreadsTC) {
            const int cx = cx0 + (i % kW), cy = cy0 + (i / kW);
            float u0 = 0.f, u1 = 0.f;
            if (cx >= 0 && cx < gx && cy >= 0 && cy < gy) {
                const float2 uv = __ldg(reinterpret_cast<const float2 *>(U) + int64_t(cy) * gx + cx);
                u0 = uv.x * scale0;
                u1 = uv.y * scale1;
            }
            reinterpret_cast<uint4 *>(x0)[i] = make_uint4(pack_bf16x2(u0, u1), 0, 0, 0);
        }
        fence_async_smem();
        __syncthreads();
        // ---- conv1 on tcgen05 -> act0 ----
        if (tid == 0) {
            fence_after();
            issue_conv1(tmem, x0, wsm + TcLayout::w1);
            mma_commit(bar);
        }
        ok = __syncthreads_and(mbar_wait(bar, phase, err)) != 0;   // uniform
        phase ^= 1;
        fence_after();
        if (ok) epilogue_conv(tmem, act0, b1, 8, false);
        fence_before();
        fence_async_smem();
        __syncthreads();
        // ---- conv2, conv3, conv4 on tcgen05 ----
        const int n_mt[3] = {7, 7, 6};      // 28, 26, 24 valid rows of 32 pixels
        uint8_t *src = act0, *dst = act1;
        for (int l = 0; l < 3 && ok; ++l) {
            if (tid == 0) {
                fence_after();
                issue_conv(tmem, src, wsm + TcLayout::bconv + l * TcLayout::bconv_bytes, n_mt[l]);
                mma_commit(bar);
            }
            ok = __syncthreads_and(mbar_wait(bar, phase, err)) != 0;   // uniform
            phase ^= 1;
            fence_after();
            if (ok) epilogue_conv(tmem, dst, cb + 32 * l, n_mt[l], l == 2);
            fence_before();
            fence_async_smem();
            __syncthreads();
            uint8_t *tmp = src;
            src = dst;
            dst = tmp;
        }
        // ---- fc1 on tcgen05 over the 576 compacted valid pixels (5 M-tiles,
        //      two per round of 256 columns each), fc2 in the epilogue ----
        for (int round = 0; round < 3 && ok; ++round) {
            if (tid == 0) {
                fence_after();
                constexpr uint32_t id = idesc_bf16(128, 256);
                const uint32_t a0 = smem_addr(src), b0 = smem_addr(wsm + TcLayout::bfc1);
                for (int h = 0; h < 2; ++h) {
                    const int mt = 2 * round + h;
                    if (mt >= kFcTiles) break;
                    for (int kk = 0; kk < 2; ++kk) {
                        const uint64_t a =
                            sdesc(a0 + uint32_t((2 * kk * kRows + 128 * mt) * 16), kRows * 16, 128);
                        const uint64_t b = sdesc(b0 + uint32_t(2 * kk * 256 * 16), 256 * 16, 128);
                        mma_bf16(tmem + uint32_t(256 * h), a, b, id, kk);
                    }
                }
                mma_commit(bar);
            }
            ok = __syncthreads_and(mbar_wait(bar, phase, err)) != 0;   // uniform
            phase ^= 1;
            fence_after();
            // warp (g, h): M-tile 2*round + (h & 1), columns [128 (h >> 1), +128)
            const int g = warp & 3, h = warp >> 2;
            const int mt = 2 * round + (h & 1), half = h >> 1;
            const int row = 128 * mt + 32 * g + lane;
            float o0 = 0.f, o1 = 0.f;
            if (ok && mt < kFcTiles) {
                if (half == 0) {
                    o0 = fc2b[0];
                    o1 = fc2b[1];
                }
                for (int j = 4 * half; j < 4 * half + 4; ++j) {
                    float v[32];
                    // M-tile (h & 1) of this round holds TMEM columns [256 (h & 1), +256)
                    tmem_ld32(tmem + (uint32_t(32 * g) << 16) + uint32_t(256 * (h & 1) + 32 * j), v);
                    const float4 *pb = reinterpret_cast<const float4 *>(fc1b + 32 * j);
                    const float4 *p0 = reinterpret_cast<const float4 *>(fc2w + 32 * j);
                    const float4 *p1 = reinterpret_cast<const float4 *>(fc2w + 256 + 32 * j);
                    #pragma unroll
                    for (int c = 0; c < 8; ++c) {
                        const float4 bb = pb[c], w0 = p0[c], w1 = p1[c];
                        const float h0 = fmaxf(v[4 * c] + bb.x, 0.f);
                        const float h1 = fmaxf(v[4 * c + 1] + bb.y, 0.f);
                        const float h2 = fmaxf(v[4 * c + 2] + bb.z, 0.f);
                        const float h3 = fmaxf(v[4 * c + 3] + bb.w, 0.f);
                        o0 = fmaf(w0.x, h0, fmaf(w0.y, h1, fmaf(w0.z, h2, fmaf(w0.w, h3, o0))));
                        o1 = fmaf(w1.x, h0, fmaf(w1.y, h1, fmaf(w1.z, h2, fmaf(w1.w, h3, o1))));
                    }
                }
            }
            // the second column half hands its partial sums to the first
            float2 *red = reinterpret_cast<float2 *>(smem + kSmRed);
            if (half == 1) red[(h & 1) * 128 + 32 * g + lane] = make_float2(o0, o1);
            fence_before();
            __syncthreads();
            if (ok && half == 0 && mt < kFcTiles) {
                const float2 p = red[(h & 1) * 128 + 32 * g + lane];
                const int y = row / kTile, x = row % kTile;
                const int cx = tx * kTile + x, cy = ty * kTile + y;
                if (row < kTile * kTile && cx < gx && cy < gy)
                    reinterpret_cast<float2 *>(dhat)[int64_t(cy) * gx + cx] =
                        make_float2(o0 + p.x, o1 + p.y);
            }
            __syncthreads();
        }
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(kTmemCols));
}

// Pack the FP32 master weights of the 2-D predictor into the smem layout.
__global__ void pack_weights_kernel(const float *__restrict__ w, uint8_t *__restrict__ out,
                                    int64_t off_w1, int64_t off_b1, int64_t off_w2,
                                    int64_t off_b2, int64_t off_w3, int64_t off_b3,
                                    int64_t off_w4, int64_t off_b4, int64_t off_f1w,
                                    int64_t off_f1b, int64_t off_f2w, int64_t off_f2b) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
    // conv1 W[o][i][t] (i < 2) -> [t][o][8] halved (each K step reads it twice)
    __nv_bfloat16 *w1 = reinterpret_cast<__nv_bfloat16 *>(out + TcLayout::w1);
    for (int e = tid; e < 9 * 32 * 8; e += nth) {
        const int t = e / 256, o = (e / 8) % 32, j = e % 8;
        w1[e] = __float2bfloat16_rn(j < 2 ? 0.5f * w[off_w1 + (o * 2 + j) * 9 + t] : 0.f);
    }
    for (int i = tid; i < 32; i += nth) {
        reinterpret_cast<float *>(out + TcLayout::b1)[i] = w[off_b1 + i];
        reinterpret_cast<float *>(out + TcLayout::cb)[i] = w[off_b2 + i];
        reinterpret_cast<float *>(out + TcLayout::cb)[32 + i] = w[off_b3 + i];
        reinterpret_cast<float *>(out + TcLayout::cb)[64 + i] = w[off_b4 + i];
    }
    // conv weights W[o][i][t] -> [t][q][o][8] with i = 8q + j
    const int64_t offs[3] = {off_w2, off_w3, off_w4};
    for (int l = 0; l < 3; ++l) {
        __nv_bfloat16 *bw =
            reinterpret_cast<__nv_bfloat16 *>(out + TcLayout::bconv + l * TcLayout::bconv_bytes);
        for (int e = tid; e < 9 * 32 * 32; e += nth) {
            const int t = e / 1024, o = (e / 32) % 32, i = e % 32;
            const int q = i / 8, j = i % 8;
            bw[((t * 4 + q) * 32 + o) * 8 + j] = __float2bfloat16_rn(w[offs[l] + (o * 32 + i) * 9 + t]);
        }
    }
    // fc1 W[n][k] (256 x 32) -> [q][n][8] with k = 8q + j
    __nv_bfloat16 *f1 = reinterpret_cast<__nv_bfloat16 *>(out + TcLayout::bfc1);
    for (int e = tid; e < 256 * 32; e += nth) {
        const int n = e / 32, k = e % 32;
        f1[((k / 8) * 256 + n) * 8 + (k % 8)] = __float2bfloat16_rn(w[off_f1w + e]);
    }
    for (int i = tid; i < 256; i += nth) {
        reinterpret_cast<float *>(out + TcLayout::fc1b)[i] = w[off_f1b + i];
        reinterpret_cast<float *>(out + TcLayout::fc2w)[i] = w[off_f2w + i];
        reinterpret_cast<float *>(out + TcLayout::fc2w)[256 + i] = w[off_f2w + 256 + i];
    }
    if (tid < 2) reinterpret_cast<float *>(out + TcLayout::fc2b)[tid] = w[off_f2b + tid];
}

}  // namespace

int64_t tc_packed_bytes() { return TcLayout::total; }

int launch_pack_tc(const float *w, const NetShape &S, uint8_t *packed, cudaStream_t st) {
    pack_weights_kernel<<<64, 256, 0, st>>>(w, packed, S.w_off[0], S.b_off[0], S.w_off[1],
                                            S.b_off[1], S.w_off[2], S.b_off[2], S.w_off[3],
                                            S.b_off[3], S.w_off[4], S.b_off[4], S.w_off[5],
                                            S.b_off[5]);
    return 1;
}

int launch_cnn2d_tc(const DevMesh &m, const float *U, double dt, const uint8_t *packed,
                    float *dhat, int *err, int sm_count, cudaStream_t st) {
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(cnn2d_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kSmTotal);
        attr = true;
    }
    const int tiles = ((m.ga[0] + kTile - 1) / kTile) * ((m.ga[1] + kTile - 1) / kTile);
    const int grid = std::min(tiles, sm_count);
    cnn2d_tc_kernel<<<grid, kThreadsTC, kSmTotal, st>>>(
        m, U, float(dt / m.sa[0]), float(dt / m.sa[1]), packed, dhat, err);
    return 1;
}

}  // namespace cs
