// Module 1 of the classifier predictor (Sec. 2.3) fused on the tensor cores:
// the pooled-centroid window of a particle, its two zero-padded 3^D
// convolutions of 32 channels with ReLU and the 2^D average pooling, in one
// CTA, with no im2col copy and no activation leaving shared memory.
//
// Layout. A particle's zero-padded window (edge E = W + 2) sits on a flat
// index q = (z E + y) E + x. A convolution output is computed at the row
// r = q - (E + 1) (2-D; q - (E^2 + E + 1) in 3-D) of the window position q it
// belongs to, and reads its input at r + shift(tap), shift = (dz E + dy) E + dx:
// a tap is a row offset of the shared-memory operand, so each convolution is
// an implicit GEMM. Output rows whose position lies outside the window (the
// wrap-around columns) are garbage and are never stored or pooled.
//
//   input  [rows][8] BF16: the D window channels and 8 - D zero channels;
//          the ring and the rows past the window stay zero
//   conv1  tcgen05.mma kind::f16, M = 128 rows, N = 32, K = 16 = two taps of
//          8 channels: the A descriptor's leading byte offset is the row
//          distance of the two taps (5 MMAs per M-tile in 2-D, 14 in 3-D; the
//          last pair's second tap has zero weights)
//   conv2  K = 32 channels of one tap in two K = 16 steps: 2 MMAs per tap
//   act    [4 chunks][rows][8] BF16: ReLU(conv1 + b1), written at the window
//          position of each valid output row (its padded layout is conv2's
//          operand, ring zero)
//   stage  [output rows][33] FP32: ReLU(conv2 + b2), read by the pooling
//   FP32 accumulation in TMEM: conv1 in columns [0, 32 MT), conv2 in
//   [32 MT, 64 MT), MT the M-tiles of a particle (1 in 2-D, 5 in 3-D).
//
// Inputs. Each window cell holds (p - x_p) / s: p is the cell's pooled
// element centroid, given as float hi + lo parts, so the difference is taken
// in FP32 to about one unit in the last place of the FP64 value; a cell
// outside the grid or without a centroid holds its centre, (e - W/2) - offset
// in cell units. x_p's cell is the FP64 formula's (certified in FP32, with the
// FP64 formula as arbiter: the same cell as the labels and the start rule);
// its offset from the cell centre is taken in FP32.
//
// Warps. Warps 0-3 compute the inputs, run both epilogues and the pooling
// (warp w reads TMEM lanes 32 w .. 32 w + 31); warp 4 issues the MMAs. A CTA
// takes particles blockIdx.x, blockIdx.x + gridDim.x, ...; the inputs of
// particle k + 1 are computed while particle k's conv2 runs, and its conv1
// runs while particle k's conv2 epilogue and pooling run. Every wait is
// bounded; one that gives up raises the CTA's abort flag and the device
// error flag.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>

#include "classifier.h"
#include "tc_common.cuh"

namespace cs {
namespace {

constexpr int kEpiC = 4;                    // epilogue warps 0..3
constexpr int kMmaC = 4;                    // the MMA-issuing warp
constexpr int kThreadsC = (kEpiC + 1) * 32;

template <int D>
struct ClsGeo {
    static constexpr int W = D == 2 ? 9 : 7;
    static constexpr int E = W + 2;                                  // padded edge
    static constexpr int P = D == 2 ? W * W : W * W * W;             // window cells
    static constexpr int S = D == 2 ? 2 * E + 2 : (2 * E + 2) * E + 2;   // largest tap shift
    static constexpr int Ro = D == 2 ? (W - 1) * E + W : ((W - 1) * E + W - 1) * E + W;
    static constexpr int MT = (Ro + 127) / 128;                      // M-tiles per particle
    static constexpr int Rows = (128 * MT + S + 8 + 7) / 8 * 8;      // operand rows
    static constexpr int Coff = D == 2 ? E + 1 : (E + 1) * E + 1;    // output row -> position
    static constexpr int Taps = D == 2 ? 9 : 27;
    static constexpr int Pairs = (Taps + 1) / 2;
    static constexpr int Wp = W / 2;
    static constexpr int Pp = D == 2 ? Wp * Wp : Wp * Wp * Wp;
    static constexpr int Ld = 33;                                    // stage row stride (floats)
    static constexpr uint32_t Cols = D == 2 ? 64 : 512;              // TMEM columns allocated
    // packed weights
    static constexpr int kW1 = 0;                                    // bf16 [Pairs][2][32][8]
    static constexpr int kB1 = kW1 + Pairs * 1024;                   // f32 [32]
    static constexpr int kW2 = kB1 + 128;                            // bf16 [Taps][4][32][8]
    static constexpr int kB2 = kW2 + Taps * 2048;                    // f32 [32]
    static constexpr int kPacked = kB2 + 128;
    // shared memory
    static constexpr int kSmIn = 0;
    static constexpr int kSmAct = kSmIn + Rows * 16;
    static constexpr int kSmW = kSmAct + 4 * Rows * 16;
    static constexpr int kSmStage = kSmW + kPacked;
    static constexpr int kSmBar = (kSmStage + Ro * Ld * 4 + 7) / 8 * 8;   // mbarriers [3]
    static constexpr int kSmCnt = kSmBar + 3 * 8;                    // u32 in_ready, act_ready
    static constexpr int kSmPart = kSmCnt + 8;                       // int c0[3], float off[3], x hi/lo [6]
    static constexpr int kSmSlot = kSmPart + 12 * 4;                 // TMEM address, abort flag
    static constexpr int kSmTotal = kSmSlot + 16;

    static_assert(64 * MT <= int(Cols), "TMEM columns");
    static_assert(128 * MT + S < Rows, "operand reads in bounds (the zero tap included)");
    static_assert(Ro - 1 + Coff < (D == 2 ? E * E : E * E * E), "outputs land in the window");
    static_assert(kSmTotal <= 232448, "shared memory of one CTA");
    static_assert(kSmW % 128 == 0 && kSmAct % 128 == 0, "operand alignment");
};

template <int D>
__device__ __forceinline__ constexpr int cls_shift(int t) {
    using G = ClsGeo<D>;
    return D == 2 ? (t / 3) * G::E + t % 3 : ((t / 9) * G::E + (t / 3) % 3) * G::E + t % 3;
}

// named barrier 1 over the epilogue warps
__device__ __forceinline__ void epi_sync() {
    asm volatile("bar.sync 1, %0;" ::"n"(kEpiC * 32) : "memory");
}
__device__ __forceinline__ bool epi_or(bool flag) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 q, %1, 0;\n\t"
        "bar.red.or.pred p, 1, %2, q;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(r)
        : "r"(uint32_t(flag)), "n"(kEpiC * 32)
        : "memory");
    return r != 0;
}

// x_p's ASG cell on axis k and its offset from the cell centre (cell units).
// The cell is the FP64 formula's (floor((x - lo) / s), clamped): taken in
// FP32 from x's hi + lo parts where the rounding bound cannot move the
// quotient across an integer, else by the FP64 formula itself (the
// certification of the walk's cell indices). The offset is the FP32
// quotient minus (cell + 1/2), within ~1e-7 of the quotient of the FP64 one.
__device__ __forceinline__ void cell_offset(const DevMesh &m, int k, double x, float xh, float xl,
                                            int &cell, float &off) {
    const float df = (xh - m.lo_h[k]) + (xl - m.lo_l[k]);
    const float ed = delta_bound(df, xh, m.lo_h[k]);
    const float q = df * m.inv_sa[k];
    const float bnd = fmaf(2.0f * ed, m.inv_sa[k], fmaf(k8U, fabsf(q), kTiny));
    const int a = __float2int_rd(q - bnd), b = __float2int_rd(q + bnd);
    int64_t i;
    if (a == b && fabsf(q) < 4.0e6f)
        i = a < 0 ? 0 : (a > m.ga[k] - 1 ? m.ga[k] - 1 : a);
    else
        i = cell_axis64(x, m.lo[k], m.sa[k], m.ga[k]);
    cell = int(i);
    off = q - (float(i) + 0.5f);
}

// The inputs of particle b into the operand rows (epilogue warps): thread
// tid < D first computes axis tid's cell, offset and the hi/lo split of x_p;
// then every window cell is one 16-byte row.
template <int D>
__device__ __forceinline__ void cls_inputs(const DevMesh &m, const float *__restrict__ pool_f,
                                           const double *__restrict__ xp, int64_t b,
                                           uint8_t *in, int *sc0, float *soff, float *sxh,
                                           float *sxl, float *__restrict__ off_out, int tid) {
    using G = ClsGeo<D>;
    if (tid < D) {
        const double x = xp[b * D + tid];
        const float h = __double2float_rn(x);
        const float l = __double2float_rn(__dsub_rn(x, double(h)));
        int c0;
        float o;
        cell_offset(m, tid, x, h, l, c0, o);
        sc0[tid] = c0;
        soff[tid] = o;
        off_out[b * D + tid] = o;
        sxh[tid] = h;
        sxl[tid] = l;
    }
    epi_sync();
    for (int e = tid; e < G::P; e += kEpiC * 32) {
        int ek[3] = {e % G::W, (e / G::W) % G::W, D == 3 ? e / (G::W * G::W) : 0};
        bool inside = true;
        int64_t flat = 0;
        int cc[3];
        #pragma unroll
        for (int k = 0; k < D; ++k) {
            cc[k] = sc0[k] - G::W / 2 + ek[k];
            inside &= cc[k] >= 0 && cc[k] < m.ga[k];
        }
        #pragma unroll
        for (int k = D - 1; k >= 0; --k) flat = flat * m.ga[k] + (inside ? cc[k] : 0);
        float v[3] = {0.f, 0.f, 0.f};
        bool has = false;
        float ph[3], pl[3];
        if (inside) {
            #pragma unroll
            for (int k = 0; k < D; ++k) {
                ph[k] = __ldg(pool_f + flat * 2 * D + 2 * k);
                pl[k] = __ldg(pool_f + flat * 2 * D + 2 * k + 1);
            }
            has = !isnan(ph[0]);
        }
        #pragma unroll
        for (int k = 0; k < D; ++k) {
            const float inv = m.inv_sa[k];
            v[k] = has ? __fmul_rn(__fadd_rn(__fsub_rn(ph[k], sxh[k]), __fsub_rn(pl[k], sxl[k])), inv)
                       : __fsub_rn(float(ek[k] - G::W / 2), soff[k]);
        }
        const int q = D == 2 ? (ek[1] + 1) * G::E + ek[0] + 1
                             : ((ek[2] + 1) * G::E + ek[1] + 1) * G::E + ek[0] + 1;
        *reinterpret_cast<uint4 *>(in + 16 * q) =
            make_uint4(pack_bf16x2(v[0], v[1]), pack_bf16x2(v[2], 0.f), 0u, 0u);
    }
}

template <int D>
__global__ void __launch_bounds__(kThreadsC, D == 2 ? 4 : 1) cls_conv_tc_kernel(
    const DevMesh m, const float *__restrict__ pool_f, int64_t B, const double *__restrict__ xp,
    const uint8_t *__restrict__ packed, float *__restrict__ cat, int64_t ldc,
    float *__restrict__ off_out, int *err) {
    using G = ClsGeo<D>;
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t *in = smem + G::kSmIn;
    uint8_t *act = smem + G::kSmAct;
    uint8_t *wsm = smem + G::kSmW;
    float *stage = reinterpret_cast<float *>(smem + G::kSmStage);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + G::kSmBar);   // conv1, conv2, final
    uint32_t *in_ready = reinterpret_cast<uint32_t *>(smem + G::kSmCnt);
    uint32_t *act_ready = in_ready + 1;
    int *sc0 = reinterpret_cast<int *>(smem + G::kSmPart);
    float *soff = reinterpret_cast<float *>(smem + G::kSmPart) + 3;
    float *sxh = soff + 3, *sxl = soff + 6;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + G::kSmSlot);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + G::kSmSlot + 4);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    // operands zero (ring, padding channels, rows past the window), barriers, TMEM
    for (int i = tid; i < G::kSmW / 16; i += kThreadsC)
        reinterpret_cast<uint4 *>(smem)[i] = make_uint4(0, 0, 0, 0);
    if (tid == 0) {
        for (int i = 0; i < 3; ++i) mbar_init(bars + i, 1u);
        *in_ready = 0;
        *act_ready = 0;
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_addr(tmem_slot)),
                     "r"(G::Cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    for (int i = tid; i < G::kPacked / 16; i += kThreadsC) cp_async16(wsm + 16 * i, packed + 16 * i);
    cp_async_wait_all();
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_slot;
    const int64_t n_mine = B > blockIdx.x ? (B - 1 - blockIdx.x) / gridDim.x + 1 : 0;

    if (warp == kMmaC) {
        const bool leader = elect_one();
        const uint64_t d_in = sdesc(smem_addr(in), 16, 128);
        const uint64_t d_act = sdesc(smem_addr(act), G::Rows * 16, 128);
        const uint64_t d_w1 = sdesc(smem_addr(wsm + G::kW1), 32 * 16, 128);
        const uint64_t d_w2 = sdesc(smem_addr(wsm + G::kW2), 32 * 16, 128);
        constexpr uint32_t id32 = idesc_bf16(128, 32);
        for (int64_t k = 0; k < n_mine; ++k) {
            // conv1 of particle k, once its inputs are in place
            if (!wait_count(in_ready, uint32_t(k + 1), abort_flag, err)) break;
            fence_after();
            if (leader) {
                for (int mt = 0; mt < G::MT; ++mt) {
                    const uint32_t dcol = tmem + uint32_t(32 * mt);
                    const int r0 = 128 * mt;
                    #pragma unroll
                    for (int i = 0; i < G::Pairs; ++i) {
                        const int t0 = 2 * i, t1 = 2 * i + 1 < G::Taps ? 2 * i + 1 : 2 * i;
                        const int sh0 = cls_shift<D>(t0), sh1 = cls_shift<D>(t1);
                        const uint64_t a = (d_in & ~(uint64_t(0x3fff) << 16)) + uint64_t(r0 + sh0) +
                                           (uint64_t(sh1 - sh0 > 0 ? sh1 - sh0 : 1) << 16);
                        mma_bf16(dcol, a, d_w1 + uint64_t(i * 64), id32, i > 0 ? 1u : 0u);
                    }
                }
                mma_commit(bars + 0);
            }
            __syncwarp();
            // conv2 of particle k, once conv1's activations are in place
            if (!wait_count(act_ready, uint32_t(k + 1), abort_flag, err)) break;
            fence_after();
            if (leader) {
                for (int mt = 0; mt < G::MT; ++mt) {
                    const uint32_t dcol = tmem + uint32_t(32 * (G::MT + mt));
                    const int r0 = 128 * mt;
                    #pragma unroll 3
                    for (int t = 0; t < G::Taps; ++t) {
                        const int sh = cls_shift<D>(t);
                        #pragma unroll
                        for (int kk = 0; kk < 2; ++kk) {
                            const uint64_t a = d_act + uint64_t(2 * kk * G::Rows + r0 + sh);
                            const uint64_t bw = d_w2 + uint64_t((t * 4 + 2 * kk) * 32);
                            mma_bf16(dcol, a, bw, id32, (t | kk) != 0 ? 1u : 0u);
                        }
                    }
                }
                mma_commit(bars + 1);
            }
            __syncwarp();
        }
    } else {
        const float *b1 = reinterpret_cast<const float *>(wsm + G::kB1);
        const float *b2 = reinterpret_cast<const float *>(wsm + G::kB2);
        const uint32_t tq = tmem + (uint32_t(32 * warp) << 16);
        bool ok = true;
        if (n_mine > 0) {
            cls_inputs<D>(m, pool_f, xp, blockIdx.x, in, sc0, soff, sxh, sxl, off_out, tid);
            fence_async_smem();
            epi_sync();
            if (tid == 0) red_release_add(in_ready, 1u);
        }
        for (int64_t k = 0; k < n_mine && ok; ++k) {
            const int64_t b = blockIdx.x + k * gridDim.x;
            const uint32_t par = uint32_t(k & 1);
            // ---- conv1 epilogue: ReLU(z + b1) in BF16 at each valid row's window position ----
            ok = __all_sync(kFull, mbar_wait(bars + 0, par, abort_flag, err)) != 0;
            if (epi_or(!ok)) break;
            fence_after();
            for (int mt = 0; mt < G::MT; ++mt) {
                float v[32];
                tmem_ld32(tq + uint32_t(32 * mt), v);
                uint32_t hv[16];
                bias_relu_bf16(v, b1, hv);
                const int r = 128 * mt + 32 * warp + lane;
                const int x = r % G::E, y = (r / G::E) % G::E, z = D == 3 ? r / (G::E * G::E) : 0;
                if (r < G::Ro && x < G::W && y < G::W && z < G::W)
                    store_act<G::Rows>(act, r + G::Coff, hv);
            }
            fence_before();
            fence_async_smem();
            epi_sync();
            if (tid == 0) red_release_add(act_ready, 1u);
            // ---- inputs of the next particle (its conv1 read of `in` is over) ----
            if (k + 1 < n_mine) {
                cls_inputs<D>(m, pool_f, xp, b + gridDim.x, in, sc0, soff, sxh, sxl, off_out, tid);
                fence_async_smem();
                epi_sync();
                if (tid == 0) red_release_add(in_ready, 1u);
            }
            // ---- conv2 epilogue: ReLU(z + b2) in FP32 to the stage, then pooling ----
            ok = __all_sync(kFull, mbar_wait(bars + 1, par, abort_flag, err)) != 0;
            if (epi_or(!ok)) break;
            fence_after();
            for (int mt = 0; mt < G::MT; ++mt) {
                float v[32];
                tmem_ld32(tq + uint32_t(32 * (G::MT + mt)), v);
                const int r = 128 * mt + 32 * warp + lane;
                if (r < G::Ro) {
                    #pragma unroll
                    for (int c = 0; c < 32; ++c) stage[r * G::Ld + c] = fmaxf(v[c] + b2[c], 0.f);
                }
            }
            fence_before();
            epi_sync();
            for (int i = tid; i < 32 * G::Pp; i += kEpiC * 32) {
                const int c = i % 32, pp = i / 32;
                const int px = pp % G::Wp, py = (pp / G::Wp) % G::Wp, pz = D == 3 ? pp / (G::Wp * G::Wp) : 0;
                float s = 0.f;
                for (int oz = 0; oz < (D == 3 ? 2 : 1); ++oz)
                    for (int oy = 0; oy < 2; ++oy)
                        for (int ox = 0; ox < 2; ++ox) {
                            const int r = D == 2 ? (2 * py + oy) * G::E + 2 * px + ox
                                                 : ((2 * pz + oz) * G::E + 2 * py + oy) * G::E + 2 * px + ox;
                            s += stage[r * G::Ld + c];
                        }
                cat[b * ldc + int64_t(c) * G::Pp + pp] = s / float(1 << D);
            }
            epi_sync();
        }
    }
    // wait (bounded) for this CTA's MMAs in flight before TMEM is released
    if (warp == kMmaC) {
        if (elect_one()) {
            mma_commit(bars + 2);
            for (uint32_t i = 0; i < (1u << 24) && !mbar_try_wait(bars + 2, 0); ++i)
                if (i > 64) __nanosleep(64);
        }
        __syncwarp();
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(G::Cols));
}

// conv1 W[o][i][t] (i < D) -> [pair p][half h][o][8] (tap 2p + h, channel j;
// zero for j >= D and past the last tap); conv2 W[o][i][t] -> [t][q][o][8]
// with i = 8 q + j; biases as FP32.
template <int D>
__global__ void cls_pack_kernel(const float *__restrict__ w, int64_t off_w1, int64_t off_b1,
                                int64_t off_w2, int64_t off_b2, uint8_t *__restrict__ out) {
    using G = ClsGeo<D>;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
    __nv_bfloat16 *w1 = reinterpret_cast<__nv_bfloat16 *>(out + G::kW1);
    for (int e = tid; e < G::Pairs * 2 * 32 * 8; e += nth) {
        const int j = e % 8, o = (e / 8) % 32, h = (e / 256) % 2, p = e / 512;
        const int t = 2 * p + h;
        w1[e] = __float2bfloat16_rn(t < G::Taps && j < D ? w[off_w1 + (o * D + j) * G::Taps + t] : 0.f);
    }
    __nv_bfloat16 *w2 = reinterpret_cast<__nv_bfloat16 *>(out + G::kW2);
    for (int e = tid; e < G::Taps * 32 * 32; e += nth) {
        const int t = e / 1024, o = (e / 32) % 32, i = e % 32;
        w2[((t * 4 + i / 8) * 32 + o) * 8 + i % 8] =
            __float2bfloat16_rn(w[off_w2 + (o * 32 + i) * G::Taps + t]);
    }
    for (int i = tid; i < 32; i += nth) {
        reinterpret_cast<float *>(out + G::kB1)[i] = w[off_b1 + i];
        reinterpret_cast<float *>(out + G::kB2)[i] = w[off_b2 + i];
    }
}

template <int D>
void launch_conv(const DevMesh &m, const float *pool_f, int64_t B, const double *xp,
                 const uint8_t *packed, float *cat, int64_t ldc, float *off, int *err,
                 int sm_count, cudaStream_t st) {
    using G = ClsGeo<D>;
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(cls_conv_tc_kernel<D>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             G::kSmTotal);
        attr = true;
    }
    const int per_sm = D == 2 ? 4 : 1;
    const int grid = int(std::min<int64_t>(B, int64_t(sm_count) * per_sm));
    cls_conv_tc_kernel<D><<<grid, kThreadsC, G::kSmTotal, st>>>(m, pool_f, B, xp, packed, cat, ldc,
                                                                off, err);
}

}  // namespace

int64_t cls_packed_bytes(int dim) { return dim == 2 ? ClsGeo<2>::kPacked : ClsGeo<3>::kPacked; }

void launch_cls_pack(int dim, const float *w, int64_t off_w1, int64_t off_b1, int64_t off_w2,
                     int64_t off_b2, uint8_t *packed, cudaStream_t st) {
    if (dim == 2)
        cls_pack_kernel<2><<<32, 256, 0, st>>>(w, off_w1, off_b1, off_w2, off_b2, packed);
    else
        cls_pack_kernel<3><<<64, 256, 0, st>>>(w, off_w1, off_b1, off_w2, off_b2, packed);
}

void launch_cls_conv_tc(const DevMesh &m, const float *pool_f, int64_t B, const double *xp,
                        const uint8_t *packed, float *cat, int64_t ldc, float *off, int *err,
                        int sm_count, cudaStream_t st) {
    if (B <= 0) return;
    if (m.dim == 2)
        launch_conv<2>(m, pool_f, B, xp, packed, cat, ldc, off, err, sm_count, st);
    else
        launch_conv<3>(m, pool_f, B, xp, packed, cat, ldc, off, err, sm_count, st);
}

}  // namespace cs
