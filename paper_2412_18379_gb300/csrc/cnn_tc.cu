// Grid inference of the 2-D start predictor on the tensor cores (tcgen05).
//
// The predictor maps the 9x9 window of the ASG-grid velocity around a cell to
// the cell's displacement (Sec. 2.3, Algorithm 2). Windows of neighbouring
// cells overlap, so the network is evaluated for all cells at once: with
// valid convolutions, the window result at cell c equals a fully
// convolutional pass over the zero-padded grid, read at c. One persistent CTA
// per SM walks over output tiles of 24 columns x TH rows (TH = 24, 13 or 8:
// the host picks the height whose tiles fill the SMs best, e.g. 13 rows for
// 144 tiles on a 200 x 200 grid):
//
//   input   32 x (TH + 8) cells (tile + 4-cell halo), channels u_k dt / s_k, BF16,
//           tap-packed: row r holds both channels of taps 0..7 at pixel r
//   conv1   tcgen05.mma kind::f16, M = 128 pixels, N = 32: one K = 16 step
//           for taps 0..7, one for tap 8 (a shifted read of the same rows)
//   conv2-4 tcgen05.mma, implicit GEMM: M = 128 pixels, N = 32 channels,
//           K = 16 channels of one tap; 9 taps x 2 K-steps per M-tile
//   fc1     tcgen05.mma, M = 128 pixels, N = 128 (two halves of 256), K = 32
//   fc2     CUDA cores in the fc1 epilogue (256 -> 2)
//   (FP32 accumulators in TMEM; bias + ReLU + BF16 in the epilogues)
//
// Activations live in shared memory as [8-channel chunk q][pixel r][8] BF16,
// with pixels on a flat 32-wide row-major index for every layer (columns past
// the valid width hold garbage that only ever feeds garbage outputs). A tap
// (dy, dx) is then a shift of dy*32 + dx pixels, i.e. an offset of the MMA's
// shared-memory descriptor: no im2col copy. The canonical no-swizzle K-major
// layout has 8x16-byte core matrices, SBO = 128 B between 8-pixel groups and
// LBO = 16 KiB between channel chunks. An MMA of N = 32 is bound by reading
// its operands from shared memory (about 4 KiB of A per step), not by the
// tensor cores' arithmetic.
//
// Pipeline. A tile is a sequence of items (layer, M-tile); with TH = 24 there
// are 38: conv1 8, conv2 7, conv3 7, conv4 6, fc1 5 x 2 column halves (TH =
// 13: 5, 5, 4, 4, 3 x 2). Warp 16 issues the conv MMAs
// and warp 18 the fc1 MMAs, each committing an item's MMAs to the item's
// "mma" mbarrier. The 16 epilogue warps form 4 groups (one warp per TMEM lane
// quarter): groups 0-1 take the conv items, groups 2-3 the fc1 items; a group
// waits for the item's MMAs, runs the epilogue and counts it in the item's
// shared-memory counter (release). Warp 19 waits for each conv item's
// counters and releases the item to warp 16 through a named barrier, so the
// issuing warp never loads from shared memory (such a load waits behind the
// MMAs it has queued, and the tensor pipe drains). Warp 17 loads the next
// tile's input while conv2..conv4 of the current one run.
// The MMAs of item (l, m) wait only for the epilogues they read (items
// (l-1, m) and (l-1, m+1)) and for the last user of their TMEM columns, so
// the tensor cores run ahead of the epilogues instead of waiting for a whole
// layer. The conv layers share TMEM columns [0, 256) (M-tile m at 32 m) and
// fc1 owns [256, 512), so fc1 of one tile overlaps the convolutions of the
// next. conv1..conv3 write their output over their input, in place: the rows
// of M-tile m are read only by the MMAs of M-tiles m-1 and m, and both have
// completed when the epilogue of m starts; conv4 writes the compacted fc1
// input, a buffer of its own. The "mma" barrier sets alternate between even
// and odd tiles, so a parity wait never sees a phase two tiles old; the
// epilogue counters only grow.
#include <cuda_bf16.h>

#include <cstdint>

#include "cnn.h"
#include "tc_common.cuh"

namespace cs {
namespace {

constexpr int kTileW = 24;           // output cells per tile row
constexpr int kW = 32;               // flat row width (= tile width + 8)
constexpr int kEpiWarps = 16;        // 4 groups x 4 TMEM lane quarters
constexpr int kConvWarp = 16;        // issues the MMAs of conv1..conv4
constexpr int kLoadWarp = 17;        // loads the tile inputs
constexpr int kFcWarp = 18;          // issues the MMAs of fc1
constexpr int kSchedWarp = 19;       // releases the conv items to the conv warp
constexpr int kThreadsTC = 20 * 32;
static_assert(kEpiWarps == kConvWarp && kLoadWarp == kConvWarp + 1 && kFcWarp == kConvWarp + 2 &&
                  kSchedWarp == kConvWarp + 3,
              "warp roles");
constexpr uint32_t kTmemCols = 512;

// packed weights (bytes); produced by pack_weights_kernel
struct TcLayout {
    static constexpr int w1 = 0;                          // bf16 [2 MMAs][2 chunks][32][8]
    static constexpr int b1 = w1 + 2 * 2 * 32 * 8 * 2;    // fp32 [32]
    static constexpr int bconv = b1 + 32 * 4;             // 3 x bf16 [9][4][32][8]
    static constexpr int bconv_bytes = 9 * 4 * 32 * 8 * 2;
    static constexpr int cb = bconv + 3 * bconv_bytes;    // fp32 [3][32] conv biases
    static constexpr int bfc1 = cb + 3 * 32 * 4;          // bf16 [4][256][8]
    static constexpr int bfc1_bytes = 4 * 256 * 8 * 2;
    static constexpr int fc1b = bfc1 + bfc1_bytes;        // fp32 [256], negated fc1 bias
    static constexpr int fc2w = fc1b + 256 * 4;           // fp32 [2][256]
    static constexpr int fc2b = fc2w + 2 * 256 * 4;       // fp32 [2], fc2 bias + W2 b1
    static constexpr int total = ((fc2b + 2 * 4) + 127) / 128 * 128;
};

// Geometry of a tile of kTileW x TH output cells. The input is TH + 8 rows
// of 32 cells (a 4-cell halo); conv1..conv4 produce TH + 6, + 4, + 2 and TH
// valid rows, each computed in M-tiles of 128 flat pixels (4 rows of 32).
// A tall tile (TH = 24) wastes the least on halos; shorter ones give more
// tiles, so that small grids still occupy every SM (the host picks TH).
template <int TH>
struct Geo {
    static_assert(TH >= 4 && TH <= 26, "tile height");
    static constexpr int kInRows = TH + 8;
    // M-tiles of conv layer l = 0..3
    __host__ __device__ static constexpr int nmt(int l) { return (TH + 6 - 2 * l + 3) / 4; }
    // first item of conv1..conv4 (l = 0..3) and fc1 (l = 4)
    __host__ __device__ static constexpr int jbase(int l) { return l == 0 ? 0 : jbase(l - 1) + nmt(l - 1); }
    static constexpr int kRowsFc = kTileW * TH;           // compacted conv4 output rows
    static constexpr int kFcTiles = (kRowsFc + 127) / 128;
    static constexpr int kItems = jbase(4) + 2 * kFcTiles;
    static constexpr int kRows = 128 * nmt(0);            // rows per chunk of the conv buffer
    // conv1 reads 128 nmt(0) rows plus the tap-8 shift of 66
    static constexpr int kRowsX0 = (128 * nmt(0) + 2 * kW + 2 + 7) / 8 * 8;
    static constexpr int kWinRows = kInRows + 6;          // window rows + zero rows
    // conv layer whose M-tile mt is the last in a tile to use the TMEM
    // columns [32 mt, +32): the next tile's conv1 M-tile mt waits for it
    __host__ __device__ static constexpr int last_user(int mt) {
        return nmt(3) > mt ? 3 : nmt(2) > mt ? 2 : nmt(1) > mt ? 1 : 0;
    }
    // conv4 M-tiles whose compacted rows [96 m, 96 m + 96) feed fc1 M-tile f,
    // i.e. rows [128 f, 128 f + 128): m in [fc_lo(f), fc_hi(f)]
    __host__ __device__ static constexpr int fc_lo(int f) { return (128 * f) / 96; }
    __host__ __device__ static constexpr int fc_hi(int f) {
        return (128 * f + 127) / 96 < nmt(3) - 1 ? (128 * f + 127) / 96 : nmt(3) - 1;
    }

    // shared memory map (bytes)
    static constexpr int kX0Bytes = 2 * kRowsX0 * 16;     // bf16 [2][kRowsX0][8] tap-packed input
    static constexpr int kSmX0 = 0;                       // input buffer
    static constexpr int kSmAct = kSmX0 + kX0Bytes;       // bf16 [4][kRows][8] conv1..conv3
    static constexpr int kSmFc = kSmAct + 4 * kRows * 16; // bf16 [4][kRowsFc][8] conv4 -> fc1
    static constexpr int kSmW = kSmFc + 4 * kRowsFc * 16; // packed weights
    static constexpr int kSmRed = kSmW + TcLayout::total; // float2 [2][kFcTiles][128] fc2 partials
    static constexpr int kSmBar = kSmRed + 2 * kFcTiles * 128 * 8;
    static constexpr int kBarMma = 0;                     // [2][kItems]
    static constexpr int kBarEmpty = 2 * kItems;          // input buffer consumed by conv1
    static constexpr int kBarFinal = kBarEmpty + 1;       // [2] each issuing warp's last MMAs
    static constexpr int kNumBars = kBarFinal + 2;
    static constexpr int kSmWin = kSmBar + kNumBars * 8;  // u32 [kWinRows][32] input window
    static constexpr int kSmCnt = kSmWin + kWinRows * kW * 4;   // u32 counters
    static constexpr int kCntX0 = kItems;                 // counter: tile inputs loaded
    static constexpr int kCntT4 = kItems + 1;             // [nmt(3)] conv4 M-tile read out of TMEM
    static constexpr int kNumCnt = kCntT4 + nmt(3);
    static constexpr int kSmSlot = kSmCnt + kNumCnt * 4;  // TMEM address, abort flag
    static constexpr int kSmTotal = kSmSlot + 16;

    static_assert(kSmTotal <= 232448, "shared memory of one CTA");
    static_assert(32 * nmt(0) <= 256, "conv layers fit TMEM columns [0, 256)");
    static_assert(nmt(0) - nmt(1) <= 1 && nmt(1) - nmt(2) <= 1 && nmt(2) - nmt(3) <= 1,
                  "each conv M-tile depends on M-tiles mt and mt + 1 of the layer before");
    // fc1 M-tile f reads rows [128 f, +128) of each chunk: past kRowsFc it reads
    // the next chunk (or, for the last chunk, the weights that follow), garbage
    // rows whose outputs are dropped
    static_assert(kSmFc + (3 * kRowsFc + 128 * kFcTiles) * 16 <= kSmTotal, "fc1 reads in bounds");
    // conv2..conv4 M-tile mt reads rows up to 128 mt + 127 + 66 of each chunk
    static_assert(kSmAct + (3 * kRows + 128 * nmt(1) + 2 * kW + 2) * 16 <= kSmTotal,
                  "conv reads in bounds");
    static_assert(kRowsX0 >= 128 * nmt(0) + 2 * kW + 2, "conv1 reads in bounds");
    static_assert(kRowsX0 - 1 + 2 * kW + 1 < kWinRows * kW, "window reads in bounds");
    static_assert(kSmBar % 8 == 0, "mbarrier alignment");
    static_assert(96 * nmt(3) <= 128 * kFcTiles + 96, "conv4 M-tiles map onto fc1 M-tiles");

    static __device__ __forceinline__ void item_decode(int j, int &l, int &m) {
        l = j < jbase(1) ? 0 : j < jbase(2) ? 1 : j < jbase(3) ? 2 : j < jbase(4) ? 3 : 4;
        m = j - jbase(l);
    }
};
static_assert(Geo<24>::kItems == 38 && Geo<24>::jbase(4) == 28 && Geo<24>::kFcTiles == 5,
              "24-row tile: 38 items");
static_assert(Geo<24>::last_user(5) == 3 && Geo<24>::last_user(6) == 2 &&
                  Geo<24>::last_user(7) == 0,
              "24-row tile: TMEM column reuse");

// Named barrier 1 between the conv warp and the scheduler warp (64 threads),
// with an OR over both warps' flags: both get the same answer.
__device__ __forceinline__ bool handoff_or(bool flag) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 q, %1, 0;\n\t"
        "bar.red.or.pred p, 1, 64, q;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(r)
        : "r"(uint32_t(flag))
        : "memory");
    return r != 0;
}

// Named barrier 2 over the 16 epilogue warps (warps 0..15)
__device__ __forceinline__ void epi_bar_sync() {
    asm volatile("bar.sync 2, %0;" ::"n"(kEpiWarps * 32) : "memory");
}

// TMEM columns of an item: every conv layer uses [32 m, +32) for M-tile m
// (so conv M-tile m of layer l reuses the columns of layer l - 1, whose
// epilogue it waits for anyway); fc1 column half h uses [256 + 128 h, +128).
__device__ __forceinline__ uint32_t item_col(int l, int m) {
    return l < 4 ? uint32_t(32 * m) : uint32_t(256 + 128 * (m & 1));
}

// MMAs of M-tile m of conv layer l (l >= 1): 9 taps x 2 K-steps, accumulate
// into TMEM columns [col, col + 32). kRows: rows per chunk of the conv buffer.
template <int kRows>
__device__ __forceinline__ void issue_conv(uint32_t dcol, uint64_t adesc, uint64_t bdesc, int m) {
    constexpr uint32_t id = idesc_bf16(128, 32);
    #pragma unroll
    for (int t = 0; t < 9; ++t) {
        const int shift = (t / 3) * kW + (t % 3);
        #pragma unroll
        for (int kk = 0; kk < 2; ++kk) {
            // offsets in 16-byte units: A chunk pair kk, pixel row 128 m + shift;
            // B tap t, chunk pair kk (32 rows of 16 B per chunk)
            const uint64_t a = adesc + uint64_t(2 * kk * kRows + 128 * m + shift);
            const uint64_t b = bdesc + uint64_t((t * 4 + 2 * kk) * 32);
            mma_bf16(dcol, a, b, id, (t | kk) != 0 ? 1u : 0u);
        }
    }
}

// MMAs of M-tile m of conv1 on the tap-packed input: row r holds, in K order,
// channels (u0, u1) of taps 0..7 at pixel r (shifts 0, 1, 2, 32, 33, 34, 64,
// 65). One K = 16 step covers taps 0..7; a second reads the rows 66 pixels
// further on, whose first tap is tap 8 of pixel r, against weights that are
// zero past K = 2.
__device__ __forceinline__ void issue_conv1(uint32_t dcol, uint64_t adesc, uint64_t bdesc, int m) {
    constexpr uint32_t id = idesc_bf16(128, 32);
    mma_bf16(dcol, adesc + uint64_t(128 * m), bdesc, id, 0u);
    mma_bf16(dcol, adesc + uint64_t(128 * m + 2 * kW + 2), bdesc + uint64_t(2 * 32), id, 1u);
}

// MMAs of column half h of fc1 M-tile f: 128 compacted pixels x 128 features,
// K = 32 in two steps. kRowsFc: rows per chunk of the fc1 input.
template <int kRowsFc>
__device__ __forceinline__ void issue_fc1(uint32_t dcol, uint64_t adesc, uint64_t bdesc, int f,
                                          int h) {
    constexpr uint32_t id = idesc_bf16(128, 128);
    #pragma unroll
    for (int kk = 0; kk < 2; ++kk)
        mma_bf16(dcol, adesc + uint64_t(2 * kk * kRowsFc + 128 * f),
                 bdesc + uint64_t(2 * kk * 256 + 128 * h), id, uint32_t(kk));
}

template <int TH>
__global__ void __launch_bounds__(kThreadsTC, 1) cnn2d_tc_kernel(
    const DevMesh m, const TcSource src, float scale0, float scale1,
    const uint8_t *__restrict__ packed, float *__restrict__ dhat, int *err, TcHold hold) {
    using G = Geo<TH>;
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t *x0 = smem + G::kSmX0;
    uint8_t *act = smem + G::kSmAct;
    uint8_t *fcin = smem + G::kSmFc;
    uint8_t *wsm = smem + G::kSmW;
    float2 *red = reinterpret_cast<float2 *>(smem + G::kSmRed);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + G::kSmBar);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + G::kSmSlot);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + G::kSmSlot + 4);
    // epi_cnt[j] counts the epilogues of item j finished over this CTA's tiles,
    // 4 per tile (one per lane-quarter warp): item j of local tile k is done
    // once epi_cnt[j] >= 4 (k + 1)
    uint32_t *epi_cnt = reinterpret_cast<uint32_t *>(smem + G::kSmCnt);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int gx = m.ga[0], gy = m.ga[1];
    const int tiles_x = (gx + kTileW - 1) / kTileW, tiles_y = (gy + TH - 1) / TH;
    const int n_tiles = tiles_x * tiles_y;

    // Set-up that touches no global memory runs first: it may overlap the end
    // of the previous kernel on the stream (programmatic dependent launch)
    // until pdl_wait() below. The conv and fc1 buffers and the window's zero
    // rows are cleared; the input buffer needs no clearing, since the
    // tap-packed rows overwrite all of it for every tile.
    for (int i = G::kSmAct / 16 + tid; i < G::kSmW / 16; i += kThreadsTC)
        reinterpret_cast<uint4 *>(smem)[i] = make_uint4(0, 0, 0, 0);
    for (int i = G::kInRows * kW + tid; i < G::kWinRows * kW; i += kThreadsTC)
        reinterpret_cast<uint32_t *>(smem + G::kSmWin)[i] = 0u;
    if (tid == 0) {
        for (int i = 0; i < G::kNumBars; ++i) mbar_init(bars + i, 1u);
        for (int i = 0; i < G::kNumCnt; ++i) epi_cnt[i] = 0;
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_addr(tmem_slot)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    // Then, once the previous kernel's writes are visible, the first tile's
    // velocity window (the 16 epilogue warps, idle until the first MMAs
    // complete, pack it after the barrier below) and the weights (once per
    // CTA), by asynchronous copies.
    pdl_wait();
    float2 *stage = reinterpret_cast<float2 *>(x0);   // staging, until tap-packed
    static_assert(G::kInRows * kW * 8 <= G::kX0Bytes, "staging fits the input buffer");
    const float2 *U2 = reinterpret_cast<const float2 *>(src.U);
    if (warp < kEpiWarps) {
        const int cx0 = (blockIdx.x % tiles_x) * kTileW - 4, cy0 = (blockIdx.x / tiles_x) * TH - 4;
        if (src.node) {
            // the resample fused: every cell of this thread first loads its
            // table entries, then its nodal velocities, then interpolates (two
            // rounds of loads in flight, not two per cell); the tile's own
            // cells are kept as the mesh's grid velocity
            constexpr int kCells = G::kInRows * kW, kPer = (kCells + kEpiWarps * 32 - 1) / (kEpiWarps * 32);
            int32_t nd[kPer][3];
            float wt[kPer][3];
            int64_t cc[kPer];
            #pragma unroll
            for (int j = 0; j < kPer; ++j) {
                const int i = tid + j * kEpiWarps * 32;
                const int cx = cx0 + i % kW, cy = cy0 + i / kW;
                const bool in = i < kCells && cx >= 0 && cx < gx && cy >= 0 && cy < gy;
                cc[j] = in ? int64_t(cy) * gx + cx : -1;
                #pragma unroll
                for (int q = 0; q < 3; ++q) {
                    nd[j][q] = in ? __ldg(src.node + cc[j] * 3 + q) : -1;
                    wt[j][q] = in ? __ldg(src.w + cc[j] * 3 + q) : 0.f;
                }
            }
            double un[kPer][3][2];
            #pragma unroll
            for (int j = 0; j < kPer; ++j)
                #pragma unroll
                for (int q = 0; q < 3; ++q)
                    #pragma unroll
                    for (int k = 0; k < 2; ++k)
                        un[j][q][k] = nd[j][0] >= 0 ? __ldg(src.un + int64_t(nd[j][q]) * 2 + k) : 0.0;
            #pragma unroll
            for (int j = 0; j < kPer; ++j) {
                const int i = tid + j * kEpiWarps * 32;
                if (i >= kCells) break;
                // the resample kernel's arithmetic, in its order
                float v0 = 0.f, v1 = 0.f;
                if (nd[j][0] >= 0) {
                    #pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        v0 = fmaf(wt[j][q], trunc_to_float(un[j][q][0]), v0);
                        v1 = fmaf(wt[j][q], trunc_to_float(un[j][q][1]), v1);
                    }
                }
                stage[i] = make_float2(v0, v1);
                const int ix = i % kW, iy = i / kW;
                if (cc[j] >= 0 && ix >= 4 && ix < 4 + kTileW && iy >= 4 && iy < 4 + TH)
                    reinterpret_cast<float2 *>(src.U_out)[cc[j]] = make_float2(v0, v1);
            }
        } else {
            for (int i = tid; i < G::kInRows * kW; i += kEpiWarps * 32) {
                const int cx = cx0 + i % kW, cy = cy0 + i / kW;
                const bool in = cx >= 0 && cx < gx && cy >= 0 && cy < gy;
                cp_async8_zfill(stage + i, in ? U2 + int64_t(cy) * gx + cx : U2, in);
            }
        }
    }
    for (int i = tid; i < TcLayout::total / 16; i += kThreadsTC)
        cp_async16(wsm + 16 * i, packed + 16 * i);
    cp_async_wait_all();
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_slot;
    uint64_t *bar_mma = bars + G::kBarMma;

    if (warp == kLoadWarp) {
        // ---- inputs: 32 x (TH + 8) cells, channels u_k dt / s_k (BF16), zero outside.
        //      One buffer: tile k + 1 is loaded while conv2..conv4 of tile k run
        //      (the epilogue warps load the first tile) ----
        for (int k = 1;; ++k) {
            const int tile = blockIdx.x + k * gridDim.x;
            if (tile >= n_tiles) break;
            if (k >= 1 &&
                !warp_wait(bars + G::kBarEmpty, uint32_t(k - 1) & 1u, abort_flag, err))
                break;
            const int tx = tile % tiles_x, ty = tile / tiles_x;
            const int cx0 = tx * kTileW - 4, cy0 = ty * TH - 4;
            // the 32 x (TH + 8) window of velocities, zero outside the grid, in
            // one round of asynchronous copies staged in the input buffer (free
            // until the tap-packed rows below overwrite it); then scaled, as
            // BF16 pairs, into the window, whose rows past it stay zero
            for (int y = 0; y < G::kInRows; ++y) {
                const int cx = cx0 + lane, cy = cy0 + y;
                const bool in = cx >= 0 && cx < gx && cy >= 0 && cy < gy;
                if (src.node) {
                    float v[2] = {0.f, 0.f};
                    if (in) interp_cell<2>(src.node, src.w, src.un, int64_t(cy) * gx + cx, v);
                    stage[y * kW + lane] = make_float2(v[0], v[1]);
                    if (in && lane >= 4 && lane < 4 + kTileW && y >= 4 && y < 4 + TH)
                        reinterpret_cast<float2 *>(src.U_out)[int64_t(cy) * gx + cx] =
                            make_float2(v[0], v[1]);
                } else {
                    cp_async8_zfill(stage + y * kW + lane, in ? U2 + int64_t(cy) * gx + cx : U2, in);
                }
            }
            cp_async_wait_all();
            uint32_t *win = reinterpret_cast<uint32_t *>(smem + G::kSmWin);
            for (int y = 0; y < G::kInRows; ++y) {
                const float2 uv = stage[y * kW + lane];
                win[y * kW + lane] = pack_bf16x2(uv.x * scale0, uv.y * scale1);
            }
            __syncwarp();
            // tap-packed rows: taps 0..7 of pixel r are pixels r + 32 dy + dx
            uint4 *xv = reinterpret_cast<uint4 *>(x0);
            #pragma unroll 2
            for (int r = lane; r < G::kRowsX0; r += kW) {
                const uint32_t *p = win + r;
                xv[r] = make_uint4(p[0], p[1], p[2], p[kW]);
                xv[G::kRowsX0 + r] = make_uint4(p[kW + 1], p[kW + 2], p[2 * kW], p[2 * kW + 1]);
            }
            __syncwarp();
            fence_async_smem();
            __syncwarp();
            if (lane == 0) red_release_add(epi_cnt + G::kCntX0, 1u);
        }
    } else if (warp == kConvWarp) {
        // ---- conv MMAs: the whole warp runs the schedule (descriptors and
        //      waits stay warp-uniform), one elected lane issues ----
        const uint64_t d_act = sdesc(smem_addr(act), G::kRows * 16, 128);
        const uint64_t d_x0 = sdesc(smem_addr(x0), G::kRowsX0 * 16, 128);
        const uint64_t d_w1 = sdesc(smem_addr(wsm + TcLayout::w1), 32 * 16, 128);
        const uint64_t d_wc = sdesc(smem_addr(wsm + TcLayout::bconv), 32 * 16, 128);
        const bool leader = elect_one();
        // The scheduler warp waits for each item's dependencies and releases it
        // through named barrier 1: a shared-memory load issued here would wait
        // behind the MMAs this warp has queued, and the tensor pipe would drain.
        bool stop = false;
        for (int k = 0; !stop; ++k) {
            const int tile = blockIdx.x + k * gridDim.x;
            if (tile >= n_tiles) break;
            uint64_t *mma_s = bar_mma + (k & 1) * G::kItems;
            for (int c = 0; c < G::jbase(4); ++c) {
                stop = handoff_or(false);
                if (stop) break;
                int l, mt;
                G::item_decode(c, l, mt);
                fence_after();
                if (leader) {
                    if (l == 0) {
                        issue_conv1(tmem + uint32_t(32 * mt), d_x0, d_w1, mt);
                    } else {
                        const uint64_t d_w = d_wc + uint64_t((l - 1) * (TcLayout::bconv_bytes / 16));
                        issue_conv<G::kRows>(tmem + uint32_t(32 * mt), d_act, d_w, mt);
                    }
                    mma_commit(mma_s + c);
                    if (c == G::nmt(0) - 1) mma_commit(bars + G::kBarEmpty);   // input buffer free again
                }
                __syncwarp();
            }
        }
        // wait (bounded) for this warp's MMAs in flight before TMEM is released
        if (leader) {
            mma_commit(bars + G::kBarFinal);
            for (uint32_t i = 0; i < (1u << 24) && !mbar_try_wait(bars + G::kBarFinal, 0); ++i)
                if (i > 64) __nanosleep(64);
        }
        __syncwarp();
    } else if (warp == kFcWarp) {
        // ---- fc1 MMAs, half h of M-tile f into columns [256 + 128 h, +128): they
        //      run while the next tile's convolutions use columns [0, 256) ----
        const uint64_t d_fc = sdesc(smem_addr(fcin), G::kRowsFc * 16, 128);
        const uint64_t d_fc1 = sdesc(smem_addr(wsm + TcLayout::bfc1), 256 * 16, 128);
        const bool leader = elect_one();
        bool ok = true;
        for (int k = 0; ok; ++k) {
            const int tile = blockIdx.x + k * gridDim.x;
            if (tile >= n_tiles) break;
            uint64_t *mma_s = bar_mma + (k & 1) * G::kItems;
            const uint32_t done = 4u * uint32_t(k + 1);
            const uint32_t done_p = 4u * uint32_t(k);
            for (int f = 0; f < G::kFcTiles && ok; ++f) {
                for (int h = 0; h < 2 && ok; ++h) {
                    // input: the conv4 M-tiles that wrote compacted rows [128 f, +128)
                    for (int q = G::fc_lo(f); q <= G::fc_hi(f) && ok && h == 0; ++q)
                        ok = wait_count(epi_cnt + G::jbase(3) + q, done, abort_flag, err);
                    // columns: last used by M-tile f - 1 (same half) or the previous tile's M-tile 4
                    if (ok && f > 0)
                        ok = wait_count(epi_cnt + G::jbase(4) + 2 * (f - 1) + h, done, abort_flag, err);
                    else if (ok && k > 0)
                        ok = wait_count(epi_cnt + G::jbase(4) + 2 * (G::kFcTiles - 1) + h,
                                        done_p, abort_flag, err);
                    if (!ok) break;
                    fence_after();
                    if (leader) {
                        issue_fc1<G::kRowsFc>(tmem + item_col(4, h), d_fc, d_fc1, f, h);
                        mma_commit(mma_s + G::jbase(4) + 2 * f + h);
                    }
                    __syncwarp();
                }
            }
        }
        if (leader) {
            mma_commit(bars + G::kBarFinal + 1);
            for (uint32_t i = 0; i < (1u << 24) && !mbar_try_wait(bars + G::kBarFinal + 1, 0); ++i)
                if (i > 64) __nanosleep(64);
        }
        __syncwarp();
    } else if (warp == kSchedWarp) {
        // ---- releases conv item c of tile k to the conv warp once its inputs
        //      are ready: conv1 M-tile mt needs the tile's input and its TMEM
        //      columns back from the previous tile (from the last layer that
        //      has an M-tile mt: with 24-row tiles conv4 for mt <= 5, conv3
        //      for mt = 6, conv1 for mt = 7); conv2..conv4 M-tile mt needs the
        //      previous layer's M-tiles mt and mt + 1 ----
        bool ok = true, stop = false;
        // test hook: a wait for a flag that nothing sets runs out; the first
        // handoff then stops the conv warp before any MMA
        if (hold.flag) ok = __all_sync(kFull, wait_flag(hold.flag, hold.polls, abort_flag, err)) != 0;
        for (int k = 0; !stop; ++k) {
            const int tile = blockIdx.x + k * gridDim.x;
            if (tile >= n_tiles) break;
            for (int c = 0; c < G::jbase(4); ++c) {
                int l, mt;
                G::item_decode(c, l, mt);
                if (ok && l == 0) {
                    if (k > 0) {
                        const int lu = G::last_user(mt);
                        const int jl = lu == 3 ? G::kCntT4 + mt : G::jbase(lu) + mt;
                        ok = wait_count(epi_cnt + jl, 4u * uint32_t(k), abort_flag, err);
                    }
                    if (ok && mt == 0)
                        ok = wait_count(epi_cnt + G::kCntX0, uint32_t(k + 1), abort_flag, err);
                } else if (ok) {
                    const uint32_t done = 4u * uint32_t(k + 1);
                    ok = wait_count(epi_cnt + G::jbase(l - 1) + mt, done, abort_flag, err);
                    if (ok && mt + 1 < G::nmt(l - 1))
                        ok = wait_count(epi_cnt + G::jbase(l - 1) + mt + 1, done, abort_flag, err);
                }
                stop = handoff_or(!ok || *abort_flag != 0);
                if (stop) break;
            }
        }
    } else {
        // ---- epilogues: groups 0 and 1 take the conv items of the CTA's sequence
        //      alternately, groups 2 and 3 the fc1 items, so a conv epilogue never
        //      queues behind the longer fc1 epilogues of the previous tile ----
        // the first tile's input (its window copies completed before the
        // barrier above): scale and round to BF16 pairs, tap-pack, release
        {
            uint32_t *win = reinterpret_cast<uint32_t *>(smem + G::kSmWin);
            for (int i = tid; i < G::kInRows * kW; i += kEpiWarps * 32) {
                const float2 uv = stage[i];
                win[i] = pack_bf16x2(uv.x * scale0, uv.y * scale1);
            }
            epi_bar_sync();
            uint4 *xv = reinterpret_cast<uint4 *>(x0);
            for (int r = tid; r < G::kRowsX0; r += kEpiWarps * 32) {
                const uint32_t *p = win + r;
                xv[r] = make_uint4(p[0], p[1], p[2], p[kW]);
                xv[G::kRowsX0 + r] = make_uint4(p[kW + 1], p[kW + 2], p[2 * kW], p[2 * kW + 1]);
            }
            fence_async_smem();
            epi_bar_sync();
            if (tid == 0) red_release_add(epi_cnt + G::kCntX0, 1u);
        }
        const int g = warp >> 2, q = warp & 3;
        constexpr int kConvItems = G::jbase(4), kFcItems = G::kItems - G::jbase(4);
        const float *b1 = reinterpret_cast<const float *>(wsm + TcLayout::b1);
        const float *cb = reinterpret_cast<const float *>(wsm + TcLayout::cb);
        const float *fc1b = reinterpret_cast<const float *>(wsm + TcLayout::fc1b);
        const float *fc2w = reinterpret_cast<const float *>(wsm + TcLayout::fc2w);
        const float *fc2b = reinterpret_cast<const float *>(wsm + TcLayout::fc2b);
        const uint32_t tq = tmem + (uint32_t(32 * q) << 16);     // this warp's lane quarter
        for (int n = g & 1;; n += 2) {
            const int k = g < 2 ? n / kConvItems : n / kFcItems;
            const int j = g < 2 ? n - k * kConvItems : G::jbase(4) + n - k * kFcItems;
            const int tile = blockIdx.x + k * gridDim.x;
            if (tile >= n_tiles) break;
            const int s = k & 1;
            const uint32_t par = uint32_t(k >> 1) & 1u;
            if (!__all_sync(kFull, mbar_wait(bar_mma + s * G::kItems + j, par, abort_flag, err)))
                break;
            fence_after();
            int l, mt;
            G::item_decode(j, l, mt);
            if (l < 4) {
                float v[32];
                tmem_ld32(tq + item_col(l, mt), v);
                if (l == 3) {
                    // conv4's columns are free for the next tile's conv1 now
                    fence_before();
                    __syncwarp();
                    if (lane == 0) red_release_add(epi_cnt + G::kCntT4 + mt, 1u);
                }
                uint32_t hv[16];
                bias_relu_bf16(v, l == 0 ? b1 : cb + 32 * (l - 1), hv);
                const int row = 128 * mt + 32 * q + lane;
                if (l < 3) {
                    store_act<G::kRows>(act, row, hv);
                } else {
                    // conv4: pixel (y, x) -> compacted row 24 y + x of the fc1 input
                    // (rows y >= TH, columns x >= 24 are dropped),
                    // once the previous tile's fc1 M-tiles that read rows [96 mt, +96)
                    // are done (their epilogues end long before, so this is one load)
                    bool ok = true;
                    for (int f = (96 * mt) / 128;
                         f <= (96 * mt + 95) / 128 && f < G::kFcTiles && ok && k > 0; ++f)
                        ok = wait_count(epi_cnt + G::jbase(4) + 2 * f + 1, 4u * uint32_t(k), abort_flag,
                                        err);
                    if (!ok) break;
                    if (row % kW < kTileW && row / kW < TH)
                        store_act<G::kRowsFc>(fcin, (row / kW) * kTileW + row % kW, hv);
                }
            } else {
                // fc1 half h of M-tile f: 128 features, their part of fc2. With the
                // packed weights holding -b1 and the fc2 bias plus W2 b1,
                // W2 ReLU(z + b1) = W2 max(z, -b1) + W2 b1 costs one max and one
                // paired FMA per feature and output.
                const int f = mt >> 1, h = mt & 1;
                float2 a0 = make_float2(h == 0 ? fc2b[0] : 0.f, 0.f), b0 = make_float2(0.f, 0.f);
                float2 a1 = make_float2(h == 0 ? fc2b[1] : 0.f, 0.f), b1v = make_float2(0.f, 0.f);
                #pragma unroll 1
                for (int c = 0; c < 4; ++c) {
                    float v[32];
                    tmem_ld32(tq + item_col(4, h) + uint32_t(32 * c), v);   // one wait per 32 columns
                    const int n0 = 128 * h + 32 * c;
                    const float4 *pb = reinterpret_cast<const float4 *>(fc1b + n0);   // -b1
                    const float4 *p0 = reinterpret_cast<const float4 *>(fc2w + n0);
                    const float4 *p1 = reinterpret_cast<const float4 *>(fc2w + 256 + n0);
                    #pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        const float4 nb = pb[e], w0 = p0[e], w1 = p1[e];
                        const float2 h01 = make_float2(fmaxf(v[4 * e], nb.x), fmaxf(v[4 * e + 1], nb.y));
                        const float2 h23 =
                            make_float2(fmaxf(v[4 * e + 2], nb.z), fmaxf(v[4 * e + 3], nb.w));
                        a0 = __ffma2_rn(make_float2(w0.x, w0.y), h01, a0);
                        b0 = __ffma2_rn(make_float2(w0.z, w0.w), h23, b0);
                        a1 = __ffma2_rn(make_float2(w1.x, w1.y), h01, a1);
                        b1v = __ffma2_rn(make_float2(w1.z, w1.w), h23, b1v);
                    }
                }
                const float o0 = (a0.x + a0.y) + (b0.x + b0.y), o1 = (a1.x + a1.y) + (b1v.x + b1v.y);
                float2 *slot = red + (s * G::kFcTiles + f) * 128 + 32 * q + lane;
                if (h == 0) {
                    *slot = make_float2(o0, o1);
                } else {
                    // the first half (the previous item) left its partial sums in `slot`
                    if (!wait_count(epi_cnt + j - 1, 4u * uint32_t(k + 1), abort_flag, err)) break;
                    const float2 p = *slot;
                    const int row = 128 * f + 32 * q + lane;
                    const int y = row / kTileW, x = row % kTileW;
                    const int tx = tile % tiles_x, ty = tile / tiles_x;
                    const int cx = tx * kTileW + x, cy = ty * TH + y;
                    if (row < G::kRowsFc && cx < gx && cy < gy)
                        reinterpret_cast<float2 *>(dhat)[int64_t(cy) * gx + cx] =
                            make_float2(p.x + o0, p.y + o1);
                }
            }
            fence_before();
            fence_async_smem();
            __syncwarp();
            if (lane == 0) red_release_add(epi_cnt + j, 1u);
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
    // conv1 W[o][i][t] -> [mma][chunk][o][8]; K index kk = 8 chunk + j is
    // (tap kk / 2, channel kk % 2) for MMA 0 (taps 0..7), (tap 8, channel kk)
    // for kk < 2 in MMA 1 and zero past it
    __nv_bfloat16 *w1 = reinterpret_cast<__nv_bfloat16 *>(out + TcLayout::w1);
    for (int e = tid; e < 2 * 2 * 32 * 8; e += nth) {
        const int mm = e / 512, o = (e / 8) % 32, kk = 8 * ((e / 256) % 2) + e % 8;
        const int t = mm == 0 ? kk / 2 : 8, i = kk % 2;
        w1[e] = __float2bfloat16_rn(mm == 0 || kk < 2 ? w[off_w1 + (o * 2 + i) * 9 + t] : 0.f);
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
        reinterpret_cast<float *>(out + TcLayout::fc1b)[i] = -w[off_f1b + i];
        reinterpret_cast<float *>(out + TcLayout::fc2w)[i] = w[off_f2w + i];
        reinterpret_cast<float *>(out + TcLayout::fc2w)[256 + i] = w[off_f2w + 256 + i];
    }
    // fc2 bias plus W2 b1 (the epilogue evaluates W2 max(z, -b1))
    if (tid < 2) {
        double acc = w[off_f2b + tid];
        for (int n = 0; n < 256; ++n) acc += double(w[off_f2w + tid * 256 + n]) * w[off_f1b + n];
        reinterpret_cast<float *>(out + TcLayout::fc2b)[tid] = float(acc);
    }
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

namespace {

template <int TH>
int tiles_of(const DevMesh &m) {
    return ((m.ga[0] + kTileW - 1) / kTileW) * ((m.ga[1] + TH - 1) / TH);
}

// Relative cost of a grid pass with TH-row tiles: waves of one tile per SM,
// each a pipeline of Geo<TH>::kItems items plus a fixed part (weights, TMEM,
// first input) worth about 8 items.
template <int TH>
int64_t tile_cost(const DevMesh &m, int sm_count) {
    const int64_t waves = (tiles_of<TH>(m) + sm_count - 1) / sm_count;
    return waves * (Geo<TH>::kItems + 8);
}

template <int TH>
int launch_rows(const DevMesh &m, const TcSource &src, double dt, const uint8_t *packed,
                float *dhat, int *err, int sm_count, cudaStream_t st, TcHold hold) {
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(cnn2d_tc_kernel<TH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             Geo<TH>::kSmTotal);
        attr = true;
    }
    const int grid = std::min(tiles_of<TH>(m), sm_count);
    launch_pdl(cnn2d_tc_kernel<TH>, dim3(grid), dim3(kThreadsTC), size_t(Geo<TH>::kSmTotal), st, m,
               src, float(dt / m.sa[0]), float(dt / m.sa[1]), packed, dhat, err, hold);
    return 1;
}

}  // namespace

int tc_pick_tile_rows(const DevMesh &m, int sm_count) {
    const int64_t c24 = tile_cost<24>(m, sm_count), c13 = tile_cost<13>(m, sm_count),
                  c8 = tile_cost<8>(m, sm_count);
    if (c24 <= c13 && c24 <= c8) return 24;
    return c13 <= c8 ? 13 : 8;
}

int launch_cnn2d_tc(const DevMesh &m, const TcSource &src, double dt, const uint8_t *packed,
                    float *dhat, int *err, int sm_count, int tile_rows, cudaStream_t st,
                    TcHold hold) {
    const int th = tile_rows ? tile_rows : tc_pick_tile_rows(m, sm_count);
    if (th == 24) return launch_rows<24>(m, src, dt, packed, dhat, err, sm_count, st, hold);
    if (th == 13) return launch_rows<13>(m, src, dt, packed, dhat, err, sm_count, st, hold);
    return launch_rows<8>(m, src, dt, packed, dhat, err, sm_count, st, hold);
}

}  // namespace cs
