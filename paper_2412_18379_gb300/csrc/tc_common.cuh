// tcgen05 building blocks shared by the tensor-core predictor kernels
// (cnn_tc.cu, 2-D; cnn3d_tc.cu, 3-D): shared-memory matrix and instruction
// descriptors, MMA issue and commit, mbarriers and counters with bounded
// waits, asynchronous copies, proxy fences, TMEM loads and the BF16
// epilogue helpers. Device code with internal linkage: each includer gets
// its own copy.
#pragma once

#include <cuda_bf16.h>

#include <cstdint>

#include "walk_common.cuh"

namespace cs {
namespace {

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// shared-memory matrix descriptor: no swizzle, K-major core matrices. The
// start address sits in the low 14 bits in 16-byte units; every operand here
// lies below 256 KiB, so adding a 16-byte offset to a descriptor never
// carries out of that field.
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

// arrive on `bar` once all MMAs issued so far by this thread have completed
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count));
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

// Bounded wait for the phase of `bar` with the given parity. Gives up (false)
// when another thread has raised the CTA's abort flag, or after 2^24 polls,
// in which case it raises the flag and the device error flag itself.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag,
                                          int *err) {
    for (uint32_t i = 0; i < (1u << 24); ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if (*abort_flag) return false;
        if (i > 64) __nanosleep(64);
    }
    *abort_flag = 1;
    atomicExch(err, 1);
    return false;
}

// warp-uniform bounded wait: every lane polls, the warp agrees on the result
__device__ __forceinline__ bool warp_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag,
                                          int *err) {
    return __all_sync(kFull, mbar_wait(bar, parity, abort_flag, err)) != 0;
}

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.cta.shared::cta.u32 %0, [%1];" : "=r"(v) : "r"(smem_addr(p)) : "memory");
    return v;
}

__device__ __forceinline__ void red_release_add(uint32_t *p, uint32_t v) {
    asm volatile("red.release.cta.shared::cta.add.u32 [%0], %1;" ::"r"(smem_addr(p)), "r"(v)
                 : "memory");
}

// Bounded wait until the counter *cnt reaches `target` (acquire). A plain
// shared-memory load is much cheaper than an mbarrier test, which matters on
// the MMA-issuing warp: the tensor pipe's issue queue is shallow, so every
// cycle that warp spends waiting is a cycle the tensor cores may idle. All
// lanes of a converged warp load the same word in one instruction, so the
// result is warp-uniform.
__device__ __forceinline__ bool wait_count(const uint32_t *cnt, uint32_t target,
                                           volatile int *abort_flag, int *err) {
    for (uint32_t i = 0; i < (1u << 26); ++i) {
        if (ld_acquire(cnt) >= target) return true;
        if (*abort_flag) return false;
        if (i > 256) __nanosleep(32);
    }
    *abort_flag = 1;
    atomicExch(err, 1);
    return false;
}

// true in exactly one lane of the (converged) warp
__device__ __forceinline__ bool elect_one() {
    uint32_t pred;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "elect.sync _|p, 0xffffffff;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(pred));
    return pred != 0;
}

// Asynchronous global -> shared copies (cp.async): a thread issues all of
// its copies before waiting once, instead of one load latency per element.
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src)
                 : "memory");
}
// 8 bytes, or 8 zero bytes when !valid (src is then not read)
__device__ __forceinline__ void cp_async8_zfill(void *dst, const void *src, bool valid) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(smem_addr(dst)), "l"(src),
                 "r"(valid ? 8u : 0u)
                 : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.wait_all;" ::: "memory");
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
// buffer in the chunked layout ([4 chunks][rows][8] BF16).
template <int ROWS>
__device__ __forceinline__ void store_act(uint8_t *buf, int row, const uint32_t *hv) {
    #pragma unroll
    for (int q = 0; q < 4; ++q)
        *reinterpret_cast<uint4 *>(buf + (size_t(q) * ROWS + row) * 16) =
            make_uint4(hv[4 * q], hv[4 * q + 1], hv[4 * q + 2], hv[4 * q + 3]);
}

// hv = BF16 pairs of ReLU(v + bias) over 32 channels. The bias is added in FP32
// pairs and ReLU taken on the rounded BF16 pairs: rounding to nearest is
// monotone and keeps 0, so this equals rounding ReLU(v + bias).
__device__ __forceinline__ void bias_relu_bf16(const float *v, const float *bias, uint32_t *hv) {
    const __nv_bfloat162 zero = __float2bfloat162_rn(0.f);
    #pragma unroll
    for (int e = 0; e < 8; ++e) {
        const float4 b = reinterpret_cast<const float4 *>(bias)[e];
        const float2 s0 = __fadd2_rn(make_float2(v[4 * e], v[4 * e + 1]), make_float2(b.x, b.y));
        const float2 s1 = __fadd2_rn(make_float2(v[4 * e + 2], v[4 * e + 3]), make_float2(b.z, b.w));
        const __nv_bfloat162 h0 = __hmax2(__floats2bfloat162_rn(s0.x, s0.y), zero);
        const __nv_bfloat162 h1 = __hmax2(__floats2bfloat162_rn(s1.x, s1.y), zero);
        hv[2 * e] = *reinterpret_cast<const uint32_t *>(&h0);
        hv[2 * e + 1] = *reinterpret_cast<const uint32_t *>(&h1);
    }
}

// Bounded wait until the device-memory flag *flag is non-zero (an acquire
// load per poll, at most `polls` polls ~256 ns apart). Gives up (false) when
// the CTA's abort flag is raised, or at the limit, raising the abort flag and
// the device error flag itself.
__device__ __forceinline__ bool wait_flag(const int *flag, uint32_t polls, volatile int *abort_flag,
                                          int *err) {
    for (uint32_t i = 0; i < polls; ++i) {
        int v;
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(flag) : "memory");
        if (v != 0) return true;
        if (*abort_flag) return false;
        __nanosleep(256);
    }
    *abort_flag = 1;
    atomicExch(err, 1);
    return false;
}

// The P1 interpolation of the nodal velocity at predictor cell c through the
// static table (node, w), with the resample kernel's arithmetic in its order
// (FP32 fused multiply-adds of the truncated nodal components, vertex by
// vertex); 0 where the cell centre has no host.
template <int D>
__device__ __forceinline__ void interp_cell(const int32_t *__restrict__ node,
                                            const float *__restrict__ w,
                                            const double *__restrict__ un, int64_t c, float *out) {
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
}

}  // namespace
}  // namespace cs
