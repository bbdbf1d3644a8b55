// Device helpers shared by the walk and the exact search: record loads, the
// FP64 barycentric arithmetic (the arbiter), the certified FP32 filter, ASG
// grid cells and the warp-cooperative exact search.
//
// Exact arithmetic. Every decision of the walk is that of FP64 barycentric
// coordinates with a pinned rounding order (no fused multiply-add):
//   x_p       = x - (u * dt)
//   delta_k   = x_p,k - v0_k
//   lambda_k  = sum_j M[k-1][j] * delta_j   (k = 1..d, left to right)
//   lambda_0  = ((1 - lambda_1) - lambda_2) - lambda_3
//   cell_k    = floor((x_k - lo_k) / s_k), clamped to [0, g_k - 1]
//
// FP32 filter. GB300 executes FP64 at 1/64 of the FP32 rate, so each step
// first evaluates the coordinates in FP32 (x_p and v0 split into float
// hi + lo parts, M rounded to float) together with a bound T_i on
// |lambda_i(FP64) - lambda_i(FP32)|, twice the worst-case rounding error of
// both evaluations. A decision is taken in FP32 only when the bound makes it
// certain; any other step is recomputed with the FP64 formula above, so every
// decision equals the FP64 one.
#pragma once

#include <cstdint>

#include "internal.h"

namespace cs {

constexpr unsigned kFull = 0xffffffffu;

// Programmatic dependent launch. launch_pdl lets the kernel be scheduled
// while the previous kernel on the stream is still finishing, which hides
// the launch gap between the kernels of a step; the kernel must call
// pdl_wait() before it touches global memory that an earlier kernel on the
// stream writes or reads (it returns once those kernels have completed and
// their writes are visible; without the launch attribute it returns at once).
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t st, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// FP32 unit roundoff u = 2^-24 and the filter's constants
constexpr float kU = 5.9604644775390625e-08f;
constexpr float k4U = 4.0f * kU;
constexpr float k8U = 8.0f * kU;
constexpr float k32UU = 32.0f * kU * kU;
constexpr float kTiny = 1e-36f;              // covers subnormal rounding
constexpr float kNegEpsIn = -0.99e-12f;      // certain: lambda >= -eps
constexpr float kNegEpsOut = -1.01e-12f;     // certain: lambda <  -eps

template <int D> struct Recs;
template <> struct Recs<2> { using W = WalkRec2; using X = ExactRec2; };
template <> struct Recs<3> { using W = WalkRec3; using X = ExactRec3; };

// walk record fields in registers
template <int D> struct WalkE {
    float vh[D], vl[D], m[D * D];
    int32_t nbr[D + 1];
    int32_t uid;
};

// walk record fields from its 16-byte words
__device__ __forceinline__ void decode_walk(const float4 a, const float4 b, const float4 c,
                                            WalkE<2> &o) {
    o.vh[0] = a.x; o.vh[1] = a.y; o.vl[0] = a.z; o.vl[1] = a.w;
    o.m[0] = b.x; o.m[1] = b.y; o.m[2] = b.z; o.m[3] = b.w;
    o.nbr[0] = __float_as_int(c.x); o.nbr[1] = __float_as_int(c.y);
    o.nbr[2] = __float_as_int(c.z); o.uid = __float_as_int(c.w);
}
__device__ __forceinline__ void decode_walk(const float4 a, const float4 b, const float4 c,
                                            const float4 d, const float4 n, WalkE<3> &o) {
    o.vh[0] = a.x; o.vh[1] = a.y; o.vh[2] = a.z; o.vl[0] = a.w;
    o.vl[1] = b.x; o.vl[2] = b.y; o.m[0] = b.z; o.m[1] = b.w;
    o.m[2] = c.x; o.m[3] = c.y; o.m[4] = c.z; o.m[5] = c.w;
    o.m[6] = d.x; o.m[7] = d.y; o.m[8] = d.z; o.uid = __float_as_int(d.w);
    o.nbr[0] = __float_as_int(n.x); o.nbr[1] = __float_as_int(n.y);
    o.nbr[2] = __float_as_int(n.z); o.nbr[3] = __float_as_int(n.w);
}

__device__ __forceinline__ void load_walk(const WalkRec2 *__restrict__ r, int32_t e,
                                          WalkE<2> &o) {
    const float4 *p = reinterpret_cast<const float4 *>(r + e);
    decode_walk(__ldg(p + 0), __ldg(p + 1), __ldg(p + 2), o);
}
__device__ __forceinline__ void load_walk(const WalkRec3 *__restrict__ r, int32_t e,
                                          WalkE<3> &o) {
    const float4 *p = reinterpret_cast<const float4 *>(r + e);
    decode_walk(__ldg(p + 0), __ldg(p + 1), __ldg(p + 2), __ldg(p + 3), __ldg(p + 4), o);
}
// FP64 coordinates from the exact record (the arbiter).
__device__ __forceinline__ void bary64(const ExactRec2 *__restrict__ r, int32_t e,
                                       const double *x, double *lam) {
    const double2 *p = reinterpret_cast<const double2 *>(r + e);
    const double2 a = __ldg(p + 0), b = __ldg(p + 1), c = __ldg(p + 2);
    const double dx = __dsub_rn(x[0], a.x), dy = __dsub_rn(x[1], a.y);
    const double l1 = __dadd_rn(__dmul_rn(b.x, dx), __dmul_rn(b.y, dy));
    const double l2 = __dadd_rn(__dmul_rn(c.x, dx), __dmul_rn(c.y, dy));
    lam[0] = __dsub_rn(__dsub_rn(1.0, l1), l2);
    lam[1] = l1;
    lam[2] = l2;
}
__device__ __forceinline__ void bary64(const ExactRec3 *__restrict__ r, int32_t e,
                                       const double *x, double *lam) {
    const double2 *p = reinterpret_cast<const double2 *>(r + e);
    const double2 a = __ldg(p + 0), b = __ldg(p + 1), c = __ldg(p + 2), d = __ldg(p + 3),
                  f = __ldg(p + 4), g = __ldg(p + 5);
    // v0 = (a.x, a.y, b.x); M rows (b.y c.x c.y) (d.x d.y f.x) (f.y g.x g.y)
    const double dx = __dsub_rn(x[0], a.x), dy = __dsub_rn(x[1], a.y),
                 dz = __dsub_rn(x[2], b.x);
    const double l1 = __dadd_rn(__dadd_rn(__dmul_rn(b.y, dx), __dmul_rn(c.x, dy)),
                                __dmul_rn(c.y, dz));
    const double l2 = __dadd_rn(__dadd_rn(__dmul_rn(d.x, dx), __dmul_rn(d.y, dy)),
                                __dmul_rn(f.x, dz));
    const double l3 = __dadd_rn(__dadd_rn(__dmul_rn(f.y, dx), __dmul_rn(g.x, dy)),
                                __dmul_rn(g.y, dz));
    lam[0] = __dsub_rn(__dsub_rn(__dsub_rn(1.0, l1), l2), l3);
    lam[1] = l1;
    lam[2] = l2;
    lam[3] = l3;
}

// |(xh + xl) - (vh + vl) - df| bound for df = (xh - vh) + (xl - vl) in FP32,
// given |x - xh - xl| <= 2^-44 |xh| and |v - vh - vl| <= 2^-48 |vh|.
__device__ __forceinline__ float delta_bound(float df, float xh, float vh) {
    return fmaf(k4U, fabsf(df), k32UU * (fabsf(xh) + fabsf(vh)));
}

// FP32 coordinates lf and their bounds T (see the file comment).
template <int D>
__device__ __forceinline__ void bary32(const WalkE<D> &e, const float *xh, const float *xl,
                                       float *lf, float *T) {
    float df[D], ed[D];
    #pragma unroll
    for (int k = 0; k < D; ++k) {
        const float dh = xh[k] - e.vh[k];
        const float dl = xl[k] - e.vl[k];
        df[k] = dh + dl;
        ed[k] = delta_bound(df[k], xh[k], e.vh[k]);
    }
    float sumT = 0.f, suml = 0.f;
    float l0 = 1.0f;
    #pragma unroll
    for (int r = 0; r < D; ++r) {
        float acc = e.m[r * D] * df[0];
        float a = fabsf(e.m[r * D]) * fmaf(k4U, fabsf(df[0]), ed[0]);
        float ms = fabsf(e.m[r * D]);
        #pragma unroll
        for (int j = 1; j < D; ++j) {
            acc = fmaf(e.m[r * D + j], df[j], acc);
            a = fmaf(fabsf(e.m[r * D + j]), fmaf(k4U, fabsf(df[j]), ed[j]), a);
            ms += fabsf(e.m[r * D + j]);
        }
        lf[r + 1] = acc;
        T[r + 1] = fmaf(2.0f, a, kTiny * (1.0f + ms));
        sumT += T[r + 1];
        suml += fabsf(acc);
        l0 = l0 - acc;
    }
    lf[0] = l0;
    T[0] = sumT + fmaf(k8U, 1.0f + suml, kTiny);
}

// The two 32-bit halves of a double's bit pattern. Through inline PTX so
// that the compiler cannot fold the integer tests below back into FP64
// comparisons: on GB300 every FP64 instruction, compares and conversions
// included, occupies the FP64 pipe for about 56 cycles per warp, while these
// integer tests cost a few cycles each.
__device__ __forceinline__ void dbits(double x, uint32_t &lo, uint32_t &hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=r"(lo), "=r"(hi) : "d"(x));
}

// x = hi + lo + r with hi = x truncated to 24 significant bits, lo = the
// remainder truncated to float, |r| <= 2^-44 |hi|, from the bit pattern of x
// (integer pipe only). Zero gives (0, 0); exponents outside [-74, 127] give
// hi = NaN, which no filter test certifies (those steps use FP64).
__device__ __forceinline__ void split_double(double x, float &hi, float &lo) {
    uint32_t bl, bh;
    dbits(x, bl, bh);
    if (((bh << 1) | bl) == 0) {
        hi = 0.f;
        lo = 0.f;
        return;
    }
    const int E = int((bh >> 20) & 0x7ffu) - 1023;
    if (E < -74 || E > 127) {
        hi = __int_as_float(0x7fc00000);
        lo = 0.f;
        return;
    }
    const unsigned sign = bh & 0x80000000u;
    // the 23 fraction bits below the leading one: bh[19:0] and bl[31:29]
    hi = __uint_as_float(sign | (unsigned(E + 127) << 23) | (((bh << 3) | (bl >> 29)) & 0x7fffffu));
    const float low = __uint2float_rz(bl & 0x1fffffffu);
    lo = __fmul_rn(sign ? -low : low, __uint_as_float(unsigned(E + 75) << 23));
}

// x truncated to float from its bit pattern (integer pipe only); magnitudes
// below 2^-126 become 0, above the float range +-inf, NaN stays NaN.
__device__ __forceinline__ float trunc_to_float(double x) {
    uint32_t bl, bh;
    dbits(x, bl, bh);
    const unsigned sign = bh & 0x80000000u;
    const int E = int((bh >> 20) & 0x7ffu) - 1023;
    if (E < -126) return __uint_as_float(sign);
    if (E > 127) {
        const bool nan = E == 1024 && ((bh & 0xfffffu) | bl) != 0;
        return __uint_as_float(sign | 0x7f800000u | (nan ? 0x400000u : 0u));
    }
    return __uint_as_float(sign | (unsigned(E + 127) << 23) | (((bh << 3) | (bl >> 29)) & 0x7fffffu));
}

__device__ __forceinline__ bool finite_bits(double x) {
    uint32_t bl, bh;
    dbits(x, bl, bh);
    return (bh & 0x7ff00000u) != 0x7ff00000u;
}

// Cell index of one axis, FP64: floor((x - lo) / s) clamped, NaN -> 0.
__device__ __forceinline__ int64_t cell_axis64(double x, double lo, double s, int32_t g) {
    const double t = floor(__ddiv_rn(__dsub_rn(x, lo), s));
    if (!(t >= 0.0)) return 0;
    if (t > double(g - 1)) return g - 1;
    return int64_t(t);
}

template <int D>
__device__ __forceinline__ int64_t grid_cell(const double *x, const double *lo, const double *s,
                                             const int32_t *g) {
    int64_t c = 0;
    #pragma unroll
    for (int k = D - 1; k >= 0; --k) c = c * g[k] + cell_axis64(x[k], lo[k], s[k], g[k]);
    return c;
}

// Same cell, certified in FP32 per axis when the rounding bound cannot move
// the quotient across an integer; otherwise the FP64 formula. inv_s is 1/s
// rounded to float.
template <int D>
__device__ __forceinline__ int64_t grid_cell_cert(const double *x, const float *xh,
                                                  const float *xl, const DevMesh &m,
                                                  const double *s, const float *inv_s,
                                                  const int32_t *g) {
    int64_t c = 0;
    #pragma unroll
    for (int k = D - 1; k >= 0; --k) {
        const float df = (xh[k] - m.lo_h[k]) + (xl[k] - m.lo_l[k]);
        const float ed = delta_bound(df, xh[k], m.lo_h[k]);
        const float q = df * inv_s[k];
        const float B = fmaf(2.0f * ed, inv_s[k], fmaf(k8U, fabsf(q), kTiny));
        // floor of both ends in int32 (the XU pipe; a float -> int64
        // conversion would take the FP64 pipe); equal ends with |q| < 4e6
        // are in range, and NaN or out-of-range ends never pass the test
        const int a = __float2int_rd(q - B), b = __float2int_rd(q + B);
        int64_t i;
        if (a == b && fabsf(q) < 4.0e6f) {
            i = a < 0 ? 0 : (a > g[k] - 1 ? g[k] - 1 : a);
        } else {
            i = cell_axis64(x[k], m.lo[k], s[k], g[k]);
        }
        c = c * g[k] + i;
    }
    return c;
}

// ASG cell of a point (seed grid, CNN grid)
template <int D>
__device__ __forceinline__ int64_t grid_cell_f(const double *x, const float *xh, const float *xl,
                                               const DevMesh &m) {
    return grid_cell_cert<D>(x, xh, xl, m, m.sa, m.inv_sa, m.ga);
}

// Cell index of one axis in FP32 (the CNN-SNS origin, reading R23):
// floor((v - lo) * inv) with each operation rounded to nearest float,
// clamped to [0, g - 1]; negative and NaN quotients give 0. lo and inv are
// the FP64 grid origin and 1 / cell size rounded to float.
__device__ __forceinline__ int cell_f32(float v, float lo, float inv, int32_t g) {
    const float q = __fmul_rn(__fsub_rn(v, lo), inv);
    const int i = __float2int_rd(q);   // saturates at the int32 range
    return q >= 0.0f ? min(i, g - 1) : 0;
}

// Monotone integer key of a non-NaN double: a < b <=> key(a) < key(b), with
// +0 and -0 equal (exact comparisons on the integer pipe).
__device__ __forceinline__ unsigned long long order_key(double x) {
    uint32_t bl, bh;
    dbits(x, bl, bh);
    if (((bh << 1) | bl) == 0) return 0x8000000000000000ull;
    const unsigned long long b = (static_cast<unsigned long long>(bh) << 32) | bl;
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

// Exact search for the point that lane j holds (xp and its hi/lo split): the
// host of x_p is the lowest user id among the elements containing it (every
// FP64 lambda >= -eps, Sec. 2.2), or -1. Candidates are the elements listed in
// x_p's cell of the bucket index. Called by all 32 lanes of a warp; each lane
// tests every 32nd candidate, then a warp-wide min. Finite x_p only.
template <int D>
__device__ __forceinline__ int32_t exact_search_lane(const DevMesh &m, const double *xp,
                                                     const float *xh, const float *xl, int j,
                                                     int lane) {
    using WR = typename Recs<D>::W;
    using XR = typename Recs<D>::X;
    const WR *__restrict__ rw = static_cast<const WR *>(m.recw);
    const XR *__restrict__ rx = static_cast<const XR *>(m.recx);
    double q[D];
    float qh[D], ql[D];
    bool outside = false;
    #pragma unroll
    for (int k = 0; k < D; ++k) {
        q[k] = __shfl_sync(kFull, xp[k], j);
        qh[k] = __shfl_sync(kFull, xh[k], j);
        ql[k] = __shfl_sync(kFull, xl[k], j);
        const unsigned long long key = order_key(q[k]);
        outside = outside || key < order_key(m.lo_m[k]) || key > order_key(m.hi_m[k]);
    }
    // no element's grown box reaches x_p
    if (outside) return -1;
    const int64_t c = grid_cell_cert<D>(q, qh, ql, m, m.sb, m.inv_sb, m.gb);
    const int32_t t0 = __ldg(m.bstart + c), t1 = __ldg(m.bstart + c + 1);
    unsigned best = 0xffffffffu;
    for (int32_t t = t0 + lane; t < t1; t += 32) {
        const int32_t el = __ldg(m.bitems + t);
        WalkE<D> e;
        load_walk(rw, el, e);
        // containment certified in FP32 when possible, else decided by the
        // FP64 coordinates
        float lf[D + 1], T[D + 1];
        bary32<D>(e, qh, ql, lf, T);
        bool cin = true, cout = false;
        #pragma unroll
        for (int i = 0; i <= D; ++i) {
            cin = cin && (lf[i] - T[i] >= kNegEpsIn);
            cout = cout || (lf[i] + T[i] < kNegEpsOut);
        }
        bool inside = cin;
        if (!cin && !cout) {
            double lam[D + 1];
            bary64(rx, el, q, lam);
            inside = true;
            #pragma unroll
            for (int i = 0; i <= D; ++i) inside = inside && (lam[i] >= -CS_EPS);
        }
        if (inside) best = min(best, unsigned(e.uid));
    }
    best = __reduce_min_sync(kFull, best);
    return best == 0xffffffffu ? -1 : int32_t(best);
}

}  // namespace cs
