// Exact search, ASG seed grid and walk statistics.
//
// The exact search realises the result definition directly: the host of x_p
// is the lowest user id among the elements that contain x_p (every FP64
// lambda >= -eps, Sec. 2.2). Candidates are the elements listed in x_p's
// cell of the bucket index (every element whose margin-grown box meets the
// cell and whose face planes do not separate it from the cell). It resolves
// walks that left the mesh or hit the step cap, and canonicalises walks that
// ended near a face, where a lower id may contain x_p as well.
#include <cstdint>

#include "walk_common.cuh"

namespace cs {
namespace {

// One warp per point: lanes test candidates, then a warp-wide min of user ids.
template <int D>
__device__ __forceinline__ int32_t exact_search_warp(const DevMesh &m, const double *xp,
                                                     int lane) {
    using WR = typename Recs<D>::W;
    using XR = typename Recs<D>::X;
    const WR *__restrict__ rw = static_cast<const WR *>(m.recw);
    const XR *__restrict__ rx = static_cast<const XR *>(m.recx);
    bool outside = false;
    #pragma unroll
    for (int k = 0; k < D; ++k)
        outside = outside || !(xp[k] >= m.lo[k] - m.margin) || !(xp[k] <= m.hi[k] + m.margin);
    if (outside) return -1;
    float xh[D], xl[D];
    #pragma unroll
    for (int k = 0; k < D; ++k) split_double(xp[k], xh[k], xl[k]);
    const int64_t c = grid_cell_cert<D>(xp, xh, xl, m, m.sb, m.inv_sb, m.gb);
    const int32_t b0 = __ldg(m.bstart + c), b1 = __ldg(m.bstart + c + 1);
    unsigned best = 0xffffffffu;
    for (int32_t t = b0 + lane; t < b1; t += 32) {
        const int32_t el = __ldg(m.bitems + t);
        WalkE<D> e;
        load_walk(rw, el, e);
        // containment certified in FP32 when possible (see walk_common.cuh),
        // else decided by the FP64 coordinates
        float lf[D + 1], T[D + 1];
        bary32<D>(e, xh, xl, lf, T);
        bool cin = true, cout = false;
        #pragma unroll
        for (int i = 0; i <= D; ++i) {
            cin = cin && (lf[i] - T[i] >= kNegEpsIn);
            cout = cout || (lf[i] + T[i] < kNegEpsOut);
        }
        bool inside = cin;
        if (!cin && !cout) {
            double lam[D + 1];
            bary64(rx, el, xp, lam);
            inside = true;
            #pragma unroll
            for (int i = 0; i <= D; ++i) inside = inside && (lam[i] >= -CS_EPS);
        }
        if (inside) best = min(best, unsigned(e.uid));
    }
    best = __reduce_min_sync(kFull, best);
    return best == 0xffffffffu ? -1 : int32_t(best);
}

// Monotone integer key of a non-NaN double: a < b <=> key(a) < key(b), with
// +0 and -0 equal (exact comparisons on the integer pipe).
__device__ __forceinline__ unsigned long long order_key(double x) {
    const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
    if ((b << 1) == 0) return 0x8000000000000000ull;
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

// Each lane prepares one listed particle (departure point, box test, bucket
// range) so the FP64 work runs with full warps; then the warp searches the
// candidates of each remaining particle together.
template <int D>
__global__ void __launch_bounds__(256) fallback_kernel(const DevMesh m, const TrackArgs a,
                                                       const int32_t *fb_count,
                                                       const int32_t *fb_list) {
    using WR = typename Recs<D>::W;
    using XR = typename Recs<D>::X;
    const WR *__restrict__ rw = static_cast<const WR *>(m.recw);
    const XR *__restrict__ rx = static_cast<const XR *>(m.recx);
    const int lane = threadIdx.x & 31;
    const int64_t warp = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
    const int32_t count = *fb_count;
    // particles per warp: spread a short list over many warps (the searches
    // of one warp run one after another), batch a long one (full-lane FP64)
    const int per = int(min(int64_t(32), max(int64_t(1), (count + nwarps - 1) / nwarps)));
    for (int64_t base = warp * per; base < count; base += nwarps * per) {
        const bool valid = lane < per && base + lane < count;
        int64_t p = 0;
        double xp[D];
        float xh[D], xl[D];
        int32_t b0 = 0, b1 = 0;
        bool work = false;
        if (valid) {
            p = fb_list[base + lane];
            bool outside = false;
            #pragma unroll
            for (int k = 0; k < D; ++k) {
                xp[k] = __dsub_rn(__ldg(a.x + p * D + k),
                                  __dmul_rn(__ldg(a.u + p * D + k), a.dt));
                const unsigned long long key = order_key(xp[k]);
                outside = outside || key < order_key(m.lo_m[k]) || key > order_key(m.hi_m[k]);
                split_double(xp[k], xh[k], xl[k]);
            }
            if (outside) {
                // no element's grown box reaches x_p: the host is -1
                a.host[p] = -1;
                if (a.status[p] != CS_FOUND) a.status[p] = CS_OUTSIDE;
            } else {
                const int64_t c = grid_cell_cert<D>(xp, xh, xl, m, m.sb, m.inv_sb, m.gb);
                b0 = __ldg(m.bstart + c);
                b1 = __ldg(m.bstart + c + 1);
                work = true;
            }
        }
        unsigned todo = __ballot_sync(kFull, work);
        while (todo) {
            const int j = __ffs(todo) - 1;
            todo &= todo - 1;
            double q[D];
            float qh[D], ql[D];
            #pragma unroll
            for (int k = 0; k < D; ++k) {
                q[k] = __shfl_sync(kFull, xp[k], j);
                qh[k] = __shfl_sync(kFull, xh[k], j);
                ql[k] = __shfl_sync(kFull, xl[k], j);
            }
            const int32_t t0 = __shfl_sync(kFull, b0, j), t1 = __shfl_sync(kFull, b1, j);
            unsigned best = 0xffffffffu;
            for (int32_t t = t0 + lane; t < t1; t += 32) {
                const int32_t el = __ldg(m.bitems + t);
                WalkE<D> e;
                load_walk(rw, el, e);
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
            if (lane == j) {
                const int32_t h = best == 0xffffffffu ? -1 : int32_t(best);
                a.host[p] = h;
                if (a.status[p] != CS_FOUND)
                    a.status[p] = h >= 0 ? CS_FOUND_VIA_FALLBACK : CS_OUTSIDE;
            }
        }
    }
}

// seed[c] = internal id of the host of the centre of ASG cell c, or -1.
template <int D>
__global__ void __launch_bounds__(256) seed_kernel(const DevMesh m, int32_t *seed) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
    for (int64_t c = warp; c < m.n_asg; c += nwarps) {
        double ctr[D];
        int64_t r = c;
        #pragma unroll
        for (int k = 0; k < D; ++k) {
            const int64_t i = r % m.ga[k];
            r /= m.ga[k];
            ctr[k] = __dadd_rn(m.lo[k], __dmul_rn(double(i) + 0.5, m.sa[k]));
        }
        const int32_t h = exact_search_warp<D>(m, ctr, lane);
        if (lane == 0) seed[c] = h >= 0 ? __ldg(m.iperm + h) : -1;
    }
}

__global__ void __launch_bounds__(256) stats_kernel(int64_t n, const int32_t *path,
                                                    const uint8_t *status, int64_t *out) {
    int64_t sum = 0, mx = 0, cnt[4] = {0, 0, 0, 0};
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += int64_t(gridDim.x) * blockDim.x) {
        const int32_t v = path[i];
        sum += v;
        mx = max(mx, int64_t(v));
        const uint8_t s = status[i];
        #pragma unroll
        for (int k = 0; k < 4; ++k) cnt[k] += (s == k);
    }
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sum += __shfl_xor_sync(kFull, sum, o);
        mx = max(mx, __shfl_xor_sync(kFull, mx, o));
        #pragma unroll
        for (int k = 0; k < 4; ++k) cnt[k] += __shfl_xor_sync(kFull, cnt[k], o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(reinterpret_cast<unsigned long long *>(out + 0), (unsigned long long)sum);
        atomicMax(reinterpret_cast<unsigned long long *>(out + 1), (unsigned long long)mx);
        for (int k = 0; k < 4; ++k)
            atomicAdd(reinterpret_cast<unsigned long long *>(out + 2 + k),
                      (unsigned long long)cnt[k]);
    }
}

}  // namespace

int launch_fallback(const DevMesh &m, const TrackArgs &a, const int32_t *count,
                    const int32_t *list, int sm_count, cudaStream_t st, Profiler *prof) {
    // The list is usually empty or nearly so (it holds particles within tau of
    // a face, walks that left the mesh or hit the cap), and its length is only
    // known on the device: one wave of resident blocks, which the kernel's
    // grid-stride loop spreads over any length, costs least to launch.
    static int occ[2] = {0, 0};
    int &o = occ[m.dim == 2 ? 0 : 1];
    if (o == 0) {
        if (m.dim == 2)
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, fallback_kernel<2>, 256, 0);
        else
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, fallback_kernel<3>, 256, 0);
        o = std::max(o, 1);
    }
    const int grid = int(std::max<int64_t>(1, std::min<int64_t>(int64_t(sm_count) * o,
                                                                (a.n + 7) / 8)));
    const int ev = prof ? prof->begin(CS_STAGE_FALLBACK, st) : -1;
    if (m.dim == 2)
        fallback_kernel<2><<<grid, 256, 0, st>>>(m, a, count, list);
    else
        fallback_kernel<3><<<grid, 256, 0, st>>>(m, a, count, list);
    if (prof) prof->end(ev, st);
    return 1;
}

int launch_seed_grid(const DevMesh &m, int32_t *seed, int sm_count, cudaStream_t st) {
    const int grid = sm_count * 8;
    if (m.dim == 2)
        seed_kernel<2><<<grid, 256, 0, st>>>(m, seed);
    else
        seed_kernel<3><<<grid, 256, 0, st>>>(m, seed);
    return 1;
}

int launch_stats(int64_t n, const int32_t *path, const uint8_t *status, int64_t *out,
                 int sm_count, cudaStream_t st) {
    cudaMemsetAsync(out, 0, 6 * sizeof(int64_t), st);
    if (n == 0) return 0;
    const int grid = int(std::min<int64_t>(int64_t(sm_count) * 4, (n + 255) / 256));
    stats_kernel<<<grid, 256, 0, st>>>(n, path, status, out);
    return 1;
}

}  // namespace cs
