// ASG seed grid and walk statistics.
//
// The seed of an ASG cell is the host of its centre, found by the exact
// search (exact_search_lane): the lowest user id among the elements that
// contain the point (every FP64 lambda >= -eps, Sec. 2.2). Candidates are the
// elements listed in the point's cell of the bucket index (every element
// whose margin-grown box meets the cell and whose face planes do not separate
// it from the cell). The walk kernel runs the same search for walks that
// left the mesh or hit the step cap, and for walks that ended near a face,
// where a lower id may contain x_p as well.
#include <cstdint>

#include "walk_common.cuh"

namespace cs {
namespace {

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
        // all lanes hold the centre; it lies inside the grown box
        float ch[D], cl[D];
        #pragma unroll
        for (int k = 0; k < D; ++k) split_double(ctr[k], ch[k], cl[k]);
        const int32_t h = exact_search_lane<D>(m, ctr, ch, cl, 0, lane);
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

// Error statistics of a finished track call (Sec. 3.1): the origin error err
// of a particle is the distance between the centroids of its tracking origin
// (the walk's start element) and of its host; the displacement error is
// |dhat * s - (x_p - x)|, the predicted displacement at the predictor cell of
// x (the cell CNN-SNS reads, in length units) against the true one. Sums and maxima go to out[0..3]
// (FP64, maxima as the bit patterns of non-negative doubles), counts to
// cnt[0..1].
template <int D>
__global__ void __launch_bounds__(256) error_stats_kernel(
    const DevMesh m, int64_t n, const int32_t *__restrict__ start, const int32_t *__restrict__ host,
    const double *__restrict__ x, const double *__restrict__ u, double dt,
    const float *__restrict__ dhat, double *out, unsigned long long *cnt) {
    double es = 0.0, em = 0.0, ds = 0.0, dm = 0.0;
    unsigned long long ne = 0, nd = 0;
    for (int64_t p = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; p < n;
         p += int64_t(gridDim.x) * blockDim.x) {
        const int32_t s = start ? start[p] : -1, h = host[p];
        if (start && s >= 0 && s < m.n_e && h >= 0 && h < m.n_e) {
            const int32_t a = __ldg(m.iperm + s), b = __ldg(m.iperm + h);
            double q = 0.0;
            #pragma unroll
            for (int k = 0; k < D; ++k) {
                const double d = __dsub_rn(m.centroid[int64_t(a) * D + k], m.centroid[int64_t(b) * D + k]);
                q = __dadd_rn(q, __dmul_rn(d, d));
            }
            const double e = __dsqrt_rn(q);
            es += e;
            em = fmax(em, e);
            ne += 1;
        }
        if (dhat) {
            double xv[D], dtrue[D];
            bool finite = true;
            #pragma unroll
            for (int k = 0; k < D; ++k) {
                xv[k] = x[p * D + k];
                const double xp = __dsub_rn(xv[k], __dmul_rn(u[p * D + k], dt));
                dtrue[k] = __dsub_rn(xp, xv[k]);
                finite = finite && isfinite(xp);
            }
            if (finite) {
                // the predictor cell the walk's CNN-SNS start rule reads (R23)
                int64_t c = 0;
                #pragma unroll
                for (int k = D - 1; k >= 0; --k)
                    c = c * m.pga[k] + cell_f32(trunc_to_float(xv[k]), m.lo_h[k], m.pinv_sa[k], m.pga[k]);
                double q = 0.0;
                #pragma unroll
                for (int k = 0; k < D; ++k) {
                    const double d =
                        __dsub_rn(__dmul_rn(double(dhat[c * D + k]), m.psa[k]), dtrue[k]);
                    q = __dadd_rn(q, __dmul_rn(d, d));
                }
                const double e = __dsqrt_rn(q);
                ds += e;
                dm = fmax(dm, e);
                nd += 1;
            }
        }
    }
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        es += __shfl_xor_sync(kFull, es, o);
        ds += __shfl_xor_sync(kFull, ds, o);
        em = fmax(em, __shfl_xor_sync(kFull, em, o));
        dm = fmax(dm, __shfl_xor_sync(kFull, dm, o));
        ne += __shfl_xor_sync(kFull, ne, o);
        nd += __shfl_xor_sync(kFull, nd, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(out + 0, es);
        atomicMax(reinterpret_cast<unsigned long long *>(out + 1),
                  static_cast<unsigned long long>(__double_as_longlong(em)));
        atomicAdd(out + 2, ds);
        atomicMax(reinterpret_cast<unsigned long long *>(out + 3),
                  static_cast<unsigned long long>(__double_as_longlong(dm)));
        atomicAdd(cnt + 0, ne);
        atomicAdd(cnt + 1, nd);
    }
}

}  // namespace

int launch_error_stats(const DevMesh &m, int64_t n, const int32_t *start, const int32_t *host,
                       const double *x, const double *u, double dt, const float *dhat,
                       double *out, unsigned long long *cnt, int sm_count, cudaStream_t st) {
    cudaMemsetAsync(out, 0, 4 * sizeof(double), st);
    cudaMemsetAsync(cnt, 0, 2 * sizeof(unsigned long long), st);
    if (n == 0) return 0;
    const int grid = int(std::min<int64_t>(int64_t(sm_count) * 4, (n + 255) / 256));
    if (m.dim == 2)
        error_stats_kernel<2><<<grid, 256, 0, st>>>(m, n, start, host, x, u, dt, dhat, out, cnt);
    else
        error_stats_kernel<3><<<grid, 256, 0, st>>>(m, n, start, host, x, u, dt, dhat, out, cnt);
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
