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

}  // namespace

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
