// Particle-location kernels: departure point, start element, the successive
// neighbour search walk (Algorithm 1), the exact search that canonicalises
// ties and resolves walks that left the mesh or hit the step cap, the ASG
// seed grid, and walk statistics.
//
// FP64 rounding is pinned with explicit _rn intrinsics (no fused multiply-
// add anywhere on the decision path) so that every barycentric coordinate is
// bit-identical to the one the host-side reference arithmetic produces:
//   delta_k   = x_p,k - v0_k
//   lambda_k  = sum_j M[k-1][j] * delta_j   (k = 1..d, left to right)
//   lambda_0  = ((1 - lambda_1) - lambda_2) - lambda_3
//   x_p       = x - (u * dt)
#include <cstdint>

#include "internal.h"

namespace cs {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kChunk = 64;          // particles a warp takes per global grab
constexpr uint8_t kPending = 0xff;  // status: exact search decides

template <int D> struct RecOf;
template <> struct RecOf<2> { using T = Rec2; };
template <> struct RecOf<3> { using T = Rec3; };

struct Elem2 { double v0[2]; double m[4]; int32_t nbr[3]; int32_t uid; };
struct Elem3 { double v0[3]; double m[9]; int32_t nbr[4]; int32_t uid; };

// One element record: 4 (2-D) or 7 (3-D) 16-byte read-only loads of one line.
__device__ __forceinline__ void load_elem(const Rec2 *__restrict__ r, int32_t e, Elem2 &o) {
    const double2 *p = reinterpret_cast<const double2 *>(r + e);
    const double2 a = __ldg(p + 0), b = __ldg(p + 1), c = __ldg(p + 2);
    const int4 n = __ldg(reinterpret_cast<const int4 *>(p + 3));
    o.v0[0] = a.x; o.v0[1] = a.y;
    o.m[0] = b.x; o.m[1] = b.y; o.m[2] = c.x; o.m[3] = c.y;
    o.nbr[0] = n.x; o.nbr[1] = n.y; o.nbr[2] = n.z; o.uid = n.w;
}
__device__ __forceinline__ void load_elem(const Rec3 *__restrict__ r, int32_t e, Elem3 &o) {
    const double2 *p = reinterpret_cast<const double2 *>(r + e);
    const double2 a = __ldg(p + 0), b = __ldg(p + 1), c = __ldg(p + 2), d = __ldg(p + 3),
                  f = __ldg(p + 4), g = __ldg(p + 5);
    const int4 n = __ldg(reinterpret_cast<const int4 *>(p + 6));
    const int4 w = __ldg(reinterpret_cast<const int4 *>(p + 7));
    o.v0[0] = a.x; o.v0[1] = a.y; o.v0[2] = b.x;
    o.m[0] = b.y; o.m[1] = c.x; o.m[2] = c.y; o.m[3] = d.x; o.m[4] = d.y;
    o.m[5] = f.x; o.m[6] = f.y; o.m[7] = g.x; o.m[8] = g.y;
    o.nbr[0] = n.x; o.nbr[1] = n.y; o.nbr[2] = n.z; o.nbr[3] = n.w; o.uid = w.x;
}

__device__ __forceinline__ void bary(const Elem2 &e, const double *x, double *lam) {
    const double dx = __dsub_rn(x[0], e.v0[0]), dy = __dsub_rn(x[1], e.v0[1]);
    const double l1 = __dadd_rn(__dmul_rn(e.m[0], dx), __dmul_rn(e.m[1], dy));
    const double l2 = __dadd_rn(__dmul_rn(e.m[2], dx), __dmul_rn(e.m[3], dy));
    lam[0] = __dsub_rn(__dsub_rn(1.0, l1), l2);
    lam[1] = l1;
    lam[2] = l2;
}
__device__ __forceinline__ void bary(const Elem3 &e, const double *x, double *lam) {
    const double dx = __dsub_rn(x[0], e.v0[0]), dy = __dsub_rn(x[1], e.v0[1]),
                 dz = __dsub_rn(x[2], e.v0[2]);
    const double l1 = __dadd_rn(__dadd_rn(__dmul_rn(e.m[0], dx), __dmul_rn(e.m[1], dy)),
                                __dmul_rn(e.m[2], dz));
    const double l2 = __dadd_rn(__dadd_rn(__dmul_rn(e.m[3], dx), __dmul_rn(e.m[4], dy)),
                                __dmul_rn(e.m[5], dz));
    const double l3 = __dadd_rn(__dadd_rn(__dmul_rn(e.m[6], dx), __dmul_rn(e.m[7], dy)),
                                __dmul_rn(e.m[8], dz));
    lam[0] = __dsub_rn(__dsub_rn(__dsub_rn(1.0, l1), l2), l3);
    lam[1] = l1;
    lam[2] = l2;
    lam[3] = l3;
}

template <int D> using ElemT = typename std::conditional<D == 2, Elem2, Elem3>::type;

// Cell of a point in a grid of g cells of size s over [lo, ...]:
// floor((x - lo) / s) clamped to [0, g-1] (NaN -> 0), x fastest.
template <int D>
__device__ __forceinline__ int64_t grid_cell(const double *x, const double *lo, const double *s,
                                             const int32_t *g) {
    int64_t c = 0;
    #pragma unroll
    for (int k = D - 1; k >= 0; --k) {
        const double t = floor(__ddiv_rn(__dsub_rn(x[k], lo[k]), s[k]));
        int64_t i;
        if (!(t >= 0.0)) i = 0;
        else if (t > double(g[k] - 1)) i = g[k] - 1;
        else i = int64_t(t);
        c = c * g[k] + i;
    }
    return c;
}

// Warp-aggregated append of particle p to the exact-search list.
__device__ __forceinline__ void push_list(bool want, int64_t p, int32_t *count, int32_t *list,
                                          int lane) {
    const unsigned m = __ballot_sync(kFull, want);
    if (!m) return;
    int base = 0;
    const int leader = __ffs(m) - 1;
    if (lane == leader) base = atomicAdd(count, __popc(m));
    base = __shfl_sync(kFull, base, leader);
    if (want) list[base + __popc(m & ((1u << lane) - 1u))] = int32_t(p);
}

// ---------------------------------------------------------------------------
// Persistent walk kernel. Each warp keeps 32 particles in flight; whenever
// lanes finish, a ballot finds them and they are refilled from the warp's
// current chunk of particle indices (a chunk of kChunk indices is taken from
// the global cursor with one atomic), so long walks never leave lanes idle
// while work remains.
// ---------------------------------------------------------------------------
template <int D>
__global__ void __launch_bounds__(256) walk_kernel(const DevMesh m, const TrackArgs a,
                                                   int32_t *cursor, int32_t *fb_count,
                                                   int32_t *fb_list) {
    using Rec = typename RecOf<D>::T;
    const Rec *__restrict__ recs = static_cast<const Rec *>(m.rec);
    const int lane = threadIdx.x & 31;
    const int64_t n = a.n;

    int64_t p = -1;              // particle of this lane, -1 = idle
    double xp[D];
    int32_t cur = -1, it = 0;
    int64_t chunk_next = 0, chunk_end = 0;   // warp-uniform
    bool drained = false;                    // warp-uniform: global cursor exhausted

    for (;;) {
        // ---- refill idle lanes ----
        unsigned idle = __ballot_sync(kFull, p < 0);
        while (idle && !drained) {
            if (chunk_next >= chunk_end) {
                int base = 0;
                if (lane == 0) base = atomicAdd(cursor, kChunk);
                base = __shfl_sync(kFull, base, 0);
                if (int64_t(base) >= n) {
                    drained = true;
                    break;
                }
                chunk_next = base;
                chunk_end = min(int64_t(base) + kChunk, n);
            }
            const int take = int(min(int64_t(__popc(idle)), chunk_end - chunk_next));
            const int rank = __popc(idle & ((1u << lane) - 1u));
            bool mine = ((idle >> lane) & 1u) && rank < take;
            bool need_search = false;
            if (mine) {
                p = chunk_next + rank;
                // departure point x_p = x - (u * dt)  (Eq. 3, first order)
                bool finite = true;
                #pragma unroll
                for (int k = 0; k < D; ++k) {
                    const double xv = __ldg(a.x + p * D + k), uv = __ldg(a.u + p * D + k);
                    xp[k] = __dsub_rn(xv, __dmul_rn(uv, a.dt));
                    finite = finite && isfinite(xp[k]);
                }
                // plain start K_m, as an internal id
                int32_t plain;
                if (a.start_user) {
                    const int32_t su = __ldg(a.start_user + p);
                    plain = (su >= 0 && su < m.n_e) ? __ldg(m.iperm + su) : -1;
                } else {
                    plain = __ldg(m.node_elem + p);
                }
                int32_t s = plain;
                if (finite && a.mode == CS_ASG_DIRECT) {
                    const int32_t sd = __ldg(m.seed + grid_cell<D>(xp, m.lo, m.sa, m.ga));
                    if (sd >= 0) s = sd;
                } else if (finite && a.mode == CS_CNN_SNS) {
                    double x0[D], y[D];
                    #pragma unroll
                    for (int k = 0; k < D; ++k) x0[k] = __ldg(a.x + p * D + k);
                    const int64_t c0 = grid_cell<D>(x0, m.lo, m.sa, m.ga);
                    #pragma unroll
                    for (int k = 0; k < D; ++k) {
                        const double dh = double(__ldg(a.dhat + c0 * D + k));
                        y[k] = __dadd_rn(x0[k], __dmul_rn(dh, m.sa[k]));
                    }
                    const int32_t sd = __ldg(m.seed + grid_cell<D>(y, m.lo, m.sa, m.ga));
                    if (sd >= 0) s = sd;
                }
                cur = s;
                it = 0;
                if (!finite) {
                    a.host[p] = -1;
                    a.path[p] = 0;
                    a.status[p] = CS_INVALID;
                    if (a.start_out) a.start_out[p] = -1;
                    p = -1;
                } else if (s < 0) {
                    a.host[p] = -1;
                    a.path[p] = 0;
                    a.status[p] = kPending;
                    if (a.start_out) a.start_out[p] = -1;
                    need_search = true;
                }
            }
            const int64_t pp = p;
            push_list(need_search, pp, fb_count, fb_list, lane);
            if (need_search) p = -1;
            chunk_next += take;
            idle = __ballot_sync(kFull, p < 0);
            if (take == 0) break;   // unreachable: a fresh chunk is never empty
        }
        if (__ballot_sync(kFull, p >= 0) == 0) break;

        // ---- one step of Algorithm 1 for every busy lane ----
        bool done = false, search = false;
        if (p >= 0) {
            ElemT<D> e;
            load_elem(recs, cur, e);
            if (it == 0 && a.start_out) a.start_out[p] = e.uid;
            ++it;
            double lam[D + 1];
            bary(e, xp, lam);
            bool inside = true, near = false;
            // argmin of lambda, lowest index on equal minima (Eq. 5); the
            // neighbour across that face is picked without dynamic indexing
            double lmin = lam[0];
            int32_t next = e.nbr[0];
            #pragma unroll
            for (int i = 0; i <= D; ++i) {
                inside = inside && (lam[i] >= -CS_EPS);
                near = near || (lam[i] < m.tau);
                if (i > 0 && lam[i] < lmin) {
                    lmin = lam[i];
                    next = e.nbr[i];
                }
            }
            if (inside) {
                a.host[p] = e.uid;
                a.path[p] = it;
                a.status[p] = CS_FOUND;
                done = true;
                search = near;      // another element may contain x_p too
            } else {
                const int32_t nb = next;
                if (nb < 0 || it >= m.cap) {
                    a.host[p] = -1;
                    a.path[p] = it;
                    a.status[p] = kPending;
                    done = true;
                    search = true;
                } else {
                    cur = nb;
                }
            }
        }
        push_list(search, p, fb_count, fb_list, lane);
        if (done) p = -1;
    }
}

// ---------------------------------------------------------------------------
// Exact search: host = lowest user id whose element contains x_p (every
// lambda >= -eps) among the candidates listed in x_p's bucket cell. One warp
// per point: lanes test candidates, then a warp-wide min of user ids.
// ---------------------------------------------------------------------------
template <int D>
__device__ __forceinline__ int32_t exact_search_warp(const DevMesh &m, const double *xp,
                                                     int lane) {
    using Rec = typename RecOf<D>::T;
    const Rec *__restrict__ recs = static_cast<const Rec *>(m.rec);
    bool outside = false;
    #pragma unroll
    for (int k = 0; k < D; ++k)
        outside = outside || !(xp[k] >= m.lo[k] - m.margin) || !(xp[k] <= m.hi[k] + m.margin);
    if (outside) return -1;
    const int64_t c = grid_cell<D>(xp, m.lo, m.sb, m.gb);
    const int32_t b0 = __ldg(m.bstart + c), b1 = __ldg(m.bstart + c + 1);
    unsigned best = 0xffffffffu;
    for (int32_t t = b0 + lane; t < b1; t += 32) {
        ElemT<D> e;
        load_elem(recs, __ldg(m.bitems + t), e);
        double lam[D + 1];
        bary(e, xp, lam);
        bool inside = true;
        #pragma unroll
        for (int i = 0; i <= D; ++i) inside = inside && (lam[i] >= -CS_EPS);
        if (inside) best = min(best, unsigned(e.uid));
    }
    best = __reduce_min_sync(kFull, best);
    return best == 0xffffffffu ? -1 : int32_t(best);
}

template <int D>
__global__ void __launch_bounds__(256) fallback_kernel(const DevMesh m, const TrackArgs a,
                                                       const int32_t *fb_count,
                                                       const int32_t *fb_list) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
    const int32_t count = *fb_count;
    for (int64_t w = warp; w < count; w += nwarps) {
        const int64_t p = fb_list[w];
        double xp[D];
        #pragma unroll
        for (int k = 0; k < D; ++k)
            xp[k] = __dsub_rn(__ldg(a.x + p * D + k), __dmul_rn(__ldg(a.u + p * D + k), a.dt));
        const int32_t h = exact_search_warp<D>(m, xp, lane);
        if (lane == 0) {
            const uint8_t st = a.status[p];
            a.host[p] = h;
            if (st != CS_FOUND) a.status[p] = h >= 0 ? CS_FOUND_VIA_FALLBACK : CS_OUTSIDE;
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

int launch_track(const DevMesh &m, const TrackArgs &a, const Scratch &s, int sm_count,
                 cudaStream_t st, Profiler *prof) {
    if (a.n == 0) return 0;
    cudaMemsetAsync(s.counters, 0, 2 * sizeof(int32_t), st);
    int per_sm = 0;
    if (m.dim == 2)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, walk_kernel<2>, 256, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, walk_kernel<3>, 256, 0);
    per_sm = per_sm > 0 ? per_sm : 1;
    const int64_t need = (a.n + 255) / 256;
    const int grid = int(std::min<int64_t>(int64_t(sm_count) * per_sm, need));
    const int fb_grid = sm_count * 4;
    int ev = prof ? prof->begin(CS_STAGE_WALK, st) : -1;
    if (m.dim == 2)
        walk_kernel<2><<<grid, 256, 0, st>>>(m, a, s.counters, s.counters + 1, s.list);
    else
        walk_kernel<3><<<grid, 256, 0, st>>>(m, a, s.counters, s.counters + 1, s.list);
    if (prof) prof->end(ev, st);
    ev = prof ? prof->begin(CS_STAGE_FALLBACK, st) : -1;
    if (m.dim == 2)
        fallback_kernel<2><<<fb_grid, 256, 0, st>>>(m, a, s.counters + 1, s.list);
    else
        fallback_kernel<3><<<fb_grid, 256, 0, st>>>(m, a, s.counters + 1, s.list);
    if (prof) prof->end(ev, st);
    return 2;
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
