// The successive neighbour search walk (Algorithm 1) as one persistent kernel,
// with the departure point (Eq. 3) and the start element (plain SNS: the
// particle's own element; ASG: the seed of the cell of x_p; CNN-SNS,
// Algorithm 2: the seed of the cell at x + predicted displacement).
//
// Work distribution. Each warp owns a queue of 32 prepared particles in
// shared memory. When the queue is empty the whole warp prepares the next 32
// particles at once, one per lane (departure point, hi/lo split, start
// element): the FP64 work of a particle runs with every lane active. Each
// step, a ballot finds the lanes whose particle finished; they pop the next
// prepared particles from the queue, so long walks never leave lanes idle
// while work remains.
//
// Exact search. A walk that leaves the mesh or reaches the step cap, a
// particle with no start element, and a walk that ends within tau of an
// interior face (where a lower id may contain x_p too) are resolved where
// they occur: the whole warp runs the bucketed exact search for that lane's
// x_p, then goes on walking. These are a few particles in a million, so the
// pause is short and the other warps keep the SM busy; a separate pass over
// a list would pay a launch and a tail for them.
#include <cstdint>
#include <mutex>
#include <string>

#include "walk_common.cuh"

namespace cs {
namespace {

constexpr int kWarps = 8;   // 256 threads per block

template <int D> struct Queue {
    int32_t p[32];          // particle index, -1 = nothing to walk
    int32_t cur[32];        // start element (internal id)
    double xp[D][32];
    float xh[D][32], xl[D][32];
};

// The warp's next batch: x, u and the plain start of its 32 particles,
// fetched with cp.async while the current batch walks, so that preparing it
// does not begin with a global round trip. 2-D only. In 3-D, holding a
// second batch per warp widens the range of particles in flight, and with it
// the mesh region the walks touch at once: L2 reuse of the element records
// drops (12% more DRAM traffic on the ABC case), which costs more than the
// round trip saves; so the 3-D walk claims a batch when its queue runs dry.
template <int D> constexpr bool kPrefetch = D == 2;

template <int D> struct Prefetch {
    double x[32 * D];
    double u[32 * D];
    int32_t start[32];      // start_user[p] if given, else node_elem[p]
};

__device__ __forceinline__ void walk_cp_async(void *dst, const void *src, int bytes, bool valid) {
    const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(dst));
    if (bytes == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(d), "l"(src),
                     "r"(valid ? 8u : 0u)
                     : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(src),
                     "r"(valid ? 4u : 0u)
                     : "memory");
}

// Issue the copies of the batch at `base` (lane l: particle base + l, zeros
// past n; an invalid lane copies nothing from its in-range source address).
template <int D>
__device__ __forceinline__ void prefetch_batch(const DevMesh &m, const TrackArgs &a, int64_t base,
                                               int64_t n, Prefetch<D> &f, int lane) {
    const bool valid = base + lane < n;
    const int64_t ps = valid ? base + lane : 0;
    #pragma unroll
    for (int k = 0; k < D; ++k) {
        walk_cp_async(&f.x[lane * D + k], a.x + ps * D + k, 8, valid);
        walk_cp_async(&f.u[lane * D + k], a.u + ps * D + k, 8, valid);
    }
    walk_cp_async(&f.start[lane], a.start_user ? a.start_user + ps : m.node_elem + ps, 4, valid);
}

// Prepare particle pp (if `valid`) into slot `lane` of the warp's queue, from
// the lane's prefetched x, u and start (copies complete). Called by all 32
// lanes of the warp.
template <int D>
__device__ __forceinline__ void prepare(const DevMesh &m, const TrackArgs &a, int64_t pp,
                                        bool valid, Queue<D> &q, const Prefetch<D> &f, int lane) {
    bool need_search = false;
    int32_t entry = -1, s = -1;
    double xp[D];
    float xh[D], xl[D];
    if (valid) {
        // CNN-SNS: Algorithm 2's origin, in FP32 (reading R23: it selects the
        // start element only, never the host, and FP64 costs GB300 1/64 of
        // the FP32 rate): x truncated to float and its predictor cell. The
        // gather of the cell's predicted displacement depends on x alone, so
        // it is issued before the departure point's FP64 arithmetic, which
        // then runs under its latency (any x gives an in-range cell; the
        // value is used only when x_p is finite).
        float xt[D], dh[D];
        if (a.mode == CS_CNN_SNS) {
            int64_t c0 = 0;
            #pragma unroll
            for (int k = D - 1; k >= 0; --k) {
                xt[k] = trunc_to_float(kPrefetch<D> ? f.x[lane * D + k] : __ldg(a.x + pp * D + k));
                c0 = c0 * m.pga[k] + cell_f32(xt[k], m.lo_h[k], m.pinv_sa[k], m.pga[k]);
            }
            if constexpr (D == 2) {
                const float2 v = __ldg(reinterpret_cast<const float2 *>(a.dhat) + c0);
                dh[0] = v.x;
                dh[D - 1] = v.y;
            } else {
                #pragma unroll
                for (int k = 0; k < D; ++k) dh[k] = __ldg(a.dhat + c0 * D + k);
            }
        }
        bool finite = true;
        #pragma unroll
        for (int k = 0; k < D; ++k) {
            const double xv = kPrefetch<D> ? f.x[lane * D + k] : __ldg(a.x + pp * D + k);
            const double uv = kPrefetch<D> ? f.u[lane * D + k] : __ldg(a.u + pp * D + k);
            xp[k] = __dsub_rn(xv, __dmul_rn(uv, a.dt));   // x_p = x - (u * dt)
            finite = finite && finite_bits(xp[k]);
            split_double(xp[k], xh[k], xl[k]);
        }
        int32_t plain;
        if (a.start_user) {
            const int32_t su = kPrefetch<D> ? f.start[lane] : __ldg(a.start_user + pp);
            plain = (su >= 0 && su < m.n_e) ? __ldg(m.iperm + su) : -1;
        } else {
            plain = kPrefetch<D> ? f.start[lane] : __ldg(m.node_elem + pp);
        }
        s = plain;
        int64_t c1 = -1;    // ASG cell whose seed starts the walk (ASG, CNN-SNS)
        if (finite && a.mode == CS_ASG_DIRECT) {
            c1 = grid_cell_f<D>(xp, xh, xl, m);
        } else if (finite && a.mode == CS_CNN_SNS) {
            // the ASG seed of y = x + dhat * (predictor cell size)
            c1 = 0;
            #pragma unroll
            for (int k = D - 1; k >= 0; --k) {
                const float y = __fadd_rn(xt[k], __fmul_rn(dh[k], m.psa_f[k]));
                c1 = c1 * m.ga[k] + cell_f32(y, m.lo_h[k], m.inv_sa[k], m.ga[k]);
            }
        }
        if (c1 >= 0) {
            const int32_t sd = __ldg(m.seed + c1);
            if (sd >= 0) s = sd;
        }
        if (!finite) {
            a.host[pp] = -1;
            a.path[pp] = 0;
            a.status[pp] = CS_INVALID;
            if (a.start_out) a.start_out[pp] = -1;
        } else if (s < 0) {
            // no start element: the exact search alone decides
            a.path[pp] = 0;
            if (a.start_out) a.start_out[pp] = -1;
            need_search = true;
        } else {
            entry = int32_t(pp);
            #pragma unroll
            for (int k = 0; k < D; ++k) {
                q.xp[k][lane] = xp[k];
                q.xh[k][lane] = xh[k];
                q.xl[k][lane] = xl[k];
            }
        }
    }
    q.p[lane] = entry;
    q.cur[lane] = s;
    for (unsigned want = __ballot_sync(kFull, need_search); want; want &= want - 1) {
        const int j = __ffs(want) - 1;
        const int32_t h = exact_search_lane<D>(m, xp, xh, xl, j, lane);
        if (lane == j) {
            a.host[pp] = h;
            a.status[pp] = h >= 0 ? CS_FOUND_VIA_FALLBACK : CS_OUTSIDE;
        }
    }
}

template <int D>
__global__ void __launch_bounds__(256, D == 2 ? 4 : 3) walk_kernel(const DevMesh m, const TrackArgs a,
                                                   int32_t *cursor, int32_t *next_cursor) {
    using WR = typename Recs<D>::W;
    using XR = typename Recs<D>::X;
    __shared__ Queue<D> queues[kWarps];
    __shared__ Prefetch<D> prefetched[kPrefetch<D> ? kWarps : 1];
    Queue<D> &q = queues[threadIdx.x >> 5];
    Prefetch<D> &f = prefetched[kPrefetch<D> ? threadIdx.x >> 5 : 0];
    const WR *__restrict__ rw = static_cast<const WR *>(m.recw);
    const XR *__restrict__ rx = static_cast<const XR *>(m.recx);
    const int lane = threadIdx.x & 31;
    const int64_t n = a.n;
    const float tau_f = static_cast<float>(m.tau) * 1.02f;

    int64_t p = -1;              // particle of this lane, -1 = idle
    double xp[D];
    float xh[D], xl[D];
    int32_t cur = -1, it = 0;
    int q_head = 0, q_n = 0;     // warp-uniform
    bool drained = false;        // warp-uniform: global cursor exhausted
    // nothing before this reads or writes global memory (launched with
    // programmatic dependent launch, the kernel may start while the kernel
    // before it, e.g. the predictor writing dhat, is finishing)
    pdl_wait();
    // the cursor of the next walk on this stream, which no one uses now
    if (blockIdx.x == 0 && threadIdx.x == 0) *next_cursor = 0;
    // Claim batches of 32 particles. Unsigned: n < 2^31 and the cursor
    // overshoots n by at most 32 per warp (one failed claim), so it cannot
    // wrap. With the prefetch the warp always holds its next batch in flight.
    unsigned nbase = 0;          // warp-uniform: base of the prefetched batch
    if (kPrefetch<D>) {
        if (lane == 0) nbase = atomicAdd(reinterpret_cast<unsigned *>(cursor), 32u);
        nbase = __shfl_sync(kFull, nbase, 0);
        if (int64_t(nbase) >= n)
            drained = true;
        else
            prefetch_batch<D>(m, a, int64_t(nbase), n, f, lane);
    }

    for (;;) {
        // ---- refill idle lanes from the warp's queue ----
        unsigned idle = __ballot_sync(kFull, p < 0);
        while (idle) {
            if (q_head >= q_n) {
                if (drained) break;
                unsigned base = nbase;
                if (!kPrefetch<D>) {
                    if (lane == 0) base = atomicAdd(reinterpret_cast<unsigned *>(cursor), 32u);
                    base = __shfl_sync(kFull, base, 0);
                    if (int64_t(base) >= n) {
                        drained = true;
                        break;
                    }
                }
                q_n = int(min(int64_t(32), n - base));
                if (kPrefetch<D>) asm volatile("cp.async.wait_all;" ::: "memory");
                __syncwarp();
                prepare<D>(m, a, int64_t(base) + lane, lane < q_n, q, f, lane);
                __syncwarp();
                if (kPrefetch<D>) {
                    // the buffer is read: claim the next batch and start its copies
                    if (lane == 0) nbase = atomicAdd(reinterpret_cast<unsigned *>(cursor), 32u);
                    nbase = __shfl_sync(kFull, nbase, 0);
                    if (int64_t(nbase) >= n)
                        drained = true;
                    else
                        prefetch_batch<D>(m, a, int64_t(nbase), n, f, lane);
                }
                q_head = 0;
            }
            const int take = min(__popc(idle), q_n - q_head);
            const int rank = __popc(idle & ((1u << lane) - 1u));
            if (((idle >> lane) & 1u) && rank < take) {
                const int slot = q_head + rank;
                const int32_t pp = q.p[slot];
                if (pp >= 0) {
                    p = pp;
                    cur = q.cur[slot];
                    it = 0;
                    #pragma unroll
                    for (int k = 0; k < D; ++k) {
                        xp[k] = q.xp[k][slot];
                        xh[k] = q.xh[k][slot];
                        xl[k] = q.xl[k][slot];
                    }
                }
            }
            q_head += take;
            idle = __ballot_sync(kFull, p < 0);
        }
        if (__ballot_sync(kFull, p >= 0) == 0) break;

        // ---- one step of Algorithm 1 for every busy lane ----
        bool done = false, search = false, found = false;
        if (p >= 0) {
            WalkE<D> e;
            load_walk(rw, cur, e);
            if (it == 0 && a.start_out) a.start_out[p] = e.uid;
            ++it;
            float lf[D + 1], T[D + 1];
            bary32<D>(e, xh, xl, lf, T);
            bool cin = true, cout = false;
            #pragma unroll
            for (int i = 0; i <= D; ++i) {
                cin = cin && (lf[i] - T[i] >= kNegEpsIn);
                cout = cout || (lf[i] + T[i] < kNegEpsOut);
            }
            // exit face in FP32: the smallest lf, certain when its upper bound is
            // below every other lower bound (then it is the unique FP64 minimum)
            int32_t next = e.nbr[0];
            float lj = lf[0], tj = T[0];
            #pragma unroll
            for (int i = 1; i <= D; ++i)
                if (lf[i] < lj) {
                    lj = lf[i];
                    tj = T[i];
                    next = e.nbr[i];
                }
            bool carg = true;
            int nmin = 0;
            #pragma unroll
            for (int i = 0; i <= D; ++i) {
                carg = carg && (lf[i] == lj || lj + tj < lf[i] - T[i]);
                nmin += (lf[i] == lj);
            }
            carg = carg && nmin == 1;

            // near: another element may contain x_p too, so the exact search
            // picks the lowest id. Not when the only face within tau is on the
            // mesh boundary: no element lies across it, and x_p is at least
            // tau inside every other face.
            bool inside, near = false;
            if (cin) {
                inside = true;
                int nnear = 0;
                bool inner = false;
                #pragma unroll
                for (int i = 0; i <= D; ++i) {
                    const bool ni = lf[i] - T[i] < tau_f;
                    nnear += ni;
                    inner = inner || (ni && e.nbr[i] >= 0);
                }
                near = nnear > 1 || inner;
            } else if (cout && carg) {
                inside = false;
            } else {
                // the filter cannot decide: FP64 arithmetic of the record
                double lam[D + 1];
                bary64(rx, cur, xp, lam);
                inside = true;
                #pragma unroll
                for (int i = 0; i <= D; ++i) inside = inside && (lam[i] >= -CS_EPS);
                if (inside) {
                    int nnear = 0;
                    bool inner = false;
                    #pragma unroll
                    for (int i = 0; i <= D; ++i) {
                        const bool ni = lam[i] < m.tau;
                        nnear += ni;
                        inner = inner || (ni && e.nbr[i] >= 0);
                    }
                    near = nnear > 1 || inner;
                } else {
                    // argmin, lowest index on equal minima (Eq. 5)
                    double lmin = lam[0];
                    next = e.nbr[0];
                    #pragma unroll
                    for (int i = 1; i <= D; ++i)
                        if (lam[i] < lmin) {
                            lmin = lam[i];
                            next = e.nbr[i];
                        }
                }
            }
            if (inside) {
                if (!near) a.host[p] = e.uid;
                a.path[p] = it;
                a.status[p] = CS_FOUND;
                done = found = true;
                search = near;      // another element may contain x_p too
            } else if (next < 0 || it >= m.cap) {
                a.path[p] = it;     // left the mesh or reached the step cap
                done = true;
                search = true;
            } else {
                cur = next;
            }
        }
        for (unsigned want = __ballot_sync(kFull, search); want; want &= want - 1) {
            const int j = __ffs(want) - 1;
            const int32_t h = exact_search_lane<D>(m, xp, xh, xl, j, lane);
            if (lane == j) {
                a.host[p] = h;
                if (!found) a.status[p] = h >= 0 ? CS_FOUND_VIA_FALLBACK : CS_OUTSIDE;
            }
        }
        if (done) p = -1;
    }
}

}  // namespace

int launch_track(const DevMesh &m, const TrackArgs &a, Scratch &s, int sm_count,
                 cudaStream_t st, Profiler *prof) {
    if (a.n == 0) return 0;
    // Two cursors used alternately: this walk's was zeroed by the walk before
    // it on the stream (or at allocation), and it zeroes the other one for
    // the walk after it. No memset node between the kernels of a step.
    int32_t *cursor = s.counters + s.parity, *next = s.counters + (s.parity ^ 1);
    s.parity ^= 1;
    static int per_sm[4] = {0, 0, 0, 0};
    if (!per_sm[m.dim]) {
        if (m.dim == 2)
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[2], walk_kernel<2>, 256, 0);
        else
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[3], walk_kernel<3>, 256, 0);
        if (per_sm[m.dim] < 1) per_sm[m.dim] = 1;
    }
    const int64_t need = (a.n + 255) / 256;
    const int grid = int(std::min<int64_t>(int64_t(sm_count) * per_sm[m.dim], need));
    const int ev = prof ? prof->begin(CS_STAGE_WALK, st) : -1;
    if (m.dim == 2)
        launch_pdl(walk_kernel<2>, dim3(grid), dim3(256), 0, st, m, a, cursor, next);
    else
        launch_pdl(walk_kernel<3>, dim3(grid), dim3(256), 0, st, m, a, cursor, next);
    // a walk that did not launch zeroed nothing: zero both cursors, so the
    // next call starts from a clean state whichever one it takes
    if (cudaPeekAtLastError() != cudaSuccess) cudaMemsetAsync(s.counters, 0, 2 * sizeof(int32_t), st);
    if (prof) prof->end(ev, st);
    return 1;
}

// ---------------------------------------------------------------------------
// Allocation-free tracking (cs_track_noalloc).
//
// Some callers cannot let this library allocate device memory during a call:
// a host solver that owns all device memory through its own pool, or a time-
// step loop that must not pay the implicit device synchronisation that
// cudaMalloc / cudaFree can cause. For them the walk's only scratch, its
// work cursor, lives in this fixed, file-scope device array instead of the
// context's scratch buffers. Every GPU that loads the library holds it (256
// bytes) until the process exits.
// ---------------------------------------------------------------------------
namespace {

// [0], [1] the walk's alternate work cursors (zero at load); the rest is
// padding to one 256-byte line
static __device__ __align__(256) int32_t g_noalloc_scratch[64];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
int32_t *g_noalloc_ptr[kMaxDevices] = {};
int g_noalloc_parity[kMaxDevices] = {};    // cursor of the next call per device

}  // namespace

}  // namespace cs

extern "C" cs_status cs_track_noalloc(cs_ctx *ctx, int32_t mesh_id, int32_t field_id, int64_t n,
                                      const double *x, const double *u, double dt,
                                      const int32_t *start, int mode, int32_t *host_out,
                                      int32_t *path_len_out, uint8_t *status_out,
                                      int32_t *start_out, void *stream) {
    using namespace cs;
    (void)field_id;   // only CS_CNN_SNS reads a field, and it is refused below
    if (!ctx) return CS_EINVAL;
    auto it = ctx->meshes.find(mesh_id);
    if (it == ctx->meshes.end()) {
        ctx->err = "cs_track_noalloc: unknown mesh id";
        return CS_ENOMESH;
    }
    const Mesh *mesh = it->second;
    if (mode != CS_SNS && mode != CS_ASG_DIRECT && mode != CS_CNN_SNS) {
        ctx->err = "cs_track_noalloc: unknown mode";
        return CS_EINVAL;
    }
    if (n < 0 || n >= (int64_t(1) << 31) - 1) {
        ctx->err = "cs_track_noalloc: n = " + std::to_string(n) +
                   " is outside [0, 2^31 - 2]";
        return CS_EINVAL;
    }
    // the start predictor writes a displacement grid the library would have
    // to allocate: use cs_track_dhat with a caller-owned grid instead
    if (mode == CS_CNN_SNS) {
        ctx->err = "cs_track_noalloc: CS_CNN_SNS is not supported (its predicted displacement "
                   "grid needs device memory); use cs_track_dhat with a caller-owned grid";
        return CS_EINVAL;
    }
    if (n == 0) return CS_OK;
    if (!x || !u || !host_out || !path_len_out || !status_out) {
        ctx->err = "cs_track_noalloc: null pointer";
        return CS_EINVAL;
    }
    if (!start && n != mesh->d.n_v) {
        ctx->err = "cs_track_noalloc: start == NULL needs n == n_vertices";
        return CS_EINVAL;
    }
    if (ctx->device < 0 || ctx->device >= kMaxDevices) {
        ctx->err = "cs_track_noalloc: device ordinal out of range";
        return CS_EINVAL;
    }
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) {
        ctx->err = std::string("cs_track_noalloc: cudaSetDevice: ") + cudaGetErrorString(e);
        return CS_ECUDA;
    }
    // once per device, with that device current: the device address of the
    // array (its name in host code is only a host-side stand-in)
    int32_t *base = nullptr;
    Scratch s;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        if (!g_noalloc_ptr[ctx->device]) {
            void *ptr = nullptr;
            e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
            if (e != cudaSuccess) {
                ctx->err = std::string("cs_track_noalloc: cudaGetSymbolAddress: ") +
                           cudaGetErrorString(e);
                return CS_ECUDA;
            }
            g_noalloc_ptr[ctx->device] = static_cast<int32_t *>(ptr);
        }
        base = g_noalloc_ptr[ctx->device];
        s.counters = base;
        s.parity = g_noalloc_parity[ctx->device];
        // n > 0 here, so launch_track launches the walk and flips the cursor
        g_noalloc_parity[ctx->device] ^= 1;
    }
    TrackArgs a{};
    a.n = n;
    a.x = x;
    a.u = u;
    a.dt = dt;
    a.start_user = start;
    a.mode = mode;
    a.dhat = nullptr;
    a.host = host_out;
    a.path = path_len_out;
    a.status = status_out;
    a.start_out = start_out;
    ctx->launches += launch_track(mesh->d, a, s, ctx->sm_count, static_cast<cudaStream_t>(stream),
                                  nullptr);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        ctx->err = std::string("cs_track_noalloc: launch: ") + cudaGetErrorString(e);
        return CS_ECUDA;
    }
    return CS_OK;
}
