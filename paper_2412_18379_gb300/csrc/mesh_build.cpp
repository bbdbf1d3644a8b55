// Host-side preprocessing of an uploaded mesh (done once per mesh).
//
// Builds, in this order: the inverse-affine matrix of every element (the
// barycentric coordinates of Sec. 2.2 solved once per element), the
// neighbour table m_i^l (Sec. 2.2), the plain-SNS start of every vertex
// (Sec. 2.1, Eq. 4), a Hilbert order of the element centroids (internal
// ids), the exact-search bucket index and the ASG grid geometry (Sec. 1,
// 2.3). Compiled with -ffp-contract=off: every rounding of the inverse-affine
// arithmetic is the one written here.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>

#include "internal.h"

namespace cs {
namespace {

// Inverse-affine form: lambda_{1..d} = M (x - v0), M = adj(T) * (1/det T),
// T = [v1 - v0, ..., vd - v0] as columns. Cofactors are (p*q) - (r*s), det is
// the first-row expansion ((a*C00 + b*C01) + c*C02). Returns false on det == 0
// or a non-finite det.
bool inverse_affine(int dim, const double *p[4], double *v0, double *m) {
    for (int k = 0; k < dim; ++k) v0[k] = p[0][k];
    if (dim == 2) {
        const double a = p[1][0] - p[0][0], b = p[2][0] - p[0][0];
        const double c = p[1][1] - p[0][1], d = p[2][1] - p[0][1];
        const double det = a * d - b * c;
        if (!(det != 0.0) || !std::isfinite(det)) return false;
        const double inv = 1.0 / det;
        m[0] = d * inv;
        m[1] = (-b) * inv;
        m[2] = (-c) * inv;
        m[3] = a * inv;
        return true;
    }
    const double t00 = p[1][0] - p[0][0], t01 = p[2][0] - p[0][0], t02 = p[3][0] - p[0][0];
    const double t10 = p[1][1] - p[0][1], t11 = p[2][1] - p[0][1], t12 = p[3][1] - p[0][1];
    const double t20 = p[1][2] - p[0][2], t21 = p[2][2] - p[0][2], t22 = p[3][2] - p[0][2];
    const double c00 = t11 * t22 - t12 * t21;
    const double c01 = t12 * t20 - t10 * t22;
    const double c02 = t10 * t21 - t11 * t20;
    const double c10 = t02 * t21 - t01 * t22;
    const double c11 = t00 * t22 - t02 * t20;
    const double c12 = t01 * t20 - t00 * t21;
    const double c20 = t01 * t12 - t02 * t11;
    const double c21 = t02 * t10 - t00 * t12;
    const double c22 = t00 * t11 - t01 * t10;
    const double det = (t00 * c00 + t01 * c01) + t02 * c02;
    if (!(det != 0.0) || !std::isfinite(det)) return false;
    const double inv = 1.0 / det;
    // M = transpose of the cofactor matrix, scaled
    m[0] = c00 * inv; m[1] = c10 * inv; m[2] = c20 * inv;
    m[3] = c01 * inv; m[4] = c11 * inv; m[5] = c21 * inv;
    m[6] = c02 * inv; m[7] = c12 * inv; m[8] = c22 * inv;
    return true;
}

// lambda of point x in the element (v0, m): same rounding order as the walk.
void bary(int dim, const double *v0, const double *m, const double *x, double *lam) {
    if (dim == 2) {
        const double dx = x[0] - v0[0], dy = x[1] - v0[1];
        const double l1 = m[0] * dx + m[1] * dy;
        const double l2 = m[2] * dx + m[3] * dy;
        lam[0] = (1.0 - l1) - l2; lam[1] = l1; lam[2] = l2;
    } else {
        const double dx = x[0] - v0[0], dy = x[1] - v0[1], dz = x[2] - v0[2];
        const double l1 = (m[0] * dx + m[1] * dy) + m[2] * dz;
        const double l2 = (m[3] * dx + m[4] * dy) + m[5] * dz;
        const double l3 = (m[6] * dx + m[7] * dy) + m[8] * dz;
        lam[0] = ((1.0 - l1) - l2) - l3; lam[1] = l1; lam[2] = l2; lam[3] = l3;
    }
}

// Hilbert index of integer coordinates x[0..n-1] of b bits each, after
// J. Skilling, "Programming the Hilbert curve" (AIP Conf. Proc. 707, 2004):
// convert the axes to the transposed Hilbert form in place, then interleave
// the bits, most significant first.
uint64_t hilbert_key(uint32_t *x, int n, int b) {
    const uint32_t top = 1u << (b - 1);
    for (uint32_t q = top; q > 1; q >>= 1) {
        const uint32_t lowmask = q - 1;
        for (int i = 0; i < n; ++i) {
            if (x[i] & q) {
                x[0] ^= lowmask;                       // invert low bits of x[0]
            } else {
                const uint32_t t = (x[0] ^ x[i]) & lowmask;  // swap low bits
                x[0] ^= t;
                x[i] ^= t;
            }
        }
    }
    for (int i = 1; i < n; ++i) x[i] ^= x[i - 1];      // Gray encode
    uint32_t t = 0;
    for (uint32_t q = top; q > 1; q >>= 1)
        if (x[n - 1] & q) t ^= q - 1;
    for (int i = 0; i < n; ++i) x[i] ^= t;
    uint64_t key = 0;
    for (int bit = b - 1; bit >= 0; --bit)
        for (int i = 0; i < n; ++i) key = (key << 1) | ((x[i] >> bit) & 1u);
    return key;
}

}  // namespace

cs_status build_host_mesh(int dim, int64_t n_v, const double *xyz, int64_t n_e,
                          const int32_t *conn_user, const int32_t *asg_grid, HostMesh &H,
                          std::string &msg) {
    const int nv = dim + 1;
    H.dim = dim;
    H.n_v = n_v;
    H.n_e = n_e;
    if (n_e >= (int64_t(1) << 31) - 1 || n_v >= (int64_t(1) << 31) - 1) {
        msg = "mesh too large for 32-bit ids";
        return CS_EINVAL;
    }
    for (int64_t k = 0; k < n_e * nv; ++k)
        if (conn_user[k] < 0 || conn_user[k] >= n_v) {
            msg = "connectivity entry " + std::to_string(k) + " out of range";
            return CS_EMESH;
        }
    for (int64_t k = 0; k < n_v * dim; ++k)
        if (!std::isfinite(xyz[k])) {
            msg = "vertex coordinate " + std::to_string(k) + " is not finite";
            return CS_EMESH;
        }

    // ---- inverse-affine matrices (user order) ----
    const int md = dim * dim;
    std::vector<double> v0(static_cast<size_t>(n_e) * dim), M(static_cast<size_t>(n_e) * md);
    double hmin = INFINITY, diam = 0.0;
    for (int64_t l = 0; l < n_e; ++l) {
        const double *p[4];
        for (int i = 0; i < nv; ++i) p[i] = xyz + int64_t(conn_user[l * nv + i]) * dim;
        if (!inverse_affine(dim, p, &v0[l * dim], &M[l * md])) {
            msg = "degenerate element " + std::to_string(l) + " (det == 0)";
            return CS_EMESH;
        }
        // height of vertex i over face i = 1 / |grad lambda_i|
        const double *m = &M[l * md];
        double g0[3] = {0, 0, 0};
        for (int k = 0; k < dim; ++k) {
            double s = 0;
            for (int j = 0; j < dim; ++j) {
                s += m[k * dim + j] * m[k * dim + j];
                g0[j] -= m[k * dim + j];
            }
            hmin = std::min(hmin, 1.0 / std::sqrt(s));
        }
        double s0 = 0;
        for (int j = 0; j < dim; ++j) s0 += g0[j] * g0[j];
        hmin = std::min(hmin, 1.0 / std::sqrt(s0));
        for (int i = 0; i < nv; ++i)
            for (int j = i + 1; j < nv; ++j) {
                double s = 0;
                for (int k = 0; k < dim; ++k) {
                    const double d = p[i][k] - p[j][k];
                    s += d * d;
                }
                diam = std::max(diam, std::sqrt(s));
            }
    }

    // ---- neighbours: faces grouped by their smallest vertex ----
    std::vector<int32_t> nbr_user(static_cast<size_t>(n_e) * nv, -1);
    {
        std::vector<int64_t> off(static_cast<size_t>(n_v) + 1, 0);
        auto face_verts = [&](int64_t l, int i, int32_t *f) {
            int q = 0;
            for (int k = 0; k < nv; ++k)
                if (k != i) f[q++] = conn_user[l * nv + k];
            for (int a = 1; a < dim; ++a)          // sort the dim face vertices
                for (int b = a; b > 0 && f[b - 1] > f[b]; --b) std::swap(f[b - 1], f[b]);
        };
        for (int64_t l = 0; l < n_e; ++l)
            for (int i = 0; i < nv; ++i) {
                int32_t f[3];
                face_verts(l, i, f);
                off[f[0] + 1]++;
            }
        for (int64_t v = 0; v < n_v; ++v) off[v + 1] += off[v];
        struct FaceRef { int32_t b, c, elem, local; };
        std::vector<FaceRef> faces(static_cast<size_t>(off[n_v]));
        std::vector<int64_t> fill(off.begin(), off.end() - 1);
        for (int64_t l = 0; l < n_e; ++l)
            for (int i = 0; i < nv; ++i) {
                int32_t f[3] = {0, 0, 0};
                face_verts(l, i, f);
                faces[fill[f[0]]++] = FaceRef{f[1], dim == 3 ? f[2] : 0, int32_t(l), i};
            }
        for (int64_t v = 0; v < n_v; ++v) {
            auto b = faces.begin() + off[v], e = faces.begin() + off[v + 1];
            std::sort(b, e, [](const FaceRef &x, const FaceRef &y) {
                return x.b != y.b ? x.b < y.b : x.c < y.c;
            });
            for (auto it = b; it != e;) {
                auto jt = it + 1;
                while (jt != e && jt->b == it->b && jt->c == it->c) ++jt;
                const auto cnt = jt - it;
                if (cnt > 2) {
                    msg = "face shared by more than two elements (element " +
                          std::to_string(it->elem) + ")";
                    return CS_EMESH;
                }
                if (cnt == 2) {
                    nbr_user[int64_t(it[0].elem) * nv + it[0].local] = it[1].elem;
                    nbr_user[int64_t(it[1].elem) * nv + it[1].local] = it[0].elem;
                }
                it = jt;
            }
        }
    }

    // ---- plain-SNS start: lowest user id owning each vertex ----
    H.node_elem.assign(size_t(n_v), -1);
    for (int64_t l = 0; l < n_e; ++l)
        for (int i = 0; i < nv; ++i) {
            int32_t &s = H.node_elem[conn_user[l * nv + i]];
            if (s < 0) s = int32_t(l);
        }

    // ---- bounding box, grids ----
    for (int k = 0; k < dim; ++k) {
        H.lo[k] = INFINITY;
        H.hi[k] = -INFINITY;
    }
    for (int64_t v = 0; v < n_v; ++v)
        for (int k = 0; k < dim; ++k) {
            H.lo[k] = std::min(H.lo[k], xyz[v * dim + k]);
            H.hi[k] = std::max(H.hi[k], xyz[v * dim + k]);
        }
    double ext = 0;
    for (int k = 0; k < dim; ++k) {
        if (!(H.hi[k] > H.lo[k])) {
            msg = "mesh has zero extent along an axis";
            return CS_EMESH;
        }
        ext = std::max(ext, H.hi[k] - H.lo[k]);
    }
    const int32_t gdef = std::max<int32_t>(1, int32_t(std::llround(std::pow(double(n_v), 1.0 / dim))) - 1);
    int64_t n_asg = 1;
    for (int k = 0; k < dim; ++k) {
        H.ga[k] = asg_grid ? asg_grid[k] : gdef;
        if (H.ga[k] < 1 || H.ga[k] > (1 << 20)) {
            msg = "ASG grid size out of range";
            return CS_EINVAL;
        }
        H.sa[k] = (H.hi[k] - H.lo[k]) / double(H.ga[k]);
        n_asg *= H.ga[k];
    }
    if (n_asg > (int64_t(1) << 31) - 1) {
        msg = "ASG grid has too many cells";
        return CS_EINVAL;
    }
    // bucket grid: about 4 triangles / 32 tetrahedra of box overlap per cell
    const double per = dim == 2 ? 4.0 : 32.0;
    const int32_t gb = std::max<int32_t>(1, int32_t(std::llround(std::pow(double(n_e) / per, 1.0 / dim))));
    for (int k = 0; k < dim; ++k) {
        H.gb[k] = gb;
        H.sb[k] = (H.hi[k] - H.lo[k]) / double(gb);
    }
    H.margin = 1e-7 * ext;
    // Walk ends in K with every lambda_i >= tau: x_p is then farther than
    // tau * h_min from every face of K, while any other element containing
    // x_p to within eps lies within (dim+1) * eps * diam of it.
    H.tau = std::max(1e-9, 10.0 * (dim + 1) * CS_EPS * diam / hmin + 1e-12);
    H.cap = int32_t(8 * std::llround(std::pow(double(n_e), 1.0 / dim)) + 64);

    // ---- Hilbert order of centroids ----
    std::vector<double> cent(static_cast<size_t>(n_e) * dim);
    std::vector<std::pair<uint64_t, int32_t>> keys(static_cast<size_t>(n_e));
    const int bits = dim == 2 ? 31 : 21;
    const double qmax = double((1u << bits) - 1);
    for (int64_t l = 0; l < n_e; ++l) {
        uint32_t q[3];
        for (int k = 0; k < dim; ++k) {
            double s = 0;
            for (int i = 0; i < nv; ++i) s += xyz[int64_t(conn_user[l * nv + i]) * dim + k];
            s /= nv;
            cent[l * dim + k] = s;
            double t = (s - H.lo[k]) / (H.hi[k] - H.lo[k]) * qmax;
            t = std::min(std::max(t, 0.0), qmax);
            q[k] = uint32_t(t);
        }
        keys[l] = {hilbert_key(q, dim, bits), int32_t(l)};
    }
    // ---- average pooling of the element centroids per ASG cell (Sec. 2.3) ----
    // The classifier's input: per cell the mean centroid of the elements
    // whose centroid lies in the cell (FP64, summed in user-id order), NaN
    // where no centroid lies in it.
    {
        std::vector<int32_t> cnt(static_cast<size_t>(n_asg), 0);
        H.pool.assign(static_cast<size_t>(n_asg) * dim, 0.0);
        for (int64_t l = 0; l < n_e; ++l) {
            int64_t c = 0;
            for (int k = dim - 1; k >= 0; --k) {
                const double t = std::floor((cent[l * dim + k] - H.lo[k]) / H.sa[k]);
                int64_t i = 0;
                if (t >= 0.0) i = t > double(H.ga[k] - 1) ? H.ga[k] - 1 : int64_t(t);
                c = c * H.ga[k] + i;
            }
            cnt[c] += 1;
            for (int k = 0; k < dim; ++k) H.pool[c * dim + k] += cent[l * dim + k];
        }
        for (int64_t c = 0; c < n_asg; ++c)
            for (int k = 0; k < dim; ++k)
                H.pool[c * dim + k] = cnt[c] > 0 ? H.pool[c * dim + k] / double(cnt[c]) : NAN;
        // the same values as float hi + lo pairs (lo = the remainder rounded)
        H.pool_f.resize(H.pool.size() * 2);
        for (size_t i = 0; i < H.pool.size(); ++i) {
            const float hi = static_cast<float>(H.pool[i]);
            H.pool_f[2 * i] = hi;
            H.pool_f[2 * i + 1] = std::isnan(H.pool[i]) ? 0.f
                                                        : static_cast<float>(H.pool[i] - double(hi));
        }
    }
    std::sort(keys.begin(), keys.end());
    H.order.resize(size_t(n_e));
    H.iperm.resize(size_t(n_e));
    for (int64_t i = 0; i < n_e; ++i) {
        H.order[i] = keys[i].second;
        H.iperm[keys[i].second] = int32_t(i);
    }
    keys.clear();
    keys.shrink_to_fit();

    // ---- records, connectivity and centroids in internal order ----
    // walk record: v0 as float hi + lo (hi = v0 rounded to float, lo = the
    // remainder v0 - hi rounded to float), M rounded to float
    const size_t wb = dim == 2 ? sizeof(WalkRec2) : sizeof(WalkRec3);
    const size_t xb = dim == 2 ? sizeof(ExactRec2) : sizeof(ExactRec3);
    H.recw.assign(size_t(n_e) * wb, 0);
    H.recx.assign(size_t(n_e) * xb, 0);
    H.conn.resize(size_t(n_e) * nv);
    H.centroid.resize(size_t(n_e) * dim);
    auto split = [](double v, float &hi, float &lo) {
        hi = static_cast<float>(v);
        lo = static_cast<float>(v - static_cast<double>(hi));
    };
    for (int64_t i = 0; i < n_e; ++i) {
        const int64_t l = H.order[i];
        if (dim == 2) {
            WalkRec2 w{};
            ExactRec2 x{};
            std::memcpy(x.v0, &v0[l * 2], sizeof(x.v0));
            std::memcpy(x.m, &M[l * 4], sizeof(x.m));
            for (int k = 0; k < 2; ++k) split(v0[l * 2 + k], w.vh[k], w.vl[k]);
            for (int k = 0; k < 4; ++k) w.m[k] = static_cast<float>(M[l * 4 + k]);
            for (int f = 0; f < 3; ++f) {
                const int32_t n = nbr_user[l * 3 + f];
                w.nbr[f] = n < 0 ? -1 : H.iperm[n];
            }
            w.uid = int32_t(l);
            std::memcpy(&H.recw[size_t(i) * wb], &w, wb);
            std::memcpy(&H.recx[size_t(i) * xb], &x, xb);
        } else {
            WalkRec3 w{};
            ExactRec3 x{};
            std::memcpy(x.v0, &v0[l * 3], sizeof(x.v0));
            std::memcpy(x.m, &M[l * 9], sizeof(x.m));
            for (int k = 0; k < 3; ++k) split(v0[l * 3 + k], w.vh[k], w.vl[k]);
            for (int k = 0; k < 9; ++k) w.m[k] = static_cast<float>(M[l * 9 + k]);
            for (int f = 0; f < 4; ++f) {
                const int32_t n = nbr_user[l * 4 + f];
                w.nbr[f] = n < 0 ? -1 : H.iperm[n];
            }
            w.uid = int32_t(l);
            std::memcpy(&H.recw[size_t(i) * wb], &w, wb);
            std::memcpy(&H.recx[size_t(i) * xb], &x, xb);
        }
        for (int k = 0; k < nv; ++k) H.conn[i * nv + k] = conn_user[l * nv + k];
        for (int k = 0; k < dim; ++k) H.centroid[i * dim + k] = cent[l * dim + k];
    }

    // ---- exact-search bucket index (internal ids) ----
    // An element is listed in every bucket cell its margin-grown bounding box
    // overlaps, unless one of its face planes separates it from the (grown)
    // cell: then lambda_i < -1e-9 on all cell corners, so no point of the
    // cell is contained in it even with the eps tolerance.
    {
        int64_t ncell = 1;
        for (int k = 0; k < dim; ++k) ncell *= H.gb[k];
        std::vector<int64_t> cnt(static_cast<size_t>(ncell) + 1, 0);
        std::vector<std::pair<int64_t, int32_t>> pairs;
        pairs.reserve(size_t(n_e) * (dim == 2 ? 4 : 8));
        for (int64_t i = 0; i < n_e; ++i) {
            const int64_t l = H.order[i];
            int32_t ia[3] = {0, 0, 0}, ib[3] = {0, 0, 0};
            for (int k = 0; k < dim; ++k) {
                double a = INFINITY, b = -INFINITY;
                for (int v = 0; v < nv; ++v) {
                    const double c = xyz[int64_t(conn_user[l * nv + v]) * dim + k];
                    a = std::min(a, c);
                    b = std::max(b, c);
                }
                int64_t x0 = int64_t(std::floor((a - H.margin - H.lo[k]) / H.sb[k]));
                int64_t x1 = int64_t(std::floor((b + H.margin - H.lo[k]) / H.sb[k]));
                ia[k] = int32_t(std::max<int64_t>(0, std::min<int64_t>(x0, H.gb[k] - 1)));
                ib[k] = int32_t(std::max<int64_t>(0, std::min<int64_t>(x1, H.gb[k] - 1)));
            }
            for (int32_t z = ia[2]; z <= ib[2]; ++z)
                for (int32_t y = ia[1]; y <= ib[1]; ++y)
                    for (int32_t x = ia[0]; x <= ib[0]; ++x) {
                        const int32_t c3[3] = {x, y, z};
                        // corners of the grown cell
                        bool separated = false;
                        double lamc[8][4];
                        const int ncorner = 1 << dim;
                        for (int cn = 0; cn < ncorner; ++cn) {
                            double pt[3];
                            for (int k = 0; k < dim; ++k) {
                                const int32_t ck = c3[k] + ((cn >> k) & 1);
                                pt[k] = H.lo[k] + double(ck) * H.sb[k] +
                                        (((cn >> k) & 1) ? H.margin : -H.margin);
                            }
                            bary(dim, &v0[l * dim], &M[l * md], pt, lamc[cn]);
                        }
                        for (int f = 0; f < nv && !separated; ++f) {
                            bool all_neg = true;
                            for (int cn = 0; cn < ncorner; ++cn)
                                if (!(lamc[cn][f] < -1e-9)) all_neg = false;
                            separated = all_neg;
                        }
                        if (separated) continue;
                        const int64_t c = dim == 2 ? int64_t(y) * H.gb[0] + x
                                                   : (int64_t(z) * H.gb[1] + y) * H.gb[0] + x;
                        pairs.emplace_back(c, int32_t(i));
                        cnt[c + 1]++;
                    }
        }
        if (pairs.size() >= size_t((int64_t(1) << 31) - 1)) {
            msg = "bucket index too large";
            return CS_ENOMEM;
        }
        for (int64_t c = 0; c < ncell; ++c) cnt[c + 1] += cnt[c];
        H.bstart.resize(size_t(ncell) + 1);
        for (int64_t c = 0; c <= ncell; ++c) H.bstart[c] = int32_t(cnt[c]);
        H.bitems.resize(pairs.size());
        std::vector<int64_t> fill(cnt.begin(), cnt.end() - 1);
        for (const auto &pr : pairs) H.bitems[fill[pr.first]++] = pr.second;
    }
    return CS_OK;
}

}  // namespace cs
