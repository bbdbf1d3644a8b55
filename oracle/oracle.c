/*
 * CPU oracle for the particle-location path of the CNN-SNS method.
 * TEST INFRASTRUCTURE ONLY -- see oracle.h. Built with -ffp-contract=off so
 * that no product is fused into an addition: every rounding is the one the
 * source text shows.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* Threads of the particle loops of or_walk and or_locate_bucketed (OpenMP,
 * when the library is built with it). The particles are independent, so the
 * results do not depend on the count; it is 1 unless or_set_threads raises
 * it (the benchmark's all-core CPU baseline). */
static int g_threads = 1;

int or_set_threads(int n)
{
#ifdef _OPENMP
    g_threads = n > 0 ? n : 1;
#else
    (void)n;
    g_threads = 1;
#endif
    return g_threads;
}

/* ------------------------------------------------------------------------ */
/* Neighbour table (Sec. 2.2: m_1^l..m_4^l, -1 for a boundary face)          */
/* ------------------------------------------------------------------------ */

typedef struct {
    int32_t v[3];   /* sorted vertex ids of the face (dim entries used) */
    int32_t elem;
    int32_t local;  /* face index = index of the opposite vertex */
} face_rec;

static int g_face_dim;

static int face_cmp(const void *a, const void *b)
{
    const face_rec *x = (const face_rec *)a, *y = (const face_rec *)b;
    for (int k = 0; k < g_face_dim; ++k) {
        if (x->v[k] < y->v[k]) return -1;
        if (x->v[k] > y->v[k]) return 1;
    }
    if (x->elem != y->elem) return x->elem < y->elem ? -1 : 1;
    return x->local - y->local;
}

static void sort_small(int32_t *a, int n)
{
    for (int i = 1; i < n; ++i)
        for (int j = i; j > 0 && a[j - 1] > a[j]; --j) {
            int32_t t = a[j]; a[j] = a[j - 1]; a[j - 1] = t;
        }
}

int or_neighbors(int dim, int64_t n_e, const int32_t *conn, int32_t *nbr)
{
    const int nv = dim + 1;
    int64_t nf = n_e * nv;
    face_rec *f = (face_rec *)malloc((size_t)(nf > 0 ? nf : 1) * sizeof(face_rec));
    if (!f) return -2;
    for (int64_t l = 0; l < n_e; ++l)
        for (int i = 0; i < nv; ++i) {
            face_rec *r = &f[l * nv + i];
            int m = 0;
            for (int k = 0; k < nv; ++k)
                if (k != i) r->v[m++] = conn[l * nv + k];
            sort_small(r->v, dim);
            r->elem = (int32_t)l;
            r->local = i;
            nbr[l * nv + i] = -1;
        }
    g_face_dim = dim;
    qsort(f, (size_t)nf, sizeof(face_rec), face_cmp);
    int64_t i = 0;
    int rc = 0;
    while (i < nf) {
        int64_t j = i + 1;
        while (j < nf && memcmp(f[j].v, f[i].v, (size_t)dim * sizeof(int32_t)) == 0) ++j;
        if (j - i == 2) {
            nbr[(int64_t)f[i].elem * nv + f[i].local] = f[i + 1].elem;
            nbr[(int64_t)f[i + 1].elem * nv + f[i + 1].local] = f[i].elem;
        } else if (j - i > 2) {
            rc = -1;
        }
        i = j;
    }
    free(f);
    return rc;
}

int or_neighbors_bruteforce(int dim, int64_t n_e, const int32_t *conn, int32_t *nbr)
{
    const int nv = dim + 1;
    for (int64_t l = 0; l < n_e; ++l)
        for (int i = 0; i < nv; ++i) {
            int found = 0;
            nbr[l * nv + i] = -1;
            for (int64_t m = 0; m < n_e; ++m) {
                if (m == l) continue;
                /* face i of l = all vertices of l but vertex i; shared iff
                 * every one of them is a vertex of m */
                int shared = 1;
                for (int k = 0; k < nv && shared; ++k) {
                    if (k == i) continue;
                    int hit = 0;
                    for (int q = 0; q < nv; ++q)
                        if (conn[m * nv + q] == conn[l * nv + k]) hit = 1;
                    shared = hit;
                }
                if (shared) {
                    ++found;
                    nbr[l * nv + i] = (int32_t)m;
                }
            }
            if (found > 1) return -1;
        }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Barycentric coordinates (Sec. 2.2)                                        */
/*                                                                          */
/* The paper defines lambda_i = |S_i|/|S_0|. Solved once per element, the   */
/* same coordinates are lambda_{1..d} = T^{-1} (x_p - v0), T the matrix of  */
/* edge columns v_k - v0, and lambda_0 = 1 - sum_k lambda_k. The reading    */
/* fixes every rounding: cofactors as (p*q) - (r*s), det by expansion along */
/* the first row, M = cofactor^T * (1/det), lambda_k summed left to right,  */
/* lambda_0 = ((1 - l1) - l2) - l3.                                          */
/* ------------------------------------------------------------------------ */

int64_t or_inverse_affine(int dim, const double *xyz, int64_t n_e,
                          const int32_t *conn, double *v0, double *M)
{
    const int nv = dim + 1;
    for (int64_t l = 0; l < n_e; ++l) {
        const int32_t *c = conn + l * nv;
        const double *p0 = xyz + (int64_t)c[0] * dim;
        double *o = v0 + l * dim;
        double *m = M + l * dim * dim;
        for (int k = 0; k < dim; ++k) o[k] = p0[k];
        if (dim == 2) {
            const double *p1 = xyz + (int64_t)c[1] * 2, *p2 = xyz + (int64_t)c[2] * 2;
            double a = p1[0] - p0[0], b = p2[0] - p0[0];
            double cc = p1[1] - p0[1], d = p2[1] - p0[1];
            double det = a * d - b * cc;
            if (!(det != 0.0) || !isfinite(det)) return l + 1;
            double inv = 1.0 / det;
            m[0] = d * inv;
            m[1] = (-b) * inv;
            m[2] = (-cc) * inv;
            m[3] = a * inv;
        } else {
            const double *p1 = xyz + (int64_t)c[1] * 3, *p2 = xyz + (int64_t)c[2] * 3,
                         *p3 = xyz + (int64_t)c[3] * 3;
            /* T = [[a b c],[d e f],[g h i]], column k-1 = v_k - v0 */
            double a = p1[0] - p0[0], b = p2[0] - p0[0], cx = p3[0] - p0[0];
            double d = p1[1] - p0[1], e = p2[1] - p0[1], f = p3[1] - p0[1];
            double g = p1[2] - p0[2], h = p2[2] - p0[2], i = p3[2] - p0[2];
            double C00 = e * i - f * h;
            double C01 = f * g - d * i;
            double C02 = d * h - e * g;
            double C10 = cx * h - b * i;
            double C11 = a * i - cx * g;
            double C12 = b * g - a * h;
            double C20 = b * f - cx * e;
            double C21 = cx * d - a * f;
            double C22 = a * e - b * d;
            double det = (a * C00 + b * C01) + cx * C02;
            if (!(det != 0.0) || !isfinite(det)) return l + 1;
            double inv = 1.0 / det;
            m[0] = C00 * inv; m[1] = C10 * inv; m[2] = C20 * inv;
            m[3] = C01 * inv; m[4] = C11 * inv; m[5] = C21 * inv;
            m[6] = C02 * inv; m[7] = C12 * inv; m[8] = C22 * inv;
        }
    }
    return 0;
}

void or_bary(int dim, const double *v0, const double *M, const double *p,
             double *lam)
{
    if (dim == 2) {
        double dx = p[0] - v0[0], dy = p[1] - v0[1];
        double l1 = M[0] * dx + M[1] * dy;
        double l2 = M[2] * dx + M[3] * dy;
        lam[1] = l1;
        lam[2] = l2;
        lam[0] = (1.0 - l1) - l2;
    } else {
        double dx = p[0] - v0[0], dy = p[1] - v0[1], dz = p[2] - v0[2];
        double l1 = (M[0] * dx + M[1] * dy) + M[2] * dz;
        double l2 = (M[3] * dx + M[4] * dy) + M[5] * dz;
        double l3 = (M[6] * dx + M[7] * dy) + M[8] * dz;
        lam[1] = l1;
        lam[2] = l2;
        lam[3] = l3;
        lam[0] = ((1.0 - l1) - l2) - l3;
    }
}

/* determinant of an n x n matrix (n <= 4) by Laplace expansion; a pin only */
static double det_n(int n, const double *a)
{
    if (n == 1) return a[0];
    if (n == 2) return a[0] * a[3] - a[1] * a[2];
    double sub[9], s = 0.0;
    for (int c = 0; c < n; ++c) {
        int q = 0;
        for (int r = 1; r < n; ++r)
            for (int k = 0; k < n; ++k)
                if (k != c) sub[q++] = a[r * n + k];
        double t = a[c] * det_n(n - 1, sub);
        s += (c & 1) ? -t : t;
    }
    return s;
}

void or_bary_det(int dim, const double *verts, const double *p, double *lam)
{
    const int n = dim + 1;
    double S0[16] = {0}, Si[16];
    for (int col = 0; col < n; ++col) {
        S0[0 * n + col] = 1.0;
        for (int k = 0; k < dim; ++k) S0[(k + 1) * n + col] = verts[col * dim + k];
    }
    double d0 = det_n(n, S0);
    for (int i = 0; i < n; ++i) {
        memcpy(Si, S0, sizeof(double) * (size_t)(n * n));
        Si[0 * n + i] = 1.0;
        for (int k = 0; k < dim; ++k) Si[(k + 1) * n + i] = p[k];
        lam[i] = det_n(n, Si) / d0;
    }
}

/* ------------------------------------------------------------------------ */
/* Departure point (Eq. 3, first order): x_p = x - (u * dt)                 */
/* ------------------------------------------------------------------------ */

void or_departure(int dim, int64_t n, const double *x, const double *u,
                  double dt, double *xp)
{
    for (int64_t k = 0; k < n * dim; ++k) {
        double s = u[k] * dt;
        xp[k] = x[k] - s;
    }
}

/* ------------------------------------------------------------------------ */
/* Containment (Sec. 2.2: x_p in K_l iff every lambda_i >= 0), with the     */
/* tolerance eps: every lambda_i >= -eps.                                   */
/* ------------------------------------------------------------------------ */

static int contains(int dim, const double *v0, const double *M, int64_t l,
                    const double *p, double eps)
{
    double lam[4];
    or_bary(dim, v0 + l * dim, M + l * dim * dim, p, lam);
    for (int i = 0; i <= dim; ++i)
        if (!(lam[i] >= -eps)) return 0;
    return 1;
}

static int finite_point(int dim, const double *p)
{
    for (int k = 0; k < dim; ++k)
        if (!isfinite(p[k])) return 0;
    return 1;
}

void or_locate_bruteforce(int dim, int64_t n_e, const double *v0,
                          const double *M, int64_t n, const double *pts,
                          double eps, int32_t *host)
{
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1024) num_threads(g_threads) if (g_threads > 1)
#endif
    for (int64_t q = 0; q < n; ++q) {
        const double *p = pts + q * dim;
        host[q] = -1;
        if (!finite_point(dim, p)) continue;
        for (int64_t l = 0; l < n_e; ++l)
            if (contains(dim, v0, M, l, p, eps)) {
                host[q] = (int32_t)l;
                break;
            }
    }
}

int or_locate_bucketed(int dim, int64_t n_v, const double *xyz, int64_t n_e,
                       const int32_t *conn, const double *v0, const double *M,
                       int64_t n, const double *pts, double eps, int g,
                       int32_t *host)
{
    const int nv = dim + 1;
    double lo[3], hi[3], w[3];
    for (int k = 0; k < dim; ++k) { lo[k] = INFINITY; hi[k] = -INFINITY; }
    for (int64_t v = 0; v < n_v; ++v)
        for (int k = 0; k < dim; ++k) {
            double c = xyz[v * dim + k];
            if (c < lo[k]) lo[k] = c;
            if (c > hi[k]) hi[k] = c;
        }
    double ext = 0.0;
    for (int k = 0; k < dim; ++k) {
        w[k] = (hi[k] - lo[k]) / g;
        if (hi[k] - lo[k] > ext) ext = hi[k] - lo[k];
    }
    /* a point with every lambda >= -eps lies within about dim*eps*diameter of
     * its element; the margin covers that with a wide factor */
    const double margin = 1e-7 * ext;
    int64_t ncell = 1;
    for (int k = 0; k < dim; ++k) ncell *= g;

    /* cell range of each element's grown bounding box */
    int32_t *rng = (int32_t *)malloc((size_t)n_e * 6 * sizeof(int32_t));
    int64_t *cnt = (int64_t *)calloc((size_t)ncell + 1, sizeof(int64_t));
    if (!rng || !cnt) { free(rng); free(cnt); return -2; }
    for (int64_t l = 0; l < n_e; ++l) {
        for (int k = 0; k < dim; ++k) {
            double a = INFINITY, b = -INFINITY;
            for (int i = 0; i < nv; ++i) {
                double c = xyz[(int64_t)conn[l * nv + i] * dim + k];
                if (c < a) a = c;
                if (c > b) b = c;
            }
            long ia = (long)floor((a - margin - lo[k]) / w[k]);
            long ib = (long)floor((b + margin - lo[k]) / w[k]);
            if (ia < 0) ia = 0;
            if (ib > g - 1) ib = g - 1;
            rng[l * 6 + 2 * k] = (int32_t)ia;
            rng[l * 6 + 2 * k + 1] = (int32_t)ib;
        }
        int32_t ia[3] = {0, 0, 0}, ib[3] = {0, 0, 0};
        for (int k = 0; k < dim; ++k) { ia[k] = rng[l * 6 + 2 * k]; ib[k] = rng[l * 6 + 2 * k + 1]; }
        for (int z = ia[2]; z <= ib[2]; ++z)
            for (int y = ia[1]; y <= ib[1]; ++y)
                for (int x = ia[0]; x <= ib[0]; ++x) {
                    int64_t c = dim == 2 ? (int64_t)y * g + x : ((int64_t)z * g + y) * g + x;
                    cnt[c + 1]++;
                }
    }
    for (int64_t c = 0; c < ncell; ++c) cnt[c + 1] += cnt[c];
    int32_t *items = (int32_t *)malloc((size_t)(cnt[ncell] > 0 ? cnt[ncell] : 1) * sizeof(int32_t));
    int64_t *fill = (int64_t *)malloc((size_t)ncell * sizeof(int64_t));
    if (!items || !fill) { free(rng); free(cnt); free(items); free(fill); return -2; }
    memcpy(fill, cnt, (size_t)ncell * sizeof(int64_t));
    /* elements are appended in increasing user id, so each cell's list is sorted */
    for (int64_t l = 0; l < n_e; ++l) {
        int32_t ia[3] = {0, 0, 0}, ib[3] = {0, 0, 0};
        for (int k = 0; k < dim; ++k) { ia[k] = rng[l * 6 + 2 * k]; ib[k] = rng[l * 6 + 2 * k + 1]; }
        for (int z = ia[2]; z <= ib[2]; ++z)
            for (int y = ia[1]; y <= ib[1]; ++y)
                for (int x = ia[0]; x <= ib[0]; ++x) {
                    int64_t c = dim == 2 ? (int64_t)y * g + x : ((int64_t)z * g + y) * g + x;
                    items[fill[c]++] = (int32_t)l;
                }
    }
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1024) num_threads(g_threads) if (g_threads > 1)
#endif
    for (int64_t q = 0; q < n; ++q) {
        const double *p = pts + q * dim;
        host[q] = -1;
        if (!finite_point(dim, p)) continue;
        int outside = 0;
        for (int k = 0; k < dim; ++k)
            if (p[k] < lo[k] - margin || p[k] > hi[k] + margin) outside = 1;
        if (outside) continue;
        int64_t c = 0;
        for (int k = dim - 1; k >= 0; --k) {
            long ik = (long)floor((p[k] - lo[k]) / w[k]);
            if (ik < 0) ik = 0;
            if (ik > g - 1) ik = g - 1;
            c = c * g + ik;
        }
        for (int64_t t = cnt[c]; t < cnt[c + 1]; ++t)
            if (contains(dim, v0, M, items[t], p, eps)) {
                host[q] = items[t];
                break;
            }
    }
    free(rng); free(cnt); free(items); free(fill);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1 (SNS). I_t counts the elements evaluated, the start          */
/* included. Containment ends the walk; otherwise the step goes across the */
/* face j of the smallest lambda (Eq. 5; equal minima -> lowest j). A -1   */
/* neighbour ends it at the boundary. The step cap ends it after `cap`     */
/* evaluations.                                                             */
/* ------------------------------------------------------------------------ */

void or_walk(int dim, const double *v0, const double *M, const int32_t *nbr,
             int64_t n, const double *pts, const int32_t *start, double eps,
             int32_t cap, int32_t *end, int32_t *path_len, uint8_t *reason)
{
    const int nv = dim + 1;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1024) num_threads(g_threads) if (g_threads > 1)
#endif
    for (int64_t q = 0; q < n; ++q) {
        const double *p = pts + q * dim;
        int32_t cur = start[q];
        if (!finite_point(dim, p) || cur < 0) {
            end[q] = -1; path_len[q] = 0; reason[q] = OR_INVALID;
            continue;
        }
        int32_t it = 0;
        for (;;) {
            double lam[4];
            ++it;
            or_bary(dim, v0 + (int64_t)cur * dim, M + (int64_t)cur * dim * dim, p, lam);
            int inside = 1;
            for (int i = 0; i < nv; ++i)
                if (!(lam[i] >= -eps)) inside = 0;
            if (inside) { reason[q] = OR_CONTAINED; break; }
            int j = 0;
            for (int i = 1; i < nv; ++i)
                if (lam[i] < lam[j]) j = i;
            int32_t next = nbr[(int64_t)cur * nv + j];
            if (next < 0) { reason[q] = OR_BOUNDARY; break; }
            if (it >= cap) { reason[q] = OR_CAP; break; }
            cur = next;
        }
        end[q] = cur;
        path_len[q] = it;
    }
}

/* ------------------------------------------------------------------------ */
/* Plain-SNS start K_m (Sec. 2.1, Eq. 4: the particle of node n_j starts in  */
/* an element that owns n_j): the lowest user id among them.               */
/* ------------------------------------------------------------------------ */

void or_node_elements(int dim, int64_t n_v, int64_t n_e, const int32_t *conn,
                      int32_t *node_elem)
{
    const int nv = dim + 1;
    for (int64_t v = 0; v < n_v; ++v) node_elem[v] = -1;
    for (int64_t l = 0; l < n_e; ++l)
        for (int i = 0; i < nv; ++i) {
            int32_t v = conn[l * nv + i];
            if (node_elem[v] < 0) node_elem[v] = (int32_t)l;
        }
}

/* ------------------------------------------------------------------------ */
/* ASG grid (Sec. 1 and 2.3: a Cartesian grid overlaid on the mesh)          */
/* ------------------------------------------------------------------------ */

void or_grid_centres(int dim, const double *lo, const double *hi,
                     const int32_t *g, double *centres)
{
    double s[3];
    int64_t n = 1;
    for (int k = 0; k < dim; ++k) {
        s[k] = (hi[k] - lo[k]) / (double)g[k];
        n *= g[k];
    }
    for (int64_t c = 0; c < n; ++c) {
        int64_t r = c;
        for (int k = 0; k < dim; ++k) {
            int64_t i = r % g[k];
            r /= g[k];
            double t = ((double)i + 0.5) * s[k];
            centres[c * dim + k] = lo[k] + t;
        }
    }
}

int64_t or_grid_cell(int dim, const double *lo, const double *hi,
                     const int32_t *g, const double *p)
{
    int64_t c = 0;
    for (int k = dim - 1; k >= 0; --k) {
        double s = (hi[k] - lo[k]) / (double)g[k];
        double t = floor((p[k] - lo[k]) / s);
        int64_t i;
        if (!(t >= 0.0)) i = 0;               /* also catches NaN */
        else if (t > (double)(g[k] - 1)) i = g[k] - 1;
        else i = (int64_t)t;
        c = c * g[k] + i;
    }
    return c;
}

void or_grid_cells(int dim, const double *lo, const double *hi,
                   const int32_t *g, int64_t n, const double *pts, int64_t *out)
{
    for (int64_t q = 0; q < n; ++q) out[q] = or_grid_cell(dim, lo, hi, g, pts + q * dim);
}

void or_p1_interpolate(int dim, const int32_t *conn, const double *v0,
                       const double *M, const double *u_nodal, int64_t n,
                       const double *pts, const int32_t *host, double *u_out)
{
    const int nv = dim + 1;
    for (int64_t q = 0; q < n; ++q) {
        int32_t l = host[q];
        if (l < 0) {
            for (int k = 0; k < dim; ++k) u_out[q * dim + k] = 0.0;
            continue;
        }
        double lam[4];
        or_bary(dim, v0 + (int64_t)l * dim, M + (int64_t)l * dim * dim, pts + q * dim, lam);
        for (int k = 0; k < dim; ++k) {
            double s = 0.0;
            for (int i = 0; i < nv; ++i)
                s = s + lam[i] * u_nodal[(int64_t)conn[l * nv + i] * dim + k];
            u_out[q * dim + k] = s;
        }
    }
}
