/*
 * CPU oracle for the particle-location path of the CNN-SNS method
 * (Luo et al., "A CNN-based particle tracking method for large-scale fluid
 * simulations with Lagrangian-Eulerian approaches").
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library. The product path never
 * links or calls it, and it shares no source with the CUDA library.
 *
 * Plain, slow, single-threaded, in user element ids (no reordering), FP64.
 * Every function names the passage of the paper it follows. Where the paper
 * leaves a choice open the fixed reading is stated beside the function.
 *
 * Arrays are row-major: xyz[n_v][dim], conn[n_e][dim+1], nbr[n_e][dim+1],
 * v0[n_e][dim], M[n_e][dim][dim], points[n][dim].
 * Local index i names vertex i of an element; face i lies opposite vertex i.
 */
#ifndef CNNSNS_ORACLE_H
#define CNNSNS_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* walk end reasons (Algorithm 1's two exits, plus the step cap) */
#define OR_CONTAINED 0
#define OR_BOUNDARY  1
#define OR_CAP       2
#define OR_INVALID   3

/* per-particle status of a full track (same codes as the library) */
#define OR_ST_FOUND     0
#define OR_ST_OUTSIDE   1
#define OR_ST_FALLBACK  2
#define OR_ST_INVALID   3

/* Neighbour table m_i^l (Sec. 2.2): nbr[l][i] = element sharing face i of l,
 * or -1 on the boundary. Returns 0, or -1 if a face is shared by more than
 * two elements, or -2 on allocation failure. */
int or_neighbors(int dim, int64_t n_e, const int32_t *conn, int32_t *nbr);

/* Pin for or_neighbors on small meshes: O(n_e^2) comparison of vertex sets. */
int or_neighbors_bruteforce(int dim, int64_t n_e, const int32_t *conn, int32_t *nbr);

/* Inverse-affine form of the barycentric coordinates (Sec. 2.2). Returns 0,
 * or 1 + index of the first element with det == 0 (or non-finite). */
int64_t or_inverse_affine(int dim, const double *xyz, int64_t n_e,
                          const int32_t *conn, double *v0, double *M);

/* lambda_0..lambda_dim of point p in one element, from (v0, M). */
void or_bary(int dim, const double *v0, const double *M, const double *p,
             double *lam);

/* The paper's literal formula lambda_i = |S_i| / |S_0| (Sec. 2.2), with S_0
 * the (dim+1)x(dim+1) matrix of [1; x; y; z] columns. Used only as a pin. */
void or_bary_det(int dim, const double *verts /* [dim+1][dim] */,
                 const double *p, double *lam);

/* Departure points x_p = x - (u * dt) (Eq. 3, first-order foot). */
void or_departure(int dim, int64_t n, const double *x, const double *u,
                  double dt, double *xp);

/* Brute force: host[p] = lowest user id l with min_i lambda_i^l >= -eps, or
 * -1 (the containment test of Sec. 2.2 with tolerance eps). */
void or_locate_bruteforce(int dim, int64_t n_e, const double *v0,
                          const double *M, int64_t n, const double *pts,
                          double eps, int32_t *host);

/* Same result through a uniform bucket grid of g cells per axis (exact:
 * every element is listed in every cell its margin-grown box touches). */
int or_locate_bucketed(int dim, int64_t n_v, const double *xyz, int64_t n_e,
                       const int32_t *conn, const double *v0, const double *M,
                       int64_t n, const double *pts, double eps, int g,
                       int32_t *host);

/* Algorithm 1 (SNS) from start[p]; end element, I_t and exit reason. */
/* Threads of the particle loops (OpenMP builds; 1 otherwise); returns the
 * count in effect. Results do not depend on it. */
int or_set_threads(int n);

void or_walk(int dim, const double *v0, const double *M, const int32_t *nbr,
             int64_t n, const double *pts, const int32_t *start, double eps,
             int32_t cap, int32_t *end, int32_t *path_len, uint8_t *reason);

/* Plain-SNS start K_m: lowest user id element incident to each vertex. */
void or_node_elements(int dim, int64_t n_v, int64_t n_e, const int32_t *conn,
                      int32_t *node_elem);

/* ASG grid of g[k] cells over [lo, hi]: cell size s_k = (hi_k - lo_k) / g_k,
 * centres c = lo_k + (i + 0.5) * s_k, cell of a point
 * floor((x_k - lo_k) / s_k) clamped to [0, g_k - 1]. */
void or_grid_centres(int dim, const double *lo, const double *hi,
                     const int32_t *g, double *centres);
int64_t or_grid_cell(int dim, const double *lo, const double *hi,
                     const int32_t *g, const double *p);
void or_grid_cells(int dim, const double *lo, const double *hi,
                   const int32_t *g, int64_t n, const double *pts, int64_t *out);

/* P1 interpolation of nodal velocity at the grid centres, given each
 * centre's host element (the Sec. 2.1 interpolation inside the host). */
void or_p1_interpolate(int dim, const int32_t *conn, const double *v0,
                       const double *M, const double *u_nodal, int64_t n,
                       const double *pts, const int32_t *host, double *u_out);

#ifdef __cplusplus
}
#endif
#endif
