/*
 * cnnsns.h -- C ABI of the GB300 particle-location library for the CNN-SNS
 * method (Luo et al., "A CNN-based particle tracking method for large-scale
 * fluid simulations with Lagrangian-Eulerian approaches").
 *
 * The library finds, for every Lagrangian particle, the host element of its
 * departure point x_p = x - (u * dt) (Sec. 2.1, Eq. 3-4) in an unstructured
 * triangle (dim 2) or tetrahedron (dim 3) mesh by the successive neighbour
 * search of Algorithm 1 (Sec. 2.2), started from the particle's own element
 * (plain SNS), from the ASG cell of x_p, or from a CNN-predicted location
 * (CNN-SNS, Algorithm 2, Sec. 2.3).
 *
 * Conventions shared by every entry point:
 *  - Return value: CS_OK (0) or a negative cs_status; cs_last_error() then
 *    holds a message. On error nothing has been written to any output.
 *  - Per-particle outcomes go to status_out, never to the return value.
 *  - Element ids across the ABI are the caller's ("user") ids: the row index
 *    of the element in the connectivity passed to cs_mesh_upload.
 *  - Local index i names vertex i of an element; face i lies opposite it.
 *  - Arrays are row-major and densely packed: xyz[n_v][dim], conn[n_e][dim+1],
 *    x[n][dim], u[n][dim].
 *  - The caller owns every array it passes; the library owns its device
 *    copies of meshes and fields (until cs_mesh_release / cs_field_release /
 *    cs_destroy).
 *  - Every device allocation of the library counts against the context's
 *    HBM budget (cs_create); an allocation that would pass it fails with
 *    CS_ENOMEM and nothing is allocated.
 *  - One context serves one thread at a time; calls on a context must not
 *    overlap (it owns one scratch arena).
 *
 * Result definition (Sec. 2.2 containment test, with tolerance CS_EPS): the
 * host of x_p is the LOWEST user id l with lambda_i^l(x_p) >= -CS_EPS for all
 * i, or -1 when no element contains x_p. Barycentric coordinates are FP64,
 * computed from a per-element inverse-affine matrix with a fixed rounding
 * order, so results are reproducible bit for bit.
 */
#ifndef CNNSNS_H
#define CNNSNS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cs_ctx cs_ctx;
typedef int32_t cs_status;

/* return codes */
#define CS_OK        0
#define CS_EINVAL   (-1)   /* bad argument (null pointer, size, id, mode)    */
#define CS_ENOMEM   (-2)   /* host or device allocation failed               */
#define CS_ENOMESH  (-3)   /* mesh id not uploaded or already released       */
#define CS_EBUSY    (-4)   /* resource in use                                */
#define CS_ECUDA    (-5)   /* CUDA runtime error (message has the CUDA text) */
#define CS_EMESH    (-6)   /* malformed mesh: index out of range, degenerate
                              element (det == 0), face shared by > 2 elements */
#define CS_ENOPRED  (-7)   /* CNN-SNS requested without a loaded predictor   */
#define CS_EDEVICE  (-8)   /* device-side wait gave up (bounded spin)        */

/* start rules of cs_track */
#define CS_SNS        0    /* start = given start, else the node's element   */
#define CS_CNN_SNS    1    /* start = seed of the ASG cell at x + CNN(d)     */
#define CS_ASG_DIRECT 2    /* start = seed of the ASG cell of x_p (control)  */

/* per-particle status */
#define CS_FOUND              0  /* the walk ended inside the host           */
#define CS_OUTSIDE            1  /* no element contains x_p; host = -1       */
#define CS_FOUND_VIA_FALLBACK 2  /* walk left the mesh or hit the step cap;
                                    the exact search found the host          */
#define CS_INVALID            3  /* x_p not finite; host = -1, path_len = 0  */

#define CS_EPS 1e-12

/* field id of calls that name no velocity field (see cs_track) */
#define CS_NO_FIELD (-1)

typedef struct cs_mesh_info {
    int32_t dim;
    int64_t n_vertices;
    int64_t n_elements;
    int32_t asg_grid[3];        /* ASG cells per axis (seed grid)            */
    int32_t bucket_grid[3];     /* cells per axis of the exact-search index  */
    int64_t bucket_items;       /* total entries of the exact-search index   */
    double  lo[3], hi[3];       /* bounding box of the vertices              */
    double  tau;                /* canonicalisation threshold (see cs_track) */
    int32_t step_cap;           /* walk stops after this many evaluations    */
    int32_t record_bytes;       /* bytes of one element record (64 or 128)   */
    size_t  device_bytes;       /* device memory held by this mesh           */
    int32_t pred_stride;        /* ASG cells per predictor cell and axis     */
    int32_t pred_grid[3];       /* predictor cells per axis (see below)      */
} cs_mesh_info;

/* Create a context on CUDA device `cuda_device`. hbm_budget_bytes caps the
 * device memory the context may hold at once (meshes, fields, predictor
 * weights and workspaces, scratch, the serving arena); 0 = no cap beyond the
 * device's own. Errors: CS_EINVAL (device out of range), CS_ENOMEM, CS_ECUDA. */
cs_status cs_create(cs_ctx **out, int cuda_device, size_t hbm_budget_bytes);

/* Release every mesh, predictor and scratch buffer of the context. */
void cs_destroy(cs_ctx *ctx);

/* Message of the last failed call on this context (owned by the context). */
const char *cs_last_error(const cs_ctx *ctx);

/* Device bytes the context holds now and its budget (0 = none); either
 * pointer may be NULL. */
cs_status cs_memory_usage(cs_ctx *ctx, size_t *used_bytes, size_t *budget_bytes);

/*
 * Upload a mesh {K_l} (Sec. 2.2). Host pointers. Builds on the host: the
 * neighbour table m_i^l, the inverse-affine matrix of every element, a
 * Hilbert order of the element centroids, the exact-search bucket index and
 * the plain-SNS start of every vertex; then on the device the ASG seed grid
 * (the host of every ASG cell centre).
 *   asg_grid: cells per axis of the ASG grid over the vertex bounding box, or
 *             NULL for round(n_v^(1/dim)) - 1 per axis.
 * Errors: CS_EINVAL (dim not 2/3, sizes < 1, null pointer), CS_EMESH
 * (vertex index out of range, degenerate element, non-manifold face),
 * CS_ENOMEM, CS_ECUDA.
 */
cs_status cs_mesh_upload(cs_ctx *ctx, int dim, int64_t n_vertices, const double *xyz,
                         int64_t n_elements, const int32_t *conn,
                         const int32_t *asg_grid, int32_t *mesh_id_out);

cs_status cs_mesh_release(cs_ctx *ctx, int32_t mesh_id);
cs_status cs_mesh_query(cs_ctx *ctx, int32_t mesh_id, cs_mesh_info *info_out);

/* Plain-SNS start K_m of every vertex (Sec. 2.1, Eq. 4: an element owning the
 * node; the lowest user id among them). Host output [n_vertices]. */
cs_status cs_node_start_elements(cs_ctx *ctx, int32_t mesh_id, int32_t *out);

/* ASG seed grid: user id of the host of every cell centre, or -1 (host
 * output, [prod asg_grid], x fastest). */
cs_status cs_seed_grid(cs_ctx *ctx, int32_t mesh_id, int32_t *out);

/*
 * Upload a velocity field of a mesh: the nodal velocity u_nodal[n_v][dim]
 * (HOST or DEVICE pointer, FP64) that Algorithm 2's start predictor reads
 * (Sec. 2.3: the CNN input is the velocity field around the particle). The
 * library keeps a device copy and its P1 resampling to the mesh's predictor
 * grid (cs_grid_velocity's arithmetic), redone at the next use after
 * cs_predictor_grid changes that grid. Synchronous.
 * Errors: CS_ENOMESH, CS_EINVAL (null pointer), CS_EBUSY (while serving),
 * CS_ENOMEM (device memory or HBM budget), CS_ECUDA.
 */
cs_status cs_field_upload(cs_ctx *ctx, int32_t mesh_id, const double *u_nodal,
                          int32_t *field_id_out);

/* Release a field (CS_EINVAL if unknown, CS_EBUSY while serving). Releasing
 * a mesh releases its fields. */
cs_status cs_field_release(cs_ctx *ctx, int32_t field_id);

/*
 * Locate n particles (Algorithm 1 / Algorithm 2). DEVICE pointers; the work
 * is enqueued on `stream` (a cudaStream_t, NULL = legacy default stream) and
 * the call returns without synchronising.
 *   field_id: the velocity field (cs_field_upload) whose grid velocity the
 *             CNN-SNS start predictor reads, or CS_NO_FIELD. Read by
 *             CS_CNN_SNS only.
 *   x[n][dim], u[n][dim]: particle position and velocity; x_p = x - (u*dt).
 *   start[n]: user ids of the plain-SNS start, or NULL when the particles are
 *             the mesh vertices in order (n == n_vertices): then start =
 *             cs_node_start_elements(). A start of -1 skips the walk.
 *   mode: CS_SNS, CS_ASG_DIRECT or CS_CNN_SNS. CS_CNN_SNS needs a loaded
 *         predictor (cs_predictor_load); the call runs the predictor over the
 *         predictor grid and then walks (Algorithm 2). The predictor reads
 *         the grid velocity of field_id. With CS_NO_FIELD the particles must
 *         be the mesh nodes (start == NULL, n == n_vertices): u is then the
 *         nodal field, resampled to the predictor grid by this call and kept
 *         as the mesh's stored grid velocity (cs_predict, cs_windows).
 *   host_out[n]  user id of the host of x_p, or -1.
 *   path_len_out[n]  I_t of Algorithm 1 (elements evaluated, start included).
 *   status_out[n]    CS_FOUND / CS_OUTSIDE / CS_FOUND_VIA_FALLBACK / CS_INVALID.
 *   start_out[n]     (may be NULL) user id of the element the walk started in.
 * The walk stops when every lambda >= -CS_EPS, steps across the face of the
 * smallest lambda (equal minima: lowest local index), stops at a -1
 * neighbour, and stops after step_cap evaluations. Particles whose walk
 * left the mesh or hit the cap, and those whose final element has some
 * lambda < tau (near a face, where a lower id may also contain x_p), go
 * through an exact search of the bucket index, run by the warp that walked
 * them; the result is the host defined at the top of this file.
 * Errors: CS_EINVAL (n outside [0, 2^31 - 2], null pointer, start == NULL
 * with n != n_v, bad mode, field_id not a field of this mesh, CS_CNN_SNS with
 * CS_NO_FIELD on particles that are not the mesh nodes), CS_ENOMESH,
 * CS_ENOPRED, CS_ENOMEM, CS_ECUDA.
 */
cs_status cs_track(cs_ctx *ctx, int32_t mesh_id, int32_t field_id, int64_t n, const double *x,
                   const double *u, double dt, const int32_t *start, int mode,
                   int32_t *host_out, int32_t *path_len_out, uint8_t *status_out,
                   int32_t *start_out, void *stream);

/* cs_track with HOST pointers: copies inputs to the device, runs, copies the
 * results back and synchronises. Same arguments, results and errors.
 * The particle range is processed in up to 4 chunks on three streams of the
 * context (copy in, compute, copy out), so that the copies of one chunk
 * overlap the walk of another; CNN-SNS without a field first copies the whole
 * nodal velocity its predictor reads. Page-locked host buffers overlap best;
 * pageable ones give the same results. The call orders itself after work
 * already queued on the legacy default stream; calls on one context must not
 * overlap (they share the streams and the device staging buffer). */
cs_status cs_track_host(cs_ctx *ctx, int32_t mesh_id, int32_t field_id, int64_t n,
                        const double *x, const double *u, double dt, const int32_t *start,
                        int mode, int32_t *host_out, int32_t *path_len_out,
                        uint8_t *status_out, int32_t *start_out);

/* cs_track_host for the mesh nodes: the departure points (Eq. 3) of all n_v
 * vertices, each particle at its vertex's coordinates as passed to
 * cs_mesh_upload (the mesh keeps a device copy, so x is not copied in) and
 * starting from its node's element. This is the step of a solver that
 * tracks its mesh nodes, whose coordinates do not change. u_nodal: HOST
 * [n_v][dim]; outputs HOST [n_v]. The same results, modes, field rule,
 * pipeline and errors as cs_track_host with n = n_v, x = those coordinates
 * and start = NULL. */
cs_status cs_track_nodes_host(cs_ctx *ctx, int32_t mesh_id, int32_t field_id,
                              const double *u_nodal, double dt, int mode, int32_t *host_out,
                              int32_t *path_len_out, uint8_t *status_out, int32_t *start_out);

/*
 * cs_track without any device allocation. (This entry point is a property of
 * the library, not of the method: the paper has no counterpart.)
 *
 * For callers that cannot let the library allocate device memory during a
 * call -- a solver that owns every byte of device memory through its own pool,
 * or a time-step loop that cannot afford the device-wide synchronisation that
 * cudaMalloc / cudaFree may cause. Same arguments, semantics, results and
 * errors as cs_track for CS_SNS and CS_ASG_DIRECT (DEVICE pointers, enqueued
 * on `stream`, returns without synchronising); the caller still provides
 * every input and output array.
 *   - CS_CNN_SNS is refused with CS_EINVAL: its start predictor writes a
 *     displacement grid this call would have to allocate. A caller that
 *     holds a displacement grid of its own uses cs_track_dhat. field_id is
 *     therefore never read.
 *   - The walk's only scratch, its work cursor, lives in one fixed 256-byte
 *     device array of this library that every GPU loading the library holds
 *     until the process exits.
 *   - n has cs_track's range, [0, 2^31 - 2]. Nothing is allocated, ever: no
 *     cudaMalloc, cudaFree or allocating library routine is called.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture.
 *   - All calls share the one array and it keeps the last call's contents;
 *     each call clears the counters it needs on its stream. Calls whose work
 *     overlaps on the GPU (other streams, other contexts, other threads on the
 *     same device) race on the array: serialise them.
 */
cs_status cs_track_noalloc(cs_ctx *ctx, int32_t mesh_id, int32_t field_id, int64_t n,
                           const double *x, const double *u, double dt, const int32_t *start,
                           int mode, int32_t *host_out, int32_t *path_len_out,
                           uint8_t *status_out, int32_t *start_out, void *stream);

/* ------------------------------------------------------------------------ */
/* Learned start predictor (Sec. 2.3 and Algorithm 2).                       */
/*                                                                          */
/* Regressor form: a window of the predictor-grid velocity (cs_predictor_  */
/* grid) around the cell of the particle (channels u_k * dt / s_k, s_k the  */
/* predictor cell size, zero outside the grid; 2-D 9x9, 3-D                 */
/* 7x7x7) goes through valid 3x3 (3x3x3) convolutions of 32 channels with    */
/* ReLU (2-D: 4 layers, 3-D: 3 layers), then fully connected 32 -> 256      */
/* (ReLU) -> dim. The output is the displacement in predictor cell units;  */
/* the walk then starts at the ASG seed of x + displacement * s (Alg. 2:    */
/* the prediction K_p replaces K_m as the origin of the walk).              */
/*                                                                          */
/* Weights: a flat float32 vector; for each conv layer W[32][C_in][taps]     */
/* then b[32] (tap t = (dz*3 +) dy*3 + dx, offsets 0..2 reading input       */
/* position (z+dz, y+dy, x+dx) for output (z, y, x)), then fc1 W[256][32],  */
/* b[256], fc2 W[dim][256], b[dim]. 37,314 floats (2-D), 67,203 (3-D).      */
/* Arithmetic: BF16 operands, FP32 accumulation, FP32 master weights.       */
/* ------------------------------------------------------------------------ */

/* Engine of grid prediction (cs_predict, CS_CNN_SNS): 1 (default) = fully
 * convolutional over the predictor grid on the tensor cores (fused tcgen05
 * kernels, 2-D and 3-D); 2 = the same fully convolutional pass in 3-D as
 * cubic tiles of implicit-GEMM layers on CUDA cores (2-D runs the tensor
 * cores); 0 = every cell's own window through the same GEMM layers (both
 * dims; the reference the grid engines are tested against). CS_EBUSY while
 * serving. */
cs_status cs_predictor_engine(cs_ctx *ctx, int engine);

/* Output rows per tile of the 2-D tensor-core grid kernel: 24, 13 or 8, or
 * 0 (default) for the height whose tiles best fill the GPU's SMs (fewest
 * waves of one tile per SM, weighted by each height's pipeline length).
 * Results do not depend on it. CS_EINVAL for any other value. */
cs_status cs_predictor_tile_rows(cs_ctx *ctx, int rows);

/* Side of the cubic output tiles of the 3-D tensor-core grid kernel: 4, 3 or
 * 2 cells, or 0 (default) for the side whose tiles best fill the GPU's SMs.
 * Results do not depend on it. CS_EINVAL for any other value. */
cs_status cs_predictor_tile3(cs_ctx *ctx, int side);

/* Test hook of the bounded device-side waits (a property of the library; the
 * paper has none): with on != 0 the tensor-core predictor kernels (2-D and
 * 3-D) first wait, for about 17 ms, for a device flag that nothing sets. The
 * wait runs out, the kernel ends through its abort path before any MMA
 * (freeing its TMEM) and raises the device error flag, which
 * cs_device_status reports as CS_EDEVICE; the context stays usable. on == 0
 * restores normal launches. Synchronises the device. */
cs_status cs_debug_hold_predictor(cs_ctx *ctx, int on);

/* Synchronise the device and report whether a bounded device-side wait gave
 * up since the last call (CS_EDEVICE, message in cs_last_error) or CS_OK. */
cs_status cs_device_status(cs_ctx *ctx);

/* Operand precision of the training and window-forward GEMMs: bf16 != 0 (the
 * default) rounds operands to BF16; 0 keeps FP32 operands, for accuracy
 * checks. Process-wide (every context). */
cs_status cs_predictor_precision(cs_ctx *ctx, int bf16);

/* Number of floats of the predictor of dimension dim (0 for other dim). */
int64_t cs_predictor_size(int dim);

/* Load (replace) the predictor of dimension dim from HOST weights; resets the
 * optimiser state. Errors: CS_EINVAL (dim, n != cs_predictor_size), CS_ENOMEM. */
cs_status cs_predictor_load(cs_ctx *ctx, int dim, const float *weights, int64_t n);

/* Copy the current FP32 master weights to HOST memory. CS_ENOPRED if none. */
cs_status cs_predictor_save(cs_ctx *ctx, int dim, float *weights_out, int64_t n);

/*
 * The grid the start predictor runs on (Sec. 2.3: the ASG pools the mesh into
 * Cartesian cells that hold several elements each). stride (odd, >= 1) ASG
 * cells per predictor cell and axis; predictor cell I spans ASG cells
 * stride*I .. stride*I + stride - 1 and shares its centre with the middle one.
 * pred_grid[k] = asg_grid[k] / stride (rounded down); a point past the last
 * whole cell belongs to the last. The grid velocity, the predictor's windows
 * and outputs (in predictor-cell units), the training pairs and the start
 * rule of CS_CNN_SNS (cell of x, then x + d_hat * cell size) all use this grid;
 * the start element is still looked up in the ASG seed grid. Default 1 (the
 * ASG grid itself). Drops the mesh's stored grid velocity and predictions.
 * Not while serving (CS_EBUSY). Errors: CS_EINVAL (even stride, or larger
 * than asg_grid on some axis), CS_ENOMESH, CS_ENOMEM.
 */
cs_status cs_predictor_grid(cs_ctx *ctx, int32_t mesh_id, int32_t stride);

/* Predictor-grid velocity of a mesh from its nodal velocity (DEVICE
 * pointers): grid[c][k] = P1 interpolation of u_nodal[n_v][dim] at the centre
 * of predictor cell c inside the centre's host element (0 where the centre is
 * outside the mesh), in FP32 with weights from the FP64 barycentric
 * coordinates. grid_out: [prod pred_grid][dim] floats, or NULL to store it in
 * the mesh (used by cs_predict / CS_CNN_SNS). Enqueued on stream. */
cs_status cs_grid_velocity(cs_ctx *ctx, int32_t mesh_id, const double *u_nodal,
                           float *grid_out, void *stream);

/* Input windows at predictor cells (DEVICE): out[b][k][w] = grid[cells[b]
 * + offset(w)][k] * dt / s_k, zero outside the grid, w over the window
 * positions (x fastest). grid = NULL uses the mesh's stored grid velocity.
 * cells = NULL means cells 0..B-1. */
cs_status cs_windows(cs_ctx *ctx, int32_t mesh_id, const float *grid, double dt,
                     const int64_t *cells, int64_t B, float *out, void *stream);

/* Predictor forward on explicit windows (DEVICE pointers): windows
 * [B][dim][S^dim] -> dhat [B][dim] (cell units). Synchronous. */
cs_status cs_predictor_forward(cs_ctx *ctx, int dim, int64_t B, const float *windows,
                               float *dhat_out);

/* Predicted displacement (cell units) at every predictor cell of a mesh from
 * its stored grid velocity and dt (DEVICE output [prod pred_grid][dim], or NULL to
 * store it in the mesh for cs_track_dhat(.., NULL ..)). Enqueued on stream. */
cs_status cs_predict(cs_ctx *ctx, int32_t mesh_id, double dt, float *dhat_out, void *stream);

/* Train the predictor of dimension dim on N (window, target) pairs (DEVICE
 * windows [N][dim][S^dim], targets [N][dim] in cell units) with Adam
 * (lr, beta1 0.9, beta2 0.999, eps 1e-8) on the mean squared error, for
 * `steps` batches of `batch` pairs drawn without replacement per epoch from a
 * generator seeded by `seed`. loss_out (HOST, may be NULL) receives the loss
 * of every step. Synchronous. CS_ENOPRED if no predictor is loaded. */
cs_status cs_predictor_train(cs_ctx *ctx, int dim, const float *windows, const float *targets,
                             int64_t N, int64_t batch, int64_t steps, float lr, uint64_t seed,
                             float *loss_out);

/* Training pairs (Sec. 2.3: the training data are produced by the tracking
 * itself) for n particles at positions x with velocities u (DEVICE pointers):
 * cells_out[p] = predictor cell of x_p's origin x, windows_out[p] = the input
 * window at that cell from the mesh's stored grid velocity (scale dt / s_k),
 * targets_out[p][k] = (x_p,k - x_k) / s_k with x_p = x - (u * dt). The host
 * element labels come from cs_track with CS_SNS. Enqueued on stream. */
cs_status cs_training_pairs(cs_ctx *ctx, int32_t mesh_id, int64_t n, const double *x,
                            const double *u, double dt, float *windows_out, float *targets_out,
                            int64_t *cells_out, void *stream);

/* Gradient of the mean squared error of the predictor of dimension dim on B
 * (window, target) pairs (DEVICE pointers; grad_out [cs_predictor_size],
 * same layout as the weights) without updating the weights; loss_out (HOST,
 * may be NULL). Synchronous. */
cs_status cs_predictor_grad(cs_ctx *ctx, int dim, int64_t B, const float *windows,
                            const float *targets, float *grad_out, float *loss_out);

/* CNN-SNS start rule with a given displacement grid (DEVICE pointers): like
 * cs_track, but the walk starts at the seed of the ASG cell of
 * x + dhat[pcell(x)] * s, pcell and s the predictor cell and cell size
 * (falling back to the plain start where that seed is -1).
 * dhat: [prod pred_grid][dim] floats in predictor cell units, or NULL for the
 * mesh's stored prediction (cs_predict). */
cs_status cs_track_dhat(cs_ctx *ctx, int32_t mesh_id, int64_t n, const double *x,
                        const double *u, double dt, const int32_t *start, const float *dhat,
                        int32_t *host_out, int32_t *path_len_out, uint8_t *status_out,
                        int32_t *start_out, void *stream);

/* ---------------------------------------------------------------------------
 * The paper's classifier predictor (Sec. 2.3, Eq. 7-8)
 *
 * A second start predictor, per particle rather than per grid cell: the CNN
 * classifies x_p among the W^dim ASG cells of a window centred on the ASG
 * cell of x_p (W = 9 in 2-D, 7 in 3-D). Its inputs are the element centroids
 * of the window, averaged per ASG cell (average pooling, computed once per
 * mesh at upload in FP64), each minus x_p in ASG cell units, with a cell
 * outside the grid or without a centroid padded by its own centre; and x_p's
 * offset from its cell's centre. Two branches read them: two zero-padded
 * 3^dim convolutions of 32 channels with ReLU and a 2^dim average pooling on
 * the window; two fully connected layers of h1 = 256 with ReLU on the offset
 * (Sec. 3.1). A fully connected layer of h2 = 512 (Sec. 3.1) with ReLU on
 * their concatenation and one to the W^dim logits follow; the softmax over
 * them is B_l of Eq. 7. K_p (Eq. 8) is the ASG seed of the most probable
 * cell. Training minimises the cross-entropy against the window cell that
 * holds the centroid of the host K_t found by plain SNS (clamped into the
 * window). Operands of every layer are BF16 with FP32 accumulation; master
 * weights, Adam state and the softmax are FP32.
 *
 * Layout of the parameters (floats): per layer W then b, layers conv1
 * [32][dim][3^dim], conv2 [32][32][3^dim], xp1 [256][dim], xp2 [256][256],
 * fuse [512][32 (W/2)^dim + 256], logits [W^dim][512]. Convolution taps are
 * ordered dz, dy, dx (dx fastest); the pooled features enter fuse as
 * [channel][z][y][x] (x fastest), followed by the 256 offset features.
 * Window cells and classes are numbered x fastest.
 * ------------------------------------------------------------------------- */

/* Number of floats of the classifier of dimension dim (0 for other dim). */
int64_t cs_classifier_size(int dim);

/* Window edge W of the classifier of dimension dim (9, 7; 0 for other dim). */
int32_t cs_classifier_window(int dim);

/* Load (replace) the classifier of dimension dim from HOST parameters; resets
 * the optimiser state. Errors: CS_EINVAL (dim, n != cs_classifier_size),
 * CS_ENOMEM. */
cs_status cs_classifier_load(cs_ctx *ctx, int dim, const float *params, int64_t n);

/* Copy the classifier's FP32 master parameters to HOST memory. CS_ENOPRED if
 * none is loaded, CS_EINVAL if n != cs_classifier_size. */
cs_status cs_classifier_save(cs_ctx *ctx, int dim, float *params_out, int64_t n);

/* Departure points x_p = x - (u * dt) (Eq. 3, FP64, no fused multiply-add)
 * of n particles (DEVICE pointers, [n][dim] each). Enqueued on stream. */
cs_status cs_departure(cs_ctx *ctx, int32_t mesh_id, int64_t n, const double *x,
                       const double *u, double dt, double *xp_out, void *stream);

/* The classifier's inputs for n departure points xp [n][dim] (DEVICE):
 * window_out [n][dim][W^dim] (FP32 of the FP64 value (p - x_p) / s_k, p the
 * pooled centroid or the padding centre, s the ASG cell size), offset_out
 * [n][dim] (FP32 of (x_p - lo) / s - (cell + 1/2)). No network needed.
 * Enqueued on stream. */
cs_status cs_classifier_features(cs_ctx *ctx, int32_t mesh_id, int64_t n, const double *xp,
                                 float *window_out, float *offset_out, void *stream);

/* Logits H [n][W^dim] of n departure points (DEVICE pointers); the softmax of
 * a row is B_l of Eq. 7. Synchronous (the batch is processed in chunks
 * through the context's workspace). CS_ENOPRED without a classifier of the
 * mesh's dimension. */
cs_status cs_classifier_forward(cs_ctx *ctx, int32_t mesh_id, int64_t n, const double *xp,
                                float *logits_out);

/* Class labels of n departure points with known hosts (DEVICE; host: user
 * ids from plain SNS): the window cell (x fastest) holding the host's
 * centroid, its coordinates clamped into the window; -1 where host < 0.
 * Enqueued on stream. */
cs_status cs_classifier_labels(cs_ctx *ctx, int32_t mesh_id, int64_t n, const double *xp,
                               const int32_t *host, int32_t *label_out, void *stream);

/* Training pairs of the classifier, by plain SNS (DEVICE pointers): for n
 * particles at x with velocities u and plain starts `start` (user ids, or
 * NULL for the mesh nodes), xp_out [n][dim] = x_p and label_out [n] = the
 * class of x_p's host (cs_classifier_labels; -1 outside the mesh). Enqueued
 * on stream. */
cs_status cs_classifier_pairs(cs_ctx *ctx, int32_t mesh_id, int64_t n, const double *x,
                              const double *u, double dt, const int32_t *start, double *xp_out,
                              int32_t *label_out, void *stream);

/* Gradient of the cross-entropy (mean over the rows whose label lies in
 * [0, W^dim); other rows count for nothing) of the classifier on B
 * (x_p, label) pairs of a mesh (DEVICE xp [B][dim], labels [B]; grad_out
 * [cs_classifier_size], same layout as the parameters), without updating the
 * parameters; loss_out (HOST, may be NULL). Synchronous. */
cs_status cs_classifier_grad(cs_ctx *ctx, int32_t mesh_id, int64_t B, const double *xp,
                             const int32_t *labels, float *grad_out, float *loss_out);

/* Train the classifier on N (x_p, label) pairs of a mesh (DEVICE) with Adam
 * (lr, beta1 0.9, beta2 0.999, eps 1e-8) on the cross-entropy, for `steps`
 * batches of `batch` pairs drawn without replacement per epoch from a
 * generator seeded by `seed` (the same draw as cs_predictor_train). loss_out
 * (HOST, may be NULL) receives every step's loss. Synchronous. */
cs_status cs_classifier_train(cs_ctx *ctx, int32_t mesh_id, const double *xp,
                              const int32_t *labels, int64_t N, int64_t batch, int64_t steps,
                              float lr, uint64_t seed, float *loss_out);

/* Start elements K_p (Eq. 8) from given logits (DEVICE): the class of the
 * largest logit (the lowest class among equal ones; a row without a finite
 * maximum has none), its window cell's ASG seed as a user id, or fallback[p]
 * where the cell lies outside the grid, its centre outside the mesh or the
 * row has no class (fallback: user ids, or NULL for the mesh nodes' plain
 * starts, n == n_vertices). class_out (may be NULL) receives the class, or
 * -1. Enqueued on stream. */
cs_status cs_classifier_start(cs_ctx *ctx, int32_t mesh_id, int64_t n, const double *xp,
                              const float *logits, const int32_t *fallback, int32_t *start_out,
                              int32_t *class_out, void *stream);

/* CNN-SNS with the classifier (Algorithm 2 with Eq. 7-8's start): departure
 * points, the classifier's start of every particle (cs_classifier_start with
 * the plain start as fallback), then Algorithm 1 from it. Arguments, results
 * and errors as cs_track with CS_SNS (DEVICE pointers); start_out receives
 * the classifier's start. Hosts are those of plain SNS. Synchronous. */
cs_status cs_track_classifier(cs_ctx *ctx, int32_t mesh_id, int64_t n, const double *x,
                              const double *u, double dt, const int32_t *start,
                              int32_t *host_out, int32_t *path_len_out, uint8_t *status_out,
                              int32_t *start_out, void *stream);

/* ------------------------------------------------------------------------ */
/* Serving: continuous batching of tracking requests over resident meshes.   */
/* (A property of the library: the paper tracks one solver step at a time.) */
/*                                                                          */
/* A worker thread owns `slots` CUDA streams and a device arena of           */
/* arena_bytes. Requests wait in arrival order; the head request is admitted */
/* as soon as a slot is free and the arena has room for its buffers (its     */
/* HBM footprint: 2*dim*8 + 17 (+4 with starts) bytes per particle, plus the */
/* prediction grid for CNN-SNS, plus a grid velocity when the request names  */
/* no field). Admitted requests run concurrently on their streams; results   */
/* are identical to cs_track_host on the same inputs. Meshes, fields and     */
/* predictor weights must be resident before cs_serve_start and unchanged    */
/* while serving (mesh, field and predictor-grid changes return CS_EBUSY).   */
/* A CNN-SNS request runs the grid predictor of its dimension on the tensor  */
/* cores (with engine 2 the 3-D tile engine, whose shared workspace           */
/* serialises the 3-D predictions while the walks still overlap) on its      */
/* field's grid velocity, or on its own u when its particles are the mesh    */
/* nodes; without a loaded predictor, or with neither, it falls back to      */
/* plain SNS.                                                                */
/* ------------------------------------------------------------------------ */
typedef struct cs_serve_cfg {
    int32_t slots;          /* concurrent requests on the GPU (1..64)        */
    size_t  arena_bytes;    /* device memory for requests' buffers           */
} cs_serve_cfg;

typedef struct cs_request {
    int32_t mesh_id;
    int32_t field_id;       /* velocity field of CNN-SNS, or CS_NO_FIELD     */
    int64_t n;
    const double *x;        /* HOST [n][dim] (pinned memory overlaps best)   */
    const double *u;        /* HOST [n][dim]                                 */
    double dt;
    const int32_t *start;   /* HOST [n] user ids, or NULL when n == n_v      */
    int32_t mode;           /* CS_SNS, CS_ASG_DIRECT, CS_CNN_SNS             */
    int32_t *host_out;      /* HOST [n], written when the request finishes   */
    int32_t *path_len_out;  /* HOST [n]                                      */
    uint8_t *status_out;    /* HOST [n]                                      */
} cs_request;

typedef struct cs_serve_stats {
    int64_t completed, rejected, particles;
    double  p50_ms, p99_ms, mean_ms, max_ms;   /* submit-to-finish latency   */
    double  wall_s;                            /* first submit to last finish */
    double  particles_per_s;
    int64_t peak_bytes;                        /* arena high-water mark      */
    int32_t max_concurrent;                    /* requests in flight at once */
} cs_serve_stats;

/* Start the worker (one server per context). CS_EBUSY if already serving;
 * CS_ENOMEM if the arena does not fit the device or the HBM budget. */
cs_status cs_serve_start(cs_ctx *ctx, const cs_serve_cfg *cfg);

/* Queue a request; returns at once with a ticket. The caller keeps the
 * request's arrays alive until cs_serve_wait reports it finished. CS_ENOMEM
 * if the request could never fit in the arena (counted as rejected). */
cs_status cs_serve_submit(cs_ctx *ctx, const cs_request *req, int64_t *ticket);

/* Wait up to timeout_ms for a ticket: CS_OK (then *result holds the request's
 * status and *mode_used the start rule it ran with) or CS_EBUSY (not yet
 * finished). A finished ticket is forgotten after it is reported. */
cs_status cs_serve_wait(cs_ctx *ctx, int64_t ticket, int32_t timeout_ms, cs_status *result,
                        int32_t *mode_used);

/* Latency percentiles and throughput of the requests finished so far. */
cs_status cs_serve_report(cs_ctx *ctx, cs_serve_stats *out);

/* One finished request of the running server. Times are milliseconds since
 * the server's first submit: submitted (cs_serve_submit returned), admitted
 * (slot and arena memory taken, inputs about to be copied in) and done (its
 * end event seen by the worker). The latency of cs_serve_report is
 * done - submit; admit - submit is its wait in the queue. */
typedef struct cs_serve_record {
    int64_t ticket;
    int64_t n;              /* particles                                     */
    int32_t mesh_id;
    int32_t mode_used;      /* start rule it ran with                        */
    int32_t slot;           /* the slot (stream) it ran on                   */
    int32_t in_flight;      /* requests on the GPU after it was admitted     */
    int32_t result;         /* its cs_status                                 */
    int32_t reserved;
    double  dt;             /* its time step                                 */
    double  submit_ms, admit_ms, done_ms;
    /* device time of its stages on its stream (CUDA events): the input
     * copies, the start predictor (0 without CNN-SNS), the walk, the output
     * copies; the gaps between admit_ms and done_ms beyond their sum are
     * host-side (launch, event polling) or waits for the GPU held by others */
    double  h2d_ms, predict_ms, walk_ms, d2h_ms;
} cs_serve_record;

/* Copy the records of the requests finished so far, in the order they
 * finished, into out[0, cap) (HOST memory the caller owns); *count = records
 * copied. With out = NULL, *count = the number of records held. The server
 * keeps every record until cs_serve_stop. CS_EINVAL when not serving, when
 * count is NULL or when cap < 0. */
cs_status cs_serve_trace(cs_ctx *ctx, int64_t cap, cs_serve_record *out, int64_t *count);

/* Drain the queue, stop the worker and free the serving resources. */
cs_status cs_serve_stop(cs_ctx *ctx);

/* Walk statistics of a finished cs_track (DEVICE pointers, synchronous):
 * out[0] = sum of path_len, out[1] = max path_len, out[2..5] = particles with
 * status 0..3. */
cs_status cs_track_stats(cs_ctx *ctx, int64_t n, const int32_t *path_len,
                         const uint8_t *status, int64_t out[6], void *stream);

/* Error statistics of a finished tracking call (Sec. 3.1), DEVICE inputs,
 * synchronous:
 *   err of a particle = distance between the centroids (mean of the
 *       vertices) of its tracking origin start[p] (the walk's start element,
 *       cs_track's start_out) and of its host host[p]; particles where either
 *       is -1 are skipped. start may be NULL (no err).
 *   displacement error = |dhat[pcell(x)] * s - (x_p - x)|, the predicted
 *       displacement at the predictor cell of x (cell units times the
 *       predictor cell size s) against the true one, x_p = x - (u*dt);
 *       computed only when dhat ([prod pred_grid][dim] floats, e.g. from
 *       cs_predict) is given, and only for finite x_p.
 * Sums are in FP64 (their order is not fixed); maxima are exact. */
typedef struct cs_error_stats {
    int64_t n_err;
    double  err_sum, err_max;
    int64_t n_disp;
    double  disp_sum, disp_max;
} cs_error_stats;
cs_status cs_track_error(cs_ctx *ctx, int32_t mesh_id, int64_t n, const double *x,
                         const double *u, double dt, const int32_t *start, const int32_t *host,
                         const float *dhat, cs_error_stats *out, void *stream);

/* Launch counter: kernels this context has launched since creation. */
int64_t cs_kernel_launches(const cs_ctx *ctx);

/* Per-stage device time, measured with CUDA events recorded on the stream
 * each kernel is launched on (enabled by cs_profile_enable; off by default). */
typedef struct cs_profile {
    int64_t launches[8];   /* per stage: calls measured                      */
    double  ms[8];         /* per stage: summed event time, milliseconds     */
} cs_profile;
#define CS_STAGE_WALK      0   /* departure + start + Algorithm 1 walk, and
                                  the exact searches, which run inside it    */
#define CS_STAGE_FALLBACK  1   /* reserved: no longer a separate kernel      */
#define CS_STAGE_RESAMPLE  2   /* nodal velocity -> predictor grid           */
#define CS_STAGE_CNN       3   /* CNN forward over the predictor grid        */
#define CS_STAGE_TRAIN     4   /* one training step (forward+backward+Adam)  */

/* Turn event timing on (1) or off (0). */
cs_status cs_profile_enable(cs_ctx *ctx, int on);

/* Synchronise the recorded events and add their times into *out (zeroed
 * first); reset != 0 clears the record afterwards. */
cs_status cs_profile_read(cs_ctx *ctx, cs_profile *out, int reset);

#ifdef __cplusplus
}
#endif
#endif
