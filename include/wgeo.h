/*
 * wgeo.h — C ABI of the GB300 (sm_103a) library that reconstructs a signed
 * distance field and surface normals on a uniform grid from an oriented point
 * cloud, and differentiates it by the adjoint method.
 *
 * What the calls compute (paper sections / equations of arXiv 2609.20964):
 *   - 27-cell normal splat, Sec. 2.3, Eqs. 23-25;
 *   - right-hand side b = <grad F_p, V>, Sec. 2.3, Eqs. 22 and 26, as a
 *     face-form divergence with zero flux through the domain faces;
 *   - Poisson solve A a = b, Sec. 2.3, Eqs. 15 and 20-21, A the cell-centred
 *     7-point Neumann operator (trilinear Galerkin with transverse lumping);
 *   - iso-value c, Sec. 2.4, Eq. 27 (mean of the interpolated indicator at the
 *     input samples);
 *   - marching cubes, Sec. 2.4, Eq. 28;
 *   - exact signed distance to the extracted triangles, Sec. 2.4, Eqs. 29-34,
 *     and unit normals grad(phi)/|grad(phi)| (Sec. 2.4, after Eq. 32);
 *   - adjoint differentiation, Sec. 2.5, Eqs. 35-39 (one extra solve with the
 *     transposed operator; no solver iterates are stored).
 *
 * Conventions shared by every call
 *   Grid: cubic, res^3 cells of edge h = max_axis(hi - lo) / res over the box
 *     [lo, lo + res*h].  Cell (node) (i,j,k) has centre lo + ((i,j,k)+1/2) h.
 *     Grids are float32, C order [z][y][x] (x fastest), linear index
 *     (k*res + j)*res + i.  Normal grids are three such planes [3][res^3].
 *   Points, normals, query points and their gradients: float32 [n][3] (AoS).
 *   Memory: every array argument is caller-owned, contiguous, 16-byte-aligned
 *     DEVICE memory unless stated otherwise.  The library never frees or
 *     retains caller arrays after a call returns.  The handle owns all
 *     workspace (allocated once by wgeo_create).
 *   Streams: every call only enqueues work on `stream` (a cudaStream_t passed
 *     as void*; NULL = legacy default stream) and returns without waiting.
 *     Calls on one handle must be ordered (same stream, or synchronised).
 *   Errors: the return value reports what the host can check (bad pointers,
 *     sizes, box, options, CUDA launch failures).  Problems found on the
 *     device set bits of a status word read with wgeo_get_info after the
 *     stream has been synchronised; kernels never trap.
 *   Thread safety: distinct handles may be used from distinct threads.
 */
#ifndef WGEO_H
#define WGEO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct wgeo_handle wgeo_handle;

/* Return codes. */
typedef enum {
  WGEO_OK = 0,
  WGEO_ERR_INVALID_ARG = 1,   /* null pointer, size over the handle's bounds, bad box/res/options */
  WGEO_ERR_OOM = 2,           /* device allocation failed in wgeo_create */
  WGEO_ERR_CUDA = 3,          /* a CUDA runtime call or kernel launch failed */
  WGEO_ERR_NO_FORWARD = 4,    /* query/backward before a forward that kept its state */
  WGEO_ERR_NOT_BUILT_FOR_DEVICE = 5 /* no sm_103a device available to this process */
} wgeo_status;

/* Device status bits (wgeo_info.status), set by kernels. */
#define WGEO_STATUS_POINT_OUTSIDE_BBOX (1u << 0) /* a point lies outside [lo, lo+res*h]; clamped */
#define WGEO_STATUS_NONFINITE_INPUT    (1u << 1) /* NaN/Inf point or normal; that point was skipped */
#define WGEO_STATUS_EMPTY_SURFACE      (1u << 2) /* no triangle: phi = +-inf, normals 0 */
#define WGEO_STATUS_NOT_CONVERGED      (1u << 3) /* solver stopped at its iteration limit */
#define WGEO_STATUS_MESH_CAPACITY      (1u << 4) /* more triangles than mesh_capacity: sdf unspecified */

/* Precision of the Poisson solve. */
#define WGEO_PREC_MIXED 0  /* iterative refinement with a float-float iterate and residual (two-sum
                              arithmetic on the FP32 pipe, ~48-bit significand) and FP64 norms and
                              sums; each step's correction is one FP32 spectral (cosine-basis) solve
                              on power-of-two grids of 32..512 with opt.spectral, else FP32
                              multigrid V-cycles */
#define WGEO_PREC_FP32  1  /* plain FP32, no refinement: one direct FP32 spectral solve on
                              power-of-two grids of 32..512 with opt.spectral (set max_vcycles >= 1),
                              else FP32 V-cycles on the iterate; FP32 residual and sums */
#define WGEO_PREC_FP64  2  /* as MIXED with a native FP64 refinement iterate and residual (the FP64
                              pipe) instead of float-float; the adjoint solve stays float-float.  A
                              comparison point: same results to ~1e-12, slower on this GPU */

typedef struct {
  double  tol_rel;           /* stop when ||b - A chi|| <= tol_rel * ||b|| (default 1e-6) */
  int32_t max_vcycles;       /* FP32 mode: maximum V-cycles, or spectral solves (default 40) */
  int32_t max_refine;        /* MIXED mode: maximum refinement steps (default 10) */
  int32_t vcycles_per_refine;/* MIXED mode: FP32 V-cycles per refinement step (default 2) */
  int32_t precision;         /* WGEO_PREC_MIXED (default), WGEO_PREC_FP32 or WGEO_PREC_FP64 */
  int32_t warm_start;        /* start the solve from the previous chi on this handle when res matches (default 0) */
  int32_t keep_for_backward; /* keep what wgeo_backward needs (closest triangles, phi copy); default 1 */
  int64_t mesh_capacity;     /* maximum triangles; 0 = default 16 * max_res^2 */
  int32_t use_graphs;        /* record the solver's fixed launch sequence once as a CUDA graph (default 1) */
  int32_t stage_timing;      /* bracket each stage with CUDA events on the call's stream (default 0) */
  int32_t galerkin;          /* 0 (default): the transverse-lumped 7-point operator and face divergence;
                                1: the unlumped trilinear Galerkin forms (27-point operator
                                A = S M M + M S M + M M S and right-hand side sum D M M V, with the
                                1-D stiffness S = {-1,2,-1}, mass M = {1,4,1}/6 and central
                                difference D, the walls mirrored; Sec. 2.3, Eqs. 20-22 and 26).
                                Needs WGEO_PREC_MIXED. */
  int32_t spectral;          /* 1 (default): when res is a power of two from 32 to 512, MIXED mode
                                takes each refinement step's correction from a direct spectral
                                solve (the operator is diagonal in the cosine basis of the mirrored
                                walls; always two steps), and FP32 mode solves once, directly;
                                0: multigrid V-cycles on every grid */
  int32_t reserved[3];
  double  tol_rel_adjoint;   /* adjoint solve: stop when ||g - A lambda|| <= tol * ||g|| (default 1e-7) */
} wgeo_options;

/* Stage ids reported by wgeo_stage_times. */
#define WGEO_STAGE_SPLAT       0   /* binning, tile sort, fused splat + divergence */
#define WGEO_STAGE_SOLVE       1   /* forward Poisson solve */
#define WGEO_STAGE_ISO         2   /* iso-value */
#define WGEO_STAGE_MC          3   /* marching cubes + box pyramid */
#define WGEO_STAGE_SDF         4   /* exact distance search and sign (float32 search) */
#define WGEO_STAGE_NORMALS     5
#define WGEO_STAGE_QUERY       6
#define WGEO_STAGE_BWD_SEED    7   /* grid seeds + query adjoint */
#define WGEO_STAGE_BWD_SURFACE 8   /* distance, marching-cubes and iso-value adjoints */
#define WGEO_STAGE_BWD_SOLVE   9   /* adjoint Poisson solve */
#define WGEO_STAGE_BWD_SPLAT   10  /* divergence transpose + splat adjoint */
#define WGEO_STAGE_SDF_TIE     11  /* float-float decisions of near-tie closest triangles */
#define WGEO_STAGE_POINT_PCA   12  /* D-PCA point-normal estimation (wgeo_estimate_normals) */
#define WGEO_STAGE_ORIENT      13  /* parity normal orientation (wgeo_orient_normals) */
#define WGEO_STAGE_QUERY_EXACT 14  /* exact off-grid signed distance (wgeo_query_exact) */
#define WGEO_NUM_STAGES        15

typedef struct {
  uint32_t status;           /* WGEO_STATUS_* bits of the last call */
  int32_t  res;              /* grid of the last forward */
  int32_t  solver_steps;     /* refinement steps (MIXED) or V-cycles (FP32) used by the last solve */
  int32_t  backward_steps;   /* the same for the adjoint solve of the last backward */
  double   residual_rel;     /* final ||b - A chi|| / ||b|| of the last forward solve */
  double   backward_residual_rel;
  double   isovalue;         /* c of the last forward */
  int64_t  n_triangles;      /* triangles extracted by the last forward */
  int64_t  n_points_used;    /* finite points used by the last forward */
  double   h;                /* cell size of the last forward */
  int64_t  sdf_node_visits;  /* with stage_timing = 2: octree nodes entered by the distance search (per warp) */
  int64_t  sdf_leaf_visits;  /* ... leaves entered (per warp) */
  int64_t  sdf_tri_tests;    /* ... point-triangle distance evaluations (per node, i.e. per lane) */
  double   backward_dc;      /* dL/dc of the last backward */
  int64_t  sdf_tie_nodes;    /* with stage_timing = 2: nodes whose nearest triangle was a float32
                                near-tie, re-decided in float-float arithmetic */
  int64_t  reserved[1];
} wgeo_info;

/* Fills `opt` with the defaults listed above.  Never fails for non-null opt. */
int wgeo_default_options(wgeo_options* opt);

/* Device bytes a handle created with these bounds would allocate (for
 * admission by memory budget).  Pure host arithmetic; 0 on invalid bounds. */
size_t wgeo_footprint_bytes(int32_t max_res, int64_t max_points, const wgeo_options* opt);

/* Creates a handle whose workspace fits grids up to max_res^3 and clouds of
 * up to max_points points, on the current CUDA device.  max_res must be >= 4
 * and coarsen by halving to a grid of at most 16^3 (res = m * 2^k, m <= 16).
 * opt may be NULL (defaults).  On failure *h is NULL and nothing is leaked.
 * Returns WGEO_ERR_OOM when a device allocation fails. */
int wgeo_create(wgeo_handle** h, int32_t max_res, int64_t max_points, const wgeo_options* opt);

/* Waits for the handle's outstanding work, frees everything it owns. */
int wgeo_destroy(wgeo_handle* h);

/* Forward (Sec. 2.3-2.4): points [n][3] and outward normals [n][3] (normals are
 * used as given, not renormalised) -> sdf_out [res^3] and, if nrm_out is not
 * NULL, unit normals nrm_out [3][res^3].  bbox is a HOST array of 6 floats
 * {lo.x, lo.y, lo.z, hi.x, hi.y, hi.z} with hi > lo on every axis.
 * 0 <= n <= max_points, 4 <= res <= max_res with the coarsening rule above.
 * sdf_out may be NULL when only the state for wgeo_query / wgeo_backward is
 * wanted. */
int wgeo_reconstruct(wgeo_handle* h, const float* points, const float* normals, int64_t n,
                     const float* bbox, int32_t res, float* sdf_out, float* nrm_out,
                     void* stream);

/* Query (Sec. 2.4 SDF on the grid; query-point differentiation, Sec. 2.5):
 * trilinear phi and the normalised trilinear stencil normal at q [m][3],
 * positions clamped into the node hull [lo+h/2, lo+(res-1/2)h].  sdf_q [m];
 * nrm_q [m][3] or NULL.  Needs a prior wgeo_reconstruct on this handle. */
int wgeo_query(wgeo_handle* h, const float* q, int64_t m, float* sdf_q, float* nrm_q, void* stream);

/* Exact query (Sec. 2.4, Eqs. 29-34 evaluated off the grid): at each point
 * q [m][3], sdf_q [m] = s(q) d(q) with d(q) the exact distance to the last
 * forward's marching-cubes surface (nearest triangle, float32 search) and
 * s(q) = -1 inside, +1 outside by the parity of the crossings of a segment
 * from q to a corner of the cube holding q (q clamped into the node hull for
 * the sign only; on a closed surface this is the parity of any ray from q).
 * grad_q [m][3] (may be NULL) receives s(q) (q - y) / d(q), y the closest
 * surface point: d(sdf_q)/dq where the closest point is unique and d > 0;
 * zero where d = 0.  Non-finite q give NaN and a zero gradient; an empty
 * surface gives +/-infinity.  Queries may lie anywhere (no clamping of the
 * distance).  The queries are sorted internally in chunks of
 * max(max_points, min(2^20, max(65536, max_res^3 / 4))), in the
 * normal-estimation workspace.  Needs a prior
 * wgeo_reconstruct on this handle (else WGEO_ERR_NO_FORWARD). */
int wgeo_query_exact(wgeo_handle* h, const float* q, int64_t m, float* sdf_q, float* grad_q, void* stream);

/* Backward (Sec. 2.5, Eqs. 35-39): given dL/dphi on the grid (d_sdf_grid
 * [res^3] or NULL), dL/dn on the grid (d_nrm_grid [3][res^3] or NULL) and/or
 * the adjoints of a wgeo_query at q [m][3] (d_sdf_q [m] or NULL, d_nrm_q
 * [m][3] or NULL), writes dL/dpoints [n][3] and dL/dnormals [n][3] of the last
 * forward's inputs, and dL/dq [m][3] if d_q is not NULL (q must then be given).
 * Requires the last forward to have run with keep_for_backward (else
 * WGEO_ERR_NO_FORWARD).  Discrete choices (central cell, marching-cubes case,
 * closest triangle) are those of the forward. */
int wgeo_backward(wgeo_handle* h, const float* d_sdf_grid, const float* d_nrm_grid,
                  const float* q, const float* d_sdf_q, const float* d_nrm_q, int64_t m,
                  float* d_points, float* d_normals, float* d_q, void* stream);

/* Normal estimation by distance-weighted PCA (Sec. 2.1, the neighbourhood,
 * weight, weighted-centroid and weighted-covariance equations and the
 * eigen-decomposition that follows them): for every point x_i of points
 * [n][3], N_i = { x_j : |x_j - x_i| <= radius } (x_i itself included),
 * w_ij = 1 / (|x_j - x_i| + eps), C_i the w-weighted covariance about the
 * w-weighted centroid, and normals[i] = the unit eigenvector of C_i with the
 * smallest eigenvalue.  The sign is arbitrary (unoriented).  A neighbourhood of
 * fewer than 3 points, a covariance with no positive eigenvalue, or a point
 * with a non-finite coordinate gives the zero vector; non-finite points belong
 * to no neighbourhood.  Membership is decided in float32 with each operation
 * rounded: ((dx*dx + dy*dy) + dz*dz) <= radius*radius, dx = x_j.x - x_i.x.
 * counts [n] (int32, may be NULL) receives |N_i| (0 for non-finite points).
 * bbox is a HOST array {lo.x, lo.y, lo.z, hi.x, hi.y, hi.z} of finite floats
 * with hi >= lo: it only places the search cells, so points outside it are
 * still handled exactly (they share the boundary cells).  radius > 0 finite,
 * eps finite with eps >= 1e-6 * radius (the float weights R / (d + eps) then
 * stay below 1e6); 0 <= n <= max_points.  Results are deterministic (sums in a
 * fixed order).  Uses the handle's normal-estimation workspace only: the
 * state kept by the last wgeo_reconstruct for wgeo_query / wgeo_backward is
 * untouched.  Enqueued on `stream`; errors WGEO_ERR_INVALID_ARG (nothing
 * enqueued) or WGEO_ERR_CUDA. */
int wgeo_estimate_normals(wgeo_handle* h, const float* points, int64_t n, const float* bbox, float radius,
                          float eps, float* normals, int32_t* counts, void* stream);

/* Parity-based normal orientation (Sec. 2.2): flips, in place, the normals
 * [n][3] of points [n][3] to point out of the closed surface the cloud samples.
 *   r_d = gamma * r_{d,0}, r_{d,0} = 1/2 max_i min_{j != i} |x_i - x_j|
 *     (Eqs. baseline_detection_radius and expanded_detection_radius);
 *   probes y_m = x_i + m r_d u_i, m = 0, 1, ..., with u_i = n_i / |n_i|, up to
 *     the first probe outside the points' bounding box widened by r_d;
 *   d_m = 1 iff some point lies within r_d of y_m;
 *   N = (number of m >= 1 with d_m = 0, d_{m-1} = 1) - 1 (Eq. N_i_define),
 *     N_one = number of leading ones of d;
 *   iteration 0: flip if N is odd (Eq. basic_parity_flip); iteration 1: flip
 *     if N != 0 or N_one > n_tol along the current normal; iteration 2: flip
 *     if N along the current normal exceeds N along its opposite.
 * Every decision is taken in float32 with each operation rounded and no
 * contraction: d2 = ((dx*dx + dy*dy) + dz*dz) <= r_d*r_d, y = x + (m r_d) u,
 * r_{d,0} = 0.5 sqrt(max d2), r_d = gamma r_{d,0}.  A flip negates the
 * normal as given.  Zero or non-finite normals, non-finite points (which are
 * not part of the cloud) and r_d = 0 (fewer than two distinct points) leave
 * normals unchanged.  Rays stop at 2^24 probes.
 * stats [n][5] int32 (may be NULL): N along +n, N_one along +n, N along -n,
 * N_one along -n, flags (1, 2, 4: flipped by iteration 0, 1, 2; 8: final
 * normal is the negated input); zeros where nothing was decided.  rd_out
 * (DEVICE float, may be NULL) receives r_d.  bbox is a HOST array as for
 * wgeo_estimate_normals (it places the search cells only).  gamma >= 1 finite
 * (the paper's default 2.5), n_tol >= 0 (default 2), 0 <= n <= max_points.
 * Uses the normal-estimation workspace only.  Enqueued on `stream`; errors
 * WGEO_ERR_INVALID_ARG (nothing enqueued) or WGEO_ERR_CUDA. */
int wgeo_orient_normals(wgeo_handle* h, const float* points, int64_t n, const float* bbox, float gamma,
                        int32_t n_tol, float* normals, int32_t* stats, float* rd_out, void* stream);

/* Backward of exact queries (Sec. 2.5 with the off-grid distance of
 * wgeo_query_exact): as wgeo_backward, with d_sdf_q [m] the seeds dL/dphi(q)
 * of exact queries at q [m][3] (no normal seeds: the exact gradient is not
 * differentiated again).  Each query's closest point y on its closest
 * triangle carries dL/dP_v = -dL/dphi beta_v (grad phi)(q) to the triangle's
 * vertices (beta the barycentric weights of y), and from there the chain is
 * that of the node seeds.  d_q [m][3] (may be NULL) receives
 * dL/dphi (grad phi)(q).  Grid seeds (d_sdf_grid, d_nrm_grid, either may be
 * NULL) are added as in wgeo_backward.  The queries are searched again
 * (chunked as in wgeo_query_exact).  Requires keep_for_backward. */
int wgeo_backward_exact(wgeo_handle* h, const float* d_sdf_grid, const float* d_nrm_grid, const float* q,
                        const float* d_sdf_q, int64_t m, float* d_points, float* d_normals, float* d_q,
                        void* stream);

/* Synchronises the stream of the handle's last call and copies the device
 * status into *out. */
int wgeo_get_info(wgeo_handle* h, wgeo_info* out);

/* Copies internal fields into caller DEVICE buffers of 4-byte elements
 * [res^3] (stage-by-stage tests, warm-start export), enqueued on `stream`:
 * which = 0 b, 1 chi, 2 phi (last forward, float32); 3 dL/dphi, 4 dL/dchi,
 * 5 lambda (adjoint solution) of the last backward (rounded to float32);
 * 6 the index of each node's closest triangle (Eq. 33) in the order of
 * wgeo_get_mesh, as int32 (-1 for an empty surface; needs keep_for_backward).
 * Returns the element count written or a negative wgeo_status. */
int64_t wgeo_get_field(wgeo_handle* h, int32_t which, float* out, void* stream);

/* Central cell of every point of the last forward (Sec. 2.3, Eq. 25): writes
 * int32 [n][3] (x, y, z) into the DEVICE array `cells`, -1 for points that
 * were skipped as non-finite.  Returns n or a negative wgeo_status. */
int64_t wgeo_get_bins(wgeo_handle* h, int32_t* cells, void* stream);

/* Triangles of the last forward: copies up to `cap` triangles into HOST
 * arrays verts [cap][3][3] (float32) and edge ids [cap][3] (int64: 3 * linear
 * index of the edge's lower node + axis); either may be NULL.  Synchronises
 * the last stream.  Returns the triangle count (may exceed cap) or a negative
 * wgeo_status. */
int64_t wgeo_get_mesh(wgeo_handle* h, float* verts, int64_t* edge_ids, int64_t cap);

/* The marching-cubes case table the library uses (host data, no GPU needed):
 * counts[256] triangles per case and tris[256][5][3] cube edge ids (-1 pad).
 * Corner k of a cube is at (k&1, k>>1&1, k>>2&1); edges 0-3 run along x at
 * (y,z) = (e&1, e>>1), 4-7 along y at (x,z), 8-11 along z at (x,y).  Bit k of
 * the case is set when corner k is inside (chi < c). */
int wgeo_mc_table(int32_t* counts, int32_t* tris);

/* Spherical-harmonic star body r(u) = base + sum_k theta_k Y_k(u) (orthonormal
 * real SH, no Condon-Shortley phase, k = l*l + l + m, K = (lmax+1)^2 <= 81)
 * sampled at unit directions dirs [n][3]: points = centre + r u and outward
 * unit normals (u - P_perp grad r / r normalised).  theta [K], centre [3] and
 * dirs are DEVICE arrays.  Differentiable shape parameterisation used for
 * parameter gradients (Sec. 2.5, last paragraph; Sec. 3.3). */
int wgeo_sh_surface(const float* theta, int32_t K, const float* dirs, int64_t n, float base,
                    const float* centre, float* points, float* normals, void* stream);

/* Adjoint of wgeo_sh_surface: d_theta [K] = sum_i dpts_i . dx_i/dtheta +
 * dnrm_i . dn_i/dtheta, reduced in a fixed order in the handle's workspace
 * (any handle; only its scratch is used).  d_theta is overwritten. */
int wgeo_sh_surface_backward(wgeo_handle* h, const float* theta, int32_t K, const float* dirs, int64_t n,
                             float base, const float* d_points, const float* d_normals,
                             float* d_theta, void* stream);

/* The same adjoint as wgeo_sh_surface_backward, computed by the same kernels
 * in the same order (identical results), without a handle and without
 * allocating any memory: the partial sums go to a fixed array of 256 x 81
 * doubles (162 KB) compiled into the library, one per device.  This entry
 * point has no counterpart in the paper; it serves callers that must not
 * allocate device memory while they run (a serving loop under a fixed memory
 * budget, or code whose allocator owns all device memory) and that hold no
 * reconstruction handle, whose creation allocates its workspace.
 *
 * Limits: K = (lmax+1)^2 <= 81 (lmax <= 8); any n >= 0.  K above 81, or not a
 * square, returns WGEO_ERR_INVALID_ARG with nothing enqueued.  Arrays as for
 * wgeo_sh_surface_backward (DEVICE pointers on the current device, d_theta
 * [K] overwritten), enqueued on `stream`.
 *
 * Set-up: the first call on a device (with that device current) looks up the
 * array's device address and checks the device is sm_103 (else
 * WGEO_ERR_NOT_BUILT_FOR_DEVICE); later calls in the same context reuse the
 * address.  The first call after the device's context has been replaced (by
 * cudaDeviceReset, for example) looks the address up again.  Make that first
 * call before any stream capture.  If the device attributes or the address
 * cannot be read, the call returns WGEO_ERR_CUDA.  No part of the array needs to start
 * at zero: each call writes every slot it reads.  The array is shared by all
 * calls on a device, so calls that may overlap in time (other streams or host
 * threads without ordering between them) race; order them on one stream or
 * with events.  Errors: WGEO_ERR_INVALID_ARG for bad arguments,
 * WGEO_ERR_CUDA if a launch fails. */
int wgeo_sh_surface_backward_noalloc(const float* theta, int32_t K, const float* dirs, int64_t n, float base,
                                     const float* d_points, const float* d_normals, float* d_theta,
                                     void* stream);

/* Number of kernels this library has launched in this process so far: those
 * enqueued from the host on any device and stream, plus those run by the
 * recorded solver graphs' device-side loops on the current device (one body
 * per iteration that ran; recording a graph counts nothing).  Reading the
 * device-side part synchronises the current device.  Never fails; take
 * differences around a region to count its launches. */
int64_t wgeo_kernel_launches(void);

/* Accumulated device time per stage (needs opt.stage_timing): synchronises the
 * handle's recorded events and ADDS, for every stage s < WGEO_NUM_STAGES, the
 * milliseconds and the number of timed calls since the last reset into ms[s]
 * and counts[s] (HOST arrays).  reset != 0 clears the accumulators after the
 * read. */
int wgeo_stage_times(wgeo_handle* h, double* ms, int64_t* counts, int32_t reset);

/* Human-readable text for a wgeo_status code or a status bit mask. */
const char* wgeo_error_string(int code);
const char* wgeo_status_string(uint32_t status_bits);

#ifdef __cplusplus
}
#endif

#endif /* WGEO_H */
