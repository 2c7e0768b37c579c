/*
 * pg.h -- C ABI of the GB300 volumetric path-graph library (libpg.so).
 *
 * The library computes the path-graph estimator of "Rendering Participating
 * Media Using Path Graphs" (Hu, Deng, Luan, Hasan, Marschner) on one GPU:
 *
 *   pg_build_graph        neighbour edges E_N of the path graph (Section 3.1)
 *   pg_aggregate          aggregation weights A+ (Eq. ag-indirect) and the
 *                         direct term A°L° (Eq. ag-direct) per vertex
 *   pg_propagate          Jacobi sweeps of L+ = P A+ L+ + P A°L° (Eq. rte-mff)
 *                         with P from Eq. volume-propagation
 *   pg_gather             per-path output into pixels (Section 4, "Final
 *                         output", "Handling direct light")
 *   pg_record_count,      the instrumented path tracer on the GPU (Section 4,
 *   pg_record_fill        "Instrumented path tracer"): the per-vertex records
 *                         the calls above take, from a voxel medium, lights
 *                         and a pinhole camera
 *   pg_gather_ex          the same with the output options: extra emitter
 *                         samples at the first vertices (Section 4, "Handling
 *                         direct light") and a final gather (Fig. 2 caption)
 *   pg_propagate_adjoint  reverse-mode gradients of an image loss through the
 *                         fixed graph (the paper has no adjoint; this follows
 *                         from differentiating the maps above)
 *
 * Conventions for every call:
 *  - Vertex arrays are indexed in CALLER order: the recorder's path order, a
 *    path's vertices contiguous from first to last (Section 4, "Instrumented
 *    path tracer"). All array pointers are DEVICE pointers allocated and owned
 *    by the caller unless a parameter says "host".
 *  - Calls are asynchronous on `stream` (a cudaStream_t; NULL = legacy
 *    default stream) unless documented to synchronise. Work stays in flight
 *    after return; keep inputs alive until the stream has passed the call.
 *  - Nothing aborts the process. Errors are returned as pg_status; device
 *    errors of earlier asynchronous work surface at the next synchronising
 *    call as PG_ERR_CUDA.
 *  - n = 0 is valid (empty outputs, PG_OK).
 *  - The library allocates its own device memory for the graph object and
 *    temporaries from a stream-ordered memory pool of its own on each device
 *    (created at the first allocation on that device, never released to the
 *    driver before exit, so repeated builds reuse it); the device's default
 *    pool is left untouched. PG_ERR_OOM when an allocation fails.
 */
#ifndef PG_H
#define PG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *pg_stream_t; /* same type as cudaStream_t */

typedef enum {
    PG_OK = 0,
    PG_ERR_INVALID_ARG = 1,  /* bad size, NULL pointer, out-of-range index */
    PG_ERR_OOM = 2,          /* device allocation failed */
    PG_ERR_CUDA = 3,         /* CUDA runtime / launch error */
    PG_ERR_NONFINITE = 4,    /* NaN or Inf in an input array */
    PG_ERR_TIMEOUT = 5,      /* reserved: a bounded device wait ran out */
    PG_ERR_UNSUPPORTED = 6,  /* parameter outside what the library supports */
    PG_ERR_STATE = 7         /* call order: e.g. propagate before aggregate */
} pg_status;

/* Storage type of the edge weights in the propagation sweep. 16-bit types
 * store each row as an FP32 scale times a 16-bit payload; accumulation is
 * FP32 in every case.
 *   PG_W_BF16, PG_W_F16  each weight divided by the row's largest weight,
 *                        rounded to nearest in that format (8 or 11
 *                        significant bits);
 *   PG_W_U16             each weight as 16-bit unsigned fixed point,
 *                        q = round(65535 w / max), scale max / 65535: the
 *                        weights are non-negative and the scale carries the
 *                        range, so every weight has an absolute error of at
 *                        most max / 131070 (the most accurate 16-bit form). */
typedef enum { PG_W_F32 = 0, PG_W_BF16 = 1, PG_W_F16 = 2, PG_W_U16 = 3 } pg_wdtype;

typedef struct pg_graph pg_graph; /* opaque; owns its device buffers */

/* Per-vertex records (caller order, length n, device pointers). They are the
 * quantities the instrumented path tracer records (Section 4):
 *   p     position x_v
 *   o     unit direction from x_v toward the previous vertex / the camera
 *   d     unit phase-sampled direction omega_v (light arrives from x_v + t d)
 *   e     unit emitter-sample direction omega^e_v
 *   g     Henyey-Greenstein asymmetry (|g| < 1), rho(o,d) with mu = -o.d
 *   sigma_s, sigma_t  scattering / extinction coefficient at x_v
 *   w_prop  tau/p_t of the segment that ENTERS x_v (Eq. volume-propagation;
 *           1/sigma_t under delta tracking); for a path's first vertex this
 *           is the camera segment
 *   Le    radiance returned by the emitter sample (transmittance included;
 *         for a delta light already divided by its selection probability)
 *   pe_e  pdf of the emitter-sampling strategy for e (selection included);
 *         ignored for delta lights
 *   e_delta  1 if the emitter sample is a delta light (cannot be hit by
 *            phase sampling), else 0
 *   Lph   emitted radiance found along d when the phase-sampled flight left
 *         the medium (0 otherwise); pe_ph its emitter-strategy pdf
 *   succ  caller index of the next vertex on the same path, or -1 at the
 *         end of a path. Every vertex has at most one predecessor.
 * pg_build_graph reads only px, py, pz; pg_aggregate reads the rest. */
typedef struct {
    const float *px, *py, *pz;
    const float *ox, *oy, *oz;
    const float *dx, *dy, *dz;
    const float *ex, *ey, *ez;
    const float *g, *sigma_s, *sigma_t, *w_prop;
    const float *Le, *pe_e, *Lph, *pe_ph;
    const uint8_t *e_delta;
    const int32_t *succ;
} pg_vertices;

typedef struct {
    int32_t k;          /* neighbours per vertex INCLUDING itself, 1..32 */
    float bbox_lo[3];   /* quantisation box; points outside are clamped */
    float bbox_hi[3];
    int64_t r2_max;     /* drop neighbours with squared quantised distance
                           > r2_max; negative = no radius limit */
    int32_t grid_level; /* hash-grid cells per axis = 2^grid_level (1..10);
                           0 = chosen from n and k */
    int32_t cluster_size; /* 0: kNN neighbourhoods (below). K > 0: the paper's
                           disjoint clusters of expected size K instead
                           (Section 3.1, Section 4 "Path graph solver"):
                           caller vertex v is a centre iff SplitMix64 output v
                           of cluster_seed is below floor((2^64-1)/K) (caller
                           vertex 0 if none is), every vertex joins its nearest
                           centre (squared quantised distance, ties by the
                           smaller caller index), and a cluster of S > k
                           members, in Morton order, is cut into ceil(S/k)
                           parts, member i going to part floor(i P / S);
                           N(s) = s, then the other members of s's part in
                           Morton order. r2_max is ignored. */
    uint64_t cluster_seed;
} pg_build_params;

/* Neighbour edges E_N (Section 3.1: points exchange information with their
 * spatial neighbourhood). Each vertex s gets N(s): itself first, then the
 * k-1 other vertices with the smallest squared distance between 21-bit
 * quantised coordinates q = min(2^21-1, floor((p - lo) * 2^21 / max_extent)),
 * ties broken by the smaller caller index; entries beyond r2_max are
 * dropped. Exact (bit-identical to brute force).
 * Synchronises `stream` twice (to size the exact search of the queries the
 * first ring around each vertex leaves open, and to report non-finite
 * positions; cluster mode synchronises more often to size its lists).
 * Errors: PG_ERR_INVALID_ARG (NULL, n < 0, n >= 2^31-1, bad box),
 * PG_ERR_UNSUPPORTED (k outside 1..32, grid_level > 10), PG_ERR_NONFINITE.
 * *out is freed with pg_graph_destroy. */
pg_status pg_build_graph(const pg_vertices *v, int64_t n, const pg_build_params *params, pg_stream_t stream,
                         pg_graph **out);

/* Copy N(s) out: nbr[s*k + i] (caller indices, row s in caller order, -1 for
 * a missing neighbour when n < k or beyond r2_max). nbr: device, n*k int32. */
pg_status pg_graph_neighbors(const pg_graph *g, int32_t *nbr, pg_stream_t stream);

typedef struct {
    int64_t n;           /* vertices */
    int32_t k;           /* neighbours per row requested */
    int32_t row_width;   /* stored row width (k rounded up to 4, 8, 16, 32) */
    int32_t grid_level;
    int32_t aggregated;  /* 1 after pg_aggregate */
    int64_t n_active;    /* vertices with a predecessor (rows a sweep updates) */
    int64_t nnz_swept;   /* edge updates per sweep: entries (s, j) with j in
                            N(s), s having a predecessor and j a successor */
    int64_t device_bytes;/* device memory held by the graph */
    int32_t weight_dtype;
    int32_t history_iters; /* sweeps stored by the last pg_propagate, -1 none */
    int64_t knn_exact;   /* queries the graph build resolved with its exact
                            (slow) neighbour search: sparse surroundings,
                            large distances or dense ties */
    int64_t clusters;    /* cluster mode: number of neighbourhoods (parts) */
} pg_graph_info;

pg_status pg_graph_get_info(const pg_graph *g, pg_graph_info *info);

/* Aggregation (Section 3.5). Each sample j (vertex j's phase sample d_j and
 * emitter sample e_j) is shared by the vertices that hold j in their
 * neighbourhood, R(j) = {r : j in N(r)}, K_j = |R(j)| (j itself included).
 * Its marginal densities are summed over those vertices' phase strategies
 * (Eq. indirect-weight's p_m; in the paper's clusters R(j) is the cluster):
 *   pm_d(j) = sum_{r in R(j)} rho_r(o_r, d_j),  pm_e(j) = sum_{r in R(j)} rho_r(o_r, e_j)
 * and for every vertex s and j in N(s):
 *   A+_{s,j} = sigma_s(s) rho_s(o_s, d_j) / pm_d(j)           (Eq. ag-indirect)
 *   c_s = sum_{j in N(s)} A°_{s,2j} Le_j + A°_{s,2j+1} Lph_j    (Eq. ag-direct)
 *     A°_{s,2j}   = sigma_s rho_s(o_s,e_j) / (pm_e(j) + K_j pe_e_j),
 *                   or sigma_s rho_s(o_s,e_j) / |N(s)| for a delta light
 *     A°_{s,2j+1} = sigma_s rho_s(o_s,d_j) / (pm_d(j) + K_j pe_ph_j)
 *   D_s = the same direct term with N(s) = {s} (the non-aggregated direct
 *     light used at output, Section 4 "Handling direct light").
 * So sample j's indirect weights over R(j) sum to sigma-weighted one (the
 * balance heuristic of Eq. indirect-weight), and every column of P A+ sums
 * to at most the largest albedo. The marginals are accumulated in 64-bit
 * fixed point (34 fraction bits), so the weights do not depend on the order
 * of the device's atomic additions.
 * The graph keeps the propagation matrix (P A+, Eq. rte-mff) in `wdtype` and
 * P c. c and D (caller order, n floats each, device) are written for the
 * caller; either may be NULL. Synchronises `stream` twice (for the count
 * of rows with a predecessor and the input checks, then for the count of
 * swept entries).
 * Errors: PG_ERR_NONFINITE, PG_ERR_INVALID_ARG (succ out of range, a vertex
 * with two predecessors, |g| >= 1, negative coefficients or pdfs). */
pg_status pg_aggregate(pg_graph *g, const pg_vertices *v, pg_wdtype wdtype, float *c, float *D, pg_stream_t stream);

/* Propagation (Eq. rte-mff, P from Eq. volume-propagation): `iters` Jacobi
 * sweeps of
 *   L+_v <- (tau/p_t)_s * ( sum_{j in N(s)} A+_{s,j} L+_j + c_s ),  s = succ(v),
 * and L+_v = 0 at the end of a path, starting from L0 (the path tracer's
 * incoming-indirect estimate, Section 4 "Path graph solver").
 *   c      caller order, n floats; NULL = the c of the last pg_aggregate
 *   L0     caller order, n floats
 *   L      out, caller order, n floats: L+ after the last sweep run
 *   tol    > 0: stop after the first sweep whose relative change
 *          ||L_t - L_{t-1}||_2 / ||L_t||_2 is < tol (each thread sums its
 *          rows' squares in float32, the threads' sums are added in FP64);
 *          later sweeps return at once on the device (no host round trip)
 *   keep_history  1: the graph keeps every iterate for pg_propagate_adjoint
 *   residual      HOST, `iters` doubles, or NULL (entries past the stop are 0)
 *   iters_done    HOST int32 or NULL
 * Asynchronous unless `residual` or `iters_done` is non-NULL (then it
 * synchronises to copy them). Errors: PG_ERR_STATE (no pg_aggregate),
 * PG_ERR_INVALID_ARG (iters < 0, NULL L0/L). */
pg_status pg_propagate(pg_graph *g, const float *c, const float *L0, int32_t iters, double tol, int32_t keep_history,
                       float *L, double *residual, int32_t *iters_done, pg_stream_t stream);

/* Output (Section 4, "Final output" and "Handling direct light"). Path p
 * with first vertex f carries
 *   val_p = bg_p + (tau/p_t)_f * ( sum_{j in N(f)} A+_{f,j} L_j + D_f )
 * (val_p = bg_p when first[p] = -1, the camera ray left the medium), and
 * pixel i averages its spp paths p = i*spp .. i*spp+spp-1:
 *   image[i] = (1/spp) sum_p val_p,   i = y*width + x.
 * L, D: caller order, n floats; first: n_paths int32 (caller vertex index
 * or -1); bg: n_paths floats; image: width*height floats (out).
 * n_paths must equal width*height*spp. Errors: PG_ERR_STATE, PG_ERR_INVALID_ARG. */
pg_status pg_gather(const pg_graph *g, const float *L, const float *D, const int32_t *first, const float *bg,
                    int64_t n_paths, int32_t spp, int32_t width, int32_t height, float *image, pg_stream_t stream);

/* Extra emitter samples recorded at each path's first vertex (Section 4,
 * "Handling direct light": a few extra emitter samples at the first bounce
 * stand in for the non-aggregated direct light in the output). m samples per
 * path, path p's at [p*m, (p+1)*m); device arrays of n_paths*m entries with
 * the meaning of the vertex fields of the same name (e unit direction toward
 * the light, Le delivered radiance with transmittance, for a delta light
 * divided by its selection probability, pe_e the continuous strategy's pdf,
 * e_delta 1 for a delta light). Entries of paths without a vertex are
 * ignored. */
typedef struct {
    int32_t m;
    const float *ex, *ey, *ez;
    const float *Le, *pe_e;
    const uint8_t *e_delta;
} pg_extra_samples;

typedef struct {
    /* 0: aggregate over N(f) with the graph's weights (pg_gather).
     * 1..32: final gather, one more aggregation at the first vertices only
     * (the optional final gather of the Fig. 2 caption): N_fg(f) = the
     * final_gather_k nearest vertices of f under the graph build's rule
     * (self first, squared quantised distance, ties by caller index, no
     * radius limit; in both neighbourhood modes), weighted by f's balance
     * heuristic over the phase strategies of N_fg(f):
     *   A^fg_{f,j} = sigma_s(f) rho_f(o_f,d_j) / sum_{l in N_fg(f)} rho_l(o_l,d_j) */
    int32_t final_gather_k;
    /* NULL: the output's direct term is D_f. Otherwise the M = extra->m
     * samples and the path's own phase sample, by the balance heuristic:
     *   D^x_f = sigma_s(f) [ sum_m rho_f(o_f,e_m) Le_m / (M pe_m + rho_f(o_f,e_m))
     *                        + rho_f(o_f,d_f) Lph_f / (M pe_ph_f + rho_f(o_f,d_f)) ]
     * where a delta-light sample contributes sigma_s rho_f(o_f,e_m) Le_m / M. */
    const pg_extra_samples *extra;
    /* optional out (device, n_paths*final_gather_k int32): N_fg(f) of each
     * path in caller indices, -1 padded (all -1 for a path without a vertex);
     * NULL to skip. Ignored when final_gather_k = 0. */
    int32_t *fg_nbr;
} pg_output_params;

/* pg_gather with output options (params NULL = pg_gather). Path p with first
 * vertex f carries
 *   val_p = bg_p + (tau/p_t)_f * ( sum_{j} A_{f,j} L_j + Dir_p )
 * with (j, A) from N(f) and A+ (final_gather_k = 0) or from N_fg(f) and
 * A^fg, and Dir_p = D_f or D^x_f; image as in pg_gather. D may be NULL when
 * extra samples are given. Synchronises `stream` once when extra samples are
 * given (to report their validation). Temporary device memory: n_paths *
 * (8 + 4 * row width) bytes for a final gather (row width = final_gather_k
 * rounded up to 4, 8, 16 or 32), plus 4 * n_paths with extra samples. A
 * final gather that searches its neighbourhoods (final_gather_k above the
 * graph's k, a cluster graph or a radius limit) adds n_paths * (4 + 8 *
 * (row width - 1)) + 16 bytes for the first-ring search's queue and the
 * saved lists its queued queries resume from.
 * Errors: PG_ERR_STATE, PG_ERR_INVALID_ARG (sizes, NULL arrays, m < 1,
 * negative Le or pe_e), PG_ERR_UNSUPPORTED (final_gather_k > 32),
 * PG_ERR_NONFINITE (an extra sample). */
pg_status pg_gather_ex(const pg_graph *g, const float *L, const float *D, const int32_t *first, const float *bg,
                       int64_t n_paths, int32_t spp, int32_t width, int32_t height, const pg_output_params *params,
                       float *image, pg_stream_t stream);

/* Adjoint of pg_aggregate -> pg_propagate -> pg_gather for a fixed graph,
 * fixed samples, fixed tau/p_t and a detached L0. Needs the last
 * pg_propagate to have run with keep_history = 1 (its iteration count is
 * used) and the gather to have used that call's L.
 *   dI        dLoss/dImage, width*height floats (device)
 *   first     as in pg_gather
 *   grad_sigma_s, grad_g  out, caller order, n floats each, or NULL:
 *             dLoss/dsigma_s(v) and dLoss/dg(v) (weights re-evaluated as
 *             functions of sigma_s and g, marginals included)
 *   voxel, sigma_t, grad_albedo_vox, n_vox: optional per-voxel albedo
 *             gradient, sigma_s = albedo[voxel(v)] * sigma_t(v):
 *             grad_albedo_vox[x] = sum_{v: voxel(v)=x} sigma_t(v) dLoss/dsigma_s(v)
 *             (overwritten, n_vox floats); pass NULL to skip
 *   recompute_weights  how W^T is applied in the reverse sweeps:
 *             0: from a transposed copy of the stored weights, built on the
 *                first call and kept in the graph (nnz * (4 + weight bytes)
 *                extra memory); deterministic summation order;
 *             1: every edge weight re-evaluated from the vertex records in
 *                each reverse sweep (no weight memory needed at all: works
 *                after pg_graph_release_weights);
 *             2: from the stored weights in their forward row layout, with
 *                atomic adds into the reverse iterate (no transposed copy).
 *             Modes 1 and 2 sum in a non-deterministic order (float atomics).
 *             grad_sigma_s of mode 0 is bitwise reproducible;
 *             grad_g (its marginal terms) and grad_albedo_vox (the sum over a
 *             voxel's vertices) are summed with float atomics, so repeated
 *             calls agree to float rounding, not bitwise.
 * With grad_g, the reverse iterates of every sweep are kept for the call
 * ((iters + 1) * (n + 1) floats of temporary memory).
 * Gradients of vertices with sigma_s = 0 are reported as 0.
 * Errors: PG_ERR_STATE (no history), PG_ERR_INVALID_ARG. */
pg_status pg_propagate_adjoint(pg_graph *g, const float *dI, const int32_t *first, int64_t n_paths, int32_t spp,
                               int32_t width, int32_t height, float *grad_sigma_s, float *grad_g,
                               const int32_t *voxel, const float *sigma_t, float *grad_albedo_vox, int64_t n_vox,
                               int32_t recompute_weights, pg_stream_t stream);

/* Build the transposed copy of the stored weights that pg_propagate_adjoint
 * with recompute_weights = 0 applies (otherwise built by its first call), on
 * `stream`, without a host round trip. It reads only the weights, so it may
 * run on a second stream concurrently with pg_propagate; order
 * pg_propagate_adjoint after it (same stream, or an event). No-op when the
 * copy exists for the current weights. Errors: PG_ERR_STATE (no
 * pg_aggregate or weights released), PG_ERR_OOM. */
pg_status pg_prepare_adjoint(pg_graph *g, pg_stream_t stream);

/* Free the stored edge weights and the transposed copy (after the forward
 * pass, when memory is tight); pg_propagate then returns PG_ERR_STATE and
 * pg_propagate_adjoint needs recompute_weights = 1. */
pg_status pg_graph_release_weights(pg_graph *g);

/* ------------------------------------------------------------------------
 * GPU path recorder (Section 4, "Instrumented path tracer": during path
 * tracing each shading point's emitter-sampling and phase-sampling records
 * and its incoming indirect radiance are recorded, a path's points stored
 * contiguously in path order). One camera path per pixel sample through a
 * pinhole camera into the unit cube [0,1]^3 holding a piecewise-constant
 * voxel medium (nearest voxel); free flights by delta tracking against the
 * grid's largest sigma_t, emitter samples with ratio-tracking transmittance,
 * exact Henyey-Greenstein phase sampling, no Russian roulette (max_depth
 * truncates). Records as described for pg_vertices, plus L0 (the path
 * tracer's incoming indirect radiance along d, the propagation's start) and
 * per path first / bg / the path tracer's value. Paths are traced in single
 * precision (positions, directions, free flights, transmittance; the records
 * are float32 anyway); L0, L0_f64 and the per-path values are then summed in
 * double from those records. Deterministic: the same scene and seed give the
 * same records on every run (and the same as the repository's host
 * recorder, which evaluates the same IEEE-rounded operations in the same
 * order). */
typedef struct {
    int32_t grid_res;        /* voxels per axis */
    const float *density;    /* device, grid_res^3 sigma_t >= 0, index x + G (y + G z) */
    const float *albedo;     /* device, grid_res^3 albedo >= 0 */
    float g;                 /* Henyey-Greenstein asymmetry, |g| < 1 */
    float sun_dir[3];        /* direction the sunlight travels (a delta light) */
    float sun_irradiance;    /* 0 = no sun */
    float sky_radiance;      /* constant environment, 0 = none */
    float area_radiance;     /* one-sided rectangle emitting toward +(u x v); 0 = none */
    float area_center[3], area_u[3], area_v[3]; /* centre and half-edge vectors */
    float p_sun;             /* probability that an emitter sample picks the sun
                                (used when both the sun and a continuous light exist) */
    float p_area;            /* share of the area light among the continuous lights */
    int32_t width, height, spp, max_depth;
    float cam_pos[3], cam_target[3], cam_fov_deg; /* vertical field of view */
    uint64_t seed;
    int32_t extra_direct;    /* extra emitter samples per path at its first vertex
                                (pg_extra_samples), 0 = none */
} pg_scene;

/* Caller-allocated device outputs of pg_record_fill: n = the vertex count
 * from pg_record_count entries per vertex array (caller order), n_paths =
 * width*height*spp per path array, n_paths*extra_direct per extra array.
 * voxel and val may be NULL; the rest are required (x_* only with
 * extra_direct > 0). */
typedef struct {
    float *px, *py, *pz, *ox, *oy, *oz, *dx, *dy, *dz, *ex, *ey, *ez;
    float *g, *sigma_s, *sigma_t, *w_prop, *Le, *pe_e, *Lph, *pe_ph, *L0;
    double *L0_f64;
    uint8_t *e_delta;
    int32_t *succ, *voxel;
    int32_t *first;         /* first vertex of each path, or -1 */
    float *bg;              /* radiance of a camera ray that left the medium */
    double *val;            /* the path tracer's value of each path */
    float *x_ex, *x_ey, *x_ez, *x_Le, *x_pe;
    uint8_t *x_delta;
} pg_recording;

/* Pass 1: trace every path and count its vertices. path_offsets (device,
 * n_paths + 1 int64) receives the exclusive scan of the counts (path p's
 * vertices are [path_offsets[p], path_offsets[p+1])); *n_vertices (host) the
 * total. Synchronises `stream`. Errors: PG_ERR_INVALID_ARG (scene fields, a
 * negative or non-finite grid value), PG_ERR_UNSUPPORTED (2^31 - 1 vertices
 * or more). */
pg_status pg_record_count(const pg_scene *scene, int64_t *path_offsets, int64_t *n_vertices, pg_stream_t stream);

/* Pass 2: trace the same paths again and write their records at the offsets
 * pass 1 produced (same scene, same seed). Asynchronous. */
pg_status pg_record_fill(const pg_scene *scene, const int64_t *path_offsets, const pg_recording *out,
                         pg_stream_t stream);

/* ------------------------------------------------------------------------
 * Sharded sweeps (one shard per GPU). The Jacobi sweep of Eq. rte-mff
 * updates every swept row from the previous iterate only, so the rows split
 * into independent parts. A shard owns a contiguous range of the graph's
 * sweep rows (sweep rows are in Morton order: a range is a spatial slab),
 * cut so that all shards hold nearly the same number of live entries, and
 * iterates a local vector z of local_len floats:
 *     z = [ own rows (row_end - row_begin) | halo (n_halo) | zero slot ]
 * The halo holds the sweep-vector entries its rows read but other shards
 * own (neighbours across the slab boundary, continuation edges leaving the
 * slab), in ascending global order, so the entries owned by shard q are the
 * halo segment [recv_begin[q], recv_begin[q+1]). Shard q sends them, in the
 * same order, as the segment [send_begin[p], send_begin[p+1]) of its packed
 * send buffer. One sweep per shard: pg_shard_pack, exchange the segments
 * (e.g. NCCL send/recv), copy each received segment into the halo, then
 * pg_shard_sweep. Every row is summed in the same order as in pg_propagate,
 * so T sharded sweeps give bitwise pg_propagate's iterate. The sweep vector
 * y (n+1 floats, sweep-row order) relates to L+ by pg_graph_y_from_L and
 * pg_graph_L_from_y; the shards' own rows, gathered into y, give L+. */
typedef struct pg_shard pg_shard;

typedef struct {
    int32_t n_shards, shard, row_width;
    int64_t row_begin, row_end; /* own sweep rows [row_begin, row_end) */
    int64_t n_halo;             /* halo entries */
    int64_t local_len;          /* floats of z: own rows + halo + 1 */
    int64_t n_send;             /* floats of the packed send buffer (all peers) */
} pg_shard_info;

/* Shard `shard` of `n_shards` of an aggregated graph (its swept rows'
 * column table is copied to the host to plan the partition; synchronises
 * `stream`). The shard keeps a pointer to g: destroy it first. Errors:
 * PG_ERR_STATE (no pg_aggregate, weights released), PG_ERR_INVALID_ARG. */
pg_status pg_shard_create(const pg_graph *g, int32_t n_shards, int32_t shard, pg_stream_t stream, pg_shard **out);

/* The same plan from a HOST column table (n_rows rows of row_width entries,
 * entry values in [0, n_rows) or zero_slot >= n_rows for an empty entry),
 * without a device: for inspecting and testing the partition. Such a shard
 * supports only pg_shard_get_info / pg_shard_get_lists / pg_shard_destroy. */
pg_status pg_shard_create_host(const int32_t *col, int64_t n_rows, int32_t row_width, int64_t zero_slot,
                               int32_t n_shards, int32_t shard, pg_shard **out);

pg_status pg_shard_get_info(const pg_shard *s, pg_shard_info *info);

/* HOST copies of the plan, each optional (NULL skips): row_begin
 * (n_shards + 1: shard q owns rows [row_begin[q], row_begin[q+1])),
 * recv_begin (n_shards + 1, halo segments by owner), send_begin
 * (n_shards + 1, send-buffer segments by receiver), halo (n_halo global
 * rows), send_idx (n_send own local rows), local_col (own rows x row_width,
 * the column table re-indexed into z). */
pg_status pg_shard_get_lists(const pg_shard *s, int64_t *row_begin, int64_t *recv_begin, int64_t *send_begin,
                             int32_t *halo, int32_t *send_idx, int32_t *local_col);

/* z (device, local_len floats) from a global sweep vector y (device, n+1):
 * own rows, halo entries, zero slot. */
pg_status pg_shard_load(const pg_shard *s, const float *y, float *z, pg_stream_t stream);

/* send[i] = z[send_idx[i]] for all peers (device, n_send floats). */
pg_status pg_shard_pack(const pg_shard *s, const float *z, float *send, pg_stream_t stream);

/* One sweep of the own rows: z_out[r] = sum_i W[r][i] z_in[local_col[r][i]]
 * (times the row scale of 16-bit weights) + b[r] for r < own rows, with the
 * graph's stored weights and P c of its last pg_aggregate. z_in's halo must
 * hold the previous iterate's values of the peers' rows. z_out's halo and
 * zero slot are not written. Asynchronous. */
pg_status pg_shard_sweep(pg_shard *s, const float *z_in, float *z_out, pg_stream_t stream);

void pg_shard_destroy(pg_shard *s);

/* y (device, n+1 floats, sweep-row order) with y[row of succ(v)] = L[v] and
 * 0 elsewhere; and back: L[v] = y[row of succ(v)], 0 at a path's end. */
pg_status pg_graph_y_from_L(const pg_graph *g, const float *L, float *y, pg_stream_t stream);
pg_status pg_graph_L_from_y(const pg_graph *g, const float *y, float *L, pg_stream_t stream);

/* ------------------------------------------------------------------------
 * The whole hot path from HOST buffers (the path-graph solver of Section 4
 * as one call): the records are copied to the device (positions first on
 * `stream`, which builds the graph from them while the other records are
 * copied on a second stream of the library's), then pg_build_graph,
 * pg_aggregate, pg_propagate, pg_gather and, with a target, the adjoint of
 * the loss 1/2 sum_p (image_p - target_p)^2 (pg_propagate_adjoint, stored
 * transpose); the image and the requested gradients are copied back.
 * Synchronises `stream` before returning; every device buffer it used is
 * released (to the library's pool) and no graph outlives the call. */
typedef struct {
    int32_t k, iters;       /* neighbours per vertex (self included), sweeps */
    pg_wdtype wdtype;
    float bbox_lo[3], bbox_hi[3];
    int32_t spp, width, height;
    int32_t adjoint;        /* 1: run the adjoint when a target is given */
    int64_t n_vox;          /* voxels of the per-voxel albedo gradient */
} pg_step_params;

/* hv: HOST pointers of the vertex records (pg_vertices fields; pinned host
 * memory lets the copies overlap the graph build); L0: host, n floats;
 * first, bg: host, n_paths; target: host width*height floats or NULL;
 * voxel: host, n int32 voxel ids (needed only for grad_albedo_vox).
 * Outputs (host): image (width*height floats), grad_sigma_s (n floats, or
 * NULL), grad_albedo_vox (n_vox floats, or NULL): as in
 * pg_propagate_adjoint. Errors: those of the calls it makes,
 * PG_ERR_INVALID_ARG (sizes, NULL inputs, a gradient without a target). */
pg_status pg_step_host(const pg_vertices *hv, int64_t n, const float *L0, const int32_t *first, const float *bg,
                       int64_t n_paths, const float *target, const int32_t *voxel, const pg_step_params *params,
                       float *image, float *grad_sigma_s, float *grad_albedo_vox, pg_stream_t stream);

void pg_graph_destroy(pg_graph *g);
const char *pg_status_string(pg_status s);

/* Propagation for callers that cannot allocate device memory at the time of
 * the call (no counterpart in the paper: it is a deployment variant of
 * pg_propagate). Examples are host applications that hand this library a
 * fixed memory budget at start-up and allow no further allocation, and
 * per-frame loops that must not allocate once set-up is done, because an
 * allocation in the middle of a frame can stall on the allocator or fail for
 * lack of memory. The graph itself is still made by pg_build_graph and
 * pg_aggregate at set-up, which do allocate.
 *
 * It runs the same Jacobi sweeps as pg_propagate with c = NULL, no history
 * and no residual output: `iters` sweeps from L0 (caller order, n floats),
 * stopping early on the device when tol > 0, writing L (caller order, n
 * floats). Its scratch (two iterates, residual partials and control words)
 * lives in one file-scope device array of 32 MiB + 96 KiB, reserved on a
 * device when the library's device code is first loaded there and held
 * until the process exits. Under CUDA's default lazy module loading that
 * can be this call's first use on the device, which then reports PG_ERR_OOM
 * if the device has no room for the array: make one call (or any other
 * library call) on each device at set-up, or set CUDA_MODULE_LOADING=EAGER.
 * The first call on each device also looks up that array's device address;
 * make that first call before any stream capture. Every call shares the array and the array keeps
 * the previous call's contents (the call resets what must start at zero), so
 * calls whose work overlaps on the GPU -- on any stream, for any graph --
 * race and corrupt each other's results: serialise them.
 * Errors: PG_ERR_UNSUPPORTED when n > PG_NOALLOC_MAX_VERTICES or
 * iters > PG_NOALLOC_MAX_ITERS; PG_ERR_STATE (no pg_aggregate, or weights
 * released); PG_ERR_INVALID_ARG; PG_ERR_OOM (the array could not be
 * reserved, see above). It calls no allocation routine. */
#define PG_NOALLOC_MAX_VERTICES 4194303
#define PG_NOALLOC_MAX_ITERS 4096
pg_status pg_propagate_noalloc(pg_graph *g, const float *L0, int32_t iters, double tol, float *L,
                               pg_stream_t stream);

/* Diagnostic (no counterpart in the paper): number of CUDA kernels this
 * library has launched in the process so far. Thread-safe; never fails. */
int64_t pg_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif /* PG_H */
