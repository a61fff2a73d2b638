/*
 * tct.h -- C ABI of libtct, point-cloud tomography on one GPU.
 *
 * Method: Yang et al., "Efficient Global Navigational Planning in 3D
 * Structures based on Point Cloud Tomography", arXiv 2403.07631.
 *   Sec. III-A / Alg. 1 (construction)  tomogram construction (tct_build)
 *   Sec. III-B / Eq. 1-6            scene evaluation (tct_evaluate)
 *   Sec. III-C / Eq. 7-9            slice simplification (tct_evaluate)
 *   Sec. III-D                      path search across slices (tct_planner_*, host)
 *   Sec. III-E / Eq. 10             cost and elevation queries (tct_sample_cost)
 *
 * Conventions shared by every entry point:
 *   - Pointers named d_* are device pointers; h_* are host pointers.  The
 *     caller owns every buffer; the library never allocates device memory
 *     (the host-side planner keeps its own host tables).
 *   - Calls are asynchronous on `stream` (NULL = the legacy default stream)
 *     and perform no host synchronisation, so a sequence of calls can be
 *     captured into a CUDA graph (tct_get_status and the autotuner excepted).
 *   - Layered outputs are dense [n_slices][H][W] row-major; row i runs along
 *     +y (cell i covers [y0 + i*res, y0 + (i+1)*res)), column j along +x.
 *   - Return value: TCT_OK (0) or a negative TCT_ERR_* code for errors the
 *     host can see (bad arguments, too small a workspace, a failed launch).
 *     Errors only the device can see (non-finite points) are OR-ed into
 *     tct_stats.status; tct_get_status reads it at a sync point.
 *   - Invalid elevations: ground -inf, ceiling +inf (Sec. III-A: a cell with
 *     no point in the group is invalid).
 */
#ifndef TCT_H
#define TCT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *tct_stream; /* a cudaStream_t */

/* ---- status codes ------------------------------------------------------ */
#define TCT_OK 0
#define TCT_ERR_INVALID_ARG (-1)       /* NULL pointer, bad size or value    */
#define TCT_ERR_WORKSPACE_TOO_SMALL (-2)
#define TCT_ERR_COVERAGE (-3)          /* d_s > d_min, see TCT_ALLOW_COARSE  */
#define TCT_ERR_UNSUPPORTED (-4)       /* beyond a documented limit          */
#define TCT_ERR_CUDA (-5)              /* a CUDA call or launch failed       */

/* device-side status bits (tct_stats.status) */
#define TCT_DEV_NONFINITE 1            /* some points were NaN/inf: skipped  */
#define TCT_DEV_BAD_QUERY 2            /* a query had a bad slice or was NaN */

/* ---- limits -------------------------------------------------------------- */
#define TCT_MAX_SLICES 127             /* N; keeps the uniqueness matrix at 128 bits per slice */
#define TCT_MAX_KERNEL_RADIUS 15       /* inflation window radius in cells   */
#define TCT_MAX_PATCH_RADIUS 4         /* p_s patch radius in cells          */
#define TCT_MAX_POINTS 2000000000LL    /* points (or queries) per call       */
#define TCT_MAX_PATH_LEN 2048          /* waypoints per path of tct_refine_paths */

#define TCT_MAX_BATCH 64               /* maps per batched call              */

/* tile shapes of the slice-stack kernel (tct_tuning.tile) */
#define TCT_TILE_AUTO 0                /* the shape with the least work per SM over whole waves */
#define TCT_TILE_64 1                  /* 64 x 64 cells, 512 threads          */
#define TCT_TILE_32 2                  /* 32 x 32 cells, 512 threads          */
#define TCT_TILE_64x56 3               /* 64 x 56 cells, 448 threads          */
#define TCT_TILE_64x40 4               /* 64 x 40 cells, 320 threads          */
#define TCT_TILE_128x56 5              /* 128 x 56 cells, 896 threads, one CTA per SM */

/* ---- geometry (Sec. III-A) ---------------------------------------------- */
#define TCT_GRID_ZMIN_FROM_DATA 1u     /* z_min = lowest finite z of the cloud (first step of Alg. 1) */

typedef struct tct_grid {
    float x0, y0;      /* world position of the corner of cell (0,0), m       */
    float res;         /* r_g, cell size, m                                    */
    int32_t W, H;      /* columns (along x) and rows (along y)                 */
    float d_s;         /* slice interval d_s, m                                */
    float z_min;       /* plane k is at fl32(z_min + (k+1) d_s), k = 0..N-1    */
    int32_t n_slices;  /* N, 1..TCT_MAX_SLICES                                 */
    uint32_t flags;    /* TCT_GRID_*                                           */
} tct_grid;

/* ---- robot and cost parameters (Sec. III-B, Table I) ------------------- */
#define TCT_KEEP_ENDS 1u               /* always keep the first and last slice   */
#define TCT_ALLOW_COARSE 2u            /* accept d_s > d_min (breaks Sec. III-A's coverage rule) */

typedef struct tct_params {
    float d_min, d_ref;                /* Eq. 1: minimum and normal body height, m   */
    float theta_b, theta_s, theta_p;   /* Eq. 3-4: barrier, slope, step-safety       */
    float c_b;                         /* c^B, cost of a barrier                     */
    float alpha_d, alpha_b, alpha_s;   /* Eq. 1, 4, 3 scaling factors, >= 0          */
    float d_inf, d_sm;                 /* Eq. 6: inflation and safe-margin radii, m  */
    int32_t patch_radius;              /* R_p: p_s patch is (2R_p+1)^2 minus centre  */
    uint32_t flags;                    /* TCT_KEEP_ENDS | TCT_ALLOW_COARSE           */
} tct_params;

/* ---- device-written statistics ----------------------------------------- */
typedef struct tct_stats {
    int32_t status;                    /* OR of TCT_DEV_* bits                       */
    int32_t n_slices;                  /* N of the last call                         */
    int64_t n_points;                  /* points read                                */
    int64_t n_dropped;                 /* finite points outside the grid             */
    int64_t n_nonfinite;               /* NaN/inf points, skipped                    */
    float z_min, z_max;                /* over the finite points                     */
    int32_t n_kept;                    /* slices kept by the simplification          */
    int32_t reserved;
    int64_t valid_cells[TCT_MAX_SLICES + 1]; /* per slice: cells with valid ground   */
    int64_t trav_cells[TCT_MAX_SLICES + 1];  /* per slice: cells with c^T < c^B      */
} tct_stats;

/* Human-readable text of a TCT_OK / TCT_ERR_* code.  Never NULL. */
const char *tct_status_string(int status);

/* ABI version (major * 10000 + minor * 100 + patch). */
int tct_version(void);

/*
 * The sync point for device-detected errors: copies d_stats->status (an OR of
 * TCT_DEV_* bits written by the calls queued before it) to *h_status and
 * waits for `stream`.  The one entry point that synchronises; it does not
 * belong in a captured graph.  TCT_ERR_INVALID_ARG for NULL pointers,
 * TCT_ERR_CUDA when the copy or the stream failed (a launch error included).
 */
int tct_get_status(const tct_stats *d_stats, int32_t *h_status, tct_stream stream);

/*
 * Table I defaults (d_min 0.5, d_ref 0.65, theta_b 1.70, theta_s 0.36,
 * theta_p 0.20, c^B 50, alpha_d 20, alpha_b 20, alpha_s 15) with the Fig. 3
 * inflation distances (d_inf 0.2, d_sm 0.4) and R_p = 2.  `p` must not be NULL.
 */
void tct_params_default(tct_params *p);

/*
 * Sec. III-A: derive a grid from the bounds of a cloud.  h_bounds6 =
 * {x_min, y_min, z_min, x_max, y_max, z_max} (e.g. from tct_bounds).  Sets
 * x0 = x_min, y0 = y_min, W and H so the maximum falls in the last cell,
 * z_min, and N = the smallest count whose last plane is at or above z_max.
 * Returns TCT_ERR_UNSUPPORTED when N would exceed TCT_MAX_SLICES.
 */
int tct_plan_grid(const float *h_bounds6, float res, float d_s, tct_grid *out);

/*
 * Bytes of device workspace tct_build / tct_build_evaluate need for n_points
 * points on `grid`, or tct_evaluate needs when n_points == 0.  `params` may
 * be NULL.  Returns 0 for an invalid grid.
 */
size_t tct_workspace_bytes(const tct_grid *grid, int64_t n_points, const tct_params *params);

/*
 * Bounds of a cloud: d_out6 receives {x_min, y_min, z_min, x_max, y_max,
 * z_max} over the finite points (float, device).  d_xyz: n points, `stride`
 * floats apart (3 = xyz, 4 = xyzw), 16-byte aligned for the vector path.
 * d_stats (may be NULL) receives n_points, n_nonfinite and TCT_DEV_NONFINITE.
 */
int tct_bounds(const float *d_xyz, int64_t n, int32_t stride, float *d_out6,
               tct_stats *d_stats, tct_stream stream);

/*
 * Sec. III-A and the construction part of Alg. 1: ground and ceiling layers.  For every slice
 * k and cell: ground = highest point z <= h_k in the cell, ceiling = lowest
 * point z > h_k, with h_k = fl32(z_min + (k+1) d_s); a point's cell is
 * (floor(fl32(fl32(y-y0)/res)), floor(fl32(fl32(x-x0)/res))).  Points off the
 * grid are dropped and counted; non-finite points are skipped and flagged.
 * d_ground, d_ceil: [N][H][W] float32, written in full.
 */
int tct_build(const float *d_xyz, int64_t n, int32_t stride, const tct_grid *grid,
              void *d_ws, size_t ws_bytes, float *d_ground, float *d_ceil,
              tct_stats *d_stats, tct_stream stream);

/*
 * Sec. III-B and III-C on given layers.  Per slice: gradient magnitudes
 * (Eq. 2, central differences; a cell on the border or next to an invalid
 * ground is a barrier), terrain cost (Eq. 3-4), interval cost (Eq. 1),
 * initial cost (Eq. 5; invalid ground -> c^B), inflation (Eq. 6, window of
 * all taps with K > 0, off-grid taps contribute nothing) into d_cost, and
 * d_mask = (c^T < c^B).  Then the sequential simplification chain (Eq. 7-9,
 * Eq. 8 against the last kept slice, Eq. 9 against the next slice) into
 * d_keep[N] (0/1).  d_ground, d_ceil: [N][H][W]; d_cost [N][H][W] float32;
 * d_mask [N][H][W] uint8; d_keep [N] uint8.  d_aux, when not NULL, receives
 * five [N][H][W] float32 layers: m^xy, m^grad, c^I, c^G, c^init.
 */
int tct_evaluate(const tct_grid *grid, const tct_params *params, const float *d_ground,
                 const float *d_ceil, void *d_ws, size_t ws_bytes, float *d_cost,
                 uint8_t *d_mask, uint8_t *d_keep, float *d_aux, tct_stats *d_stats,
                 tct_stream stream);

/*
 * tct_build followed by tct_evaluate in one pass over the slices (the
 * layers are produced and consumed tile by tile on chip).  Same outputs as
 * the two calls.
 */
int tct_build_evaluate(const float *d_xyz, int64_t n, int32_t stride, const tct_grid *grid,
                       const tct_params *params, void *d_ws, size_t ws_bytes,
                       float *d_ground, float *d_ceil, float *d_cost, uint8_t *d_mask,
                       uint8_t *d_keep, tct_stats *d_stats, tct_stream stream);

/* ---- host buffers in, host buffers out --------------------------------- */

#define TCT_HOST_KEPT_ONLY 1u          /* return only the slices the simplification kept */

/* The host side of tct_build_evaluate_host; host arrays, pinned for asynchronous copies. */
typedef struct tct_host_io {
    const float *h_xyz;                  /* n points, `stride` floats apart           */
    float *h_ground, *h_ceil, *h_cost;   /* [N][H][W] or [M][H][W]; any may be NULL    */
    uint8_t *h_mask;                     /* likewise; may be NULL                      */
    uint8_t *h_keep;                     /* [N]; needed with TCT_HOST_KEPT_ONLY        */
    uint32_t flags;                      /* TCT_HOST_*                                 */
    int32_t n_kept;                      /* out: M, the slices copied (N without KEPT_ONLY) */
} tct_host_io;

/*
 * tct_build_evaluate from host memory to host memory: copies the cloud into
 * d_xyz (device staging of n * stride floats), runs the fused path into the
 * caller's device layers and copies the layers back, one cudaMemcpyAsync
 * per copy, all on `stream`.  Without TCT_HOST_KEPT_ONLY nothing waits: the
 * host arrays are complete when the stream is, and calls on two streams with
 * two sets of buffers overlap one map's copies with the next map's work.
 * With TCT_HOST_KEPT_ONLY the call reads the keep flags (it waits for the
 * stream once), then copies only the kept slices, packed in slice order into
 * [M][H][W] (the simplified tomogram of Sec. III-C) and sets io->n_kept = M.
 * Errors as tct_build_evaluate; TCT_ERR_INVALID_ARG also for a NULL io,
 * h_xyz (n > 0), d_xyz, or h_keep with TCT_HOST_KEPT_ONLY.
 */
int tct_build_evaluate_host(tct_host_io *io, int64_t n, int32_t stride, const tct_grid *grid,
                            const tct_params *params, void *d_ws, size_t ws_bytes, float *d_xyz,
                            float *d_ground, float *d_ceil, float *d_cost, uint8_t *d_mask,
                            uint8_t *d_keep, tct_stats *d_stats, tct_stream stream);

/* ---- queries (Sec. III-E, Eq. 10: C(q), e^G(q)) ------------------------- */

/*
 * Cost and ground elevation at q query points: query t reads slice
 * d_slice[t] (an original slice index) at d_xy[2t], d_xy[2t+1] (world x, y),
 * interpolating bilinearly between cell centres (u = (x-x0)/res - 1/2,
 * v = (y-y0)/res - 1/2, clamped to the grid).  Invalid ground reads as
 * h_k - d_s, so grid->z_min must be the z_min the layers were built with
 * (tct_stats.z_min when TCT_GRID_ZMIN_FROM_DATA).  d_cost / d_ground are the
 * [N][H][W] layers; either output may be NULL.  A query with a slice outside
 * [0, N) or a non-finite coordinate gives NaN and sets TCT_DEV_BAD_QUERY in
 * d_stats (may be NULL).
 */
int tct_sample_cost(const tct_grid *grid, const float *d_cost, const float *d_ground,
                    const float *d_xy, const int32_t *d_slice, int64_t q, float *d_cost_out,
                    float *d_elev_out, tct_stats *d_stats, tct_stream stream);

/*
 * Adjoint of tct_sample_cost: d_gxy[t] = d_gcost[t] * grad C(q_t) +
 * d_gelev[t] * grad e^G(q_t), the gradient of the bilinear interpolant (zero
 * along an axis where the query was clamped).  Either of d_gcost / d_gelev
 * may be NULL (treated as zero).  d_gxy: [q][2].
 */
int tct_sample_cost_backward(const tct_grid *grid, const float *d_cost, const float *d_ground,
                             const float *d_xy, const int32_t *d_slice, int64_t q,
                             const float *d_gcost, const float *d_gelev, float *d_gxy,
                             tct_stream stream);

/*
 * Gradient refinement of waypoint paths on an evaluated tomogram (an
 * objective of this library that uses the queries above): for each of
 * `paths` paths of `len` waypoints (d_xy [paths][len][2], updated in place;
 * d_slice [paths][len]), `steps` descent steps of size eta on
 *   J = sum_w C(x_w) + lambda sum_{w=1}^{len-2} |x_{w+1} - 2 x_w + x_{w-1}|^2
 * with both end points fixed.  One launch for all steps.  len <=
 * TCT_MAX_PATH_LEN.
 */
int tct_refine_paths(const tct_grid *grid, const float *d_cost, const int32_t *d_slice,
                     int32_t paths, int32_t len, int32_t steps, float eta, float lambda,
                     float *d_xy, tct_stream stream);

/* ---- batches of maps ---------------------------------------------------- */

/* One map of a batch: its cloud, its grid and its own output buffers. */
typedef struct tct_map {
    const float *d_xyz;      /* n points, `stride` floats apart (3 or 4)          */
    int64_t n;
    int32_t stride;
    int32_t reserved;        /* 0                                                 */
    tct_grid grid;
    float *d_ground, *d_ceil, *d_cost;   /* [N][H][W] float32                    */
    uint8_t *d_mask;                     /* [N][H][W]                            */
    uint8_t *d_keep;                     /* [N]                                  */
    tct_stats *d_stats;                  /* may be NULL                          */
} tct_map;

/* Launch choices for a batch, from tct_autotune_batched or by hand. */
typedef struct tct_tuning {
    int32_t tile;              /* TCT_TILE_*                                      */
    int32_t ctas_per_sm;       /* persistent CTAs per SM; 0 = as many as fit      */
    int32_t points_per_block;  /* points per block of the two point passes, % 4   */
    int32_t reserved;
} tct_tuning;

/* Workspace of tct_build_evaluate_batched; 0 for an invalid batch. */
size_t tct_workspace_bytes_batched(const tct_map *h_maps, int32_t n_maps,
                                   const tct_params *params);

/*
 * tct_build_evaluate on up to TCT_MAX_BATCH independent maps at once (the
 * batching extension of the method: many maps of uneven size, one set of
 * launches).  h_maps is a host array; the pointers inside it are device
 * pointers.  The point passes run over all clouds together, the per-tile
 * slice stack is one persistent launch that takes (map, tile) items from a
 * queue, largest maps first, and one launch runs every map's chain.  The
 * launch sequence does not depend on the data, so it can be captured into a
 * CUDA graph and replayed.  All maps share the robot parameters; when they
 * also share r_g and the window radii have a specialised kernel the slice
 * stack is one persistent launch, otherwise it runs map after map (each with
 * its own window, the generic kernel where no specialised one exists).
 * tuning may be NULL (defaults).  Each map's outputs are those of
 * tct_build_evaluate on that map alone.
 */
int tct_build_evaluate_batched(const tct_map *h_maps, int32_t n_maps, const tct_params *params,
                               const tct_tuning *tuning, void *d_ws, size_t ws_bytes,
                               tct_stream stream);

/*
 * The construction alone (tct_build) for up to TCT_MAX_BATCH maps: the two
 * point passes over all clouds together, then one launch that walks every
 * cell of every map up its slices; writes each map's d_ground and d_ceil
 * (d_cost, d_mask and d_keep are not used and may be NULL) and its stats
 * (points, dropped, non-finite, z bounds).  The workspace is that of
 * tct_workspace_bytes_batched (params may be NULL there); tuning may be
 * NULL, only its points_per_block is used.  Graph-capturable.  Each map's
 * layers are those of tct_build on that map alone.
 */
int tct_build_batched(const tct_map *h_maps, int32_t n_maps, const tct_tuning *tuning,
                      void *d_ws, size_t ws_bytes, tct_stream stream);

/* Workspace of tct_evaluate_batched: the largest tct_evaluate workspace of the maps. */
size_t tct_workspace_bytes_evaluate_batched(const tct_map *h_maps, int32_t n_maps,
                                            const tct_params *params);

/*
 * The evaluation alone (tct_evaluate) for up to TCT_MAX_BATCH maps whose
 * d_ground / d_ceil already hold layers: writes each map's d_cost, d_mask,
 * d_keep and stats.  The maps run one after another on `stream`, reusing one
 * workspace (an evaluation reads no points, so there is nothing to merge);
 * each map's outputs are those of tct_evaluate on that map alone.  The first
 * failing map's status is returned and the maps after it are not run.
 */
int tct_evaluate_batched(const tct_map *h_maps, int32_t n_maps, const tct_params *params,
                         void *d_ws, size_t ws_bytes, tct_stream stream);

/*
 * Times tct_build_evaluate_batched on this batch for each candidate tuning
 * (tile shape, persistent CTAs per SM, points per block) and writes the
 * fastest into *out.  Runs the batch several times (the outputs are written)
 * and synchronises the stream; call it once per kind of batch, before any
 * capture.
 */
int tct_autotune_batched(const tct_map *h_maps, int32_t n_maps, const tct_params *params,
                         void *d_ws, size_t ws_bytes, tct_stream stream, tct_tuning *out);

/* ---- no-allocation variant ---------------------------------------------- */

/* Scratch compiled into the library for tct_build_evaluate_noalloc, per device. */
#define TCT_NOALLOC_SCRATCH_BYTES (32u << 20)

/*
 * tct_build_evaluate without a workspace argument, for callers that cannot
 * allocate device memory when they need the tomogram (a control loop whose
 * memory is reserved at start-up, a plug-in whose host owns the allocator).
 * The paper has no counterpart; this is an interface convenience.
 *
 * The scratch is a fixed array of TCT_NOALLOC_SCRATCH_BYTES inside the
 * library, held by every GPU that loads the library until the process exits.
 * Returns TCT_ERR_WORKSPACE_TOO_SMALL when tct_workspace_bytes(grid, n,
 * params) exceeds it (about 12 bytes per cell plus 10 per point: the 200 x 200,
 * 200k-point building fits, the 1000 x 1000, 5M-point parking structure does
 * not), and otherwise exactly what tct_build_evaluate returns.  It calls no
 * allocation routine.  The first call on a device looks up the array's device
 * address (with that device current) and should come before any stream
 * capture.  The address is kept for the life of the process: after
 * cudaDeviceReset (or any teardown of the device's primary context) it is
 * stale, so do not call this entry point on that device again.  Every call uses the same array and leaves its contents behind;
 * the call clears what it needs zeroed itself.  Calls that overlap on the GPU
 * race on the array: serialise them.
 */
int tct_build_evaluate_noalloc(const float *d_xyz, int64_t n, int32_t stride,
                               const tct_grid *grid, const tct_params *params, float *d_ground,
                               float *d_ceil, float *d_cost, uint8_t *d_mask, uint8_t *d_keep,
                               tct_stats *d_stats, tct_stream stream);

/* ---- path search across slices (Sec. III-D), a host stage -------------- */

/*
 * A planner over an evaluated tomogram in HOST memory: h_ground and h_cost
 * are the [N][H][W] e^G and c^T layers (grid->n_slices = N), h_keep the keep
 * flags (NULL: every slice).  The planner copies what it reads into a table
 * of 12 bytes per (kept slice, cell): ground, c^T and node cost; the
 * caller's arrays are not used after this call.  Only grid->H, W, n_slices
 * and res are used; c_b is the barrier cost c^B.  TCT_ERR_UNSUPPORTED when
 * the table cannot be allocated.
 *
 * The graph is that of Sec. III-D on the kept slices: a state is a cell on
 * one kept slice and connects to its 8 neighbours on that slice; cells of
 * adjacent kept slices with equal ground are one node, whose cost c^N is
 * the minimum of their c^T; moving onto a node costs c^N plus the Euclidean
 * distance between the nodes in cell units (elevation change / res); nodes
 * with c^N >= c^B cannot be entered; a gateway moves at no cost to the same
 * node on the adjacent kept slice where c^T is lower.  Search: A* with the
 * octile distance to the goal cell as heuristic (optimal path costs).
 * Returns TCT_ERR_INVALID_ARG for a bad grid, NULL arrays or no kept slice.
 */
typedef struct tct_planner tct_planner;
int tct_planner_create(const tct_grid *grid, const float *h_ground, const float *h_cost,
                       const uint8_t *h_keep, float c_b, tct_planner **out);
void tct_planner_destroy(tct_planner *planner);

/*
 * Plans n_queries paths, in parallel on n_threads host threads (<= 0: one
 * per hardware thread).  h_starts / h_goals: [n][3] int32 (i, j, slice); the
 * slice is an original index and must be kept, else TCT_ERR_INVALID_ARG
 * (nothing planned).  Outputs, all host arrays: h_paths [n][max_len][3] the
 * states (i, j, slice) from start to goal, a gateway appearing as two
 * consecutive states of the same cell; h_lens [n] the number of states
 * (0 when the goal cannot be reached or an end point lies on a node with
 * c^N >= c^B); h_costs [n] the path cost (+inf when unreachable);
 * h_expanded [n] states expanded (may be NULL).  A path longer than max_len
 * is cut to its first max_len states, its full length still goes to h_lens,
 * and the call returns TCT_ERR_WORKSPACE_TOO_SMALL.  Each thread holds
 * about 13 bytes per (kept slice, cell) of search state, kept in the
 * planner for later calls.  Calls on one planner may run concurrently.
 */
int tct_plan_paths(tct_planner *planner, int32_t n_queries, const int32_t *h_starts,
                   const int32_t *h_goals, int32_t max_len, int32_t *h_paths, int32_t *h_lens,
                   double *h_costs, int64_t *h_expanded, int32_t n_threads);

/* ---- profiling --------------------------------------------------------- */

/*
 * Turns per-phase timing on (on != 0) or off for the following calls made by
 * the calling thread.  While on, tct_build, tct_evaluate and
 * tct_build_evaluate record CUDA events on their stream around each phase
 * (Sec. IV-A times construction and evaluation separately in the same way).
 * The events are created by the thread's first call that turns timing on, on
 * the device then current; calls on another device are not timed (and
 * tct_timing_read then reports no timed call).
 */
int tct_timing_enable(int on);

/*
 * Phase times of the last timed call, in milliseconds: ms[0] the partition
 * of the points (count, scan, scatter, per-cell sort; 0 for tct_evaluate),
 * ms[1] the per-tile slice-stack kernel (the elevation kernel for
 * tct_build), ms[2] the simplification chain.  Blocks until the call's last
 * event has completed.  Returns the number of values written (<= cap) or a
 * negative TCT_ERR_* code.
 */
int tct_timing_read(float *ms, int cap);

/* Kernels launched by the library since it was loaded (a host-side count). */
int64_t tct_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif /* TCT_H */
