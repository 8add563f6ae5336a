/*
 * fgb: periodic neighbor query, radial distribution function and Steinhardt order
 * parameters on one GB300 GPU (sm_103a).  C ABI of libfgb.so.
 *
 * The operations follow freud (arXiv 1906.06317):
 *   - Box and NeighborQuery: Section "Implementation" (a triclinic box with three
 *     linearly independent vectors, centred on the origin; a NeighborQuery built from
 *     (box, points) answers queries by cutoff r_max or by neighbor count, with
 *     exclude_ii), and Section "General Utilities" (cell-list subclass, periodicity at
 *     the lowest level, NeighborList as stored query results).
 *   - RDF: the density module ("Analysis Modules"), histogram accumulated over frames
 *     with reset=False ("Implementation", Compute classes).
 *   - PMFT(x, y): the pmft module (Section "Potentials of Mean Force and Torque").
 *   - Steinhardt q_l: the order module ("Analysis Modules", bond-orientational order
 *     parameters of Steinhardt et al. 1983).
 *
 * Conventions for every call:
 *   - Box params (Lx, Ly, Lz, xy, xz, yz): a1 = (Lx,0,0), a2 = (xy Ly, Ly, 0),
 *     a3 = (xz Lz, yz Lz, Lz); the box spans M (s - 1/2) for s in [0,1)^3.
 *     Lz = 0 is a 2D box (Section "Implementation": two- or three-dimensional boxes):
 *     xz = yz = 0 (INVALID_ARG otherwise), there is no periodicity along z, the
 *     smallest width is the parallelogram's, and every point and query point must have
 *     z = 0 (results for other z are unspecified but memory-safe).  The RDF of a 2D
 *     system uses the box area and annulus shells.
 *   - Points are device pointers to float32 arrays of shape (n, 3), row-major
 *     (x0 y0 z0 x1 ...), owned by the caller; they must stay valid and unchanged for
 *     the lifetime of any handle built from them.  Points may lie outside the box.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls enqueue work on
 *     it; a call that must return a size to the host (fgb_nq_query) synchronises it.
 *   - Handles own the device memory they allocate (stream-ordered allocations on the
 *     stream of the call that made them); *_destroy frees it and accepts NULL.
 *   - Every call returns FGB_OK (0) or a negative FGB_ERR_* code and records a message
 *     for fgb_last_error() (thread-local).  No C++ exception crosses this boundary.
 *   - Distances use the minimum image; a pair (i, j) is a neighbor when its distance r
 *     satisfies r < r_max (strict).  r is defined by one fixed FP64 sequence: d = x_j - x_i
 *     reduced along a3, a2, a1 by rint(component / box length), r = sqrt((dx dx + dy dy)
 *     + dz dz).  Kernels decide in FP32 and re-decide every pair within a proven
 *     error band of an edge with that FP64 sequence, so neighbor sets and histogram
 *     counts are exact with respect to it.
 */
#ifndef FGB_H
#define FGB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FGB_OK 0
#define FGB_ERR_INVALID_ARG (-1)   /* bad pointer, size or parameter */
#define FGB_ERR_BOX_TOO_SMALL (-2) /* r_max (or the k-th neighbor distance) >= half the smallest box width */
#define FGB_ERR_OOM (-3)           /* device allocation failed */
#define FGB_ERR_CUDA (-4)          /* a CUDA runtime call or kernel launch failed */
#define FGB_ERR_UNSUPPORTED (-5)   /* valid request outside what this build implements */
#define FGB_ERR_CAPACITY (-6)      /* a documented size limit was exceeded */

typedef struct fgb_box {
    double Lx, Ly, Lz, xy, xz, yz;
} fgb_box;

/* Query arguments (freud's query dict): exactly one of r_max > 0 (ball query) or
 * num_neighbors > 0 (k nearest) is set.  exclude_ii drops pairs whose query index equals
 * the point index. */
typedef struct fgb_query_args {
    double r_max;
    int32_t num_neighbors;
    int32_t exclude_ii;
} fgb_query_args;

typedef struct fgb_nq fgb_nq;
typedef struct fgb_nlist fgb_nlist;
typedef struct fgb_rdf fgb_rdf;
typedef struct fgb_steinhardt fgb_steinhardt;
typedef struct fgb_clusters fgb_clusters;
typedef struct fgb_batch fgb_batch;
typedef struct fgb_pmft fgb_pmft;

/* ------------------------------------------------------------- library state */

/* Message of the last failed call on this host thread ("" if none). */
const char *fgb_last_error(void);
/* Library ABI version (major*10000 + minor*100 + patch). */
int32_t fgb_version(void);

/* Diagnostics.  fgb_kernel_launches: kernels launched by this library since it was
 * loaded (all threads).  fgb_timing_enable(1) brackets every later launch with CUDA
 * events on its stream; fgb_timing_read waits for the recorded events and returns the
 * summed device time (ms) and launch count of kernels named `name` (the __global__
 * function name, e.g. "k_ball_write"); fgb_timing_reset clears the totals. */
int64_t fgb_kernel_launches(void);

/* Device memory of the library comes from a memory pool of its own on each device (the
 * device's default pool, shared with torch and other libraries, is left as it is).
 * Device blocks of 1 MB or more freed by the library (neighbor lists, sort buffers) are
 * kept, up to the cache limit, and handed to later allocations of a similar size on
 * any stream (ordered by an event recorded when they were freed); the pool also keeps
 * up to the cache limit of freed memory mapped.  fgb_trim_memory waits for the kept
 * blocks' last use and returns them and the pool's unused memory to the device.
 * fgb_set_memory_cache sets the cache limit in bytes (default 4 GB, or the environment
 * variable FGB_MEMORY_CACHE_MB read at load) and releases kept blocks beyond it. */
int fgb_trim_memory(void);
int fgb_set_memory_cache(uint64_t bytes);
int fgb_timing_enable(int32_t on);
int fgb_timing_read(const char *name, double *total_ms, int64_t *count);
int fgb_timing_reset(void);

/* --------------------------------------------------------- NeighborQuery (cell list) */

/*
 * Builds a cell-list NeighborQuery over `n` points (Section "General Utilities": the
 * cell-list NeighborQuery subclass).  Work on `stream`: box wrap and fractional
 * transform, cell index per point, stable radix sort by cell index, cell start offsets.
 * Cells are at least `r_cell` wide along every reciprocal axis; any later query with
 * r_max > r_cell widens its stencil instead of failing.
 * n may be 0.  Errors: INVALID_ARG (n < 0, points NULL with n > 0, r_cell <= 0,
 * degenerate box), OOM, CUDA.
 */
int fgb_nq_create(const fgb_box *box, const float *points, int64_t n, double r_cell, void *stream,
                  fgb_nq **out);
void fgb_nq_destroy(fgb_nq *nq);

/*
 * A NeighborQuery of the box and the points only, with no search structure: for the
 * computes that take a NeighborList (Steinhardt forward and backward, W_l, averages,
 * descriptors, RDF / PMFT from a list, clusters, solid-liquid), e.g. a Q_l evaluated
 * every step of a biased-sampling loop over a fixed list.  No device work, no
 * allocation; fgb_nq_query on it is UNSUPPORTED.  points must outlive the handle.
 */
int fgb_nq_create_points(const fgb_box *box, const float *points, int64_t n, fgb_nq **out);

/* ----------------------------------------------------- NeighborQuery (AABB tree) */

/*
 * Builds a tree NeighborQuery over `n` points (Section "General Utilities": the AABBQuery
 * subclass of NeighborQuery, benchmarked in Fig. 3): a bounding-volume hierarchy over the
 * points wrapped into the box, ordered by 30-bit Morton code (radix tree built in
 * parallel, boxes refit bottom-up).  The handle is an fgb_nq: fgb_nq_query answers ball
 * (r_max) and k-nearest (num_neighbors <= 32) queries with the same NeighborList, bit for
 * bit in the pairs and their order, as the cell list (kNN with exclude_ii over separate
 * query points needs more than k points: UNSUPPORTED otherwise), and fgb_rdf_compute /
 * fgb_steinhardt_compute take it together with a NeighborList.  The call synchronises `stream` once (it checks the coordinates).
 * Points (and query points) must lie within two box lengths of the box centre
 * (|s - 1/2| <= 2 in fractional coordinates); points inside the box keep their exact
 * coordinates.  n may be 0.  Errors: INVALID_ARG (n < 0, points NULL with n > 0,
 * degenerate box, points out of range), CAPACITY (n >= 2^31), OOM, CUDA.
 */
int fgb_aabb_create(const fgb_box *box, const float *points, int64_t n, void *stream, fgb_nq **out);

/* Cell grid of a NeighborQuery: cells per axis (x, y, z) and number of points (a tree
 * NeighborQuery reports 0 cells). */
int fgb_nq_dims(const fgb_nq *nq, int32_t ncell[3], int64_t *n_points);

/*
 * Device views of the cell list (owned by nq, valid until fgb_nq_destroy):
 *   sorted      (n, 4) float32: cell-local x, y, z and the original point index stored
 *               as the bit pattern of the 4th float, in (cell, index) order;
 *   sorted_cell (n) uint32: cell index of each sorted entry;
 *   cell_start  (ncells + 1) uint32: entries of cell c are cell_start[c] .. cell_start[c+1].
 * Cell index = (cz * ny + cy) * nx + cx.  UNSUPPORTED for a tree NeighborQuery.
 */
int fgb_nq_cells(const fgb_nq *nq, const float **sorted, const uint32_t **sorted_cell,
                 const uint32_t **cell_start);

/*
 * Query (Section "Implementation": queries by cutoff distance or by number of
 * neighbors) producing a NeighborList sorted by (query index, point index) for ball
 * queries and by (query index, distance, point index) for k-nearest queries.
 * query_points == NULL queries the NeighborQuery's own points (n_query ignored).
 * Ball query: count pass, exclusive scan into int64 segment offsets, write pass; the
 * call synchronises `stream` once to size the output.  kNN: min(k, available)
 * neighbors per query; FGB_ERR_BOX_TOO_SMALL if a selected neighbor is at distance
 * >= w_min/2 (the minimum image would be ambiguous) or if r_max >= w_min/2.
 */
int fgb_nq_query(fgb_nq *nq, const float *query_points, int64_t n_query, const fgb_query_args *args,
                 void *stream, fgb_nlist **out);

/*
 * The self ball query of fgb_nq_query (same Section; query_points = the NeighborQuery's
 * own points, args->r_max > 0, args->num_neighbors = 0) without a host synchronisation:
 * the list's arrays are allocated for `capacity` pairs up front (0: an estimate for
 * uniformly spread points, n(n-1)·ball volume/box volume + 10 % + 8 per point), the
 * count, scan and write passes are queued on `stream`, and the call returns.  The list
 * is then pending: fgb_nlist_wait completes it, and every call that reads a list
 * (fgb_nlist_size, fgb_nlist_arrays, fgb_nlist_escalations and the analyses that take a
 * NeighborList) waits for it first.  Completing waits for the queued work; when the
 * list turned out larger than `capacity`, or held a row longer than 128 in a cell whose
 * candidates exceed the write kernel's stage, the write pass runs again by the
 * synchronous route into arrays of the exact size (the result is the same list;
 * fgb_nlist_wait reports that it happened).  The result is identical to fgb_nq_query's.
 * nq must stay alive and unchanged until the list is completed or destroyed; destroying
 * a pending list is allowed.  Queries without the cell-tile route (a tree NeighborQuery,
 * grids with fewer than 2s+1 cells per axis, the thread-per-query kernels) run
 * fgb_nq_query and return a complete list.  Errors: FGB_ERR_INVALID_ARG (NULL argument,
 * not a ball query, capacity < 0), FGB_ERR_BOX_TOO_SMALL, FGB_ERR_OOM; errors of the
 * queued work are reported by the call that completes the list.
 */
int fgb_nq_query_async(fgb_nq *nq, const fgb_query_args *args, int64_t capacity, void *stream,
                       fgb_nlist **out);

/* Completes a pending list (no-op for a complete one).  *rewritten (may be NULL) is set
 * to 1 when the write pass had to run again (capacity too small, or a long row in a
 * cell beyond the write kernel's stage), else 0. */
int fgb_nlist_wait(fgb_nlist *nl, int32_t *rewritten);

/* --------------------------------------------------------------- NeighborList */

int fgb_nlist_size(const fgb_nlist *nl, int64_t *n_pairs, int64_t *n_query);

/*
 * Device arrays of a NeighborList (owned by nl; any pointer argument may be NULL):
 *   query_point_indices, point_indices: int32 (n_pairs);  distances: float32 (n_pairs);
 *   segments: int64 (n_query + 1), pairs of query i are segments[i] .. segments[i+1];
 *   counts: int32 (n_query).
 */
int fgb_nlist_arrays(const fgb_nlist *nl, const int32_t **query_point_indices, const int32_t **point_indices,
                     const float **distances, const int64_t **segments, const int32_t **counts);

/* Number of pair decisions that fell inside the FP32 error band and were re-decided in
 * FP64 while building this list (a diagnostic). */
int fgb_nlist_escalations(const fgb_nlist *nl, int64_t *n);

/*
 * NeighborList from caller arrays (device; query_point_indices must be non-decreasing;
 * distances may be NULL).  The arrays are copied.  symmetric != 0 promises that (j, i) is
 * present whenever (i, j) is (a self ball query), which lets the Steinhardt backward use
 * its deterministic gather form.
 */
int fgb_nlist_from_arrays(int64_t n_query, int64_t n_points, const int32_t *query_point_indices,
                          const int32_t *point_indices, const float *distances, int64_t n_pairs,
                          int32_t symmetric, void *stream, fgb_nlist **out);
void fgb_nlist_destroy(fgb_nlist *nl);

/* ------------------------------------------------------------------------ RDF */

/*
 * Radial distribution function (density module; Section "Potentials of Mean Force and
 * Torque" relates g(r) = exp(-beta F(r))).  Bin b holds R_b <= r < R_{b+1},
 * R_b = r_min + b ((r_max - r_min)/bins), R_bins = r_max.  Errors: INVALID_ARG for
 * bins <= 0, r_min < 0, r_max <= r_min.
 */
int fgb_rdf_create(int32_t bins, double r_max, double r_min, fgb_rdf **out);
void fgb_rdf_destroy(fgb_rdf *rdf);

/*
 * Adds the ordered-pair distance histogram of one frame to the accumulator (reset != 0
 * clears it first: freud's compute(..., reset=False) accumulation).
 * nlist == NULL: fused cell-list query; pairs are never stored; query_points == NULL
 * means the NeighborQuery's own points with exclude_ii (each unordered pair is visited
 * once and counted twice).  nlist != NULL: histogram of the list's pairs (distances
 * recomputed and decided exactly).  Frames of one accumulation share a dimension (2D or
 * 3D; INVALID_ARG otherwise).  Asynchronous on `stream`.
 */
int fgb_rdf_compute(fgb_rdf *rdf, fgb_nq *nq, const float *query_points, int64_t n_query,
                    const fgb_nlist *nlist, int32_t reset, void *stream);

/*
 * Copies the accumulated counts (uint64, bins), g(r) (float64, bins; counts divided by
 * sum over frames of N_query (N_points / V) (4 pi/3)(R_{b+1}^3 - R_b^3); for 2D frames
 * V is the box area and the shell pi (R_{b+1}^2 - R_b^2)) and bin centres
 * r_min + (b + 1/2) (r_max - r_min)/bins to host arrays (any may be NULL).  Synchronises
 * `stream`.
 */
int fgb_rdf_result(fgb_rdf *rdf, uint64_t *counts, double *rdf_values, double *bin_centers, void *stream);

/* Device pointer of the uint64 accumulator (bins entries), for graph-captured use and
 * for summing the partial histograms of sharded frames across ranks. */
int fgb_rdf_counts_device(const fgb_rdf *rdf, const uint64_t **counts);

/* The RDF's bins and range (any pointer may be NULL). */
int fgb_rdf_params(const fgb_rdf *rdf, int32_t *bins, double *r_max, double *r_min);

/* Number of pairs re-decided in FP64 by the last compute (synchronises `stream`). */
int fgb_rdf_escalations(fgb_rdf *rdf, int64_t *n, void *stream);

/*
 * Allocation-free RDF of one frame (self query, exclude_ii), for callers that cannot
 * allocate device memory while they run: a simulation engine analysing inside its time
 * step with a fixed memory budget, a runtime whose memory pool owns the device and
 * treats an outside cudaMalloc (which may synchronise the device) as an error.  The
 * paper has no counterpart; it is the same computation as fgb_rdf_compute with
 * reset != 0 and no NeighborList.
 *   points: device float32 (n, 3); counts: device uint64 (bins), overwritten with the
 *   ordered-pair counts of bins [r_min + b (r_max - r_min)/bins, ...).
 * Limits: n <= 262144 points, bins <= 8192 (FGB_ERR_CAPACITY beyond), and the
 * FGB_ERR_BOX_TOO_SMALL / FGB_ERR_INVALID_ARG rules of the other RDF calls.
 * All working memory (cell list, sort buffers, thresholds, band-pair list; about 24 MB)
 * is one static device array of the library, held by every GPU that loads it until the
 * process exits.  The first call on a device looks up that array's device address, so
 * make the first call on each device before any stream capture; that address lives as
 * long as the device's context, so use after a cudaDeviceReset of a device already used
 * here is not supported.  Every call shares the
 * array and leaves its contents behind (each call clears what must start at zero):
 * calls whose work overlaps on the GPU (different streams, other threads) race and must
 * be serialised by the caller.  No cudaMalloc, cudaFree or allocating library routine is
 * called.
 */
int fgb_rdf_noalloc(const fgb_box *box, const float *points, int64_t n, int32_t bins, double r_max, double r_min,
                    uint64_t *counts, void *stream);

/* ----------------------------------------------- one frame split across ranks */

/*
 * One frame sharded by contiguous ranges of query cells (Section "Implementation": the
 * parallel wrappers split per-particle work across workers; here a worker is one GPU
 * holding every point of the frame, so no halo is exchanged).  Cells are numbered
 * (z * ny + y) * nx + x on the grid of fgb_nq_dims, so a range is a stack of z slabs.
 * The ranges of all ranks must partition [0, nx*ny*nz).  Between the calls the caller
 * sums the ranks' partial counts and histograms (an all-reduce); the library does no
 * communication.  These calls take the cell-tile route (self query, exclude_ii as
 * given, every axis at least 2s+1 cells and at most 128 stencil cells; UNSUPPORTED
 * otherwise) and synchronise `stream` where noted.
 *
 * fgb_nq_count_cells: overwrites counts[n] (uint32, device, caller's point order) with
 * this range's partial neighbor counts of the ball query r_max: each unordered pair whose
 * half-stencil cell lies in the range adds one to both of its points (plus one for the
 * self pair of the range's own points when exclude_ii == 0).  The sum over the ranges is
 * every point's neighbor count.  Asynchronous.
 */
int fgb_nq_count_cells(fgb_nq *nq, double r_max, int32_t exclude_ii, int64_t cell_lo, int64_t cell_hi,
                       uint32_t *counts, void *stream);

/*
 * From the summed counts (device, n): local_segments (device int64, n + 1) = exclusive
 * scan of the counts of the points in cells [cell_lo, cell_hi) (other points get empty
 * rows), global_segments (device int64, n + 1, may be NULL) = exclusive scan of all
 * counts (the row starts of the whole frame's NeighborList), and on the host the
 * range's number of pairs and its largest count (either pointer may be NULL).
 * Synchronises `stream`.
 */
int fgb_nq_shard_segments(const fgb_nq *nq, int64_t cell_lo, int64_t cell_hi, const uint32_t *counts,
                          int64_t *local_segments, int64_t *global_segments, int64_t *n_local_pairs,
                          uint32_t *max_count, void *stream);

/*
 * Writes the rows of the range's query points, each sorted by point index as in
 * fgb_nq_query, at segments[i] (device int64, n + 1; e.g. the local segments above) into
 * caller-allocated device arrays qi, pj (int32) and dist (float32) of the range's pair
 * count.  counts: the summed counts; max_count: their largest value over the range.
 * Synchronises `stream`; CUDA if a row disagrees with its count.
 */
int fgb_nq_write_cells(fgb_nq *nq, double r_max, int32_t exclude_ii, int64_t cell_lo, int64_t cell_hi,
                       const int64_t *segments, const uint32_t *counts, uint32_t max_count, int32_t *qi,
                       int32_t *pj, float *dist, void *stream);

/*
 * fgb_rdf_compute of the NeighborQuery's own points restricted to the pairs whose
 * half-stencil cell lies in [cell_lo, cell_hi) (each unordered pair counted twice, as
 * there); the ranges' accumulators sum to the frame's histogram.  The normalisation
 * counts the whole frame, so g(r) of the summed counts is the frame's.  At most 1024
 * bins.  Asynchronous.
 */
int fgb_rdf_compute_cells(fgb_rdf *rdf, fgb_nq *nq, int64_t cell_lo, int64_t cell_hi, int32_t reset,
                          void *stream);

/* ------------------------------------------------------------------------ PMFT */

/*
 * Potential of mean force and torque in the plane, PMFT(x, y) (pmft module; Section
 * "Potentials of Mean Force and Torque": the PMFT relation, a histogram of the relative
 * configurations accumulated over frames and its negative logarithm; Fig. 6 benchmarks
 * it against the RDF on a 2D system).  Bins cover [-x_max, x_max) x [-y_max, y_max)
 * with bins_x x bins_y cells (x major).  Errors: INVALID_ARG for non-positive or
 * non-finite extents, bin counts <= 0 or more than 2^26 bins.
 */
int fgb_pmftxy_create(double x_max, double y_max, int32_t bins_x, int32_t bins_y, fgb_pmft **out);
void fgb_pmftxy_destroy(fgb_pmft *pmft);

/*
 * Adds one frame: every bond (i, j), d = x_j - q_i (minimum image), turned by -theta_i
 * into the frame of query particle i:
 *   x' = cos(theta_i) d_x + sin(theta_i) d_y,   y' = cos(theta_i) d_y - sin(theta_i) d_x,
 * is counted in bin (floor((x' + x_max)/dx), floor((y' + y_max)/dy)), dx = 2 x_max/bins_x,
 * dy = 2 y_max/bins_y, when it lies inside the bin rectangle; every bond is decided in
 * FP64 from the defining displacement (cos and sin of the float32 angle in FP64).
 *   nq: a NeighborQuery over a 2D box (INVALID_ARG otherwise).
 *   query_points: device float32 (n_query, 3), or NULL for nq's own points (then
 *     n_query must equal the point count and bonds exclude i == j).
 *   query_orientations: device float32 (n_query) angles theta_i about z, in radians.
 *   nlist: the bonds (query indices address the query points, point indices nq's
 *     points), or NULL for every pair (i != j for self queries): all bonds within
 *     R = (1 + 1e-6) sqrt(x_max^2 + y_max^2), which holds every bond that can land in a
 *     bin.  Self queries on a cell list take a fused kernel (pairs never stored; FP32
 *     with a proven margin from every edge, the rest in FP64); others build that list
 *     internally (which synchronises `stream` once).
 *   reset != 0 clears the histogram first (freud's compute(..., reset=False) otherwise).
 * Errors: BOX_TOO_SMALL when R >= half the smallest box width; INVALID_ARG for NULL or
 * mismatched arguments.  Asynchronous on `stream` otherwise.
 */
int fgb_pmftxy_compute(fgb_pmft *pmft, fgb_nq *nq, const float *query_points, const float *query_orientations,
                       int64_t n_query, const fgb_nlist *nlist, int32_t reset, void *stream);

/*
 * Host copies (any may be NULL) of the accumulated counts (uint64), the pair
 * correlation pcf = counts / (norm * bin area), norm = sum over frames of
 * N_query N_points / (box area), and PMFT = -log(pcf) in units of k_B T (+infinity for
 * an empty bin); each bins_x * bins_y, x major.  Synchronises `stream`.
 */
int fgb_pmftxy_result(const fgb_pmft *pmft, uint64_t *counts, double *pcf, double *pmft_values, void *stream);

/* Device pointer of the uint64 accumulator (bins_x * bins_y entries, x major). */
int fgb_pmftxy_counts_device(const fgb_pmft *pmft, const uint64_t **counts);

/* Bonds the last compute's fused kernel left to its FP64 pass (0 for the list route);
 * synchronises `stream`. */
int fgb_pmftxy_escalations(fgb_pmft *pmft, int64_t *n, void *stream);

/* ----------------------------------------------------------------- Steinhardt */

/*
 * Steinhardt q_l (order module): Q_lm(i) = (1/n_i) sum_j Y_lm(u_ij),
 * q_l(i) = sqrt(4 pi/(2l+1) sum_m |Q_lm(i)|^2); q_l = 0 for a particle without
 * neighbors.  0 <= l <= 12.
 */
int fgb_steinhardt_create(int32_t l, fgb_steinhardt **out);
void fgb_steinhardt_destroy(fgb_steinhardt *st);

/*
 * q_out: device float32 (n points).  Neighbors come from `nlist` when it is not NULL
 * (its query indices address nq's points), otherwise from a fused self ball query with
 * qargs->r_max (no list is stored).  Keeps Q_lm (m = 0..l) and the neighbor counts for
 * fgb_steinhardt_backward.  Asynchronous on `stream`.
 */
int fgb_steinhardt_compute(fgb_steinhardt *st, fgb_nq *nq, const fgb_nlist *nlist, const fgb_query_args *qargs,
                           float *q_out, void *stream);

/* Device views of the last compute: Q_lm as float32 (n, l+1, 2) (re, im) and int32
 * neighbor counts (n). */
int fgb_steinhardt_state(const fgb_steinhardt *st, const float **qlm, const int32_t **n_neighbors);

/*
 * Gradient of Q = (1/n) sum_i q_l(i) times `upstream` with respect to the positions,
 * neighbor list fixed (requires the nlist used by the last compute; q from that
 * compute).  grad_out: device float32 (n, 3), overwritten.  A symmetric list (self ball
 * query) uses a deterministic gather over each particle's neighbors; other lists use
 * a scatter with float atomics.
 */
int fgb_steinhardt_backward(fgb_steinhardt *st, fgb_nq *nq, const fgb_nlist *nlist, const float *q,
                            float upstream, float *grad_out, void *stream);

/*
 * W_l, the third-order invariant of the Steinhardt order parameters (order module,
 * Section "Analysis Modules"; Steinhardt, Nelson and Ronchetti 1983), from the Q_lm held
 * by the last fgb_steinhardt_compute (or fgb_steinhardt_average):
 *   w_l(i) = sum_{m1+m2+m3=0} (l l l; m1 m2 m3) Q_lm1(i) Q_lm2(i) Q_lm3(i)   (real),
 * with Wigner 3j symbols and Q_{l,-m} = (-1)^m conj(Q_lm).  normalize != 0 divides by
 * (sum_m |Q_lm(i)|^2)^{3/2} (0 for a particle without neighbors).  w_out: float32 (n)
 * device.  Errors: INVALID_ARG (no compute yet).  Asynchronous on `stream` after the
 * first call for a given l (which uploads the 3j table once).
 */
int fgb_steinhardt_wl(fgb_steinhardt *st, int32_t normalize, float *w_out, void *stream);

/*
 * Neighbor-averaged q_l (Lechner and Dellago 2008; freud's `average` option):
 *   Qbar_lm(i) = (Q_lm(i) + sum_{k in nb(i)} Q_lm(k)) / (n_i + 1),
 *   qbar_l(i) = sqrt(4 pi / (2l+1) sum_m |Qbar_lm(i)|^2),
 * nb(i) from `nlist` (a self list over the points of the last compute).  The state then
 * holds Qbar_lm: fgb_steinhardt_wl gives the averaged w_l, fgb_steinhardt_state returns
 * Qbar_lm, and fgb_steinhardt_backward returns UNSUPPORTED until the next compute.
 * q_out: float32 (n) device.  Asynchronous on `stream`.
 */
int fgb_steinhardt_average(fgb_steinhardt *st, const fgb_nlist *nlist, float *q_out, void *stream);

/* -------------------------------------------------------------------- Clusters */

/*
 * Clusters of points joined by the bonds of a NeighborList (cluster module, Section
 * "Analysis Modules": cluster membership defined by neighbor bonds): connected
 * components over the n points (a point without bonds is a cluster of its own), bonds
 * with bond_mask[e] == 0 ignored (bond_mask NULL: all).  Clusters are numbered by
 * decreasing size, ties by their smallest member.  The call synchronises `stream` once
 * (to size the outputs).  Errors: INVALID_ARG (NULL, n out of range, list indexes
 * beyond n), OOM, CUDA.
 */
int fgb_cluster_compute(int64_t n, const fgb_nlist *nlist, const uint8_t *bond_mask, void *stream,
                        fgb_clusters **out);
/* Device views owned by the handle: cluster index per point (int32, n), sizes per
 * cluster (int32, num_clusters, non-increasing). */
int fgb_cluster_result(const fgb_clusters *c, int64_t *num_clusters, const int32_t **cluster_idx,
                       const int32_t **sizes);
/*
 * Per-cluster properties (ClusterProperties): every member is unwrapped to the image
 * nearest the cluster's smallest member; centers (num_clusters, 3) = that member plus the
 * mean unwrapped offset, wrapped into the box; gyration (num_clusters, 3, 3) = mean outer
 * product of the unwrapped offsets from the centre.  Meaningful for clusters smaller
 * than half the box.  Device float32 outputs; asynchronous on `stream`.
 */
int fgb_cluster_properties(const fgb_clusters *c, const fgb_box *box, const float *points, float *centers,
                           float *gyration, void *stream);
void fgb_cluster_destroy(fgb_clusters *c);

/*
 * Solid-liquid order parameter (order module, Section "Analysis Modules": a solid-liquid
 * order parameter for generic ordered phases, after ten Wolde, Ruiz-Montero and Frenkel
 * 1996) over a self NeighborList of `points`:
 *   s_ij = Re sum_{m=-l..l} Q_lm(i) conj(Q_lm(j)) / (|Q_l(i)| |Q_l(j)|)  per bond
 * (unnormalised dot product when normalize_q == 0; 0 for a particle without bonds),
 * with Q_lm(i) = (1/n_i) sum_j Y_lm over the list's bonds; a bond is solid-like when
 * s_ij > q_threshold, a particle is solid with at least solid_threshold solid-like bonds,
 * and *clusters_out joins solid particles through solid-like bonds (as
 * fgb_cluster_compute; every other particle is a cluster of its own).  Decided in FP64
 * on the device.  ql_ij: float32 (n_pairs) device or NULL; num_connections: int32 (n)
 * device.  Synchronises `stream` once (in the clustering).  Errors: INVALID_ARG (l
 * outside [0, 12], not a self list, NULL arrays, degenerate box), OOM, CUDA.
 */
int fgb_solid_liquid(const fgb_box *box, const float *points, const fgb_nlist *nlist, int32_t l, double q_threshold,
                     int32_t solid_threshold, int32_t normalize_q, float *ql_ij, int32_t *num_connections,
                     void *stream, fgb_clusters **clusters_out);

/* ------------------------------------------------------------ LocalDescriptors */

/*
 * Spherical harmonics of every bond of a NeighborList (environment module's
 * LocalDescriptors, Section "Analysis Modules"; global orientation): for pair e with
 * query point i and point j, the minimum-image bond d = x_j - q_i and, for l = 0..l_max,
 * Y_lm(d / |d|) with m = -l..l (negative_m != 0) or m = 0..l, in that order, the same
 * orthonormal harmonics with the Condon-Shortley phase as the Steinhardt parameters
 * (all zero for coincident points).  out: complex64 as float32 pairs, (n_pairs, n_sph, 2)
 * device, n_sph = (l_max+1)^2 or (l_max+1)(l_max+2)/2.  query_points NULL means the
 * points.  Errors: INVALID_ARG (l_max outside [0, 12], NULL arrays, degenerate box).
 * Asynchronous on `stream`.
 */
int fgb_local_descriptors(const fgb_box *box, const float *points, const float *query_points,
                          const fgb_nlist *nlist, int32_t l_max, int32_t negative_m, float *out, void *stream);

/* -------------------------------------------------------------- batched frames */

typedef struct fgb_batch_params {
    double r_max;        /* ball query radius feeding q_l */
    int32_t l;           /* Steinhardt l (0..12), or -1 for none */
    int32_t rdf_bins;    /* RDF bins (0 for none) */
    double rdf_r_max;
    double rdf_r_min;
    int32_t cell_div;    /* cells per r_max along each axis: 1 or 2; 0 = autotune */
    int32_t block;       /* threads per block of the per-point kernel: 64..512; 0 = autotune */
    int32_t hist_copies; /* its shared histogram copies per block: 1, 2 or 4; 0 = autotune */
    int32_t tile_cells;  /* largest work item of the cell-tile kernels, in cells: 1..4096;
                            0 = autotune; -1 = every frame on the per-point kernel */
    int32_t cells_per_warp; /* query cells per warp of the cell-tile kernels (x-adjacent
                               cells of a row walked together over the union of their
                               stencils): 1, 2, 4 or 8, i.e. 1 to 1/8 warp per query
                               cell; a frame whose grid is too narrow, or whose block
                               union would exceed 128 stencil cells, takes fewer;
                               0 = autotune */
} fgb_batch_params;

/*
 * Many frames of uneven size and different boxes analysed together (the per-frame
 * trajectory loops of the paper's listings).  frame_offsets (host, n_frames + 1): frame f
 * owns points frame_offsets[f] .. frame_offsets[f+1] of the packed (total, 3) array.
 * All device buffers are allocated here, so fgb_batch_run enqueues a fixed sequence of
 * kernels with no allocation and no host synchronisation (it can be captured in a CUDA
 * graph; fgb_batch_run_graph does that itself).
 */
int fgb_batch_create(int32_t n_frames, const int64_t *frame_offsets, const fgb_box *boxes,
                     const fgb_batch_params *params, void *stream, fgb_batch **out);
void fgb_batch_destroy(fgb_batch *b);

/* One pass over all frames: per-frame binning and one sort over all frames, then every
 * frame's RDF counts and q_l.  A frame whose RDF half stencil and ball stencil are both
 * on the fixed-offset route with at most 128 cells (and rdf_bins <= 1024) takes the
 * persistent cell-tile kernels (a warp per query cell, work items of up to tile_cells
 * cells); the others take the persistent per-point kernel (a thread per point).  The RDF
 * counts are the same either way; q_l may differ in the last bits (summation order). */
int fgb_batch_run(fgb_batch *b, const float *points, void *stream);

/* Same work replayed from a CUDA graph captured on the first call for this `points`
 * pointer (recaptured when it changes). */
int fgb_batch_run_graph(fgb_batch *b, const float *points, void *stream);

/* Times the candidate (cell_div, tile_cells, cells_per_warp, block, hist_copies) settings
 * on `points` and keeps the fastest (the parameters set to 0 at create).  Synchronises
 * `stream`. */
int fgb_batch_tune(fgb_batch *b, const float *points, void *stream, fgb_batch_params *chosen);

/* Device outputs: RDF counts uint64 (n_frames, bins), q_l float32 (total points, in
 * input order), neighbor counts int32 (total). */
int fgb_batch_outputs(const fgb_batch *b, const uint64_t **rdf_counts, const float **q,
                      const int32_t **n_neighbors);

/* Number of frames on the cell-tile kernels and on the per-point kernel in the current
 * configuration (host values; either pointer may be NULL). */
int fgb_batch_routes(const fgb_batch *b, int32_t *tile_frames, int32_t *point_frames);

#ifdef __cplusplus
}
#endif
#endif /* FGB_H */
