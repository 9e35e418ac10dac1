/*
 * si.h -- C ABI of the B300 spherical-index neighborhood queries.
 *
 * Method: N. Brodu, "Spherical Indexing for Neighborhood Queries".
 *   Problem statement (Sec. I, Sec. II.A): a query center C, a radius d, the
 *   objects X with |X - C| <= d; optionally only the K nearest (Sec. II.A,
 *   last paragraph; Sec. IV.B).  Space is a power-of-two lattice of cubic
 *   cells (Sec. II.B) whose axes are each cyclic or not (Sec. II.B,
 *   Appendix), with one extra cell for every object outside the region.
 *
 * Conventions shared by every call
 *   - Points are float32 quadruples (x, y, z, unused): an array of n * 4
 *     floats, 16-byte aligned.  The fourth lane is never read.
 *   - "d_" pointers are device pointers, "h_" pointers host pointers.  The
 *     caller owns every buffer it passes and the stream; the library owns
 *     only the opaque objects it returns (si_grid, si_batch).
 *   - Every call is ordered on `stream` (a cudaStream_t; NULL = legacy
 *     default stream) and returns without synchronising unless stated.
 *   - A grid's calls share its device work buffers (queues, scratch, the
 *     center buffers): calls on one grid must not overlap on the GPU (issue
 *     them on one stream, or order the streams); different grids are
 *     independent.  A grid is not safe to use from two host threads at once.
 *   - Errors are returned as si_status; no call aborts or throws.
 *     si_last_error() gives a one-line message for the calling host thread.
 *   - Distances follow one canonical predicate, identical on every path:
 *       a_k = |x_jk - x_ik| in FP64; on a cyclic axis a_k = min(a_k, L_k - a_k);
 *       D2  = (a_x^2 + a_y^2) + a_z^2 in FP64 (round to nearest, no FMA);
 *       neighbor  <=>  D2 <= (double)r * (double)r.
 *     The kernels filter in FP32 and re-test in FP64 every pair whose FP32
 *     value lies inside a guard band around r^2, so the sets are exact.
 *   - Neighbor ids are indices into the point array given to si_grid_build.
 */
#ifndef SI_H
#define SI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SI_OK = 0,
  SI_ERR_INVALID = 1,   /* bad argument, descriptor, or input value        */
  SI_ERR_OOM = 2,       /* device or host allocation failed                */
  SI_ERR_CUDA = 3,      /* a CUDA runtime call failed (see si_last_error)  */
  SI_ERR_CAPACITY = 4,  /* output buffer too small; required size reported */
  SI_ERR_TIMEOUT = 5,   /* a bounded device-side wait gave up              */
  SI_ERR_INTERNAL = 6   /* a device-side consistency check failed          */
} si_status;

/* Query flags */
#define SI_METHOD_SPHERE   0u  /* spherical index walk (Sec. II-III)            */
#define SI_METHOD_CUBE     1u  /* bin-lattice cube scan (Sec. I, Sec. IV.A)     */
#define SI_INCLUDE_SELF    2u  /* all-agents mode: keep the querying point      */
#define SI_NO_SORT         4u  /* radius lists left in walk order (not by id)   */
#define SI_WALK_PAPER      8u  /* radius: walk the 64 direction-bit tables of
                                  Sec. III.A with the run-time test (Eq. 1)
                                  instead of the sub-cell class tables         */
#define SI_METHOD_LIST    16u  /* radius: the non-empty cell list method of
                                  Sec. III.B / IV.A: every object tested      */
#define SI_SPHERE_ONLY    32u  /* radius: the spherical index without the volume
                                  comparison (Sec. IV.A, Fig. 8): never switch
                                  to the list method                           */
#define SI_WALK_PLANES    64u  /* radius: stacked circle-indexed z-planes (Sec. V),
                                  each plane skipped when empty, taken as its
                                  point list when sparse, else walked by rows:
                                  for points concentrated on a few planes      */
#define SI_FAST_D2       256u  /* K nearest: report the kernel's FP32 squared
                                  distance (within 12u D2 + 16u L sqrt(D2) of
                                  the canonical D2, u = 2^-24) instead of the
                                  FP32 rounding of the canonical FP64 D2
                                  (formed in FP32 by error-free transforms,
                                  FP64 only next to a rounding midpoint)      */
#define SI_NO_GROUPS     128u  /* radius: serve every crowded cell on its own
                                  (by default neighbouring crowded cells of an
                                  aligned 2x2x2 block share one candidate
                                  gather and sort); the lists are the same     */

/* Region, lattice and table extent (Sec. II.B).  The box side on axis a is
 * L_a = cell_size * 2^log2_cells[a] (exact in float32).  A cyclic axis wraps
 * at L_a; positions on it must lie in [origin_a, origin_a + L_a).  On a
 * non-cyclic axis points may lie anywhere (finite); those outside the region
 * go to the single outside cell.
 * r_max bounds every radius queried on the grid (it sizes the offset tables).
 * r_max = +inf (or <= 0) means "the whole region" and is accepted only when
 * no axis is cyclic.  On a cyclic axis the tables must not wrap onto
 * themselves: 2 * (floor(r_max / cell_size) + 1) + 1 <= 2^log2_cells[a].
 * Constraints: 2 <= log2_cells[a] <= 10, sum <= 27. */
typedef struct {
  float origin[3];
  float cell_size;
  uint8_t log2_cells[3];
  uint8_t reserved;
  uint32_t cyclic_mask;   /* bit 0 = x, bit 1 = y, bit 2 = z */
  float r_max;
} si_grid_desc;

typedef struct si_grid si_grid;

/* Grid state that tests and tools may read (all device pointers are owned by
 * the grid and valid until the next build or destroy). */
typedef struct {
  int64_t n;               /* points in the last build                       */
  int64_t n_cells;         /* 2^W + 1 (the last one is the outside cell)     */
  const int32_t *d_cell_start; /* n_cells + 1 entries: cell c holds sorted
                                  points cell_start[c] .. cell_start[c+1]-1  */
  const float *d_sorted_pos;   /* n float4, points in cell order            */
  const int32_t *d_perm;       /* n: sorted slot -> input index             */
  int64_t table_entries;   /* offsets in the sorted table                    */
  int32_t table_n_max;     /* largest floor(d^2) the table covers            */
  int32_t spec_shells;     /* shells with specialized tables (0..spec_shells-1) */
} si_grid_info;

/* Create a grid for up to n_capacity points: validates the descriptor,
 * builds the sorted offset table (Sec. II.A), its index by floor(d^2) and the
 * 64 specialized tables (Sec. III.A, Eq. 1-2) on the host, and allocates and
 * uploads every device array.  The grid owns its device memory (no caller
 * workspace): the query paths size part of it from data known only on the
 * device (records of crowded cells, centers' staging, the point list of the
 * list method), so a query call may grow it (eagerly, outside any stream
 * capture; bench code captures only after a first eager call), and it is
 * freed by si_grid_destroy.  Callers that cannot allocate at all have
 * si_neighbor_energy_noalloc. */
si_status si_grid_create(const si_grid_desc *desc, int64_t n_capacity, si_grid **out);

/* Bin n points (n <= capacity) into the lattice: cell key by mask and shift
 * (Sec. II.B), histogram, exclusive scan, scatter into cell order.  Re-binning
 * moved points (Sec. I: objects move freely) reuses the grid's memory.
 * d_pos: n * 4 floats, device, 16-byte aligned.  A cyclic-axis coordinate
 * outside its box or a non-finite coordinate makes the build fail with
 * SI_ERR_INVALID; this is detected on the device and reported by the next
 * call that synchronises (si_grid_sync). */
si_status si_grid_build(si_grid *g, const float *d_pos, int64_t n, void *stream);

/* Convenience: si_grid_create(desc, n) followed by si_grid_build. */
si_status si_build_grid(const si_grid_desc *desc, const float *d_pos, int64_t n,
                        void *stream, si_grid **out);

/* Wait for the grid's work on `stream` and return any device-side status
 * recorded since the last call (SI_ERR_INVALID from a build, SI_ERR_CAPACITY
 * from an asynchronous radius query, SI_ERR_INTERNAL).  Clears it. */
si_status si_grid_sync(si_grid *g, void *stream);

si_status si_grid_get_info(const si_grid *g, si_grid_info *info);

/* Run-time method selection of the radius queries (Appendix: a weighting
 * factor for the volume comparison, and an optional reversal to the bin
 * lattice below a distance, off by default).  list_weight (>= 0): with
 * SI_METHOD_SPHERE the non-empty list method is taken when list_weight times
 * its estimated cost is below the spherical index's (default 1.2; 0: always
 * the list, +inf: never).  cube_below (>= 0, cell units): a radius query with
 * r / s below it takes the bin-lattice cube scan instead of the spherical
 * index (default 0: never).  knn_cube_below (>= 0, cell units): the
 * Appendix's distinct reversal distance of the K-nearest query, whose
 * r_max / s below it takes the bin lattice (every cell of the bounding cube
 * of the r_max sphere, the list of the K nearest kept per query, the cut
 * shrinking as they are found; default 0: never).  Every choice returns the
 * same lists. */
si_status si_grid_set_method(si_grid *g, float list_weight, float cube_below, float knn_cube_below);
si_status si_grid_destroy(si_grid *g);

/* Fixed-radius query (Sec. I: every agent queries its neighborhood;
 * Sec. II.A: x <= d).
 * Method: with SI_METHOD_SPHERE (0) the call compares volumes as the paper
 * does (Sec. III.B, Sec. IV.A): when the estimated cost of walking the query
 * sphere's cells exceeds that of testing every object of the region (large
 * radius, low load), it uses the non-empty list method (SI_METHOD_LIST)
 * instead; SI_SPHERE_ONLY disables the comparison.  Every method returns the
 * same lists.
 * d_centers NULL: all agents; query k is point k of the last build, m must
 * equal the grid's n, and a point's own index is excluded unless
 * SI_INCLUDE_SELF.
 * d_centers non-NULL: m query centers (m * 4 floats, device, 16-byte
 * aligned, the fourth lane unread); no index is excluded (SI_INCLUDE_SELF
 * has no effect).  A center outside the region on a non-cyclic axis is
 * answered like any other.  A center with a non-finite coordinate, or
 * outside its box on a cyclic axis, gets an empty list and makes the grid
 * record SI_ERR_INVALID (returned by the next si_grid_sync).  The first call
 * with more centers than any before allocates the grid's center buffers
 * (about 44 bytes per center, plus 128 with the class tables in use).
 * Output: CSR in input order, d_offsets[m + 1] (int64, device) and d_ids
 * (int32, device, capacity ids_capacity); ids ascending per query unless
 * SI_NO_SORT.  r must satisfy 0 <= r <= r_max.
 * h_total (nullable, host): when given, the call synchronises after counting,
 * stores the total there and returns SI_ERR_CAPACITY without writing ids if
 * total > ids_capacity.  When NULL the call stays asynchronous; an overflow
 * then writes only the ids that fit and is reported by si_grid_sync. */
si_status si_query_radius(si_grid *g, const float *d_centers, int64_t m, float r,
                          uint32_t flags, int64_t *d_offsets, int32_t *d_ids,
                          int64_t ids_capacity, int64_t *h_total, void *stream);

/* End to end with host buffers: the all-agents radius query of n points
 * held in host memory.  Copies h_pos (n * 4 floats, host; page-locked memory
 * makes the copy direct and fast) into the grid's own device buffer, bins
 * it (si_grid_build), runs the all-agents si_query_radius into the grid's
 * own device output buffers, copies the CSR result to h_offsets[n + 1]
 * (int64, host) and h_ids (int32, host, capacity ids_capacity), and waits
 * for the copies: on return the host buffers hold the result.  *h_total
 * (host, required) receives the number of ids; SI_ERR_CAPACITY, with
 * nothing written to h_ids, when it exceeds ids_capacity.  The first call,
 * and a call with more points or a larger ids_capacity than before,
 * allocates those device buffers (16 n + 8 (n + 1) + 4 ids_capacity bytes);
 * si_grid_destroy frees them. */
si_status si_query_radius_host(si_grid *g, const float *h_pos, int64_t n, float r, uint32_t flags,
                               int64_t *h_offsets, int32_t *h_ids, int64_t ids_capacity,
                               int64_t *h_total, void *stream);

/* K-nearest query (Sec. II.A, last paragraph: once K neighbors are found
 * the search radius shrinks to the K-th distance; Sec. IV.B), for all agents
 * (d_centers NULL, m = the grid's n; own index excluded unless
 * SI_INCLUDE_SELF) or for m query centers (as in si_query_radius; a center
 * with invalid coordinates gets count 0, ids -1 and d2 +inf).
 * Up to k (1 <= k <= 64) nearest points within r_max_query (inclusive), ordered
 * by (canonical D2, index); d_ids[m * k] int32 padded with -1, d_d2[m * k]
 * float (nullable; the FP32 rounding of the canonical FP64 D2, evaluated for
 * the reported neighbors only, or with SI_FAST_D2 the kernel's FP32 value;
 * +inf padding), and
 * d_counts[m] int32 (number found).  r_max_query <= the grid's r_max
 * (+inf allowed when the grid's r_max is +inf). */
/* flags: SI_INCLUDE_SELF, SI_FAST_D2, and SI_METHOD_CUBE for the bin-lattice
 * walk (every cell of the bounding cube of the r_max sphere) instead of the
 * spherical index; the results do not change. */
si_status si_query_knn(si_grid *g, const float *d_centers, int64_t m, int k,
                       float r_max_query, uint32_t flags, int32_t *d_ids, float *d_d2,
                       int32_t *d_counts, void *stream);

/* Smooth neighbor reduction: the "functor applied to each neighbor" of
 * Sec. IV.A made concrete.  kernel 0 (SI_KERNEL_POLY6_CUBED):
 *   E = sum_i sum_{j != i, D_ij < r} (1 - D_ij^2 / r^2)^3
 *   dE/dx_i = -(12 / r^2) sum_{j != i, D_ij < r} (1 - D_ij^2 / r^2)^2 (x_i - x_j)
 * (shortest displacement on cyclic axes).  d_energy: one double (device,
 * nullable).  d_grad: n * 4 floats in input order (device, nullable; the
 * fourth lane is written 0), multiplied by *d_grad_scale when that device
 * pointer is given.  FP32 arithmetic, FP64 accumulation of E. */
#define SI_KERNEL_POLY6_CUBED 0
si_status si_neighbor_reduce(si_grid *g, float r, int kernel, double *d_energy,
                             float *d_grad, const float *d_grad_scale, void *stream);

/* Smooth-kernel energy E (as si_neighbor_reduce, kernel SI_KERNEL_POLY6_CUBED)
 * of n points, for callers that cannot allocate device memory.  The paper has
 * no counterpart: this entry point exists because some callers cannot call
 * cudaMalloc where they need the energy -- code running under a framework
 * that owns every device allocation, plug-ins with a fixed device-memory
 * budget, a real-time step that must never touch the allocator -- and cannot
 * create a grid.  It allocates nothing: its scratch (2,364,416 bytes =
 * 2.25 MiB: cell keys, counts and starts, points in cell order, partial
 * sums, a status word) is one static device array that every GPU loading the
 * library holds until the process exits.  Limits: n <= 65536 points and at most 2^16 cells
 * (sum of log2_cells <= 16); larger inputs return SI_ERR_INVALID.
 * desc: lattice as for si_grid_create (r_max ignored; r validated the same
 * way).  d_pos: n * 4 floats, device, 16-byte aligned.  d_energy: one double,
 * device; NaN when a point lies outside a cyclic axis' box or is not finite.
 * Neighbors come from the bin-lattice walk (no tables needed), so the result
 * equals si_neighbor_reduce's up to summation order; it is not bit-
 * reproducible from call to call (the order of the points inside a cell
 * follows the binning's atomic arrival; each thread sums its FP32 terms in
 * FP64, which keeps the spread at the last few bits).
 * The first call on a device looks up the scratch array's device address
 * (with that device current) and keeps it for the life of the process; make
 * that first call before any stream capture, and do not call this entry
 * point on a device whose context was reset (cudaDeviceReset) after that
 * first call, since the kept address would be stale.  Every call shares the scratch and leaves its contents there; the
 * call clears what must start at zero, and calls whose work overlaps on the
 * GPU (other streams, other host threads) race on it. */
si_status si_neighbor_energy_noalloc(const si_grid_desc *desc, const float *d_pos, int64_t n,
                                     float r, double *d_energy, void *stream);

/* Discretization tuning (Sec. IV.A, Fig. 9 and 10: for a fixed region, fixed
 * objects and fixed query centers there is a best cell size, which depends on
 * the number of objects, the query distance and on K).  Candidate i cuts the
 * region of *desc into 2^(log2_cells[a] + h_shifts[i]) cells on every axis
 * (cell side cell_size * 2^-h_shifts[i], same origin and box); for each, a
 * grid is created for the n points (d_pos, device) and `reps` rounds of
 * si_grid_build plus one query are timed with CUDA events on `stream`: the
 * radius query of radius r when k == 0, else the k nearest within r
 * (1 <= k <= 64), from d_centers (m centers, device; NULL = all agents,
 * m = n) with default flags.  h_ms[i] (host, n_cand floats) receives the
 * median milliseconds per round, +inf for a candidate that is not a valid
 * lattice (log2 out of [2, 10], or tables that would wrap a cyclic axis);
 * *h_best (host) the index of the fastest.  One warm-up round per candidate
 * is not timed.  Synchronises; allocates and frees its own grids and
 * buffers.  SI_ERR_INVALID when no candidate is valid. */
si_status si_tune_lattice(const si_grid_desc *desc, const float *d_pos, int64_t n, const float *d_centers,
                          int64_t m, float r, int k, const int32_t *h_shifts, int n_cand, int reps,
                          float *h_ms, int32_t *h_best, void *stream);

/* ---------------------------------------------------------------------------
 * Batched scenes: many independent grids served together.
 * Each scene has its own lattice, cyclic mask, radius and points.  Scenes
 * with short expected lists are binned and queried together by a fixed,
 * small number of launches (one persistent query kernel pulls (scene, query
 * tile) items from a device work queue); scenes with long lists each run the
 * single-scene pipeline of si_grid_build + si_query_radius on a grid of
 * their own, on concurrent branches.  The whole batch is captured once in a
 * CUDA graph and replayed.
 * ------------------------------------------------------------------------- */
typedef struct {
  si_grid_desc desc;       /* r_max is ignored; the scene's r sizes its tables */
  const float *d_pos;      /* n * 4 floats, device                            */
  int64_t n;
  float r;                 /* all-agents radius of this scene                 */
  int64_t *d_offsets;      /* n + 1, device                                   */
  int32_t *d_ids;          /* ids_capacity, device                            */
  int64_t ids_capacity;
} si_scene;

typedef struct si_batch si_batch;

/* The batch planner's choices (the paper's discretization tuning, Sec.
 * IV.A, carried over to the batch: the best split depends on the scenes).
 *   heavy_hits     expected list length (load x sphere volume in cells) from
 *                  which a scene runs the single-scene pipeline instead of
 *                  the fused launches (default 24; 0: every non-empty scene)
 *   q_tile         queries per work item, and threads per block, of the
 *                  fused query kernels (one thread per query): 64, 128 or 256
 *                  (default 128)
 *   branches       concurrent graph branches of the single-scene pipelines,
 *                  1..32 (default 8)
 *   blocks_per_sm  resident blocks per SM of the fused persistent query
 *                  kernels, 1..2048 / q_tile (default 8) */
typedef struct {
  float heavy_hits;
  int32_t q_tile;
  int32_t branches;
  int32_t blocks_per_sm;
} si_batch_params;

/* The defaults above, into *p (host). */
si_status si_batch_default_params(si_batch_params *p);

/* Plan a batch: validates every scene, builds each scene's tables and
 * allocates the batch's device memory (cell arrays of all scenes, sorted
 * points, work queue).  Scene pointers are captured: later runs read the
 * scenes' current point data and write their outputs.  si_batch_create uses
 * the default planner choices; si_batch_create_params takes them from
 * *params (host, nullable = defaults; SI_ERR_INVALID when out of range). */
si_status si_batch_create(const si_scene *scenes, int n_scenes, uint32_t flags, si_batch **out);
si_status si_batch_create_params(const si_scene *scenes, int n_scenes, uint32_t flags,
                                 const si_batch_params *params, si_batch **out);

/* Time planner choices on these scenes: for each of the n_cand candidates
 * (host array) a batch is created, run once eagerly, captured, replayed twice
 * and then timed over `reps` graph replays with CUDA events on a stream of
 * its own; h_ms[i] (host) receives the median milliseconds, *h_best (host)
 * the index of the fastest.  The runs write the scenes' outputs.
 * Synchronises; allocates and frees each candidate's batch.  Errors:
 * SI_ERR_INVALID (bad arguments, a candidate out of range), and those of
 * si_batch_create_params / si_batch_run / si_batch_sync (e.g.
 * SI_ERR_CAPACITY when an id buffer is too small). */
si_status si_batch_tune(const si_scene *scenes, int n_scenes, uint32_t flags, const si_batch_params *cands,
                        int n_cand, int reps, float *h_ms, int32_t *h_best);

/* Run the batch on `stream`: bin all scenes, count, scan, write, sort.
 * Capacity overflow is reported by si_batch_sync.  The first call runs
 * eagerly and waits for the GPU (the long-list scenes build their radius
 * tables and size their scratch from the list totals); later calls are
 * asynchronous.  use_graph != 0: the first call also captures the launches
 * into a CUDA graph, and every later call replays it. */
si_status si_batch_run(si_batch *b, int use_graph, void *stream);

/* Wait, then report the per-scene totals (h_totals[n_scenes], host,
 * nullable) and any device-side status. */
si_status si_batch_sync(si_batch *b, int64_t *h_totals, void *stream);
si_status si_batch_destroy(si_batch *b);

/* Number of kernel launches issued by this library (all calls, this process):
 * lets a benchmark count the launches inside its timed region. */
int64_t si_launch_count(void);

/* Per-kernel device timing, for benchmarks.  While enabled, every kernel
 * launch of the library (and every batch graph replay) is bracketed by two
 * CUDA events recorded on its own stream; launches made during a stream
 * capture are not timed.  While enabled, a query issues all its kernels in
 * order on the caller's stream (no second stream for the per-query kernels),
 * so that each launch is timed alone.  Not thread-safe with concurrent
 * library calls. */
si_status si_kernel_timing_enable(int enable);

/* Synchronise the device, aggregate the launches timed since the last report
 * and write one line per kernel, "name launches total_ms\n", into buf (host,
 * cap bytes, always NUL-terminated).  Clears the records. */
si_status si_kernel_timing_report(char *buf, size_t cap);

/* Measured pair-test rate of the current device, for the arithmetic
 * roofline of the radius kernels (not part of the paper's method).  A pair
 * test is the FP32 filter of the canonical predicate: three coordinate
 * differences, a square and two fused multiply-adds, and the sign of
 * d^2 - t moved into a hit mask, with the candidates read from shared
 * memory by broadcast, as in the cell kernels' test phase.  variant 0:
 * scalar FP32 operations; 1: packed f32x2 operations (two pairs per
 * instruction).  Launches its own kernel on a stream of its own (the whole
 * GPU, about a millisecond, six launches), synchronises, and writes the best
 * rate in pair tests per second to *pairs_per_second (host).  Allocates and
 * frees a small device buffer; errors: SI_ERR_INVALID (null output, unknown
 * variant), SI_ERR_CUDA. */
si_status si_measure_pair_rate(uint32_t variant, double *pairs_per_second);

const char *si_status_string(si_status s);
const char *si_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SI_H */
