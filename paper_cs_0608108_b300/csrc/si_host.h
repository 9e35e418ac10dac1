// Host-side internals shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "si.h"
#include "si_internal.cuh"

namespace si {

constexpr int kCounterInts = 8;
constexpr long long kClassCapMax = 1ll << 22;   // class-table entries a grid may hold
constexpr size_t kClassSmemMax = 48 * 1024;      // class tables staged in shared memory up to this

// Record a message for si_last_error() (per host thread) and return `s`.
si_status fail(si_status s, const std::string &msg);
si_status cuda_fail(cudaError_t e, const char *what);
void count_launch(int k = 1);

#define SI_CUDA_TRY(expr)                                   \
  do {                                                      \
    cudaError_t _e = (expr);                                \
    if (_e != cudaSuccess) return ::si::cuda_fail(_e, #expr); \
  } while (0)

#define SI_LAUNCH_CHECK(name)                               \
  do {                                                      \
    ::si::count_launch();                                   \
    cudaError_t _e = cudaGetLastError();                    \
    if (_e != cudaSuccess) return ::si::cuda_fail(_e, name); \
  } while (0)

// Optional per-kernel event timing (si_kernel_timing_enable).
void prof_begin(cudaStream_t st);
void prof_end(cudaStream_t st, const char *name);

// Launch a kernel with error check and optional timing:
//   SI_KLAUNCH("name", stream, kernel<<<grid, block, smem, stream>>>(args));
#define SI_KLAUNCH(name, st, ...)  \
  do {                             \
    ::si::prof_begin(st);          \
    __VA_ARGS__;                   \
    SI_LAUNCH_CHECK(name);         \
    ::si::prof_end(st, name);      \
  } while (0)

// Host copy of the offset tables of one lattice / cyclic mask / extent.
struct HostTables {
  std::vector<TabEntry> tab;
  std::vector<int> tab_end;        // n_max + 1
  std::vector<TabEntry> spec;
  std::vector<int> spec_begin;     // spec_shells * 64
  std::vector<int> spec_end;       // 64 * spec_shells^2
  int n_max = 0;
  int spec_shells = 0;
  std::vector<RowEntry> rows;      // x-rows of the sphere, by b2 of their y-z offset
  std::vector<int> row_end;        // row_end[n] = rows with b2 <= n, n = 0..n_max
  int row_lim_x = 0;
};

// Largest shell with specialized tables: 64 copies of a shell cost memory
// (64 x its entries); beyond this the run-time cell test does the same job.
constexpr int kSpecShellsMax = 8;

// Build the sorted table for b2 <= n_max (Sec. II.A) and the specialized
// tables (Sec. III.A, Eq. 2).  Fails (returns false) if a cyclic axis would
// wrap onto itself.
bool build_tables(const int w[3], unsigned cyc, int n_max, HostTables &out, std::string &err);

// Device copies of the tables.
struct DevTables {
  TabEntry *tab = nullptr;
  int *tab_end = nullptr;
  TabEntry *spec = nullptr;
  int *spec_begin = nullptr;
  int *spec_end = nullptr;
  RowEntry *rows = nullptr;
  std::vector<int> row_end;        // host copy: row_end[n] = rows with b2 <= n
  int n_max = 0, spec_shells = 0, n_rows = 0, row_lim_x = 0;
  int64_t entries = 0;
};
si_status upload_tables(const HostTables &h, DevTables &d);
void free_tables(DevTables &d);

// Geometry derived from a descriptor.
struct Lattice {
  int w[3];
  int W;
  unsigned cyc;
  float origin[3];
  float s, inv_s;
  float L[3];
  double eps;          // cell-unit margin for conservative culling
  int n_max;           // table extent
  bool unbounded;
};
si_status make_lattice(const si_grid_desc &d, double r_for_tables, Lattice &lat);
void fill_griddev(const Lattice &lat, const DevTables &t, GridDev &g);

// Inclusive prefix sum of n values, in place allowed (in == out).
// Scratch must hold scan_scratch_elems(n) values: one per tile of kScanTile
// values, plus one.
constexpr int kScanTile = 4096;
constexpr int64_t scan_scratch_count(int64_t n) { return (n + kScanTile - 1) / kScanTile + 1; }
int64_t scan_scratch_elems(int64_t n);
si_status scan_inclusive_i32(const int *in, int *out, int64_t n, int *scratch, cudaStream_t st);
si_status scan_inclusive_i64(const long long *in, long long *out, int64_t n, long long *scratch,
                             cudaStream_t st);

// FP32 guard band around r^2 for a lattice (see si_grid.cu for the bound).
Band make_band(const Lattice &lat, float r);
// Band coefficients for comparing two FP32 squared distances (KNN order).
struct PairBand {
  // two FP32 squared distances of one query further apart than
  // c2 * d2 + c1 * sqrt(d2) are in the order of their canonical FP64 values;
  // the c1 term (the rounding of a coordinate shifted by a box side) is
  // needed only when one of them came through a wrapped image
  float c2, c1;
};
PairBand make_pair_band(const Lattice &lat);

// Sub-cell class tables (si_class.cu).
int class_q_for(double dmax);
int64_t class_capacity(const Lattice &lat, int64_t table_entries);
void build_class_tables(const Lattice &lat, double dg, int q, std::vector<unsigned long long> &ent,
                        std::vector<int> &begin);
void build_box_rows(const Lattice &lat, double dg, int B, std::vector<unsigned long long> &ent);
constexpr int kGroupTCap = 128;   // runs of a cell group's rows (two per row at most, and the outside cell)

// Outputs a query-center call gives a center it cannot query (a non-finite
// coordinate, or one outside its box on a cyclic axis): an empty result.
struct CenterOut {
  long long *rad_counts = nullptr;   // radius: per-center counts (offsets + 1)
  int K = 0;                         // K nearest: ids (-1), d2 (+inf, nullable), counts (0)
  int *ids = nullptr;
  float *d2 = nullptr;
  int *counts = nullptr;
};

// Query centers (si_centers.cu): sort the m centers (device float4) by
// coarse cell into the grid's center buffers and list them (clist0: the
// centers of light cells, or every valid center unless `split`; clist1: the
// rest), then set dv to the grid's view with that query set.
si_status prepare_centers(si_grid *g, const float *d_centers, int64_t m, bool split, bool stage,
                          const CenterOut &out, GridDev &dv, cudaStream_t st);

}  // namespace si

struct si_grid {
  si_grid_desc desc;
  si::Lattice lat;
  int64_t cap = 0, n = 0;
  // run-time method selection (si_grid_set_method): the weight of the list
  // method's estimated cost, and the radius (cell units) below which radius
  // queries take the bin-lattice cube scan
  double list_weight = 1.2;
  double cube_below = 0.0;
  double knn_cube_below = 0.0;   // the same reversal for K-nearest queries (r_max, cell units)
  int64_t n_cells = 0;
  si::DevTables tables;
  // device arrays
  uint2 *key_slot = nullptr;     // cap: (cell, rank in cell)
  int *cell_count = nullptr;     // n_cells
  int *cell_start = nullptr;     // n_cells + 1
  float4 *spos = nullptr;        // cap
  int *perm = nullptr;           // cap
  int *scan_i32 = nullptr;       // scan scratch for cells
  long long *scan_i64 = nullptr; // scan scratch for offsets
  int *status = nullptr;         // device status word
  int *longq = nullptr;          // cap + 1: [0] = count, then query ids of long lists
  int *hugeq = nullptr;          // cap + 1: lists too long for a warp sort
  int *heavy = nullptr;          // [0] = count, then heavy cells (heavy_cell; set by build)
  int *heavy_big = nullptr;      // [0] = count, then heavy cells for the large cell kernel (build + overflow)
  int *heavy_big_built = nullptr;   // heavy_big[0] as the build left it
  int *over = nullptr;           // [0] = count, then sorted slots of queries the cell kernel handed back
  int *denseq = nullptr;         // [0] = count, then sorted slots of the queries of dense cells (set by build)
  int *lightq = nullptr;         // [0] = count, then sorted slots of the queries of light cells (set by build)
  int *lstage = nullptr;         // kInlineSort x cap: short lists kept by the count pass (allocated on first use)
  unsigned char *cell_cls = nullptr;   // per cell: kCellLight / kCellHeavy / kCellDense (set by build)
  unsigned char *slot_cls = nullptr;   // per sorted slot: its cell's class (set by build)
  long long *cell_rec = nullptr; // per heavy cell: its record in the scratch buffer (-1: per-query path)
  int *scratch = nullptr;        // cell records (ordered candidate ids, hit masks) written before the prefix sum
  long long scr_cap = 0;
  unsigned long long *scr_top = nullptr;   // bump allocator of the scratch (also the size needed)
  int *counters = nullptr;       // kCounterInts work counters
  std::vector<int> tab_end_host; // host copy of the table's end[] index
  // sub-cell class tables for the current radius (see si_class.cu)
  unsigned long long *cls = nullptr;
  int *cls_begin = nullptr;
  int64_t cls_cap = 0;
  float cls_dg = -1.f;
  int cls_q = 0;
  size_t cls_smem_bytes = 0;     // > 0: the current tables fit a block's shared memory
  std::vector<unsigned long long> cls_host;
  std::vector<int> cls_begin_host;
  bool ensure_classes(float dg, cudaStream_t st);
  unsigned long long *crow = nullptr;   // cell-level x-row runs (class table with q = 1) for crow_dg
  int64_t crow_cap = 0;
  int n_crow = 0;
  float crow_dg = -1.f;
  std::vector<unsigned long long> crow_host;
  bool ensure_cell_rows(float dg, cudaStream_t st);
  unsigned long long *grow = nullptr;   // x-row runs of the cells within d of a 2 x 2 x 2 cell group
  int64_t grow_cap = 0;
  int n_grow = 0;
  float grow_dg = -1.f;
  std::vector<unsigned long long> grow_host;
  bool ensure_group_rows(float dg, cudaStream_t st);
  int *groups = nullptr;         // [0] = count, then the lowest cell key of each group of >= 2 heavy cells
  int *hsolo = nullptr;          // [0] = count, then heavy cells served one at a time
  int4 *xitems = nullptr;        // expansion items ([0].x = count): record, first slot, queries of one cell
  int *xblock = nullptr;         // [0] = count, then heavy cells expanded a block per cell
  double *partial = nullptr;     // reduce partial sums
  int64_t partial_len = 0;
  long long *h_pinned = nullptr; // pinned host scratch (2 values)
  // a second stream for the per-query kernels of a radius query, which run
  // beside the crowded cells' kernels (forked from and joined to the
  // caller's stream by events, so CUDA graph capture follows them)
  cudaStream_t side = nullptr;
  cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
  bool fork = true;              // false: one stream (the batch's scene pipelines run on branches already)
  bool ensure_side();
  // query centers in coarse cell order (si_centers.cu), grown on demand
  int64_t ccap = 0;
  float4 *cpos = nullptr;        // ccap: positions
  int *cid = nullptr;            // ccap: input index of each
  uint2 *ckey = nullptr;         // ccap: (bucket, rank in bucket)
  int *cbuck = nullptr;          // bucket starts ([0] = 0, then inclusive counts)
  int *cscan = nullptr;          // their scan scratch
  long long *cscan64 = nullptr;  // scan scratch for ccap per-center counts
  int *clist0 = nullptr;         // ccap + 1: [0] = count, then slots (light group)
  int *clist1 = nullptr;         // ccap + 1: the warp-per-center group
  int *clong = nullptr;          // ccap + 1: long lists to sort; K nearest: the per-thread fallback queue
  int *chuge = nullptr;          // ccap + 1: lists too long for a warp sort
  int *cstage = nullptr;         // kInlineSort x cstage_cap: short lists kept by the count pass
  int64_t cstage_cap = 0;
  si_status ensure_centers(int64_t m, bool stage);
  float4 *ipos = nullptr;        // cap: points in input order (non-empty list method; allocated on first use)
  // si_query_radius_host: the points and the CSR result on the device,
  // grown on demand
  float4 *io_pos = nullptr;
  int64_t io_pos_cap = 0;
  long long *io_off = nullptr;
  int64_t io_off_cap = 0;
  int *io_ids = nullptr;
  int64_t io_ids_cap = 0;
  si::GridDev dev() const;
};
