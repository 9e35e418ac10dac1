// Internal definitions shared by the CUDA translation units of the library.
// Method: Brodu, "Spherical Indexing for Neighborhood Queries" (Sec. II-III).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "si.h"

namespace si {

// ---------------------------------------------------------------------------
// Offset table entry (Sec. II.A, Sec. II.B): one cell offset of the sorted
// center-to-edge array.  16 bytes so a warp reads whole sectors.
//   unp   offset in the unpacked layout (Y field above Z and X, see below),
//         each field in (w+1)-bit two's complement: after the SWAR add the
//         field's bit w is set exactly when that coordinate left [0, G).
//   ox..  the offset itself (cell units), for the exact cell test (Eq. 1)
//   dirs  6 direction bits: bit 2a for +axis a, bit 2a+1 for -axis a
//   b2    minimum-bound squared distance sum_a max(|o_a|-1, 0)^2 (Fig. 2)
// ---------------------------------------------------------------------------
struct __align__(16) TabEntry {
  unsigned long long unp;
  signed char ox, oy, oz;
  unsigned char dirs;
  int b2;
};
static_assert(sizeof(TabEntry) == 16, "table entry must be 16 bytes");

// One x-row of the sphere's cells (for the K-nearest walk): the row's (0, oy,
// oz) offset in unpacked form and its minimum-bound squared y-z distance.
struct __align__(16) RowEntry {
  unsigned long long unp;
  short oy, oz;
  int b2;
};
static_assert(sizeof(RowEntry) == 16, "row entry must be 16 bytes");

// Everything a query kernel needs, passed by value (kernel parameter space).
struct GridDev {
  const float4 *spos;        // sorted positions (cell order)
  const int *perm;           // sorted slot -> input index
  const int *cell_start;     // n_cells + 1
  const unsigned char *cell_cls;   // per non-empty cell: kCellLight / kCellHeavy(Big) / kCellDense
  const unsigned char *slot_cls;   // per sorted slot: its cell's class
  int n;
  float ox, oy, oz;          // region origin
  float inv_s;               // 1 / cell side (float32)
  float Lx, Ly, Lz;          // box sides (float32, exact: s * 2^w)
  int wx, wy, wz, W;
  unsigned cyc;              // cyclic mask
  unsigned outside;          // 1 << W, the outside cell
  unsigned long long valid;  // bits of the three fields in unpacked form
  unsigned long long gx, gy, gz;   // guard bit of each field
  unsigned long long guard_non;    // guard bits of the non-cyclic fields
  const TabEntry *tab;       // main sorted table
  const int *tab_end;        // tab_end[n] = entries with b2 <= n, n = 0..n_max
  int n_max;
  const TabEntry *spec;      // specialized tables, concatenated
  const int *spec_begin;     // [shell * 64 + mask]
  const int *spec_end;       // [64 * shell^2 + mask * (2 shell + 1) + (n - shell^2)]
  int spec_shells;           // shells 0 .. spec_shells-1 have specialized tables
  float eps;                 // conservative margin in cell units
  int *status;               // device status word (bit flags below)
  // sub-cell class tables (refinement of the specialized tables): class
  // c = (k q + j) q + i of the query's sub-cell position lists, center to
  // edge, every offset whose cell lies within d of the class's sub-box
  const unsigned long long *cls;   // entries: unpacked offset | bit 63 = whole cell inside
  const int *cls_begin;            // q^3 + 1
  int cls_q;                       // 0: no class tables
  const unsigned long long *crow;  // x-row runs of the cells within d of a whole cell (class table with q = 1)
  int n_crow;
  const RowEntry *rows;            // x-rows sorted by b2 (K-nearest walk)
  int n_rows;
  int row_lim_x;                   // |ox| bound of the rows' x extent
  // the query set: positions in walk order and the output row of each; the
  // grid's own sorted points (all-agents mode, q_agents = 1: query s is
  // point s and leaves itself out of its list unless SI_INCLUDE_SELF) or
  // caller-given centers sorted by cell (q_agents = 0)
  const float4 *qpos;
  const int *qid;
  int q_agents;
};

enum : int { ST_INVALID = 1, ST_CAPACITY = 2, ST_INTERNAL = 4, ST_TIMEOUT = 8 };

// The sorted slot query s must leave out of its own list, or -1.
__device__ __forceinline__ int query_self(const GridDev &g, unsigned flags, int s) {
  return (g.q_agents && !(flags & SI_INCLUDE_SELF)) ? s : -1;
}

// Inclusive warp scan of one int per lane (all 32 lanes take part).
__device__ __forceinline__ int warp_incl_scan_i(int v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

// Exclusive block scan of one int per thread (every thread of the block takes
// part; scan holds blockDim.x / 32 ints of shared memory); returns the block
// total in `total`.
__device__ __forceinline__ int block_excl_scan_i(int v, int &total, int *scan) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int inc = warp_incl_scan_i(v);
  if (lane == 31) scan[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    const int x = lane < nw ? scan[lane] : 0;
    const int y = warp_incl_scan_i(x);
    if (lane < nw) scan[lane] = y;
  }
  __syncthreads();
  total = scan[nw - 1];
  const int before = wid > 0 ? scan[wid - 1] : 0;
  __syncthreads();
  return before + inc - v;
}

// Heavy cells take the cell-at-a-time radius kernel: at least kHeavyMin
// points, or at least kHeavyMinDense points in a dense x-row (the cell and
// its two x neighbours hold kHeavyRowDense or more), where sharing one walk
// pays even for few queries.  The binning lists them and the per-query
// kernels skip their queries with this same predicate; either path gives
// the same lists.
constexpr int kHeavyMin = 8;
constexpr int kHeavyMinDense = 3;
constexpr int kHeavyRowDense = 12;

__device__ __forceinline__ bool heavy_cell(const int *start, unsigned key, unsigned outside) {
  if (key >= outside) return false;
  const int m = __ldg(start + key + 1) - __ldg(start + key);
  if (m >= kHeavyMin) return true;
  if (m < kHeavyMinDense || key < 1u || key + 2u > outside) return false;
  return __ldg(start + key + 2) - __ldg(start + key - 1) >= kHeavyRowDense;
}

// Which radius kernels serve a cell's queries, decided once per cell at
// binning: heavy cells (heavy_cell) one block per cell; dense cells (light,
// but with at least kDenseN27 points in the 27 cells around them, i.e. long
// lists) one warp per query; the rest one thread per query.  Heavy cells
// with at least kBigN27 points around them are marked for the large
// configuration of the cell kernel.  The outside cell is dense when it holds
// kDenseN27 points.  Only the work split
// depends on it; every path gives the same lists.
enum : int { kCellLight = 0, kCellHeavy = 1, kCellDense = 2, kCellHeavyBig = 3 };
constexpr int kDenseN27 = 24;
constexpr int kBigN27 = 768;   // heavy cells this crowded go straight to the large cell kernel

__device__ __forceinline__ int cell_class(const int *start, unsigned key, unsigned outside, int wx, int wy,
                                          int wz) {
  if (key >= outside) return __ldg(start + key + 1) - __ldg(start + key) >= kDenseN27 ? kCellDense : kCellLight;
  const bool heavy = heavy_cell(start, key, outside);
  // the 3 x 3 rows of 3 cells around it (y, z wrapped, x clipped)
  const unsigned Gx = 1u << wx, Gy = 1u << wy, Gz = 1u << wz;
  const unsigned x = key & (Gx - 1u), y = (key >> wx) & (Gy - 1u), z = key >> (wx + wy);
  const unsigned x0 = x > 0u ? x - 1u : 0u, x1 = min(x + 1u, Gx - 1u);
  int sum = 0;
#pragma unroll
  for (int dz = -1; dz <= 1; ++dz) {
    const unsigned zz = (z + (unsigned)dz) & (Gz - 1u);
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy) {
      const unsigned row = (zz << (wx + wy)) | (((y + (unsigned)dy) & (Gy - 1u)) << wx);
      sum += __ldg(start + row + x1 + 1u) - __ldg(start + row + x0);
    }
  }
  if (heavy) return sum >= kBigN27 ? kCellHeavyBig : kCellHeavy;
  return sum >= kDenseN27 ? kCellDense : kCellLight;
}

// ---------------------------------------------------------------------------
// Cell of one coordinate (Sec. II.B: power-of-two lattice; Sec. II.B last
// paragraph: one outside cell for objects out of the region).  The same
// function bins points and locates query centers, so both agree bit for bit.
// rel * inv_s is >= 0 here, so truncation is floor; the clamp to G-1 keeps a
// coordinate that rounds up to G (rel just below L) in the last cell.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int axis_cell(float x, float o, float L, float inv_s, int w,
                                         bool cyclic, bool &outside, bool &bad) {
  const float rel = x - o;
  if (!(rel >= 0.f && rel < L)) {          // false for NaN too
    if (cyclic || !(fabsf(x) <= 3.0e38f)) bad = true;
    outside = true;
    return 0;
  }
  const int c = (int)(rel * inv_s);
  return min(c, (1 << w) - 1);
}

// Packed location: bits z | y | x (Sec. II.B), also the cell's memory index.
__device__ __forceinline__ unsigned pack3(int cx, int cy, int cz, const GridDev &g) {
  return ((unsigned)cz << (g.wx + g.wy)) | ((unsigned)cy << g.wx) | (unsigned)cx;
}

// Unpacked location: Y moved up by the packed width W, leaving carry gaps.
__device__ __forceinline__ unsigned long long unpack3(int cx, int cy, int cz, const GridDev &g) {
  return ((unsigned long long)cy << (g.W + g.wx)) |
         ((unsigned long long)cz << (g.wx + g.wy)) | (unsigned long long)cx;
}

// Pack a masked unpacked location: shift Y back down and OR the low part.
__device__ __forceinline__ unsigned repack(unsigned long long u, const GridDev &g) {
  return (unsigned)(u >> g.W) | (unsigned)(u & ((1ull << g.W) - 1ull));
}

// ---------------------------------------------------------------------------
// Canonical FP64 predicate value (identical definition on every path):
//   a = |xj - xi|, cyclic: min(a, L - a);  D2 = (ax*ax + ay*ay) + az*az,
// each operation rounded to nearest, no fused multiply-add.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double canon_gap(float a, float b, float L, bool cyclic) {
  double d = fabs((double)b - (double)a);
  if (cyclic) {
    const double w = (double)L - d;
    if (w < d) d = w;
  }
  return d;
}

__device__ __forceinline__ double canon_d2_raw(const float4 &q, const float4 &p, float Lx, float Ly, float Lz,
                                               unsigned cyc) {
  const double ax = canon_gap(q.x, p.x, Lx, cyc & 1u);
  const double ay = canon_gap(q.y, p.y, Ly, (cyc >> 1) & 1u);
  const double az = canon_gap(q.z, p.z, Lz, (cyc >> 2) & 1u);
  double s = __dmul_rn(ax, ax);
  s = __dadd_rn(s, __dmul_rn(ay, ay));
  s = __dadd_rn(s, __dmul_rn(az, az));
  return s;
}
__device__ __forceinline__ double canon_d2(const float4 &q, const float4 &p, const GridDev &g) {
  return canon_d2_raw(q, p, g.Lx, g.Ly, g.Lz, g.cyc);
}
// The same value behind a real call: for rare uses inside hot loops, where
// an inlined copy would be predicated and issue its FP64 instructions (at a
// small fraction of the FP32 rate on this GPU) for every warp.
static __device__ __noinline__ double canon_d2_call(float4 q, float4 p, float Lx, float Ly, float Lz, unsigned cyc) {
  return canon_d2_raw(q, p, Lx, Ly, Lz, cyc);
}

// ---------------------------------------------------------------------------
// The FP32 rounding of canon_d2, mostly without FP64 (the FP64 pipe of this
// GPU is slow).  The exact squared distance E of the two points is formed as
// an unevaluated sum H + lo of two floats by error-free transformations
// (Knuth's TwoSum, Dekker's Fast2Sum, the rounding error of a product by one
// fused multiply-add): each axis gap exactly as a float pair (its cyclic
// image L - gap exactly too, by Sterbenz's lemma, wherever it is the shorter
// one), its square to within 2^-45 relative, the sum of the three to within
// 2^-43 (every term is >= 0: no cancellation).  canon_d2 differs from E by a
// few FP64 roundings (under 2^-49 relative).  H is the float nearest to
// H + lo; the float nearest to canon_d2 is H as well unless H + lo lies
// within 2^-40 H of the midpoint between H and its neighbour on lo's side,
// and those distances (about one in 2^15) take canon_d2 itself, as do
// coordinates outside a cyclic box (gap > L), values below 2^-70 (where
// flushed subnormals could matter) or above 2^120.  The result equals
// __double2float_rn(canon_d2(q, p, g)) for every pair.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e) {   // |a| >= |b|
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}
// Gap of one axis as a float pair (h, l), h + l = |b - a| exactly (or the
// shorter way round a cyclic axis), then its square as a float pair (sh, sl);
// false for a cyclic gap longer than L.
__device__ __forceinline__ bool gap_sq(float a, float b, float L, bool cyclic, float &sh, float &sl) {
  float s, t;
  two_sum(b, -a, s, t);
  float h = fabsf(s), l = s < 0.f ? -t : t;
  if (cyclic) {
    if (!(h <= L)) return false;
    float u, v;
    two_sum(L, -h, u, v);   // v = 0 whenever h >= L / 2
    float wh, wl;
    fast_two_sum(u, __fsub_rn(v, l), wh, wl);
    if (wh < h || (wh == h && wl < l)) {   // both pairs normalised: lexicographic order is the order of the sums
      h = wh;
      l = wl;
    }
  }
  sh = __fmul_rn(h, h);
  float e = __fmaf_rn(h, h, -sh);
  e = __fmaf_rn(__fmul_rn(2.f, h), l, e);
  sl = __fmaf_rn(l, l, e);
  return true;
}
// true with v = the FP32 rounding of canon_d2 when the FP32 form settles
// it; false (v unset) for the pairs that need canon_d2 itself
__device__ __forceinline__ bool canon_d2_f32_try(const float4 &q, const float4 &p, const GridDev &g, float &v) {
  if (q.x == p.x && q.y == p.y && q.z == p.z) {   // every gap exactly 0
    v = 0.f;
    return true;
  }
  float xh, xl, yh, yl, zh, zl;
  const bool ok = gap_sq(q.x, p.x, g.Lx, g.cyc & 1u, xh, xl) & gap_sq(q.y, p.y, g.Ly, (g.cyc >> 1) & 1u, yh, yl) &
                  gap_sq(q.z, p.z, g.Lz, (g.cyc >> 2) & 1u, zh, zl);
  float s, e, H, lo;
  two_sum(xh, yh, s, e);
  fast_two_sum(s, __fadd_rn(e, __fadd_rn(xl, yl)), H, lo);
  two_sum(H, zh, s, e);
  fast_two_sum(s, __fadd_rn(e, __fadd_rn(lo, zl)), H, lo);
  if (ok && H >= 0x1p-70f && H <= 0x1p120f) {
    // half the gap from H to its neighbour on lo's side (exact; H is a
    // positive normal float, so its neighbours are one encoding step away)
    const unsigned hb = __float_as_uint(H);
    const float m = 0.5f * (lo >= 0.f ? __fsub_rn(__uint_as_float(hb + 1u), H) : __fsub_rn(H, __uint_as_float(hb - 1u)));
    if (__fsub_rn(m, fabsf(lo)) > H * 0x1p-40f) {
      v = H;
      return true;
    }
  }
  return false;
}
__device__ __forceinline__ float canon_d2_f32(const float4 &q, const float4 &p, const GridDev &g) {
  float v;
  return canon_d2_f32_try(q, p, g, v) ? v : __double2float_rn(canon_d2(q, p, g));
}

// ---------------------------------------------------------------------------
// Query geometry: the center's cell, its unpacked location and the distances
// zeta from the center to its own cell faces (Sec. III.A, Fig. 3), in cell
// units, shrunk by the margin eps so every cell rejection stays conservative
// under float32 binning (a point may sit a few ulps outside its cell).
// ---------------------------------------------------------------------------
struct QueryGeom {
  float4 q;                  // query position
  float u[3];                // query position in cell units (relative to origin)
  int c[3];                  // query cell (valid when !outside)
  float phi[3];              // sub-cell position in [0, 1] (cell units)
  float zp[3], zn[3];        // zeta toward +axis and -axis, shrunk by eps
  unsigned long long cu;     // unpacked center cell
  bool outside;              // query center outside the region
};

__device__ __forceinline__ QueryGeom make_geom(const float4 &q, const GridDev &g) {
  QueryGeom Q;
  Q.q = q;
  bool out = false, bad = false;
  Q.c[0] = axis_cell(q.x, g.ox, g.Lx, g.inv_s, g.wx, g.cyc & 1u, out, bad);
  Q.c[1] = axis_cell(q.y, g.oy, g.Ly, g.inv_s, g.wy, (g.cyc >> 1) & 1u, out, bad);
  Q.c[2] = axis_cell(q.z, g.oz, g.Lz, g.inv_s, g.wz, (g.cyc >> 2) & 1u, out, bad);
  Q.outside = out;
  Q.u[0] = (q.x - g.ox) * g.inv_s;
  Q.u[1] = (q.y - g.oy) * g.inv_s;
  Q.u[2] = (q.z - g.oz) * g.inv_s;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float phi = fminf(fmaxf(Q.u[a] - (float)Q.c[a], 0.f), 1.f);
    Q.phi[a] = phi;
    Q.zp[a] = fmaxf(1.f - phi - g.eps, 0.f);
    Q.zn[a] = fmaxf(phi - g.eps, 0.f);
  }
  Q.cu = unpack3(Q.c[0], Q.c[1], Q.c[2], g);
  return Q;
}

// Exact minimum squared distance (cell units) from the query center to the
// cell at offset o (Sec. III.A, Eq. 1 left side): sum over non-zero offset
// axes of (b_a + zeta_a)^2.  With zeta shrunk by eps this never exceeds the
// true value.
__device__ __forceinline__ float cell_t2(const TabEntry &e, const QueryGeom &Q) {
  float t2 = 0.f;
  const int o[3] = {e.ox, e.oy, e.oz};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    float gap = 0.f;
    if (o[a] > 0) gap = (float)(o[a] - 1) + Q.zp[a];
    else if (o[a] < 0) gap = (float)(-o[a] - 1) + Q.zn[a];
    t2 = fmaf(gap, gap, t2);
  }
  return t2;
}

// Farthest squared distance (cell units) from the query to any point of the
// cell at offset o, grown by eps: a cell below this bound lies wholly inside
// the sphere (Sec. III.A, unconditional inclusion, exact-corner reading).
__device__ __forceinline__ float cell_far2(const TabEntry &e, const QueryGeom &Q, float eps) {
  float f2 = 0.f;
  const int o[3] = {e.ox, e.oy, e.oz};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float lo = fabsf((float)o[a] - Q.phi[a]), hi = fabsf((float)(o[a] + 1) - Q.phi[a]);
    const float far = fmaxf(lo, hi) + eps;
    f2 = fmaf(far, far, f2);
  }
  return f2;
}

// Result of translating a table entry to the query's cell (Sec. II.B): the
// packed cell key, or the outside cell, and the image shift of each cyclic
// axis whose coordinate wrapped (-1, 0, +1 box lengths).
struct Target {
  unsigned key;
  bool outside;
  bool wrapped;
  float qx, qy, qz;          // query position moved by the image shift
};

__device__ __forceinline__ Target translate(const TabEntry &e, const QueryGeom &Q, const GridDev &g) {
  Target t;
  const unsigned long long s = Q.cu + e.unp;          // SWAR add of all fields
  t.outside = (s & g.guard_non) != 0ull;
  t.key = t.outside ? g.outside : repack(s & g.valid, g);
  const bool wx = (s & g.gx) != 0ull, wy = (s & g.gy) != 0ull, wz = (s & g.gz) != 0ull;
  t.wrapped = !t.outside && (wx | wy | wz);
  // wrapped on +a: the candidate's near image is x + L, so compare against q - L
  t.qx = Q.q.x - (wx ? (e.ox > 0 ? g.Lx : -g.Lx) : 0.f);
  t.qy = Q.q.y - (wy ? (e.oy > 0 ? g.Ly : -g.Ly) : 0.f);
  t.qz = Q.q.z - (wz ? (e.oz > 0 ? g.Lz : -g.Lz) : 0.f);
  return t;
}

// Translation of a class-table entry: the same SWAR add as translate(); the
// sign of a wrapped coordinate's offset is the top bit of its (w+1)-bit field.
__device__ __forceinline__ Target translate_raw(unsigned long long e, const QueryGeom &Q, const GridDev &g) {
  Target t;
  const unsigned long long s = Q.cu + e;
  t.outside = (s & g.guard_non) != 0ull;
  t.key = t.outside ? g.outside : repack(s & g.valid, g);
  const bool wx = (s & g.gx) != 0ull, wy = (s & g.gy) != 0ull, wz = (s & g.gz) != 0ull;
  t.wrapped = !t.outside && (wx | wy | wz);
  t.qx = Q.q.x - (wx ? ((e & g.gx) ? -g.Lx : g.Lx) : 0.f);
  t.qy = Q.q.y - (wy ? ((e & g.gy) ? -g.Ly : g.Ly) : 0.f);
  t.qz = Q.q.z - (wz ? ((e & g.gz) ? -g.Lz : g.Lz) : 0.f);
  return t;
}

__device__ __forceinline__ int isqrt_small(int n) {
  int r = (int)sqrtf((float)n);
  while (r * r > n) --r;
  while ((r + 1) * (r + 1) <= n) ++r;
  return r;
}

// FP32 guard band around r^2 (absolute, world units squared): pairs with an
// FP32 squared distance inside [lo, hi] are re-tested with canon_d2.
struct Band {
  float lo, hi;        // pairs not crossing a cyclic boundary
  float lo_w, hi_w;    // pairs compared through a wrapped image
  double r2;           // canonical (double)r * (double)r
};

}  // namespace si
