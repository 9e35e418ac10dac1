// All-agents fixed-radius query (Sec. I, Sec. II.A): count pass, prefix sum,
// write pass, per-list id sort.  One thread per query point, queries taken in
// cell order so that neighbouring threads walk neighbouring cells (their
// candidate cells are shared through L1/L2).
#include <cmath>

#include "si_host.h"
#include "si_walk.cuh"

namespace si {

constexpr int kQueryThreads = 128;
constexpr int kInlineSort = 32;      // lists up to this length are sorted while written
constexpr int kSortThreads = 512;
constexpr int kSortSmem = 8192;      // longer lists are sorted in global memory

struct CountVisitor {
  const GridDev &g;
  const QueryGeom &Q;
  const Band &B;
  int self;
  long long count;
  __device__ __forceinline__ void operator()(const Target &t, bool full) {
    const int b = __ldg(g.cell_start + t.key), e = __ldg(g.cell_start + t.key + 1);
    if (full) {
      count += e - b - ((self >= b && self < e) ? 1 : 0);
      return;
    }
    for (int j = b; j < e; ++j) {
      const float4 p = g.spos[j];
      if (j != self && pair_hit(g, Q, t, B, p)) ++count;
    }
  }
};

struct WriteVisitor {
  const GridDev &g;
  const QueryGeom &Q;
  const Band &B;
  int self;
  int *out;        // this query's list
  int len;         // its final length
  int k;           // ids written so far
  bool sort_inline;
  __device__ __forceinline__ void emit(int id) {
    if (k >= len) return;           // defensive: never write past the list
    if (sort_inline) {
      int p = k;
      while (p > 0) {
        const int prev = out[p - 1];
        if (prev <= id) break;
        out[p] = prev;
        --p;
      }
      out[p] = id;
    } else {
      out[k] = id;
    }
    ++k;
  }
  __device__ __forceinline__ void operator()(const Target &t, bool full) {
    const int b = __ldg(g.cell_start + t.key), e = __ldg(g.cell_start + t.key + 1);
    for (int j = b; j < e; ++j) {
      if (j == self) continue;
      if (full || pair_hit(g, Q, t, B, g.spos[j])) emit(__ldg(g.perm + j));
    }
  }
};

template <bool CUBE>
__global__ void __launch_bounds__(kQueryThreads) k_radius_count(GridDev g, WalkParams P, Band B,
                                                                unsigned flags,
                                                                long long *__restrict__ counts) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= g.n) return;
  const QueryGeom Q = make_geom(g.spos[s], g);
  CountVisitor v{g, Q, B, (flags & SI_INCLUDE_SELF) ? -1 : s, 0};
  if (CUBE || Q.outside) walk_cube(g, Q, P.dg, v);
  else walk_sphere(g, Q, P, v);
  counts[__ldg(g.perm + s)] = v.count;
}

template <bool CUBE>
__global__ void __launch_bounds__(kQueryThreads) k_radius_write(GridDev g, WalkParams P, Band B,
                                                                unsigned flags,
                                                                const long long *__restrict__ offsets,
                                                                int *__restrict__ ids, long long cap,
                                                                int *__restrict__ longq) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= g.n) return;
  const int orig = __ldg(g.perm + s);
  const long long base = offsets[orig];
  const int len = (int)(offsets[orig + 1] - base);
  if (len == 0) return;
  if (base + len > cap) {
    atomicOr(g.status, ST_CAPACITY);
    return;
  }
  const bool sort_all = !(flags & SI_NO_SORT);
  const QueryGeom Q = make_geom(g.spos[s], g);
  WriteVisitor v{g, Q, B, (flags & SI_INCLUDE_SELF) ? -1 : s, ids + base, len, 0,
                 sort_all && len <= kInlineSort};
  if (CUBE || Q.outside) walk_cube(g, Q, P.dg, v);
  else walk_sphere(g, Q, P, v);
  if (v.k != len) atomicOr(g.status, ST_INTERNAL);
  if (sort_all && len > kInlineSort) {
    const int slot = atomicAdd(longq, 1);
    longq[1 + slot] = orig;
  }
}

// Ascending bitonic sort of a[0..n) by one block, with virtual +inf padding
// up to the next power of two.  Every compare-exchange puts the smaller value
// at the lower index (first step of each merge compares mirrored pairs), so a
// pair whose upper index is past n never moves anything.
__device__ void block_bitonic(int *a, int n) {
  int P = 1;
  while (P < n) P <<= 1;
  for (int k = 2; k <= P; k <<= 1) {
    for (int i = threadIdx.x; i < P / 2; i += blockDim.x) {
      const int lo = (i / (k / 2)) * k + (i % (k / 2));
      const int hi = (lo / k) * k + (k - 1 - (lo % k));
      if (hi < n && a[hi] < a[lo]) {
        const int t = a[lo];
        a[lo] = a[hi];
        a[hi] = t;
      }
    }
    __syncthreads();
    for (int h = k / 4; h >= 1; h >>= 1) {
      for (int i = threadIdx.x; i < P / 2; i += blockDim.x) {
        const int lo = (i / h) * 2 * h + (i % h);
        const int hi = lo + h;
        if (hi < n && a[hi] < a[lo]) {
          const int t = a[lo];
          a[lo] = a[hi];
          a[hi] = t;
        }
      }
      __syncthreads();
    }
  }
}

__global__ void __launch_bounds__(kSortThreads) k_sort_long(const long long *__restrict__ offsets,
                                                           int *ids, const int *__restrict__ longq) {
  __shared__ int buf[kSortSmem];
  const int nq = longq[0];
  for (int item = blockIdx.x; item < nq; item += gridDim.x) {
    const int q = longq[1 + item];
    const long long base = offsets[q];
    const int len = (int)(offsets[q + 1] - base);
    int *list = ids + base;
    if (len <= kSortSmem) {
      for (int i = threadIdx.x; i < len; i += blockDim.x) buf[i] = list[i];
      __syncthreads();
      block_bitonic(buf, len);
      for (int i = threadIdx.x; i < len; i += blockDim.x) list[i] = buf[i];
    } else {
      block_bitonic(list, len);
    }
    __syncthreads();
  }
}

}  // namespace si

using namespace si;

// Culling parameters for radius r on grid g (cell units).
static WalkParams walk_params(const Lattice &lat, float r, bool inclusion) {
  WalkParams P;
  const float d = r * lat.inv_s;
  P.dg = d + (float)lat.eps;
  // run-time exact test above d - 1 (Sec. III.A heuristic): b > d - 1
  const float thr = d - 1.f;
  P.rt_b2 = thr <= 0.f ? 0 : (int)floorf(thr * thr) + 1;
  // a cell can lie wholly inside only if b <= d - 1 (its far corner is at
  // least b + 1 away); test those cells' far corners exactly
  const float dm = d - (float)lat.eps;
  if (inclusion && d >= 1.f) {
    P.incl_b2 = (int)floorf((d - 1.f) * (d - 1.f));
    P.incl_d2 = dm * dm;
  } else {
    P.incl_b2 = -1;
    P.incl_d2 = 0.f;
  }
  return P;
}

extern "C" si_status si_query_radius(si_grid *g, const float *d_centers, int64_t m, float r,
                                     uint32_t flags, int64_t *d_offsets, int32_t *d_ids,
                                     int64_t ids_capacity, int64_t *h_total, void *stream) {
  if (!g) return fail(SI_ERR_INVALID, "null grid");
  if (d_centers) return fail(SI_ERR_INVALID, "only the all-agents mode is supported (centers must be NULL)");
  if (m != g->n) return fail(SI_ERR_INVALID, "all-agents mode: m must equal the grid's point count");
  if (!(r >= 0.f) || !std::isfinite(r)) return fail(SI_ERR_INVALID, "radius must be finite and >= 0");
  if (!g->lat.unbounded && (double)r > (double)g->desc.r_max)
    return fail(SI_ERR_INVALID, "radius exceeds the grid's r_max");
  if (!d_offsets) return fail(SI_ERR_INVALID, "null offsets");
  if (ids_capacity < 0 || (ids_capacity > 0 && !d_ids)) return fail(SI_ERR_INVALID, "bad ids buffer");
  if (flags & ~(SI_METHOD_CUBE | SI_INCLUDE_SELF | SI_NO_SORT))
    return fail(SI_ERR_INVALID, "unknown flags");
  cudaStream_t st = (cudaStream_t)stream;
  const bool cube = flags & SI_METHOD_CUBE;
  const double load = g->n_cells > 1 ? (double)g->n / (double)(g->n_cells - 1) : 0.0;
  const WalkParams P = walk_params(g->lat, r, load >= 4.0);
  const Band B = make_band(g->lat, r);
  const GridDev dv = g->dev();
  long long *off = (long long *)d_offsets;
  SI_CUDA_TRY(cudaMemsetAsync(off, 0, sizeof(long long), st));
  const unsigned blocks = (unsigned)((m + kQueryThreads - 1) / kQueryThreads);
  if (m > 0) {
    if (cube)
      SI_KLAUNCH("k_radius_count_cube", st,
                 k_radius_count<true><<<blocks, kQueryThreads, 0, st>>>(dv, P, B, flags, off + 1));
    else
      SI_KLAUNCH("k_radius_count", st,
                 k_radius_count<false><<<blocks, kQueryThreads, 0, st>>>(dv, P, B, flags, off + 1));
    si_status s = scan_inclusive_i64(off + 1, off + 1, m, g->scan_i64, st);
    if (s != SI_OK) return s;
  }
  if (h_total) {
    SI_CUDA_TRY(cudaMemcpyAsync(g->h_pinned, off + m, sizeof(long long), cudaMemcpyDeviceToHost, st));
    SI_CUDA_TRY(cudaStreamSynchronize(st));
    *h_total = g->h_pinned[0];
    if (*h_total > ids_capacity) return fail(SI_ERR_CAPACITY, "neighbor id buffer too small");
  }
  if (m == 0) return SI_OK;
  SI_CUDA_TRY(cudaMemsetAsync(g->longq, 0, sizeof(int), st));
  if (cube)
    SI_KLAUNCH("k_radius_write_cube", st,
               k_radius_write<true><<<blocks, kQueryThreads, 0, st>>>(dv, P, B, flags, off, d_ids,
                                                                      ids_capacity, g->longq));
  else
    SI_KLAUNCH("k_radius_write", st,
               k_radius_write<false><<<blocks, kQueryThreads, 0, st>>>(dv, P, B, flags, off, d_ids,
                                                                       ids_capacity, g->longq));
  if (!(flags & SI_NO_SORT)) {
    SI_KLAUNCH("k_sort_long", st, k_sort_long<<<2 * 148, kSortThreads, 0, st>>>(off, d_ids, g->longq));
  }
  return SI_OK;
}
