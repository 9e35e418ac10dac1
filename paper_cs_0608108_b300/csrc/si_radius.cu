// All-agents fixed-radius query (Sec. I, Sec. II.A): count pass, prefix sum,
// write pass, ids ascending per list.
//
// Queries in lightly loaded cells: one thread per query point, queries in cell
// order so that neighbouring threads walk neighbouring cells (their candidate
// cells are shared through L1/L2); lists of up to 32 ids are sorted while
// written, longer ones are queued for a warp (or block) bitonic sort.
// Queries in cells holding at least kHeavyMin points: one block per cell
// (si_cell.cu), lists written already sorted.
#include <algorithm>
#include <cmath>

#include "si_host.h"
#include "si_radius.cuh"
#include "si_sort.cuh"

namespace si {

struct CountVisitor {
  const GridDev &g;
  const QueryGeom &Q;
  const Band &B;
  int self;
  long long count;
  __device__ __forceinline__ void operator()(const Target &t, bool full, int b, int e) {
    if (full) {
      count += e - b - ((self >= b && self < e) ? 1 : 0);
      return;
    }
    for (int j = b; j < e; ++j) {
      const float4 p = g.spos[j];
      if (j != self && pair_hit(g, Q, t, B, p)) ++count;
    }
  }
  __device__ __forceinline__ void operator()(const Target &t, bool full) {
    (*this)(t, full, __ldg(g.cell_start + t.key), __ldg(g.cell_start + t.key + 1));
  }
};

struct WriteVisitor {
  const GridDev &g;
  const QueryGeom &Q;
  const Band &B;
  int self;
  int *out;        // this query's list (global), or its staging slots (shared)
  int stride;      // distance between consecutive slots of `out`
  int len;         // its final length
  int k;           // ids written so far
  bool sort_inline;
  __device__ __forceinline__ void emit(int id) {
    if (k >= len) return;           // defensive: never write past the list
    if (sort_inline) {
      int p = k;
      while (p > 0) {
        const int prev = out[(p - 1) * stride];
        if (prev <= id) break;
        out[p * stride] = prev;
        --p;
      }
      out[p * stride] = id;
    } else {
      out[k * stride] = id;
    }
    ++k;
  }
  __device__ __forceinline__ void operator()(const Target &t, bool full, int b, int e) {
    for (int j = b; j < e; ++j) {
      if (j == self) continue;
      if (full || pair_hit(g, Q, t, B, g.spos[j])) emit(__ldg(g.perm + j));
    }
  }
  __device__ __forceinline__ void operator()(const Target &t, bool full) {
    (*this)(t, full, __ldg(g.cell_start + t.key), __ldg(g.cell_start + t.key + 1));
  }
};

// Cell walks of the per-query kernels.
enum Walk : int { kWalkPaper = 0, kWalkClasses = 1, kWalkCube = 2 };

template <int WALK, class V>
__device__ __forceinline__ void walk_one(const GridDev &g, const QueryGeom &Q, const WalkParams &P, V &v) {
  if (WALK == kWalkCube || Q.outside) walk_cube(g, Q, P.dg, v);
  else if (WALK == kWalkClasses) walk_classes_in(g, Q, g.cls, g.cls_begin, g.cls_q, v);
  else walk_sphere(g, Q, P, v);
}

// One query by one thread.  heavy_min > 0: queries of heavy cells
// (heavy_cell) are left to the cell kernel.
// stage (nullable): this thread's kInlineSort shared slots, `stride` apart;
// short lists are sorted there and stored once.
template <bool WRITE, int WALK>
__device__ __forceinline__ void radius_one(const GridDev &g, const WalkParams &P, const Band &B,
                                           unsigned flags, int s, int heavy_min, long long *counts,
                                           const long long *offsets, int *ids, long long cap,
                                           int *longq, int *stage = nullptr, int stride = 0) {
  const QueryGeom Q = make_geom(g.spos[s], g);
  if (heavy_min > 0 && !Q.outside && heavy_cell(g.cell_start, pack3(Q.c[0], Q.c[1], Q.c[2], g), g.outside))
    return;
  const int self = (flags & SI_INCLUDE_SELF) ? -1 : s;
  const int orig = __ldg(g.perm + s);
  if (!WRITE) {
    CountVisitor v{g, Q, B, self, 0};
    walk_one<WALK>(g, Q, P, v);
    counts[orig] = v.count;
  } else {
    const long long base = offsets[orig];
    const int len = (int)(offsets[orig + 1] - base);
    if (len == 0) return;
    if (base + len > cap) {
      atomicOr(g.status, ST_CAPACITY);
      return;
    }
    const bool sort_all = !(flags & SI_NO_SORT);
    const bool inl = sort_all && len <= kInlineSort;
    const bool staged = inl && stage != nullptr;
    WriteVisitor v{g, Q, B, self, staged ? stage : ids + base, staged ? stride : 1, len, 0, inl};
    walk_one<WALK>(g, Q, P, v);
    if (v.k != len) atomicOr(g.status, ST_INTERNAL);
    if (staged)
      for (int i = 0; i < len; ++i) ids[base + i] = stage[i * stride];
    if (sort_all && len > kInlineSort) {
      const int slot = atomicAdd(longq, 1);
      longq[1 + slot] = orig;
    }
  }
}

template <bool WRITE, int WALK>
__global__ void __launch_bounds__(kQueryThreads) k_radius(GridDev g, WalkParams P, Band B, unsigned flags,
                                                          int heavy_min, long long *counts,
                                                          const long long *offsets, int *ids,
                                                          long long cap, int *longq) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= g.n) return;
  radius_one<WRITE, WALK>(g, P, B, flags, s, heavy_min, counts, offsets, ids, cap, longq);
}

// Per-query kernel with the class tables staged in shared memory: a
// persistent grid, each block copies the tables once and then walks queries
// in cell order (grid-stride), so the divergent per-lane table reads hit
// shared memory instead of L2.
template <bool WRITE>
__global__ void __launch_bounds__(kClassThreads) k_radius_cls(GridDev g, WalkParams P, Band B,
                                                              unsigned flags, int heavy_min,
                                                              int n_entries, long long *counts,
                                                              const long long *offsets, int *ids,
                                                              long long cap, int *longq) {
  extern __shared__ __align__(16) unsigned long long cls_smem[];
  const int nbeg = g.cls_q * g.cls_q * g.cls_q + 1;
  int *beg_smem = reinterpret_cast<int *>(cls_smem + n_entries);
  // write pass: short lists are sorted in shared slots, column-interleaved
  int *stage = WRITE ? beg_smem + ((nbeg + 3) & ~3) + threadIdx.x : nullptr;
  for (int i = threadIdx.x; i < n_entries; i += blockDim.x) cls_smem[i] = __ldg(g.cls + i);
  for (int i = threadIdx.x; i < nbeg; i += blockDim.x) beg_smem[i] = __ldg(g.cls_begin + i);
  __syncthreads();
  GridDev gs = g;
  gs.cls = cls_smem;
  gs.cls_begin = beg_smem;
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < g.n; s += gridDim.x * blockDim.x)
    radius_one<WRITE, kWalkClasses>(gs, P, B, flags, s, heavy_min, counts, offsets, ids, cap, longq,
                                    stage, kClassThreads);
}

// Queries the cell kernel handed back (listed by sorted slot): per query.
template <bool WRITE>
__global__ void __launch_bounds__(kQueryThreads) k_radius_over(GridDev g, WalkParams P, Band B,
                                                               unsigned flags, const int *over,
                                                               long long *counts,
                                                               const long long *offsets, int *ids,
                                                               long long cap, int *longq) {
  const int nover = over[0];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nover; i += gridDim.x * blockDim.x)
    radius_one<WRITE, kWalkPaper>(g, P, B, flags, over[1 + i], 0, counts, offsets, ids, cap, longq);
}

// One warp per queued list (up to kSortWarpCap ids, in shared memory); longer
// lists are passed on to the block sort.
__global__ void __launch_bounds__(kSortWarps * 32) k_sort_warp(const long long *__restrict__ offsets,
                                                              int *ids, const int *__restrict__ longq,
                                                              int *hugeq) {
  extern __shared__ int sbuf[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int *buf = sbuf + w * kSortWarpCap;
  const int nq = longq[0];
  const int gw = blockIdx.x * kSortWarps + w, nwarps = gridDim.x * kSortWarps;
  for (int item = gw; item < nq; item += nwarps) {
    const int q = longq[1 + item];
    const long long base = offsets[q];
    const int len = (int)(offsets[q + 1] - base);
    int *list = ids + base;
    if (len > kSortWarpCap) {
      if (lane == 0) {
        const int slot = atomicAdd(hugeq, 1);
        hugeq[1 + slot] = q;
      }
      continue;
    }
    for (int i = lane; i < len; i += 32) buf[i] = list[i];
    __syncwarp();
    bitonic_padded(buf, len, lane, 32, WarpSync());
    for (int i = lane; i < len; i += 32) list[i] = buf[i];
    __syncwarp();
  }
}

__global__ void __launch_bounds__(512) k_sort_block(const long long *__restrict__ offsets, int *ids,
                                                   const int *__restrict__ hugeq) {
  extern __shared__ int sbuf[];
  const int nq = hugeq[0];
  for (int item = blockIdx.x; item < nq; item += gridDim.x) {
    const int q = hugeq[1 + item];
    const long long base = offsets[q];
    const int len = (int)(offsets[q + 1] - base);
    int *list = ids + base;
    if (len <= kSortBlockCap) {
      for (int i = threadIdx.x; i < len; i += blockDim.x) sbuf[i] = list[i];
      __syncthreads();
      bitonic_padded(sbuf, len, threadIdx.x, blockDim.x, BlockSync());
      for (int i = threadIdx.x; i < len; i += blockDim.x) list[i] = sbuf[i];
    } else {
      bitonic_padded(list, len, threadIdx.x, blockDim.x, BlockSync());
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

template <bool WRITE>
static si_status launch_light(int walk, const si_grid *gr, const GridDev &dv, const WalkParams &P,
                              const Band &B, unsigned flags, int heavy_min, long long *counts,
                              const long long *off, int *ids, long long cap, int *longq,
                              unsigned blocks, cudaStream_t st) {
  if (walk == kWalkCube) {
    SI_KLAUNCH(WRITE ? "k_radius_write_cube" : "k_radius_count_cube", st,
               k_radius<WRITE, kWalkCube><<<blocks, kQueryThreads, 0, st>>>(dv, P, B, flags, 0, counts,
                                                                            off, ids, cap, longq));
  } else if (walk == kWalkClasses && gr->cls_smem_bytes > 0) {
    const int nbeg = gr->cls_q * gr->cls_q * gr->cls_q + 1;
    const size_t smem = gr->cls_host.size() * sizeof(unsigned long long) +
                        (size_t)((nbeg + 3) & ~3) * sizeof(int) +
                        (WRITE ? (size_t)kInlineSort * kClassThreads * sizeof(int) : 0);
    SI_CUDA_TRY(cudaFuncSetAttribute(k_radius_cls<WRITE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
    int per_sm = 0;
    SI_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_radius_cls<WRITE>,
                                                              kClassThreads, smem));
    const unsigned grid = (unsigned)std::max(1, std::min<int>(per_sm, 8) * 148);
    SI_KLAUNCH(WRITE ? "k_radius_write" : "k_radius_count", st,
               k_radius_cls<WRITE><<<grid, kClassThreads, smem, st>>>(
                   dv, P, B, flags, heavy_min, (int)gr->cls_host.size(), counts, off, ids, cap, longq));
  } else if (walk == kWalkClasses) {
    SI_KLAUNCH(WRITE ? "k_radius_write_cls_l2" : "k_radius_count_cls_l2", st,
               k_radius<WRITE, kWalkClasses><<<blocks, kQueryThreads, 0, st>>>(
                   dv, P, B, flags, heavy_min, counts, off, ids, cap, longq));
  } else {
    SI_KLAUNCH(WRITE ? "k_radius_write_eq2" : "k_radius_count_eq2", st,
               k_radius<WRITE, kWalkPaper><<<blocks, kQueryThreads, 0, st>>>(
                   dv, P, B, flags, heavy_min, counts, off, ids, cap, longq));
  }
  return SI_OK;
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
  if (flags & ~(SI_METHOD_CUBE | SI_INCLUDE_SELF | SI_NO_SORT | SI_WALK_PAPER))
    return fail(SI_ERR_INVALID, "unknown flags");
  cudaStream_t st = (cudaStream_t)stream;
  const bool cube = flags & SI_METHOD_CUBE;
  const double load = g->n_cells > 1 ? (double)g->n / (double)(g->n_cells - 1) : 0.0;
  const WalkParams P = walk_params(g->lat, r, load >= 4.0);
  const Band B = make_band(g->lat, r);
  const int walk = cube ? kWalkCube
                        : ((!(flags & SI_WALK_PAPER) && g->ensure_classes(P.dg, st)) ? kWalkClasses
                                                                                    : kWalkPaper);
  const GridDev dv = g->dev();
  // the cell path holds the whole cell-level sphere (entries with b^2 <= n)
  const int n_tab = std::min((int)std::floor((double)P.dg * (double)P.dg), g->tables.n_max);
  const bool heavy = !cube && n_tab >= 0 && g->tab_end_host[n_tab] <= kCellTCap;
  const int heavy_min = heavy ? kHeavyMin : 0;
  long long *off = (long long *)d_offsets;
  const unsigned blocks = (unsigned)((m + kQueryThreads - 1) / kQueryThreads);
  si_status s;
  // count phase: per-query counts of light cells, the cell kernel's counts
  // and scratch lists for heavy cells, per-query counts of what it handed back
  auto count_phase = [&]() -> si_status {
    SI_CUDA_TRY(cudaMemsetAsync(off, 0, sizeof(long long), st));
    SI_CUDA_TRY(cudaMemsetAsync(g->counters, 0, kCounterInts * sizeof(int), st));
    SI_CUDA_TRY(cudaMemsetAsync(g->over, 0, sizeof(int), st));
    SI_CUDA_TRY(cudaMemsetAsync(g->scr_top, 0, sizeof(unsigned long long), st));
    if (m == 0) return SI_OK;
    si_status r;
    if ((r = launch_light<false>(walk, g, dv, P, B, flags, heavy_min, off + 1, nullptr, nullptr, 0,
                                 nullptr, blocks, st)) != SI_OK)
      return r;
    if (heavy) {
      if ((r = launch_cell_pass(dv, P, B, flags, g->heavy, g->counters, g->over, off + 1, g->scr_off,
                                g->scratch, g->scr_cap, g->scr_top, st)) != SI_OK)
        return r;
      SI_KLAUNCH("k_radius_over_count", st,
                 k_radius_over<false><<<148 * 4, kQueryThreads, 0, st>>>(dv, P, B, flags, g->over,
                                                                         off + 1, nullptr, nullptr, 0,
                                                                         nullptr));
    }
    return scan_inclusive_i64(off + 1, off + 1, m, g->scan_i64, st);
  };
  if ((s = count_phase()) != SI_OK) return s;
  if (h_total) {
    SI_CUDA_TRY(cudaMemcpyAsync(g->h_pinned, off + m, sizeof(long long), cudaMemcpyDeviceToHost, st));
    SI_CUDA_TRY(cudaMemcpyAsync(g->h_pinned + 1, g->scr_top, sizeof(long long), cudaMemcpyDeviceToHost, st));
    SI_CUDA_TRY(cudaStreamSynchronize(st));
    // cells whose lists did not fit the scratch took the per-query path;
    // make room and count again so that the cell kernel serves them
    if (heavy && g->h_pinned[1] > g->scr_cap) {
      const long long want = g->h_pinned[1] + g->h_pinned[1] / 4 + 1024;
      int *fresh = nullptr;
      if (cudaMalloc((void **)&fresh, want * sizeof(int)) == cudaSuccess) {
        cudaFree(g->scratch);
        g->scratch = fresh;
        g->scr_cap = want;
        if ((s = count_phase()) != SI_OK) return s;
        SI_CUDA_TRY(cudaMemcpyAsync(g->h_pinned, off + m, sizeof(long long), cudaMemcpyDeviceToHost, st));
        SI_CUDA_TRY(cudaStreamSynchronize(st));
      } else {
        cudaGetLastError();   // keep the old scratch; results stay exact
      }
    }
    *h_total = g->h_pinned[0];
    if (*h_total > ids_capacity) return fail(SI_ERR_CAPACITY, "neighbor id buffer too small");
  }
  if (m == 0) return SI_OK;
  SI_CUDA_TRY(cudaMemsetAsync(g->longq, 0, sizeof(int), st));
  SI_CUDA_TRY(cudaMemsetAsync(g->hugeq, 0, sizeof(int), st));
  if ((s = launch_light<true>(walk, g, dv, P, B, flags, heavy_min, nullptr, off, d_ids, ids_capacity,
                              g->longq, blocks, st)) != SI_OK)
    return s;
  if (heavy) {
    if ((s = launch_cell_copy(dv, g->heavy, g->scr_off, g->scratch, off, d_ids, ids_capacity, st)) != SI_OK)
      return s;
    SI_KLAUNCH("k_radius_over_write", st,
               k_radius_over<true><<<148 * 4, kQueryThreads, 0, st>>>(dv, P, B, flags, g->over, nullptr,
                                                                      off, d_ids, ids_capacity,
                                                                      g->longq));
  }
  if (!(flags & SI_NO_SORT)) {
    const size_t wsm = (size_t)kSortWarps * kSortWarpCap * sizeof(int);
    SI_CUDA_TRY(cudaFuncSetAttribute(k_sort_warp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)wsm));
    SI_KLAUNCH("k_sort_warp", st,
               k_sort_warp<<<148 * 2, kSortWarps * 32, wsm, st>>>(off, d_ids, g->longq, g->hugeq));
    const size_t bsm = (size_t)kSortBlockCap * sizeof(int);
    SI_CUDA_TRY(cudaFuncSetAttribute(k_sort_block, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bsm));
    SI_KLAUNCH("k_sort_block", st, k_sort_block<<<148, 512, bsm, st>>>(off, d_ids, g->hugeq));
  }
  return SI_OK;
}
