// All-agents fixed-radius query (Sec. I, Sec. II.A): count pass, prefix sum,
// write pass, ids ascending per list.
//
// Queries in lightly loaded cells: one thread per query point, queries in cell
// order so that neighbouring threads walk neighbouring cells (their candidate
// cells are shared through L1/L2); lists of up to 24 ids are sorted while
// written, longer ones are queued for a warp (or block) bitonic sort.
// Queries in dense cells: one warp per query over the flattened class walk.
// Queries in heavy cells (heavy_cell): one block per 2 x 2 x 2 group of heavy
// cells (si_group.cu) or per cell (si_cell.cu), hit masks over id-ordered
// candidates, expanded into sorted lists after the scan.  When heavy cells
// exist, the per-query kernels run on a second stream of the grid beside the
// heavy cells' kernels (forked and joined by events, so graph capture
// follows them).
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
    int j = b;
    for (; j < e; ++j) {
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
    int j = b;
    for (; j < e; ++j) {
      if (j == self) continue;
      if (full || pair_hit(g, Q, t, B, g.spos[j])) emit(__ldg(g.perm + j));
    }
  }
  __device__ __forceinline__ void operator()(const Target &t, bool full) {
    (*this)(t, full, __ldg(g.cell_start + t.key), __ldg(g.cell_start + t.key + 1));
  }
};

// Count pass that also keeps a short list: hits are counted, and the first
// kInlineSort ids are kept sorted in the thread's shared slots (`stride`
// apart), so that the write pass can copy a list of up to kInlineSort ids
// instead of walking the cells again.
struct StageVisitor {
  const GridDev &g;
  const QueryGeom &Q;
  const Band &B;
  int self;
  int *out;
  int stride;
  int k;           // hits so far
  __device__ __forceinline__ void hit(int id) {
    if (k < kInlineSort) {
      int p = k;
      while (p > 0) {
        const int prev = out[(p - 1) * stride];
        if (prev <= id) break;
        out[p * stride] = prev;
        --p;
      }
      out[p * stride] = id;
    }
    ++k;
  }
  __device__ __forceinline__ void operator()(const Target &t, bool full, int b, int e) {
    for (int j = b; j < e; ++j) {
      if (j == self) continue;
      if (full || pair_hit(g, Q, t, B, g.spos[j])) hit(__ldg(g.perm + j));
    }
  }
  __device__ __forceinline__ void operator()(const Target &t, bool full) {
    (*this)(t, full, __ldg(g.cell_start + t.key), __ldg(g.cell_start + t.key + 1));
  }
};

// Cell walks of the per-query kernels.
enum Walk : int { kWalkPaper = 0, kWalkClasses = 1, kWalkCube = 2, kWalkPlanes = 3 };

template <int WALK, class V>
__device__ __forceinline__ void walk_one(const GridDev &g, const QueryGeom &Q, const WalkParams &P, V &v) {
  if (WALK == kWalkCube || Q.outside) walk_cube(g, Q, P.dg, v);
  else if (WALK == kWalkClasses) walk_classes_in(g, Q, g.cls, g.cls_begin, g.cls_q, v);
  else if (WALK == kWalkPlanes) walk_planes(g, Q, P.dg, v);
  else walk_sphere(g, Q, P, v);
}

// One query by one thread.  skip: bit 0 leaves the queries of heavy cells to
// the cell kernel, bit 1 those of dense cells to the warp-per-query kernels
// (the class byte of the query's cell, copied to every slot at binning).
// stage (nullable): this thread's kInlineSort shared slots, `stride` apart;
// short lists are sorted there and stored once.
template <bool WRITE, int WALK>
// lstage (nullable, with stage): the short-list staging area, column
// `column` of kInlineSort rows `lstride` apart; the count pass stores lists of
// up to kInlineSort ids there, sorted, and the write pass copies them.
__device__ __forceinline__ void radius_one(const GridDev &g, const WalkParams &P, const Band &B,
                                           unsigned flags, int s, unsigned skip, long long *counts,
                                           const long long *offsets, int *ids, long long cap,
                                           int *longq, int *stage = nullptr, int stride = 0,
                                           int *lstage = nullptr, long long lstride = 0, int column = 0) {
  if (skip) {
    const int c = g.slot_cls[s];
    if (((c == kCellHeavy || c == kCellHeavyBig) && (skip & 1u)) || (c == kCellDense && (skip & 2u))) return;
  }
  const QueryGeom Q = make_geom(g.qpos[s], g);
  const int self = query_self(g, flags, s);
  const int orig = __ldg(g.qid + s);
  if (!WRITE) {
    if (lstage && stage) {
      StageVisitor v{g, Q, B, self, stage, stride, 0};
      walk_one<WALK>(g, Q, P, v);
      counts[orig] = v.k;
      if (v.k <= kInlineSort)
        for (int i = 0; i < v.k; ++i) lstage[i * lstride + column] = stage[i * stride];
    } else {
      CountVisitor v{g, Q, B, self, 0};
      walk_one<WALK>(g, Q, P, v);
      counts[orig] = v.count;
    }
  } else {
    const long long base = offsets[orig];
    const int len = (int)(offsets[orig + 1] - base);
    if (len == 0) return;
    if (base + len > cap) {
      atomicOr(g.status, ST_CAPACITY);
      return;
    }
    if (lstage && len <= kInlineSort) {   // kept, sorted, by the count pass
      for (int i = 0; i < len; ++i) ids[base + i] = lstage[i * lstride + column];
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

// list (nullable): [0] = count, then the sorted slots to serve; else every slot.
template <bool WRITE, int WALK>
__global__ void __launch_bounds__(kQueryThreads) k_radius(GridDev g, WalkParams P, Band B, unsigned flags,
                                                          unsigned skip, long long *counts,
                                                          const long long *offsets, int *ids,
                                                          long long cap, int *longq,
                                                          const int *__restrict__ list) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (list ? list[0] : g.n)) return;
  radius_one<WRITE, WALK>(g, P, B, flags, list ? list[1 + t] : t, skip, counts, offsets, ids, cap, longq);
}

// Per-query kernel with the class tables staged in shared memory: a
// persistent grid, each block copies the tables once and then walks queries
// in cell order (grid-stride), so the divergent per-lane table reads hit
// shared memory instead of L2.  Up to six blocks per SM (40 registers; at
// d = 1.5 cells the tables and 24 staged ids a thread fit six blocks' shared
// memory): the walk waits on dependent loads, and more resident warps hide
// more of them.
template <bool WRITE>
__global__ void __launch_bounds__(kClassThreads, 6) k_radius_cls(GridDev g, WalkParams P, Band B,
                                                              unsigned flags, unsigned skip,
                                                              int n_entries, long long *counts,
                                                              const long long *offsets, int *ids,
                                                              long long cap, int *longq,
                                                              const int *__restrict__ list, int *lstage,
                                                              long long lstride) {
  extern __shared__ __align__(16) unsigned long long cls_smem[];
  const int nbeg = g.cls_q * g.cls_q * g.cls_q + 1;
  int *beg_smem = reinterpret_cast<int *>(cls_smem + n_entries);
  // short lists are sorted in shared slots, column-interleaved (write pass;
  // with lstage, the count pass, which keeps them for the write pass)
  int *stage = (WRITE || lstage) ? beg_smem + ((nbeg + 3) & ~3) + threadIdx.x : nullptr;
  for (int i = threadIdx.x; i < n_entries; i += blockDim.x) cls_smem[i] = __ldg(g.cls + i);
  for (int i = threadIdx.x; i < nbeg; i += blockDim.x) beg_smem[i] = __ldg(g.cls_begin + i);
  __syncthreads();
  GridDev gs = g;
  gs.cls = cls_smem;
  gs.cls_begin = beg_smem;
  // list: the light cells' slots (the other cells have their own kernels);
  // else every slot, skipping by class byte
  const int nl = list ? list[0] : g.n;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nl; t += gridDim.x * blockDim.x)
    radius_one<WRITE, kWalkClasses>(gs, P, B, flags, list ? list[1 + t] : t, list ? 0u : skip, counts, offsets,
                                    ids, cap, longq, stage, kClassThreads, lstage, lstride, t);
}

// Queries of dense cells (queued at binning): one warp per query.
//
// Flattened class walk: lane r decodes row r of each batch of 32 rows of the
// query's class list into its runs of points (two if the row crosses the
// cyclic x boundary), so that all run bounds are fetched at once; a warp
// prefix of the run lengths numbers the batch's candidates and the lanes
// take them 32 at a time.  fn(hit, j) is called by every lane for each group
// of 32 (j < 0: no candidate).  The outside cell, if a row reaches it, is
// taken last, every pair in FP64.  Query points outside the region walk the
// bounding cube instead (warp visitors below).
struct FlatRuns {
  int b[64];
  int len[64];
  float qx[64], qy[64], qz[64];
  unsigned char flags[64];   // bit 0: whole run inside the sphere, bit 1: wrapped image
  int pre[33];
};

template <class F>
__device__ __forceinline__ void warp_class_walk(const GridDev &g, const QueryGeom &Q, const Band &B, int self,
                                                int lane, FlatRuns &R, F &fn) {
  const int q = g.cls_q;
  const int ci = min((int)(Q.phi[0] * (float)q), q - 1);
  const int cj = min((int)(Q.phi[1] * (float)q), q - 1);
  const int ck = min((int)(Q.phi[2] * (float)q), q - 1);
  const int c = (ck * q + cj) * q + ci;
  const int cb = g.cls_begin[c], ce = g.cls_begin[c + 1];
  const int Gx = 1 << g.wx;
  const bool cyc_x = g.cyc & 1u;
  bool out_any = false;
  for (int base = cb; base < ce; base += 32) {
    const int t = base + lane;
    int b0 = 0, l0 = 0, b1 = 0, l1 = 0;
    float qx0 = 0.f, qy0 = 0.f, qz0 = 0.f, qx1 = 0.f;
    unsigned f0 = 0u, f1 = 0u;
    bool out = false;
    if (t < ce) {
      const unsigned long long E = g.cls[t];
      const int lo = (int)(signed char)((E >> 48) & 0xffull);
      const int len = (int)((E >> 56) & 127ull);
      const unsigned full = (unsigned)(E >> 63);
      const Target tg = translate_raw(E & ((1ull << 48) - 1ull), Q, g);
      if (tg.outside) {
        out = true;
      } else {
        const unsigned row = tg.key - (unsigned)Q.c[0];
        int x0 = Q.c[0] + lo, x1 = x0 + len - 1;
        qx0 = tg.qx;
        qy0 = tg.qy;
        qz0 = tg.qz;
        f0 = full | (tg.wrapped ? 2u : 0u);
        if (!cyc_x) {
          if (x0 < 0 || x1 >= Gx) out = true;
          x0 = max(x0, 0);
          x1 = min(x1, Gx - 1);
        } else if (x0 < 0 || x1 >= Gx) {
          const int wa = x0 < 0 ? x0 + Gx : 0;
          const int wb = x0 < 0 ? Gx - 1 : x1 - Gx;
          b1 = __ldg(g.cell_start + row + wa);
          l1 = __ldg(g.cell_start + row + wb + 1) - b1;
          qx1 = Q.q.x + (x0 < 0 ? g.Lx : -g.Lx);
          f1 = full | 2u;
          x0 = max(x0, 0);
          x1 = min(x1, Gx - 1);
        }
        if (x0 <= x1) {
          b0 = __ldg(g.cell_start + row + x0);
          l0 = __ldg(g.cell_start + row + x1 + 1) - b0;
        }
      }
    }
    out_any |= __any_sync(0xffffffffu, out);
    R.b[2 * lane] = b0;
    R.len[2 * lane] = l0;
    R.qx[2 * lane] = qx0;
    R.qy[2 * lane] = qy0;
    R.qz[2 * lane] = qz0;
    R.flags[2 * lane] = (unsigned char)f0;
    R.b[2 * lane + 1] = b1;
    R.len[2 * lane + 1] = l1;
    R.qx[2 * lane + 1] = qx1;
    R.qy[2 * lane + 1] = qy0;
    R.qz[2 * lane + 1] = qz0;
    R.flags[2 * lane + 1] = (unsigned char)f1;
    int inc = l0 + l1;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += v;
    }
    R.pre[lane + 1] = inc;
    if (lane == 0) R.pre[0] = 0;
    __syncwarp();
    const int total = __shfl_sync(0xffffffffu, inc, 31);
    for (int f = lane; f - lane < total; f += 32) {
      int j = -1;
      bool hit = false;
      if (f < total) {
        // the lane whose runs hold candidate f: the last L with pre[L] <= f
        int L = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1)
          if (R.pre[L + step] <= f) L += step;
        int off = f - R.pre[L];
        int slot = 2 * L;
        if (off >= R.len[slot]) {
          off -= R.len[slot];
          ++slot;
        }
        j = R.b[slot] + off;
        if (j != self) {
          const unsigned fl = R.flags[slot];
          if (fl & 1u) {
            hit = true;
          } else {
            const float4 p = g.spos[j];
            const float dx = p.x - R.qx[slot], dy = p.y - R.qy[slot], dz = p.z - R.qz[slot];
            const float d2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
            const float blo = (fl & 2u) ? B.lo_w : B.lo, bhi = (fl & 2u) ? B.hi_w : B.hi;
            hit = d2 <= blo || (!(d2 > bhi) && canon_d2(Q.q, p, g) <= B.r2);
          }
        }
      }
      fn(hit, j);
    }
    __syncwarp();   // the next batch rewrites R
  }
  if (out_any) {
    const int b = __ldg(g.cell_start + g.outside), e = __ldg(g.cell_start + g.outside + 1);
    for (int j0 = b; j0 < e; j0 += 32) {
      const int j = j0 + lane;
      const bool hit = j < e && j != self && canon_d2(Q.q, g.spos[j], g) <= B.r2;
      fn(hit, j < e ? j : -1);
    }
  }
}

struct WarpCountVisitor {
  const GridDev &g;
  const QueryGeom &Q;
  const Band &B;
  int self, lane;
  long long count;
  __device__ __forceinline__ void operator()(const Target &t, bool full, int b, int e) {
    for (int j0 = b; j0 < e; j0 += 32) {
      const int j = j0 + lane;
      bool h = j < e && j != self;
      if (h && !full) h = pair_hit(g, Q, t, B, g.spos[j]);
      count += __popc(__ballot_sync(0xffffffffu, h));
    }
  }
  __device__ __forceinline__ void operator()(const Target &t, bool full) {
    (*this)(t, full, __ldg(g.cell_start + t.key), __ldg(g.cell_start + t.key + 1));
  }
};

struct WarpWriteVisitor {
  const GridDev &g;
  const QueryGeom &Q;
  const Band &B;
  int self, lane;
  int *list;       // the warp's shared list (len <= kDenseCap) or the output list
  int len, k;
  __device__ __forceinline__ void add(bool h, int j) {
    const unsigned m = __ballot_sync(0xffffffffu, h);
    if (h) {
      const int p = k + __popc(m & ((1u << lane) - 1u));
      if (p < len) list[p] = __ldg(g.perm + j);
    }
    k += __popc(m);
  }
  __device__ __forceinline__ void operator()(const Target &t, bool full, int b, int e) {
    for (int j0 = b; j0 < e; j0 += 32) {
      const int j = j0 + lane;
      bool h = j < e && j != self;
      if (h && !full) h = pair_hit(g, Q, t, B, g.spos[j]);
      add(h, j);
    }
  }
  __device__ __forceinline__ void operator()(const Target &t, bool full) {
    (*this)(t, full, __ldg(g.cell_start + t.key), __ldg(g.cell_start + t.key + 1));
  }
};

// Up to six blocks per SM (40 registers): more resident warps to wait on
// the walk's dependent loads, and room beside the heavy cells' kernels.
template <bool WRITE>
__global__ void __launch_bounds__(kClassThreads, 6) k_radius_dense(GridDev g, WalkParams P, Band B,
                                                                   unsigned flags, int n_entries,
                                                                   const int *__restrict__ denseq,
                                                                   long long *counts, const long long *offsets,
                                                                   int *ids, long long cap, int *longq) {
  extern __shared__ __align__(16) unsigned long long cls_smem[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nwb = blockDim.x >> 5;
  const int nq = denseq[0];
  if (blockIdx.x * nwb >= nq) return;   // no work for this block
  const int nbeg = g.cls_q * g.cls_q * g.cls_q + 1;
  int *beg_smem = reinterpret_cast<int *>(cls_smem + n_entries);
  FlatRuns *runs = reinterpret_cast<FlatRuns *>(beg_smem + ((nbeg + 3) & ~3));
  int *buf = reinterpret_cast<int *>(runs + nwb) + w * kDenseCap;   // write pass only
  for (int i = threadIdx.x; i < n_entries; i += blockDim.x) cls_smem[i] = __ldg(g.cls + i);
  for (int i = threadIdx.x; i < nbeg; i += blockDim.x) beg_smem[i] = __ldg(g.cls_begin + i);
  __syncthreads();
  GridDev gs = g;
  gs.cls = cls_smem;
  gs.cls_begin = beg_smem;
  FlatRuns &R = runs[w];
  for (int item = blockIdx.x * nwb + w; item < nq; item += gridDim.x * nwb) {
    const int s = denseq[1 + item];
    const QueryGeom Q = make_geom(g.qpos[s], g);
    const int self = query_self(g, flags, s);
    const int orig = __ldg(g.qid + s);
    if (!WRITE) {
      long long count = 0;
      if (Q.outside) {
        WarpCountVisitor v{gs, Q, B, self, lane, 0};
        walk_cube(gs, Q, P.dg, v);
        count = v.count;
      } else {
        auto fn = [&](bool hit, int) { count += __popc(__ballot_sync(0xffffffffu, hit)); };
        warp_class_walk(gs, Q, B, self, lane, R, fn);
      }
      if (lane == 0) counts[orig] = count;
    } else {
      const long long base = offsets[orig];
      const int len = (int)(offsets[orig + 1] - base);
      if (len == 0) continue;
      if (base + len > cap) {
        if (lane == 0) atomicOr(g.status, ST_CAPACITY);
        continue;
      }
      const bool staged = len <= kDenseCap;
      WarpWriteVisitor v{gs, Q, B, self, lane, staged ? buf : ids + base, len, 0};
      if (Q.outside) {
        walk_cube(gs, Q, P.dg, v);
      } else {
        auto fn = [&](bool hit, int j) { v.add(hit, j); };
        warp_class_walk(gs, Q, B, self, lane, R, fn);
      }
      if (v.k != len && lane == 0) atomicOr(g.status, ST_INTERNAL);
      const bool sort_all = !(flags & SI_NO_SORT);
      if (staged) {
        __syncwarp();
        if (sort_all) warp_sort(buf, len, lane, 0x7fffffff);
        __syncwarp();
        for (int i = lane; i < len; i += 32) ids[base + i] = buf[i];
        __syncwarp();
      } else if (sort_all && lane == 0) {
        const int slot = atomicAdd(longq, 1);
        longq[1 + slot] = orig;
      }
    }
  }
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
    warp_sort(buf, len, lane, 0x7fffffff);
    __syncwarp();
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

// The class walk with its tables in shared memory: the walk of the
// warp-per-query kernels for dense cells.
static bool dense_path(int walk, const si_grid *gr) { return walk == kWalkClasses && gr->cls_smem_bytes > 0; }

// The per-thread query kernels.  list (nullable): [0] = count, then the
// slots to serve; else every slot of dv's query set, skipping by class byte.
// lstage (nullable): the short-list staging area, lstride slots per row.
template <bool WRITE>
static si_status launch_light(int walk, const si_grid *gr, const GridDev &dv, const WalkParams &P,
                              const Band &B, unsigned flags, unsigned skip, long long *counts,
                              const long long *off, int *ids, long long cap, int *longq,
                              unsigned blocks, const int *list, int *lstage, long long lstride,
                              cudaStream_t st) {
  if (walk == kWalkCube) {
    SI_KLAUNCH(WRITE ? "k_radius_write_cube" : "k_radius_count_cube", st,
               k_radius<WRITE, kWalkCube><<<blocks, kQueryThreads, 0, st>>>(dv, P, B, flags, 0, counts,
                                                                            off, ids, cap, longq, list));
  } else if (walk == kWalkClasses && gr->cls_smem_bytes > 0) {
    const int nbeg = gr->cls_q * gr->cls_q * gr->cls_q + 1;
    const size_t smem = gr->cls_host.size() * sizeof(unsigned long long) +
                        (size_t)((nbeg + 3) & ~3) * sizeof(int) +
                        ((WRITE || lstage) ? (size_t)kInlineSort * kClassThreads * sizeof(int) : 0);
    SI_CUDA_TRY(cudaFuncSetAttribute(k_radius_cls<WRITE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
    int per_sm = 0;
    SI_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_radius_cls<WRITE>,
                                                              kClassThreads, smem));
    const unsigned grid = (unsigned)std::max(1, std::min<int>(per_sm, 8) * 148);
    SI_KLAUNCH(WRITE ? "k_radius_write" : "k_radius_count", st,
               k_radius_cls<WRITE><<<grid, kClassThreads, smem, st>>>(
                   dv, P, B, flags, skip, (int)gr->cls_host.size(), counts, off, ids, cap, longq,
                   list, lstage, lstride));
  } else if (walk == kWalkPlanes) {
    SI_KLAUNCH(WRITE ? "k_radius_write_planes" : "k_radius_count_planes", st,
               k_radius<WRITE, kWalkPlanes><<<blocks, kQueryThreads, 0, st>>>(
                   dv, P, B, flags, skip, counts, off, ids, cap, longq, list));
  } else if (walk == kWalkClasses) {
    SI_KLAUNCH(WRITE ? "k_radius_write_cls_l2" : "k_radius_count_cls_l2", st,
               k_radius<WRITE, kWalkClasses><<<blocks, kQueryThreads, 0, st>>>(
                   dv, P, B, flags, skip, counts, off, ids, cap, longq, list));
  } else {
    SI_KLAUNCH(WRITE ? "k_radius_write_eq2" : "k_radius_count_eq2", st,
               k_radius<WRITE, kWalkPaper><<<blocks, kQueryThreads, 0, st>>>(
                   dv, P, B, flags, skip, counts, off, ids, cap, longq, list));
  }
  return SI_OK;
}

// The warp-per-query kernels over the slots listed in q ([0] = count).
template <bool WRITE>
static si_status launch_dense(const si_grid *gr, const GridDev &dv, const WalkParams &P, const Band &B,
                              unsigned flags, const int *q, long long *counts, const long long *off, int *ids,
                              long long cap, int *longq, cudaStream_t st) {
  const int nbeg = gr->cls_q * gr->cls_q * gr->cls_q + 1;
  const size_t smem = gr->cls_host.size() * sizeof(unsigned long long) +
                      (size_t)((nbeg + 3) & ~3) * sizeof(int) + (kClassThreads / 32) * sizeof(FlatRuns) +
                      (WRITE ? (size_t)kDenseCap * (kClassThreads / 32) * sizeof(int) : 0);
  SI_CUDA_TRY(cudaFuncSetAttribute(k_radius_dense<WRITE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)smem));
  int per_sm = 0;
  SI_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_radius_dense<WRITE>, kClassThreads,
                                                            smem));
  const unsigned grid = (unsigned)std::max(1, std::min<int>(per_sm, 8) * 148);
  SI_KLAUNCH(WRITE ? "k_radius_dense_write" : "k_radius_dense_count", st,
             k_radius_dense<WRITE><<<grid, kClassThreads, smem, st>>>(
                 dv, P, B, flags, (int)gr->cls_host.size(), q, counts, off, ids, cap, longq));
  return SI_OK;
}

// Sort every queued list (ids ascending): a warp per list up to
// kSortWarpCap ids, a block per longer one.
static si_status launch_sorts(const long long *off, int *ids, int *longq, int *hugeq, cudaStream_t st) {
  const size_t wsm = (size_t)kSortWarps * kSortWarpCap * sizeof(int);
  SI_CUDA_TRY(cudaFuncSetAttribute(k_sort_warp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)wsm));
  SI_KLAUNCH("k_sort_warp", st, k_sort_warp<<<148 * 2, kSortWarps * 32, wsm, st>>>(off, ids, longq, hugeq));
  const size_t bsm = (size_t)kSortBlockCap * sizeof(int);
  SI_CUDA_TRY(cudaFuncSetAttribute(k_sort_block, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bsm));
  SI_KLAUNCH("k_sort_block", st, k_sort_block<<<148, 512, bsm, st>>>(off, ids, hugeq));
  return SI_OK;
}

// The non-empty list method (si_list.cu) for all agents or for centers:
// every (query, point) pair tested, points in input order, so the lists come
// out ascending without a sort.
static si_status query_radius_list(si_grid *g, const float *d_centers, int64_t m, float r, uint32_t flags,
                                   int64_t *d_offsets, int32_t *d_ids, int64_t ids_capacity, int64_t *h_total,
                                   cudaStream_t st) {
  if (!g->ipos) {
    if (cudaMalloc((void **)&g->ipos, (size_t)std::max<int64_t>(g->cap, 1) * sizeof(float4)) != cudaSuccess) {
      g->ipos = nullptr;
      cudaGetLastError();
      return fail(SI_ERR_OOM, "input-order point buffer");
    }
  }
  const Band B = make_band(g->lat, r);
  long long *off = (long long *)d_offsets;
  GridDev dv = g->dev();
  const int *list = nullptr;
  long long *scan = g->scan_i64;
  si_status s;
  if (d_centers) {
    CenterOut eo;
    eo.rad_counts = off + 1;
    if ((s = prepare_centers(g, d_centers, m, false, false, eo, dv, st)) != SI_OK) return s;
    list = g->clist0;
    scan = g->cscan64;
  }
  if ((s = gather_input(g, dv, g->ipos, st)) != SI_OK) return s;
  SI_CUDA_TRY(cudaMemsetAsync(off, 0, sizeof(long long), st));
  if (m > 0) {
    if ((s = launch_list(dv, B, flags, list, m, g->ipos, off + 1, nullptr, nullptr, 0, false, st)) != SI_OK) return s;
    if ((s = scan_inclusive_i64(off + 1, off + 1, m, scan, st)) != SI_OK) return s;
  }
  if (h_total) {
    SI_CUDA_TRY(cudaMemcpyAsync(g->h_pinned, off + m, sizeof(long long), cudaMemcpyDeviceToHost, st));
    SI_CUDA_TRY(cudaStreamSynchronize(st));
    *h_total = g->h_pinned[0];
    if (*h_total > ids_capacity) return fail(SI_ERR_CAPACITY, "neighbor id buffer too small");
  }
  if (m == 0) return SI_OK;
  return launch_list(dv, B, flags, list, m, g->ipos, nullptr, off, d_ids, ids_capacity, true, st);
}

// Volume comparison (Sec. III.B, Sec. IV.A): the paper walks the sphere
// unless its list of non-empty cells is shorter.  Here the two methods'
// estimated costs per query are compared, in nanoseconds on B300 (a fit to
// both methods measured on 20k to 1.3M uniform points, 16^3 to 128^3
// lattices, d = 0.7 to 24 cells, 100k centers):
//   sphere: 0.019 per x-row run of the class walk (0.015 per cell of the
//           table walk) + 0.0041 per candidate + 0.069 per hit + 0.85
//   list:   0.0019 per point + 0.0028 per hit + 1.2
// with candidates = load x the Steiner volume 1 + 6d + 3 pi d^2 + 4/3 pi d^3
// (cells meeting the sphere around a random center) and hits = load x
// 4/3 pi d^3.  The list is taken when its estimate times the grid's weight
// (the Appendix's weighting factor, 1.2 by default) is below the sphere's.
static bool list_cheaper(const si_grid *g, float r, int walk) {
  if (g->n <= 0 || g->n_cells <= 1) return false;
  const double d = (double)r * (double)g->lat.inv_s;
  const double load = (double)g->n / (double)(g->n_cells - 1);
  const double steiner = 1.0 + 6.0 * d + 3.0 * M_PI * d * d + 4.0 / 3.0 * M_PI * d * d * d;
  const double hits = load * 4.0 / 3.0 * M_PI * d * d * d;
  double sphere = 0.0041 * load * steiner + 0.069 * hits + 0.85;
  if (walk == kWalkClasses && g->cls_q > 0) {
    const double q3 = (double)g->cls_q * g->cls_q * g->cls_q;
    sphere += 0.019 * (double)g->cls_host.size() / q3;
  } else {
    sphere += 0.015 * steiner;
  }
  const double list = 0.0019 * (double)g->n + 0.0028 * hits + 1.2;
  return g->list_weight * list < sphere;
}

// Radius query from caller-given centers (sorted by coarse cell first; see
// si_centers.cu): the per-thread kernel for centers in light cells, the
// warp-per-query kernel for the rest; no self exclusion.
static si_status query_radius_centers(si_grid *g, const float *d_centers, int64_t m, float r, uint32_t flags,
                                      int64_t *d_offsets, int32_t *d_ids, int64_t ids_capacity, int64_t *h_total,
                                      cudaStream_t st) {
  const bool cube = flags & SI_METHOD_CUBE;
  const double load = g->n_cells > 1 ? (double)g->n / (double)(g->n_cells - 1) : 0.0;
  const WalkParams P = walk_params(g->lat, r, load >= 4.0);
  const Band B = make_band(g->lat, r);
  const int walk = cube ? kWalkCube
                        : ((flags & SI_WALK_PLANES) ? kWalkPlanes
                           : ((!(flags & SI_WALK_PAPER) && g->ensure_classes(P.dg, st)) ? kWalkClasses
                                                                                       : kWalkPaper));
  const bool split = dense_path(walk, g);
  long long *off = (long long *)d_offsets;
  CenterOut eo;
  eo.rad_counts = off + 1;
  GridDev dv;
  si_status s = prepare_centers(g, d_centers, m, split, split, eo, dv, st);
  if (s != SI_OK) return s;
  int *lstage = split ? g->cstage : nullptr;
  const long long lstride = g->cstage_cap;
  const unsigned blocks = (unsigned)((std::max<int64_t>(m, 1) + kQueryThreads - 1) / kQueryThreads);
  SI_CUDA_TRY(cudaMemsetAsync(off, 0, sizeof(long long), st));
  // the warp-per-center kernel on the side stream, beside the thread-per-center one
  const bool fork = split && g->fork && g->ensure_side();
  cudaStream_t sq = fork ? g->side : st;
  auto fork_side = [&]() -> si_status {
    if (fork) {
      SI_CUDA_TRY(cudaEventRecord(g->fork_ev, st));
      SI_CUDA_TRY(cudaStreamWaitEvent(sq, g->fork_ev, 0));
    }
    return SI_OK;
  };
  auto join_side = [&]() -> si_status {
    if (fork) {
      SI_CUDA_TRY(cudaEventRecord(g->join_ev, sq));
      SI_CUDA_TRY(cudaStreamWaitEvent(st, g->join_ev, 0));
    }
    return SI_OK;
  };
  if (m > 0) {
    if ((s = fork_side()) != SI_OK) return s;
    if ((s = launch_light<false>(walk, g, dv, P, B, flags, 0u, off + 1, nullptr, nullptr, 0, nullptr, blocks,
                                 g->clist0, lstage, lstride, st)) != SI_OK)
      return s;
    if (split && (s = launch_dense<false>(g, dv, P, B, flags, g->clist1, off + 1, nullptr, nullptr, 0, nullptr,
                                          sq)) != SI_OK)
      return s;
    if ((s = join_side()) != SI_OK) return s;
    if ((s = scan_inclusive_i64(off + 1, off + 1, m, g->cscan64, st)) != SI_OK) return s;
  }
  if (h_total) {
    SI_CUDA_TRY(cudaMemcpyAsync(g->h_pinned, off + m, sizeof(long long), cudaMemcpyDeviceToHost, st));
    SI_CUDA_TRY(cudaStreamSynchronize(st));
    *h_total = g->h_pinned[0];
    if (*h_total > ids_capacity) return fail(SI_ERR_CAPACITY, "neighbor id buffer too small");
  }
  if (m == 0) return SI_OK;
  SI_CUDA_TRY(cudaMemsetAsync(g->clong, 0, sizeof(int), st));
  SI_CUDA_TRY(cudaMemsetAsync(g->chuge, 0, sizeof(int), st));
  if ((s = fork_side()) != SI_OK) return s;
  if ((s = launch_light<true>(walk, g, dv, P, B, flags, 0u, nullptr, off, d_ids, ids_capacity, g->clong, blocks,
                              g->clist0, lstage, lstride, st)) != SI_OK)
    return s;
  if (split && (s = launch_dense<true>(g, dv, P, B, flags, g->clist1, nullptr, off, d_ids, ids_capacity, g->clong,
                                       sq)) != SI_OK)
    return s;
  if ((s = join_side()) != SI_OK) return s;
  if (!(flags & SI_NO_SORT)) return launch_sorts(off, d_ids, g->clong, g->chuge, st);
  return SI_OK;
}

extern "C" si_status si_query_radius(si_grid *g, const float *d_centers, int64_t m, float r,
                                     uint32_t flags, int64_t *d_offsets, int32_t *d_ids,
                                     int64_t ids_capacity, int64_t *h_total, void *stream) {
  if (!g) return fail(SI_ERR_INVALID, "null grid");
  if (d_centers) {
    if (m < 0 || m > (int64_t)INT32_MAX - 1) return fail(SI_ERR_INVALID, "m out of range");
    if ((uintptr_t)d_centers & 15u) return fail(SI_ERR_INVALID, "centers must be a 16-byte aligned float4 array");
  } else if (m != g->n) {
    return fail(SI_ERR_INVALID, "all-agents mode: m must equal the grid's point count");
  }
  if (!(r >= 0.f) || !std::isfinite(r)) return fail(SI_ERR_INVALID, "radius must be finite and >= 0");
  if (!g->lat.unbounded && (double)r > (double)g->desc.r_max)
    return fail(SI_ERR_INVALID, "radius exceeds the grid's r_max");
  if (!d_offsets) return fail(SI_ERR_INVALID, "null offsets");
  if (ids_capacity < 0 || (ids_capacity > 0 && !d_ids)) return fail(SI_ERR_INVALID, "bad ids buffer");
  if (flags & ~(SI_METHOD_CUBE | SI_INCLUDE_SELF | SI_NO_SORT | SI_WALK_PAPER | SI_METHOD_LIST | SI_SPHERE_ONLY |
                SI_WALK_PLANES | SI_NO_GROUPS))
    return fail(SI_ERR_INVALID, "unknown flags");
  if ((flags & SI_METHOD_CUBE) && (flags & SI_METHOD_LIST))
    return fail(SI_ERR_INVALID, "SI_METHOD_CUBE and SI_METHOD_LIST are exclusive");
  cudaStream_t st = (cudaStream_t)stream;
  if (flags & SI_METHOD_LIST)
    return query_radius_list(g, d_centers, m, r, flags, d_offsets, d_ids, ids_capacity, h_total, st);
  // the optional reversal to the bin lattice below a radius (Appendix; off
  // unless si_grid_set_method sets it)
  if (!(flags & (SI_WALK_PAPER | SI_SPHERE_ONLY | SI_WALK_PLANES)) && (double)r * (double)g->lat.inv_s < g->cube_below)
    flags |= SI_METHOD_CUBE;
  if (!(flags & (SI_METHOD_CUBE | SI_WALK_PAPER | SI_SPHERE_ONLY | SI_WALK_PLANES))) {
    // the walk the sphere method would take (class tables when they can be
    // built for this radius), then the volume comparison
    const WalkParams P0 = walk_params(g->lat, r, false);
    const int walk0 = g->ensure_classes(P0.dg, st) ? kWalkClasses : kWalkPaper;
    if (list_cheaper(g, r, walk0))
      return query_radius_list(g, d_centers, m, r, flags, d_offsets, d_ids, ids_capacity, h_total, st);
  }
  if (d_centers) return query_radius_centers(g, d_centers, m, r, flags, d_offsets, d_ids, ids_capacity, h_total, st);
  const bool cube = flags & SI_METHOD_CUBE;
  const double load = g->n_cells > 1 ? (double)g->n / (double)(g->n_cells - 1) : 0.0;
  const WalkParams P = walk_params(g->lat, r, load >= 4.0);
  const Band B = make_band(g->lat, r);
  const bool planes = !cube && (flags & SI_WALK_PLANES);
  const int walk = cube ? kWalkCube
                        : (planes ? kWalkPlanes
                                  : ((!(flags & SI_WALK_PAPER) && g->ensure_classes(P.dg, st)) ? kWalkClasses
                                                                                              : kWalkPaper));
  // the cell path holds the runs of the whole cell-level sphere (rows of
  // cells with b^2 <= floor(d^2), at most two runs per row and the outside cell);
  // the stacked-plane walk serves every query itself
  const bool heavy = !cube && !planes && g->ensure_cell_rows(P.dg, st) && 2 * g->n_crow + 1 <= kCellTCap;
  // groups of heavy cells when the lattice holds a group's rows without
  // wrapping onto itself (SI_NO_GROUPS serves every heavy cell on its own)
  const bool group = heavy && !(flags & SI_NO_GROUPS) && g->ensure_group_rows(P.dg, st);
  // the count pass keeps short lists for the write pass in a staging area
  // (allocated on first use; without it the write pass walks every list again)
  if (walk == kWalkClasses && g->cls_smem_bytes > 0 && !g->lstage && g->cap > 0) {
    if (cudaMalloc((void **)&g->lstage, (size_t)kInlineSort * (size_t)g->cap * sizeof(int)) != cudaSuccess) {
      g->lstage = nullptr;
      cudaGetLastError();
    }
  }
  const GridDev dv = g->dev();
  const unsigned skip = (heavy ? 1u : 0u) | (dense_path(walk, g) ? 2u : 0u);
  // with both other paths on, the light cells' slots are listed at binning
  const int *light_list = (walk == kWalkClasses && g->cls_smem_bytes > 0 && skip == 3u) ? g->lightq : nullptr;
  long long *off = (long long *)d_offsets;
  const unsigned blocks = (unsigned)((m + kQueryThreads - 1) / kQueryThreads);
  si_status s;
  // count phase: per-query counts of light cells, the cell kernel's counts
  // and scratch records (ordered candidate ids, hit masks) for heavy cells,
  // per-query counts of what it handed back
  auto count_phase = [&]() -> si_status {
    SI_CUDA_TRY(cudaMemsetAsync(off, 0, sizeof(long long), st));
    SI_CUDA_TRY(cudaMemsetAsync(g->counters, 0, kCounterInts * sizeof(int), st));
    SI_CUDA_TRY(cudaMemsetAsync(g->over, 0, sizeof(int), st));
    SI_CUDA_TRY(cudaMemcpyAsync(g->heavy_big, g->heavy_big_built, sizeof(int), cudaMemcpyDeviceToDevice, st));
    SI_CUDA_TRY(cudaMemsetAsync(g->scr_top, 0, sizeof(unsigned long long), st));
    if (m == 0) return SI_OK;
    si_status r;
    // the per-query kernels (light and dense cells) on the side stream when
    // the crowded cells' kernels run beside them on this one
    const bool fork = heavy && g->fork && g->ensure_side();
    cudaStream_t sq = fork ? g->side : st;
    if (fork) {
      SI_CUDA_TRY(cudaEventRecord(g->fork_ev, st));
      SI_CUDA_TRY(cudaStreamWaitEvent(sq, g->fork_ev, 0));
    }
    if ((r = launch_light<false>(walk, g, dv, P, B, flags, skip, off + 1, nullptr, nullptr, 0,
                                 nullptr, blocks, light_list, g->lstage, (long long)g->cap, sq)) != SI_OK)
      return r;
    if (dense_path(walk, g) &&
        (r = launch_dense<false>(g, dv, P, B, flags, g->denseq, off + 1, nullptr, nullptr, 0, nullptr, sq)) !=
            SI_OK)
      return r;
    if (heavy) {
      // groups of neighbouring heavy cells first (they share one gather and
      // sort), then the heavy cells served one at a time
      const int *solo = g->heavy;
      if (group) {
        SI_CUDA_TRY(cudaMemsetAsync(g->groups, 0, sizeof(int), st));
        SI_CUDA_TRY(cudaMemsetAsync(g->hsolo, 0, sizeof(int), st));
        if ((r = launch_cell_group(dv, P, B, flags, g->heavy, g->groups, g->hsolo, g->counters + 2, g->heavy_big,
                                   g->over, off + 1, g->cell_rec, g->scratch, g->scr_cap, g->scr_top, g->grow,
                                   g->n_grow, st)) != SI_OK)
          return r;
        solo = g->hsolo;
      }
      if ((r = launch_cell_pass(dv, P, B, flags, solo, g->heavy_big, g->counters, g->over, off + 1, g->cell_rec,
                                g->scratch, g->scr_cap, g->scr_top, st)) != SI_OK)
        return r;
      SI_KLAUNCH("k_radius_over_count", st,
                 k_radius_over<false><<<148 * 4, kQueryThreads, 0, st>>>(dv, P, B, flags, g->over,
                                                                         off + 1, nullptr, nullptr, 0,
                                                                         nullptr));
    }
    if (fork) {
      SI_CUDA_TRY(cudaEventRecord(g->join_ev, sq));
      SI_CUDA_TRY(cudaStreamWaitEvent(st, g->join_ev, 0));
    }
    return scan_inclusive_i64(off + 1, off + 1, m, g->scan_i64, st);
  };
  if ((s = count_phase()) != SI_OK) return s;
  if (h_total) {
    SI_CUDA_TRY(cudaMemcpyAsync(g->h_pinned, off + m, sizeof(long long), cudaMemcpyDeviceToHost, st));
    SI_CUDA_TRY(cudaMemcpyAsync(g->h_pinned + 1, g->scr_top, sizeof(long long), cudaMemcpyDeviceToHost, st));
    SI_CUDA_TRY(cudaStreamSynchronize(st));
    // cells whose records did not fit the scratch took the per-query path;
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
  // write pass: the per-query kernels on the side stream again, beside the
  // expansion of the crowded cells' masks (every kernel writes its own
  // queries' lists; the long-list queue is filled with atomics)
  const bool fork = heavy && g->fork && g->ensure_side();
  cudaStream_t sq = fork ? g->side : st;
  if (fork) {
    SI_CUDA_TRY(cudaEventRecord(g->fork_ev, st));
    SI_CUDA_TRY(cudaStreamWaitEvent(sq, g->fork_ev, 0));
  }
  if ((s = launch_light<true>(walk, g, dv, P, B, flags, skip, nullptr, off, d_ids, ids_capacity,
                              g->longq, blocks, light_list, g->lstage, (long long)g->cap, sq)) != SI_OK)
    return s;
  if (dense_path(walk, g) &&
      (s = launch_dense<true>(g, dv, P, B, flags, g->denseq, nullptr, off, d_ids, ids_capacity, g->longq, sq)) !=
          SI_OK)
    return s;
  if (heavy) {
    if ((s = launch_cell_expand(dv, g->heavy, g->cell_rec, g->scratch, g->xitems, g->xblock, off, d_ids, ids_capacity,
                                st)) != SI_OK)
      return s;
    SI_KLAUNCH("k_radius_over_write", st,
               k_radius_over<true><<<148 * 4, kQueryThreads, 0, st>>>(dv, P, B, flags, g->over, nullptr,
                                                                      off, d_ids, ids_capacity,
                                                                      g->longq));
  }
  if (fork) {
    SI_CUDA_TRY(cudaEventRecord(g->join_ev, sq));
    SI_CUDA_TRY(cudaStreamWaitEvent(st, g->join_ev, 0));
  }
  if (!(flags & SI_NO_SORT)) return launch_sorts(off, d_ids, g->longq, g->hugeq, st);
  return SI_OK;
}

// All-agents radius query from host memory to host memory (the end-to-end
// form of the path): H2D copy, binning, query, D2H copy, all on `stream`.
extern "C" si_status si_query_radius_host(si_grid *g, const float *h_pos, int64_t n, float r, uint32_t flags,
                                          int64_t *h_offsets, int32_t *h_ids, int64_t ids_capacity,
                                          int64_t *h_total, void *stream) {
  if (!g) return fail(SI_ERR_INVALID, "null grid");
  if (!h_pos || !h_offsets || !h_total) return fail(SI_ERR_INVALID, "null host buffer");
  if (ids_capacity < 0 || (ids_capacity > 0 && !h_ids)) return fail(SI_ERR_INVALID, "bad ids buffer");
  if (n < 0 || n > g->cap) return fail(SI_ERR_INVALID, "n out of range (0 .. capacity)");
  cudaStream_t st = (cudaStream_t)stream;
  auto grow = [](auto *&p, int64_t &cap, int64_t want, size_t elem) -> si_status {
    if (want <= cap) return SI_OK;
    cudaFree(p);
    p = nullptr;
    cap = 0;
    const cudaError_t e = cudaMalloc((void **)&p, (size_t)std::max<int64_t>(want, 1) * elem);
    if (e != cudaSuccess) {
      p = nullptr;
      return cuda_fail(e, "si_query_radius_host buffers");
    }
    cap = want;
    return SI_OK;
  };
  si_status s;
  if ((s = grow(g->io_pos, g->io_pos_cap, n, sizeof(float4))) != SI_OK) return s;
  if ((s = grow(g->io_off, g->io_off_cap, n + 1, sizeof(long long))) != SI_OK) return s;
  if ((s = grow(g->io_ids, g->io_ids_cap, ids_capacity, sizeof(int))) != SI_OK) return s;
  if (n > 0) SI_CUDA_TRY(cudaMemcpyAsync(g->io_pos, h_pos, (size_t)n * sizeof(float4), cudaMemcpyHostToDevice, st));
  if ((s = si_grid_build(g, reinterpret_cast<const float *>(g->io_pos), n, stream)) != SI_OK) return s;
  // the call waits after counting, stores the total and refuses an ids
  // buffer that is too small
  if ((s = si_query_radius(g, nullptr, n, r, flags, reinterpret_cast<int64_t *>(g->io_off), g->io_ids, ids_capacity,
                           h_total, stream)) != SI_OK)
    return s;
  SI_CUDA_TRY(cudaMemcpyAsync(h_offsets, g->io_off, (size_t)(n + 1) * sizeof(long long), cudaMemcpyDeviceToHost, st));
  if (*h_total > 0)
    SI_CUDA_TRY(cudaMemcpyAsync(h_ids, g->io_ids, (size_t)*h_total * sizeof(int), cudaMemcpyDeviceToHost, st));
  return si_grid_sync(g, stream);
}
