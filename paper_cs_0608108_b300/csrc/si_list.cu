// Non-empty cell list method (Sec. III.B, Sec. IV.A): when the query sphere
// holds more cells than the region has objects (large distance, low load),
// walking the sphere costs more than testing every object, and the paper
// switches to its list of non-empty cells.  On the GPU that list is the
// whole sorted point array, so the method becomes a tiled test of every
// (query, point) pair: a block stages 2048 points at a time in shared memory
// and each warp tests them, 32 at a time, against its kAllQ queries.  The
// points are taken in input order, so every list comes out ascending by id
// and needs no sort.
//
// Distances: per axis a = fl(|xj - xi|) in FP32, on a cyclic axis
// fl(h - fl(|fl(a - h)|)) with h = L / 2, i.e. min(a, L - a).  Its absolute
// error is at most u a + u h + u h' (each rounding at most u times its
// result, a <= L, both h terms <= L / 2): within u (Qmax + L) + u |dx|, the
// per-axis bound of pairs compared through a wrapped image, so the FP32 test
// with that band plus the FP64 canonical recheck inside it gives the exact
// set.
#include <algorithm>
#include <cmath>

#include "si_host.h"
#include "si_radius.cuh"

namespace si {

constexpr int kAllWarps = 8;
constexpr int kAllQ = 8;          // queries per warp
constexpr int kAllTile = 2048;    // points staged per round (32 KB)

// Points in input order: ipos[perm[s]] = spos[s].
__global__ void __launch_bounds__(256) k_gather_input(GridDev g, float4 *__restrict__ ipos) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < g.n) ipos[__ldg(g.perm + s)] = g.spos[s];
}

// The canonical FP64 test of one pair, for the rare pairs inside the guard
// band: kept out of line so that it runs only when called.
__device__ __noinline__ bool canon_within(float qx, float qy, float qz, float px, float py, float pz, float Lx,
                                          float Ly, float Lz, unsigned cyc, double r2) {
  const double ax = canon_gap(qx, px, Lx, cyc & 1u);
  const double ay = canon_gap(qy, py, Ly, (cyc >> 1) & 1u);
  const double az = canon_gap(qz, pz, Lz, (cyc >> 2) & 1u);
  double s = __dmul_rn(ax, ax);
  s = __dadd_rn(s, __dmul_rn(ay, ay));
  s = __dadd_rn(s, __dmul_rn(az, az));
  return s <= r2;
}

// FP32 gap on one axis: |x - q|, and on a cyclic axis the shorter way round,
// min(a, L - a) = h - |a - h| with h = L / 2 (three additions, no select).
template <bool CYCLIC>
__device__ __forceinline__ float gap32(float x, float q, float h) {
  const float a = fabsf(x - q);
  return CYCLIC ? h - fabsf(a - h) : a;
}

// list (nullable): [0] = count, then the query slots; else every slot.
// CYC: the grid's cyclic mask.  A query outside the list, and a point past
// the end of the array, are NaN, which no test accepts.
template <bool WRITE, unsigned CYC>
__global__ void __launch_bounds__(kAllWarps * 32) k_radius_all(GridDev g, Band B, unsigned flags,
                                                              const int *__restrict__ list,
                                                              const float4 *__restrict__ ipos,
                                                              long long *counts, const long long *offsets,
                                                              int *ids, long long cap) {
  __shared__ float4 tile[kAllTile];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int nq = list ? list[0] : g.n;
  if (blockIdx.x * kAllWarps * kAllQ >= nq) return;   // the whole block is idle
  const unsigned lt = (1u << lane) - 1u;
  const float hx = 0.5f * g.Lx, hy = 0.5f * g.Ly, hz = 0.5f * g.Lz;
  const float nan = __int_as_float(0x7fc00000);
  // all agents: query s is input point orig and, unless SI_INCLUDE_SELF,
  // leaves itself out (it is always found, at distance 0)
  const bool drop_self = g.q_agents && !(flags & SI_INCLUDE_SELF);
  float qx[kAllQ], qy[kAllQ], qz[kAllQ];
  int orig[kAllQ], k[kAllQ], len[kAllQ];
  long long base[kAllQ];
#pragma unroll
  for (int i = 0; i < kAllQ; ++i) {
    const int item = (blockIdx.x * kAllWarps + w) * kAllQ + i;
    bool act = item < nq;
    const int s = act ? (list ? list[1 + item] : item) : 0;
    const float4 q = g.qpos[s];
    orig[i] = act ? __ldg(g.qid + s) : -1;
    base[i] = 0;
    len[i] = 0;
    if (WRITE && act) {
      base[i] = offsets[orig[i]];
      len[i] = (int)(offsets[orig[i] + 1] - base[i]);
      if (base[i] + len[i] > cap) {
        if (lane == 0) atomicOr(g.status, ST_CAPACITY);
        act = false;
      }
    }
    qx[i] = act ? q.x : nan;
    qy[i] = act ? q.y : nan;
    qz[i] = act ? q.z : nan;
    k[i] = 0;
  }
  const int n = g.n;
  for (int j0 = 0; j0 < n; j0 += kAllTile) {
    const int te = min(kAllTile, n - j0);
    __syncthreads();   // the previous tile is no longer read
    for (int i = tid; i < kAllTile; i += blockDim.x)
      tile[i] = i < te ? ipos[j0 + i] : make_float4(nan, nan, nan, 0.f);
    __syncthreads();
    const int nb = (te + 31) & ~31;
    for (int i0 = 0; i0 < nb; i0 += 32) {
      const float4 p = tile[i0 + lane];
      const int j = j0 + i0 + lane;
#pragma unroll
      for (int a = 0; a < kAllQ; ++a) {
        const float ax = gap32<(CYC & 1u) != 0>(p.x, qx[a], hx);
        const float ay = gap32<(CYC & 2u) != 0>(p.y, qy[a], hy);
        const float az = gap32<(CYC & 4u) != 0>(p.z, qz[a], hz);
        const float d2 = fmaf(az, az, fmaf(ay, ay, ax * ax));
        bool hit = d2 <= B.lo_w;
        if (!hit && d2 <= B.hi_w)
          hit = canon_within(qx[a], qy[a], qz[a], p.x, p.y, p.z, g.Lx, g.Ly, g.Lz, CYC, B.r2);
        if (WRITE) {
          hit = hit && !(drop_self && j == orig[a]);
          const unsigned m = __ballot_sync(0xffffffffu, hit);
          if (hit) {
            const int at = k[a] + __popc(m & lt);
            if (at < len[a]) ids[base[a] + at] = j;
          }
          k[a] += __popc(m);
        } else {
          k[a] += hit ? 1 : 0;
        }
      }
    }
  }
#pragma unroll
  for (int a = 0; a < kAllQ; ++a) {
    if (!WRITE) {
      int c = k[a];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
      k[a] = c - (drop_self ? 1 : 0);
    }
    if (lane == 0 && orig[a] >= 0) {
      if (!WRITE) counts[orig[a]] = k[a];
      else if (k[a] != len[a] && base[a] + len[a] <= cap) atomicOr(g.status, ST_INTERNAL);
    }
  }
}

template <bool WRITE>
static si_status launch_all(const GridDev &dv, const Band &B, unsigned flags, const int *list, unsigned blocks,
                            const float4 *ipos, long long *counts, const long long *off, int *ids, long long cap,
                            cudaStream_t st) {
  using K = void (*)(GridDev, Band, unsigned, const int *, const float4 *, long long *, const long long *, int *,
                     long long);
  static const K table[8] = {k_radius_all<WRITE, 0>, k_radius_all<WRITE, 1>, k_radius_all<WRITE, 2>,
                             k_radius_all<WRITE, 3>, k_radius_all<WRITE, 4>, k_radius_all<WRITE, 5>,
                             k_radius_all<WRITE, 6>, k_radius_all<WRITE, 7>};
  SI_KLAUNCH(WRITE ? "k_radius_all_write" : "k_radius_all_count", st,
             table[dv.cyc & 7u]<<<blocks, kAllWarps * 32, 0, st>>>(dv, B, flags, list, ipos, counts, off, ids, cap));
  return SI_OK;
}

si_status launch_list(const GridDev &dv, const Band &B, unsigned flags, const int *list, int64_t m,
                      const float4 *ipos, long long *counts, const long long *off, int *ids, long long cap,
                      bool write, cudaStream_t st) {
  const unsigned blocks = (unsigned)std::max<int64_t>(1, (m + kAllWarps * kAllQ - 1) / (kAllWarps * kAllQ));
  return write ? launch_all<true>(dv, B, flags, list, blocks, ipos, counts, off, ids, cap, st)
               : launch_all<false>(dv, B, flags, list, blocks, ipos, counts, off, ids, cap, st);
}

si_status gather_input(const si_grid *g, const GridDev &dv, float4 *ipos, cudaStream_t st) {
  if (g->n == 0) return SI_OK;
  SI_KLAUNCH("k_gather_input", st,
             k_gather_input<<<(unsigned)((g->n + 255) / 256), 256, 0, st>>>(dv, ipos));
  return SI_OK;
}

}  // namespace si
