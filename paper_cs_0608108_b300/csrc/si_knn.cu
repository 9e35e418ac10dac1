// All-agents K-nearest query (Sec. II.A, last paragraph; Sec. IV.B): walk the
// sorted offset table from the center outwards and, once K neighbors are
// held, shrink the search radius to the K-th distance; the walk stops at the
// first table entry whose minimum bound b exceeds it (early cut-off).
//
// Order is (canonical FP64 D2, index).  Candidates are compared in FP32; two
// FP32 values closer than the proven FP32 error bound are compared again in
// FP64, so the kept set and its order are exact while almost every
// comparison stays in FP32.
//
// Three kernels.  With a bounded r_max and K <= kLaneKMax, k_knn_lane serves
// a query with one thread: the lanes of a warp hold neighbouring queries and
// walk the same x-rows of the sphere (rows of cells whose y-z bound is within
// the cut, each cut to the x-interval the query's exact y-z distance allows)
// in step, keeping the K + 1 smallest FP32 distances and shrinking the cut
// as described above.  For larger K, and for the queries whose K-th
// neighbour the lane kernel's list cannot settle, k_knn_warp serves a query
// with one warp: the lanes decode 32 x-rows at a time, every candidate
// within the cut (the exact predicate) goes to the warp's shared buffer as an
// FP32 key, and a warp bitonic sort orders the buffer.  Both take a first
// cut expected to hold a little more than K points and widen it to r_max
// when it holds fewer; runs of adjacent values closer than the FP32 error
// bound are put in canonical order.  k_knn, one thread per query with the
// shrinking cut from r_max, serves unbounded r_max, query points outside the
// region and queries whose candidates overflow the warp's buffer.
#include <cmath>

#include "si_host.h"
#include "si_sort.cuh"
#include "si_walk.cuh"

namespace si {

constexpr int kKnnThreads = 128;

struct KnnList {
  // column layout [k * T + t]: thread t's k-th entry; conflict-free
  float *d;      // FP32 squared distance
  int *j;        // sorted slot of the candidate
  int T, t;
  __device__ __forceinline__ int at(int k) const { return k * T + t; }
};

struct Cand {
  float d;
  int j;
  double D;      // canonical D2, NaN until needed
};

__device__ __forceinline__ double cand_D(Cand &c, const GridDev &g, const QueryGeom &Q) {
  if (isnan(c.D)) c.D = canon_d2(Q.q, g.spos[c.j], g);
  return c.D;
}

// a < b in the exact (D2, index) order, deciding in FP32 when the values are
// further apart than their combined error bound; near-ties are decided by the
// canonical FP64 values (recomputed: they are rare) and then by index.
__device__ __forceinline__ bool cand_less(Cand &a, const KnnList &L, int kb, const GridDev &g,
                                          const QueryGeom &Q, const PairBand &pb) {
  const float bd = L.d[L.at(kb)];
  const float m = fmaxf(a.d, bd) * 1.000001f;
  const float band = fmaf(pb.c2, m, pb.c1 * sqrtf(m)) + 1e-37f;
  if (a.d + band < bd) return true;
  if (bd + band < a.d) return false;
  const int jb = L.j[L.at(kb)];
  const double Da = cand_D(a, g, Q);
  const double Db = canon_d2(Q.q, g.spos[jb], g);
  if (Da != Db) return Da < Db;
  return __ldg(g.perm + a.j) < __ldg(g.perm + jb);
}

// list (nullable): [0] = count, then the sorted slots to serve; else every slot.
__global__ void __launch_bounds__(kKnnThreads) k_knn(GridDev g, int K, float dmax_g, int n_query,
                                                     Band B, PairBand pb, unsigned flags,
                                                     int *__restrict__ out_ids,
                                                     float *__restrict__ out_d2,
                                                     int *__restrict__ out_counts,
                                                     const int *__restrict__ list) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int T = blockDim.x;
  KnnList L;
  L.d = (float *)smem;
  L.j = (int *)(L.d + (size_t)K * T);
  L.T = T;
  L.t = threadIdx.x;
  const int ti = blockIdx.x * T + threadIdx.x;
  if (ti >= (list ? list[0] : g.n)) return;
  const int s = list ? list[1 + ti] : ti;
  const QueryGeom Q = make_geom(g.qpos[s], g);
  const int self = query_self(g, flags, s);
  int cnt = 0;
  float cut2 = dmax_g * dmax_g;          // cell units: walk cut on b2 and t2
  float kth_hi = fmaxf(B.hi, B.hi_w);    // world units: candidate filter
  const float hi_max = kth_hi;

  auto insert = [&](Cand c) {
    int p;
    if (cnt == K) {
      if (!cand_less(c, L, K - 1, g, Q, pb)) return;
      p = K - 1;
    } else {
      p = cnt++;
    }
    while (p > 0 && cand_less(c, L, p - 1, g, Q, pb)) {
      L.d[L.at(p)] = L.d[L.at(p - 1)];
      L.j[L.at(p)] = L.j[L.at(p - 1)];
      --p;
    }
    L.d[L.at(p)] = c.d;
    L.j[L.at(p)] = c.j;
    if (cnt == K) {
      // shrink: anything that can still enter has D2 <= D2_K, and D2_K is
      // at most d_K + its error; cells further than that are skipped and the
      // walk ends at the first b beyond it (Sec. II.A, K nearest)
      const float dk = L.d[L.at(K - 1)];
      const float m = dk * 1.000001f;
      kth_hi = fminf(hi_max, dk + fmaf(pb.c2, m, pb.c1 * sqrtf(m)) + 1e-37f);
      const float rc = sqrtf(kth_hi) * g.inv_s + g.eps;
      cut2 = rc * rc;
    }
  };

  auto cell = [&](const Target &tg, int b, int e) {
    for (int j = b; j < e; ++j) {
      if (j == self) continue;
      const float4 p = g.spos[j];
      Cand c;
      c.j = j;
      c.D = __longlong_as_double(0x7ff8000000000000ll);
      if (tg.outside) {
        const double D = canon_d2(Q.q, p, g);
        if (D > B.r2) continue;
        c.D = D;
        c.d = (float)D;
      } else {
        const float dx = p.x - tg.qx, dy = p.y - tg.qy, dz = p.z - tg.qz;
        c.d = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
        if (c.d > kth_hi) continue;
        const float lo = tg.wrapped ? B.lo_w : B.lo, hi = tg.wrapped ? B.hi_w : B.hi;
        if (c.d > hi) continue;
        if (c.d > lo) {
          const double D = canon_d2(Q.q, p, g);
          if (D > B.r2) continue;
          c.D = D;
        }
      }
      insert(c);
    }
  };

  if (!Q.outside && !(flags & SI_METHOD_CUBE)) {
    // Center to edge over x-rows (y-z minimum bound b2 ascending).  For each
    // row the exact y-z distance of the query and the current cut give the
    // x-interval of cells that can still hold a closer point: one contiguous
    // range of sorted points (consecutive x cells are consecutive packed
    // indices, Sec. II.B).  The walk ends at the first row whose bound
    // exceeds the cut (early cut-off, Sec. II.A).
    bool out_seen = false;
    const int Gx = 1 << g.wx;
    const bool cyc_x = g.cyc & 1u;
    auto outside = [&]() {
      if (out_seen) return;
      out_seen = true;
      Target t;
      t.key = g.outside;
      t.outside = true;
      t.wrapped = false;
      t.qx = Q.q.x;
      t.qy = Q.q.y;
      t.qz = Q.q.z;
      cell(t, __ldg(g.cell_start + g.outside), __ldg(g.cell_start + g.outside + 1));
    };
    for (int r = 0; r < g.n_rows; ++r) {
      const RowEntry R = g.rows[r];
      if ((float)R.b2 > cut2) break;
      if (R.b2 > n_query) break;
      const float ty = R.oy > 0 ? (float)(R.oy - 1) + Q.zp[1] : (R.oy < 0 ? (float)(-R.oy - 1) + Q.zn[1] : 0.f);
      const float tz = R.oz > 0 ? (float)(R.oz - 1) + Q.zp[2] : (R.oz < 0 ? (float)(-R.oz - 1) + Q.zn[2] : 0.f);
      const float rem = cut2 - fmaf(ty, ty, tz * tz);
      if (rem < 0.f) continue;
      const float h = sqrtf(rem) + g.eps;
      const int lo = max((int)floorf(Q.u[0] - h) - Q.c[0], -g.row_lim_x);
      const int hi = min((int)floorf(Q.u[0] + h) - Q.c[0], g.row_lim_x);
      if (lo > hi) continue;
      Target tg = translate_raw(R.unp, Q, g);
      if (tg.outside) {
        outside();
        continue;
      }
      const unsigned row = tg.key - (unsigned)Q.c[0];
      int x0 = Q.c[0] + lo, x1 = Q.c[0] + hi;
      if (!cyc_x) {
        if (x0 < 0 || x1 >= Gx) outside();
        x0 = max(x0, 0);
        x1 = min(x1, Gx - 1);
        if (x0 > x1) continue;
      } else if (x0 < 0 || x1 >= Gx) {
        const int wa = x0 < 0 ? x0 + Gx : 0;
        const int wb = x0 < 0 ? Gx - 1 : x1 - Gx;
        Target tw = tg;
        tw.qx = Q.q.x + (x0 < 0 ? g.Lx : -g.Lx);
        tw.wrapped = true;
        cell(tw, __ldg(g.cell_start + row + wa), __ldg(g.cell_start + row + wb + 1));
        x0 = max(x0, 0);
        x1 = min(x1, Gx - 1);
      }
      cell(tg, __ldg(g.cell_start + row + x0), __ldg(g.cell_start + row + x1 + 1));
    }
  } else {
    auto v = [&](const Target &tg, bool) {
      cell(tg, __ldg(g.cell_start + tg.key), __ldg(g.cell_start + tg.key + 1));
    };
    walk_cube(g, Q, dmax_g, v);
  }

  const int orig = __ldg(g.qid + s);
  int *oi = out_ids + (size_t)orig * K;
  for (int k = 0; k < K; ++k) oi[k] = k < cnt ? __ldg(g.perm + L.j[L.at(k)]) : -1;
  if (out_d2) {   // the FP32 rounding of the canonical FP64 D2 of each reported neighbor, or the FP32 value
    float *od = out_d2 + (size_t)orig * K;
    const bool fast = flags & SI_FAST_D2;
    for (int k = 0; k < K; ++k)
      od[k] = k >= cnt ? __int_as_float(0x7f800000)
                       : (fast ? L.d[L.at(k)] : canon_d2_f32(Q.q, g.spos[L.j[L.at(k)]], g));
  }
  out_counts[orig] = cnt;
}

constexpr int kKnnWarps = 8;      // warps per block of k_knn_warp
constexpr int kKnnCap = 512;      // candidates a warp holds

// First pass within dmax1 (rows1, B1: the x-rows whose y-z bound is within
// it and its guard band), a radius expected to hold about K + 2 sqrt(K) + 4
// points: exact whenever it holds at least K (the K nearest then all lie
// within it); else a second pass within r_max (dmax_g, rows_q, B).  dmax1 ==
// dmax_g: one pass.  list (nullable): [0] =
// count, then the sorted slots to serve; else every slot.
// One query (sorted slot s) served by the calling warp; key is the warp's
// candidate buffer (kKnnCap keys).
__device__ __forceinline__ void knn_warp_query(const GridDev &g, int s, unsigned long long *key, int K,
                                               float dmax_g, int rows_q, const Band &B, float dmax1, int rows1,
                                               const Band &B1, const PairBand &pb, unsigned flags,
                                               int *__restrict__ out_ids, float *__restrict__ out_d2,
                                               int *__restrict__ out_counts, int *__restrict__ fallq) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  const QueryGeom Q = make_geom(g.qpos[s], g);
  if (Q.outside) {   // the bounding-cube walk of the per-thread kernel
    if (lane == 0) fallq[1 + atomicAdd(fallq, 1)] = s;
    return;
  }
  const int self = query_self(g, flags, s);
  const int Gx = 1 << g.wx;
  const bool cyc_x = g.cyc & 1u;
  int cnt = 0;
  bool overflow = false, out_any = false;
  // key: FP32 d2 above, then bit 31 set for a candidate compared through a
  // wrapped image (its FP32 value carries the absolute error term of the
  // pair bound), then the sorted slot
  auto add = [&](bool in, float d, int j, bool wr) {
    const unsigned m = __ballot_sync(0xffffffffu, in);
    const int at = cnt + __popc(m & lt);
    if (in && at < kKnnCap)
      key[at] = ((unsigned long long)__float_as_uint(d) << 32) | (unsigned)j | (wr ? 0x80000000u : 0u);
    cnt += __popc(m);
  };
  // every candidate within the cut (cut2 = its square in cell units, nrows
  // the rows whose y-z bound is within it, Bc its guard band), decided
  // exactly, into the buffer.  Lane i decodes row base + i of a 32-row batch:
  // its x-interval of cells is one run of sorted points (and a second run
  // where it wraps a cyclic x axis); the lanes then take the batch's
  // candidates 32 at a time, whichever rows they lie in.
  auto gather = [&](float cut2, int nrows, const Band &B) {
  cnt = 0;
  overflow = false;
  out_any = false;
  for (int base = 0; base < nrows && !overflow; base += 32) {
    const int r = base + lane;
    int b0 = 0, l0 = 0, b1 = 0, l1 = 0;
    float qx0 = 0.f, qy0 = 0.f, qz0 = 0.f, qx1 = 0.f;
    bool w0 = false, out = false;
    if (r < nrows) {
      const RowEntry E = g.rows[r];
      const float ty = E.oy > 0 ? (float)(E.oy - 1) + Q.zp[1] : (E.oy < 0 ? (float)(-E.oy - 1) + Q.zn[1] : 0.f);
      const float tz = E.oz > 0 ? (float)(E.oz - 1) + Q.zp[2] : (E.oz < 0 ? (float)(-E.oz - 1) + Q.zn[2] : 0.f);
      const float rem = cut2 - fmaf(ty, ty, tz * tz);
      if (rem >= 0.f) {
        const float h = sqrtf(rem) + g.eps;
        const int lo = max((int)floorf(Q.u[0] - h) - Q.c[0], -g.row_lim_x);
        const int hi = min((int)floorf(Q.u[0] + h) - Q.c[0], g.row_lim_x);
        if (lo <= hi) {
          const Target tg = translate_raw(E.unp, Q, g);
          if (tg.outside) {
            out = true;
          } else {
            const unsigned row = tg.key - (unsigned)Q.c[0];
            int x0 = Q.c[0] + lo, x1 = Q.c[0] + hi;
            qx0 = tg.qx;
            qy0 = tg.qy;
            qz0 = tg.qz;
            w0 = tg.wrapped;
            if (!cyc_x) {
              if (x0 < 0 || x1 >= Gx) out = true;
              x0 = max(x0, 0);
              x1 = min(x1, Gx - 1);
            } else if (x0 < 0 || x1 >= Gx) {
              const int wa = x0 < 0 ? x0 + Gx : 0, wb = x0 < 0 ? Gx - 1 : x1 - Gx;
              b1 = __ldg(g.cell_start + row + wa);
              l1 = __ldg(g.cell_start + row + wb + 1) - b1;
              qx1 = Q.q.x + (x0 < 0 ? g.Lx : -g.Lx);
              x0 = max(x0, 0);
              x1 = min(x1, Gx - 1);
            }
            if (x0 <= x1) {
              b0 = __ldg(g.cell_start + row + x0);
              l0 = __ldg(g.cell_start + row + x1 + 1) - b0;
            }
          }
        }
      }
    }
    out_any |= __any_sync(0xffffffffu, out);
    // the batch's candidates numbered across the lanes' runs (prefix of the
    // run lengths) and taken 32 at a time: lane t takes candidate f0 + t of
    // the lane L that owns it (the last lane whose runs start at or before
    // it), fetching L's run bounds and frame by shuffle
    const int nt = l0 + l1;
    const int ninc = warp_incl_scan_i(nt);
    const int ntot = __shfl_sync(0xffffffffu, ninc, 31);
    const int nexc = ninc - nt;
    for (int f0 = 0; f0 < ntot; f0 += 32) {
      const int f = f0 + lane;
      int L = 0;
#pragma unroll
      for (int sh = 16; sh > 0; sh >>= 1) {
        const int e = __shfl_sync(0xffffffffu, nexc, L + sh);
        if (e <= f) L += sh;
      }
      const int k = f - __shfl_sync(0xffffffffu, nexc, L);
      const int ob0 = __shfl_sync(0xffffffffu, b0, L), ol0 = __shfl_sync(0xffffffffu, l0, L);
      const int ob1 = __shfl_sync(0xffffffffu, b1, L);
      const float oqx0 = __shfl_sync(0xffffffffu, qx0, L), oqx1 = __shfl_sync(0xffffffffu, qx1, L);
      const float oqy = __shfl_sync(0xffffffffu, qy0, L), oqz = __shfl_sync(0xffffffffu, qz0, L);
      const bool ow0 = __shfl_sync(0xffffffffu, (int)w0, L) != 0;
      bool in = false, band = false, wr = false;
      float d = 0.f;
      int j = 0;
      float4 p = make_float4(0.f, 0.f, 0.f, 0.f);
      if (f < ntot) {
        const bool second = k >= ol0;   // the run through the x wrap
        j = second ? ob1 + (k - ol0) : ob0 + k;
        wr = second || ow0;
        if (j != self) {
          p = g.spos[j];
          const float dx = p.x - (second ? oqx1 : oqx0), dy = p.y - oqy, dz = p.z - oqz;
          d = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
          const float blo = wr ? B.lo_w : B.lo, bhi = wr ? B.hi_w : B.hi;
          in = d <= blo;
          band = !in && !(d > bhi);
        }
      }
      // the guard band in FP64, behind a warp-uniform branch and a real
      // call: FP64 issues only when some lane needs it (rare)
      if (__any_sync(0xffffffffu, band)) {
        if (band) in = canon_d2_call(Q.q, p, g.Lx, g.Ly, g.Lz, g.cyc) <= B.r2;
      }
      add(in, d, j, wr);
    }
    if (cnt > kKnnCap) overflow = true;
  }
  if (out_any && !overflow) {   // the outside cell: every pair in FP64
    const int b = __ldg(g.cell_start + g.outside), e = __ldg(g.cell_start + g.outside + 1);
    for (int j0 = b; j0 < e; j0 += 32) {
      const int j = j0 + lane;
      bool in = false;
      float d = 0.f;
      if (j < e && j != self) {
        const double D = canon_d2(Q.q, g.spos[j], g);
        in = D <= B.r2;
        d = (float)D;
      }
      add(in, d, j, false);
    }
    if (cnt > kKnnCap) overflow = true;
  }
  };
  // one call site, so the gather inlines: the first pass, then the second
  // when the first held fewer than K
  for (int pass = 0; pass < 2; ++pass) {
    if (pass == 1 && (overflow || cnt >= K || !(dmax1 < dmax_g))) break;
    const float dm = pass ? dmax_g : dmax1;
    gather(dm * dm, pass ? rows_q : rows1, pass ? B : B1);
  }
  if (overflow) {   // the per-thread kernel takes it
    if (lane == 0) fallq[1 + atomicAdd(fallq, 1)] = s;
    return;
  }
  __syncwarp();
  warp_sort(key, cnt, lane, ~0ull);
  __syncwarp();
  // runs of keys closer than the FP32 error bound, up to the K-th (and the
  // first one past it, which decides who is in), in canonical order.  Two
  // FP32 values further apart than both their bounds are in canonical order
  // already; the absolute term of the bound applies only when one of them
  // came through a wrapped image (the rounding of q + L), otherwise each is
  // within a relative c2 / 2 of its canonical value.
  auto close = [&](unsigned long long xa, unsigned long long xb) {
    const float da = __uint_as_float((unsigned)(xa >> 32));
    const float db = __uint_as_float((unsigned)(xb >> 32));
    const float m = db * 1.000001f;
    const bool wr = ((unsigned)xa | (unsigned)xb) >> 31;
    return !(db - da > fmaf(pb.c2, m, wr ? pb.c1 * sqrtf(m) : 0.f) + 1e-37f);
  };
  const int top = min(cnt, K + 1);
  bool ties = false;   // an adjacent pair within the bound, up to the (K+1)-th
  for (int e0 = 1; e0 < min(top + 1, cnt); e0 += 32) {
    const int e = e0 + lane;
    bool t = false;
    if (e < min(top + 1, cnt)) t = close(key[e - 1], key[e]);
    ties |= __any_sync(0xffffffffu, t);
  }
  if (ties && lane == 0) {
    int a = 0;
    while (a < top) {
      int e = a + 1;
      while (e < cnt && close(key[e - 1], key[e])) ++e;
      if (e - a > 1) {   // insertion sort of [a, e) by (D2, index)
        for (int i = a + 1; i < e; ++i) {
          const unsigned long long x = key[i];
          const int jx = (int)(x & 0x7fffffffu);
          const double Dx = canon_d2(Q.q, g.spos[jx], g);
          const int ix = __ldg(g.perm + jx);
          int p = i;
          while (p > a) {
            const int jy = (int)(key[p - 1] & 0x7fffffffu);
            const double Dy = canon_d2(Q.q, g.spos[jy], g);
            if (Dy < Dx || (Dy == Dx && __ldg(g.perm + jy) < ix)) break;
            key[p] = key[p - 1];
            --p;
          }
          key[p] = x;
        }
      }
      a = e;
    }
  }
  __syncwarp();
  const int kept = min(cnt, K);
  const int orig = __ldg(g.qid + s);
  int *oi = out_ids + (size_t)orig * K;
  float *od = out_d2 ? out_d2 + (size_t)orig * K : nullptr;
  for (int k0 = 0; k0 < K; k0 += 32) {
    const int k = k0 + lane;
    const bool have = k < kept;
    const unsigned long long x = have ? key[k] : 0ull;
    if (k < K) oi[k] = have ? __ldg(g.perm + (int)(x & 0x7fffffffu)) : -1;
    // the FP32 rounding of the canonical FP64 D2 of each reported neighbor,
    // or (SI_FAST_D2) the FP32 value the kernel sorted by; the rare pairs
    // the FP32 form cannot settle take FP64 behind a call
    if (od) {
      float v = __int_as_float(0x7f800000);
      bool hard = false;
      float4 p = make_float4(0.f, 0.f, 0.f, 0.f);
      if (have) {
        if (flags & SI_FAST_D2) {
          v = __uint_as_float((unsigned)(x >> 32));
        } else {
          p = g.spos[(int)(x & 0x7fffffffu)];
          hard = !canon_d2_f32_try(Q.q, p, g, v);
        }
      }
      if (__any_sync(0xffffffffu, hard)) {
        if (hard) v = __double2float_rn(canon_d2_call(Q.q, p, g.Lx, g.Ly, g.Lz, g.cyc));
      }
      if (k < K) od[k] = v;
    }
  }
  if (lane == 0) out_counts[orig] = kept;
}

__global__ void __launch_bounds__(kKnnWarps * 32, 4) k_knn_warp(GridDev g, int K, float dmax_g, int rows_q,
                                                            Band B, float dmax1, int rows1, Band B1,
                                                            PairBand pb, unsigned flags,
                                                            int *__restrict__ out_ids,
                                                            float *__restrict__ out_d2,
                                                            int *__restrict__ out_counts,
                                                            int *__restrict__ fallq,
                                                            const int *__restrict__ list) {
  __shared__ unsigned long long keys[kKnnWarps][kKnnCap];
  const int w = threadIdx.x >> 5;
  const int count = list ? list[0] : g.n;
  for (int item = blockIdx.x * kKnnWarps + w; item < count; item += gridDim.x * kKnnWarps) {
    __syncwarp();   // the previous query's buffer is no longer read
    knn_warp_query(g, list ? list[1 + item] : item, keys[w], K, dmax_g, rows_q, B, dmax1, rows1, B1, pb, flags,
                   out_ids, out_d2, out_counts, fallq);
  }
}

// One thread per query, for K <= kLaneKMax with a bounded r_max.  The lanes
// of a warp serve consecutive sorted queries, which lie in neighbouring cells
// of one x-row, so they walk the same x-rows (the rows table, centre to edge)
// in step and their loads of cell starts and points fall close together.
// Each lane keeps its K + 1 smallest FP32 distances, sorted, in its column of
// shared memory; once it holds K + 1 the cut shrinks to the (K+1)-th value
// plus the FP32 error bound (the running radius of Sec. II.A), which skips
// later rows, cells and candidates.  A candidate that is dropped beyond the
// list is remembered by the smallest FP32 value dropped: when that value lies
// within the error bound of the K-th, the list alone does not settle the K-th
// neighbour and the query goes to the warp kernel's queue (warpq), which
// keeps every candidate.  Runs of list entries closer than the bound are put
// in canonical (D2, index) order, as in the warp kernel.
constexpr int kLaneT = 128;
constexpr int kLaneKMax = 16;   // measured: faster than the warp kernel up to K = 16, slower at K = 64

__global__ void __launch_bounds__(kLaneT) k_knn_lane(GridDev g, int K, float dmax_g, int rows_q, Band B,
                                                     float dmax1, int rows1, Band B1, PairBand pb,
                                                     unsigned flags, int *__restrict__ out_ids,
                                                     float *__restrict__ out_d2, int *__restrict__ out_counts,
                                                     int *__restrict__ fallq, int *__restrict__ warpq,
                                                     const int *__restrict__ list) {
  extern __shared__ __align__(16) unsigned char lane_smem[];
  const int T = blockDim.x, t = threadIdx.x;
  const int KP = K + 1;
  float *Ld = reinterpret_cast<float *>(lane_smem);              // [k * T + t]: FP32 d2, ascending
  unsigned *Lj = reinterpret_cast<unsigned *>(Ld + (size_t)KP * T);   // sorted slot | wrapped << 31
  const int ti = blockIdx.x * T + t;
  if (ti >= (list ? list[0] : g.n)) return;
  const int s = list ? list[1 + ti] : ti;
  const QueryGeom Q = make_geom(g.qpos[s], g);
  if (Q.outside) {   // the bounding-cube walk of the per-thread kernel
    fallq[1 + atomicAdd(fallq, 1)] = s;
    return;
  }
  const int self = query_self(g, flags, s);
  const int Gx = 1 << g.wx;
  const bool cyc_x = g.cyc & 1u;
  auto bound = [&](float d) {   // FP32 error bound of a pair of values near d (wrapped or not)
    const float m = d * 1.000001f;
    return fmaf(pb.c2, m, pb.c1 * sqrtf(m)) + 1e-37f;
  };
  int cnt = 0;
  float dmin_drop = INFINITY;
  for (int pass = 0; pass < 2; ++pass) {
    if (pass == 1 && (cnt >= K || !(dmax1 < dmax_g))) break;
    const Band Bp = pass ? B : B1;
    const float dm = pass ? dmax_g : dmax1;
    const int nrows = pass ? rows_q : rows1;
    const float hi0 = fmaxf(Bp.hi, Bp.hi_w);
    cnt = 0;
    dmin_drop = INFINITY;
    float cut2 = dm * dm;   // cell units: rows and cells beyond it are skipped
    float hi = hi0;         // world units: candidates beyond it are skipped
    // an accepted candidate into the sorted list of the K + 1 smallest
    auto insert = [&](float d, unsigned code) {
      int at;
      if (cnt == KP) {
        const float last = Ld[K * T + t];
        if (!(d < last)) {
          dmin_drop = fminf(dmin_drop, d);
          return;
        }
        dmin_drop = fminf(dmin_drop, last);   // the old (K+1)-th leaves the list
        at = K;
      } else {
        at = cnt++;
      }
      while (at > 0 && Ld[(at - 1) * T + t] > d) {
        Ld[at * T + t] = Ld[(at - 1) * T + t];
        Lj[at * T + t] = Lj[(at - 1) * T + t];
        --at;
      }
      Ld[at * T + t] = d;
      Lj[at * T + t] = code;
      if (cnt == KP) {   // shrink: only values below the (K+1)-th, or within its bound, still matter
        const float dl = Ld[K * T + t];
        hi = fminf(hi0, dl + bound(dl));
        const float rc = sqrtf(hi) * g.inv_s + g.eps;
        cut2 = fminf(cut2, rc * rc);
      }
    };
    auto consider = [&](float d, int j, bool wr, const float4 &p) {
      if (d > hi) return;
      const float blo = wr ? Bp.lo_w : Bp.lo, bhi = wr ? Bp.hi_w : Bp.hi;
      bool in = d <= blo;
      if (!in && !(d > bhi)) in = canon_d2_call(Q.q, p, g.Lx, g.Ly, g.Lz, g.cyc) <= Bp.r2;
      if (in) insert(d, (unsigned)j | (wr ? 0x80000000u : 0u));
    };
    bool out_any = false;
    for (int r = 0; r < nrows; ++r) {
      const RowEntry E = g.rows[r];
      if ((float)E.b2 > cut2) break;   // rows by b2: every later row lies beyond the cut
      const float ty = E.oy > 0 ? (float)(E.oy - 1) + Q.zp[1] : (E.oy < 0 ? (float)(-E.oy - 1) + Q.zn[1] : 0.f);
      const float tz = E.oz > 0 ? (float)(E.oz - 1) + Q.zp[2] : (E.oz < 0 ? (float)(-E.oz - 1) + Q.zn[2] : 0.f);
      const float rem = cut2 - fmaf(ty, ty, tz * tz);
      if (rem < 0.f) continue;
      const float h = sqrtf(rem) + g.eps;
      const int lo = max((int)floorf(Q.u[0] - h) - Q.c[0], -g.row_lim_x);
      const int hx = min((int)floorf(Q.u[0] + h) - Q.c[0], g.row_lim_x);
      if (lo > hx) continue;
      const Target tg = translate_raw(E.unp, Q, g);
      if (tg.outside) {
        out_any = true;
        continue;
      }
      const unsigned row = tg.key - (unsigned)Q.c[0];
      int x0 = Q.c[0] + lo, x1 = Q.c[0] + hx;
      if (!cyc_x) {
        if (x0 < 0 || x1 >= Gx) out_any = true;
      } else if (x0 < 0 || x1 >= Gx) {   // the part through the x wrap
        const int wa = x0 < 0 ? x0 + Gx : 0, wb = x0 < 0 ? Gx - 1 : x1 - Gx;
        const int b = __ldg(g.cell_start + row + wa), e = __ldg(g.cell_start + row + wb + 1);
        const float qx = Q.q.x + (x0 < 0 ? g.Lx : -g.Lx);
        for (int j = b; j < e; ++j) {
          if (j == self) continue;
          const float4 p = g.spos[j];
          const float dx = p.x - qx, dy = p.y - tg.qy, dz = p.z - tg.qz;
          consider(fmaf(dz, dz, fmaf(dy, dy, dx * dx)), j, true, p);
        }
      }
      x0 = max(x0, 0);
      x1 = min(x1, Gx - 1);
      if (x0 > x1) continue;
      const int b = __ldg(g.cell_start + row + x0), e = __ldg(g.cell_start + row + x1 + 1);
      for (int j = b; j < e; ++j) {
        if (j == self) continue;
        const float4 p = g.spos[j];
        const float dx = p.x - tg.qx, dy = p.y - tg.qy, dz = p.z - tg.qz;
        consider(fmaf(dz, dz, fmaf(dy, dy, dx * dx)), j, tg.wrapped, p);
      }
    }
    if (out_any) {   // the outside cell: every pair in FP64 (its FP32 rounding is within the relative bound)
      const int b = __ldg(g.cell_start + g.outside), e = __ldg(g.cell_start + g.outside + 1);
      for (int j = b; j < e; ++j) {
        if (j == self) continue;
        const double D = canon_d2_call(Q.q, g.spos[j], g.Lx, g.Ly, g.Lz, g.cyc);
        if (D <= Bp.r2 && (float)D <= hi) insert((float)D, (unsigned)j);
      }
    }
  }
  // the K-th is settled by the list unless a dropped candidate lies within
  // the error bound of it
  if (cnt == KP && dmin_drop <= Ld[(K - 1) * T + t] + bound(Ld[(K - 1) * T + t])) {
    warpq[1 + atomicAdd(warpq, 1)] = s;
    return;
  }
  // runs of adjacent entries closer than the bound, in canonical order
  auto close = [&](int a) {   // entries a and a + 1
    const float da = Ld[a * T + t], db = Ld[(a + 1) * T + t];
    const bool wr = (Lj[a * T + t] | Lj[(a + 1) * T + t]) >> 31;
    const float m = db * 1.000001f;
    return !(db - da > fmaf(pb.c2, m, wr ? pb.c1 * sqrtf(m) : 0.f) + 1e-37f);
  };
  for (int a = 0; a + 1 < cnt; ++a) {
    if (!close(a)) continue;
    int e = a + 1;
    while (e + 1 < cnt && close(e)) ++e;
    // insertion sort of [a, e] by (D2, index)
    for (int i = a + 1; i <= e; ++i) {
      const float dx = Ld[i * T + t];
      const unsigned cx = Lj[i * T + t];
      const int jx = (int)(cx & 0x7fffffffu);
      const double Dx = canon_d2_call(Q.q, g.spos[jx], g.Lx, g.Ly, g.Lz, g.cyc);
      const int ix = __ldg(g.perm + jx);
      int p = i;
      while (p > a) {
        const int jy = (int)(Lj[(p - 1) * T + t] & 0x7fffffffu);
        const double Dy = canon_d2_call(Q.q, g.spos[jy], g.Lx, g.Ly, g.Lz, g.cyc);
        if (Dy < Dx || (Dy == Dx && __ldg(g.perm + jy) < ix)) break;
        Ld[p * T + t] = Ld[(p - 1) * T + t];
        Lj[p * T + t] = Lj[(p - 1) * T + t];
        --p;
      }
      Ld[p * T + t] = dx;
      Lj[p * T + t] = cx;
    }
    a = e;
  }
  const int kept = min(cnt, K);
  const int orig = __ldg(g.qid + s);
  int *oi = out_ids + (size_t)orig * K;
  float *od = out_d2 ? out_d2 + (size_t)orig * K : nullptr;
  for (int k = 0; k < K; ++k) {
    const bool have = k < kept;
    const int j = have ? (int)(Lj[k * T + t] & 0x7fffffffu) : 0;
    oi[k] = have ? __ldg(g.perm + j) : -1;
    if (od) {
      float v = __int_as_float(0x7f800000);
      if (have) {
        if (flags & SI_FAST_D2) {
          v = Ld[k * T + t];
        } else {
          const float4 p = g.spos[j];
          if (!canon_d2_f32_try(Q.q, p, g, v)) v = __double2float_rn(canon_d2_call(Q.q, p, g.Lx, g.Ly, g.Lz, g.cyc));
        }
      }
      od[k] = v;
    }
  }
  out_counts[orig] = kept;
}

}  // namespace si

using namespace si;

extern "C" si_status si_query_knn(si_grid *g, const float *d_centers, int64_t m, int k,
                                  float r_max_query, uint32_t flags, int32_t *d_ids, float *d_d2,
                                  int32_t *d_counts, void *stream) {
  if (!g) return fail(SI_ERR_INVALID, "null grid");
  if (d_centers) {
    if (m < 0 || m > (int64_t)INT32_MAX - 1) return fail(SI_ERR_INVALID, "m out of range");
    if ((uintptr_t)d_centers & 15u) return fail(SI_ERR_INVALID, "centers must be a 16-byte aligned float4 array");
  } else if (m != g->n) {
    return fail(SI_ERR_INVALID, "all-agents mode: m must equal the grid's point count");
  }
  if (k < 1 || k > 64) return fail(SI_ERR_INVALID, "k must be in [1, 64]");
  if (!d_ids || !d_counts) return fail(SI_ERR_INVALID, "null output");
  if (flags & ~(SI_INCLUDE_SELF | SI_FAST_D2 | SI_METHOD_CUBE)) return fail(SI_ERR_INVALID, "unknown flags");
  const bool unb = !(r_max_query > 0.f) || std::isinf(r_max_query);
  if (unb && !g->lat.unbounded) return fail(SI_ERR_INVALID, "unbounded r_max needs an unbounded grid");
  if (!unb && !g->lat.unbounded && (double)r_max_query > (double)g->desc.r_max)
    return fail(SI_ERR_INVALID, "r_max exceeds the grid's r_max");
  if (m == 0) return SI_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const Lattice &lat = g->lat;
  float dmax_g;
  int n_query;
  Band B;
  if (unb) {
    n_query = g->tables.n_max;
    dmax_g = std::sqrt((float)n_query + 1.f) + 2.f;
    // every point of the region qualifies: a band that accepts everything
    B.lo = B.lo_w = B.hi = B.hi_w = INFINITY;
    B.r2 = INFINITY;
    for (int a = 0; a < 3; ++a) dmax_g = std::max(dmax_g, (float)(1 << lat.w[a]) * 2.f);
  } else {
    dmax_g = r_max_query * lat.inv_s + (float)lat.eps;
    n_query = std::min((int)std::floor(dmax_g * dmax_g), g->tables.n_max);
    B = make_band(lat, r_max_query);
  }
  const PairBand pb = make_pair_band(lat);
  const size_t smem = (size_t)k * kKnnThreads * 8;
  SI_CUDA_TRY(cudaFuncSetAttribute(k_knn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  // the query set: the grid's points, or the caller's centers in coarse
  // cell order (listed; those with invalid coordinates get empty results)
  GridDev dv = g->dev();
  const int *list = nullptr;
  int *fallq = g->longq;   // idle during a K-nearest call
  if (d_centers) {
    CenterOut eo;
    eo.K = k;
    eo.ids = d_ids;
    eo.d2 = d_d2;
    eo.counts = d_counts;
    si_status s = prepare_centers(g, d_centers, m, false, false, eo, dv, st);
    if (s != SI_OK) return s;
    list = g->clist0;
    fallq = g->clong;
  }
  // the bin lattice (SI_METHOD_CUBE, or the reversal distance of
  // si_grid_set_method): every cell of the bounding cube of the r_max sphere
  if (!unb && (double)r_max_query * (double)lat.inv_s < g->knn_cube_below) flags |= SI_METHOD_CUBE;
  if (unb || (flags & SI_METHOD_CUBE)) {
    // no bound, or the cube: the per-thread walk with the shrinking cut
    const unsigned blocks = (unsigned)((m + kKnnThreads - 1) / kKnnThreads);
    SI_KLAUNCH((flags & SI_METHOD_CUBE) ? "k_knn_cube" : "k_knn", st,
               k_knn<<<blocks, kKnnThreads, smem, st>>>(dv, k, dmax_g, n_query, B, pb, flags, d_ids, d_d2, d_counts,
                                                        list));
    return SI_OK;
  }
  // first cut: the radius expected to hold `want` points at the mean load
  // (exact when it holds K; the kernels widen it to r_max otherwise).  The
  // warp kernel takes K + 2 sqrt(K) + 4, two standard deviations of a
  // Poisson count above K; the lane kernel, whose lanes wait for the warp's
  // slowest, K + 3 sqrt(K) + 8, so that a second pass is rare in any warp
  // (its cut shrinks as soon as K + 1 are held, so the wider start costs
  // little).
  const double load = (double)g->n / (double)std::max<int64_t>(g->n_cells - 1, 1);
  const std::vector<int> &row_end = g->tables.row_end;   // rows with b2 <= n
  const int rows_q = row_end[(size_t)std::min(n_query, g->tables.n_max)];
  auto first_cut = [&](double want, float &dmax1, int &rows1, Band &B1) {
    dmax1 = dmax_g;
    rows1 = rows_q;
    B1 = B;
    if (load <= 0.0) return;
    const double r1 = std::cbrt(3.0 * want / (4.0 * M_PI * load)) / (double)lat.inv_s;   // world units
    if (r1 < 0.9 * (double)r_max_query) {
      B1 = make_band(lat, (float)r1);
      dmax1 = (float)r1 * lat.inv_s + (float)lat.eps;
      rows1 = row_end[(size_t)std::min((int)std::floor(dmax1 * dmax1), g->tables.n_max)];
    }
  };
  float dmax1w;
  int rows1w;
  Band B1w;
  first_cut(k + 2.0 * std::sqrt((double)k) + 4.0, dmax1w, rows1w, B1w);
  SI_CUDA_TRY(cudaMemsetAsync(fallq, 0, sizeof(int), st));
  if (k <= kLaneKMax) {
    // a thread per query; the queries whose K-th it cannot settle go to the
    // warp kernel (warpq), those outside the region to the per-thread kernel
    int *warpq = d_centers ? g->chuge : g->hugeq;   // idle during a K-nearest call
    SI_CUDA_TRY(cudaMemsetAsync(warpq, 0, sizeof(int), st));
    float dmax1l;
    int rows1l;
    Band B1l;
    first_cut(k + 3.0 * std::sqrt((double)k) + 8.0, dmax1l, rows1l, B1l);
    const size_t lsmem = (size_t)(k + 1) * kLaneT * (sizeof(float) + sizeof(unsigned));
    SI_CUDA_TRY(cudaFuncSetAttribute(k_knn_lane, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lsmem));
    const unsigned lblocks = (unsigned)((m + kLaneT - 1) / kLaneT);
    SI_KLAUNCH("k_knn_lane", st, k_knn_lane<<<lblocks, kLaneT, lsmem, st>>>(dv, k, dmax_g, rows_q, B, dmax1l, rows1l,
                                                                           B1l, pb, flags, d_ids, d_d2, d_counts,
                                                                           fallq, warpq, list));
    const unsigned wblocks = (unsigned)std::min<int64_t>((m + kKnnWarps - 1) / kKnnWarps, 148 * 4);
    SI_KLAUNCH("k_knn_warp (lane queue)", st, k_knn_warp<<<wblocks, kKnnWarps * 32, 0, st>>>(dv, k, dmax_g, rows_q, B, dmax1w,
                                                                                rows1w, B1w, pb, flags, d_ids, d_d2,
                                                                                d_counts, fallq, warpq));
  } else {
    // a warp per query; the queries it hands back go to the per-thread kernel
    const unsigned wblocks = (unsigned)((m + kKnnWarps - 1) / kKnnWarps);
    SI_KLAUNCH("k_knn_warp", st, k_knn_warp<<<wblocks, kKnnWarps * 32, 0, st>>>(dv, k, dmax_g, rows_q, B, dmax1w,
                                                                                rows1w, B1w, pb, flags, d_ids, d_d2,
                                                                                d_counts, fallq, list));
  }
  // sized for every query; blocks past the queue's length exit at once
  const unsigned fblocks = (unsigned)((m + kKnnThreads - 1) / kKnnThreads);
  SI_KLAUNCH("k_knn", st, k_knn<<<fblocks, kKnnThreads, smem, st>>>(dv, k, dmax_g, n_query, B, pb, flags,
                                                                   d_ids, d_d2, d_counts, fallq));
  return SI_OK;
}
