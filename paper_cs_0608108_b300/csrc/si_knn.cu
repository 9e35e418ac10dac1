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
// Two kernels.  With a bounded r_max, k_knn_warp serves a query with one
// warp: the x-rows of the r_max sphere (rows of cells whose y-z bound is
// within r_max, each cut to the x-interval the query's exact y-z distance
// allows) are decoded by the lanes in parallel, every candidate within r_max
// (the exact predicate) goes to the warp's shared buffer as an FP32 key, and
// a warp bitonic sort orders the buffer; runs of adjacent keys closer than
// the FP32 error bound are then put in canonical order.  r_max is the cut
// here from the start: on these workloads it is close to the K-th distance,
// so shrinking it saves little.  k_knn, one thread per query with the
// shrinking cut described above, serves unbounded r_max, query points outside
// the region and queries whose candidates overflow the warp's buffer.
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

  if (!Q.outside) {
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

struct KnnRuns {                  // up to two runs per row of a 32-row batch
  int b[64];
  int len[64];
  float qx[64], qy[64], qz[64];
  unsigned char wrapped[64];
  int pre[33];
};

// First pass within dmax1 (n1, B1: its table bound and guard band), a radius
// expected to hold about K + 2 sqrt(K) + 4 points: exact whenever it holds at least K
// (the K nearest then all lie within it); else a second pass within r_max
// (dmax_g, n_query, B).  dmax1 == dmax_g: one pass.  list (nullable): [0] =
// count, then the sorted slots to serve; else every slot.
__global__ void __launch_bounds__(kKnnWarps * 32, 4) k_knn_warp(GridDev g, int K, float dmax_g, int n_query,
                                                            Band B, float dmax1, int n1, Band B1,
                                                            PairBand pb, unsigned flags,
                                                            int *__restrict__ out_ids,
                                                            float *__restrict__ out_d2,
                                                            int *__restrict__ out_counts,
                                                            int *__restrict__ fallq,
                                                            const int *__restrict__ list) {
  __shared__ unsigned long long keys[kKnnWarps][kKnnCap];
  __shared__ KnnRuns runs[kKnnWarps];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int item = blockIdx.x * kKnnWarps + w;
  if (item >= (list ? list[0] : g.n)) return;
  const int s = list ? list[1 + item] : item;   // the warp's query (sorted slot)
  unsigned long long *key = keys[w];
  KnnRuns &R = runs[w];
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
  // every candidate within the cut (cut2 = its square in cell units, n_q its
  // table bound, Bc its guard band), decided exactly, into the buffer
  auto gather = [&](float cut2, int n_query, const Band &B) {
  cnt = 0;
  overflow = false;
  out_any = false;
  for (int base = 0; base < g.n_rows && !overflow; base += 32) {
    const int r = base + lane;
    int b0 = 0, l0 = 0, b1 = 0, l1 = 0;
    float qx0 = 0.f, qy0 = 0.f, qz0 = 0.f, qx1 = 0.f;
    bool w0 = false, out = false, live = false;
    if (r < g.n_rows) {
      const RowEntry E = g.rows[r];
      live = E.b2 <= n_query && (float)E.b2 <= cut2;   // rows are sorted by b2
      if (live) {
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
    }
    out_any |= __any_sync(0xffffffffu, out);
    const bool more = __any_sync(0xffffffffu, live);
    R.b[2 * lane] = b0;
    R.len[2 * lane] = l0;
    R.qx[2 * lane] = qx0;
    R.qy[2 * lane] = qy0;
    R.qz[2 * lane] = qz0;
    R.wrapped[2 * lane] = w0 ? 1 : 0;
    R.b[2 * lane + 1] = b1;
    R.len[2 * lane + 1] = l1;
    R.qx[2 * lane + 1] = qx1;
    R.qy[2 * lane + 1] = qy0;
    R.qz[2 * lane + 1] = qz0;
    R.wrapped[2 * lane + 1] = 1;
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
      bool in = false, band = false, wr = false;
      float d = 0.f;
      int j = 0;
      float4 p = make_float4(0.f, 0.f, 0.f, 0.f);
      if (f < total) {
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
          p = g.spos[j];
          const float dx = p.x - R.qx[slot], dy = p.y - R.qy[slot], dz = p.z - R.qz[slot];
          d = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
          wr = R.wrapped[slot];
          const float blo = wr ? B.lo_w : B.lo, bhi = wr ? B.hi_w : B.hi;
          in = d <= blo;
          band = !in && !(d > bhi);
        }
      }
      // the guard band in FP64, behind a warp-uniform branch: FP64 issues
      // only when some lane needs it (rare), never predicated for all
      if (__any_sync(0xffffffffu, band)) {
        if (band) in = canon_d2_call(Q.q, p, g.Lx, g.Ly, g.Lz, g.cyc) <= B.r2;
      }
      add(in, d, j, wr);
    }
    __syncwarp();   // the next batch rewrites R
    if (cnt > kKnnCap) overflow = true;
    if (!more) break;   // every later row lies beyond r_max
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
    gather(dm * dm, pass ? n_query : n1, pass ? B : B1);
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
  if (flags & ~(SI_INCLUDE_SELF | SI_FAST_D2)) return fail(SI_ERR_INVALID, "unknown flags");
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
  if (unb) {
    // no bound: the per-thread walk with the shrinking cut
    const unsigned blocks = (unsigned)((m + kKnnThreads - 1) / kKnnThreads);
    SI_KLAUNCH("k_knn", st, k_knn<<<blocks, kKnnThreads, smem, st>>>(dv, k, dmax_g, n_query, B, pb, flags,
                                                                     d_ids, d_d2, d_counts, list));
    return SI_OK;
  }
  // first cut: the radius expected to hold K + 2 sqrt(K) + 4 points at the
  // mean load, two standard deviations of a Poisson count above K (exact when
  // it holds K; the kernel widens it to r_max otherwise)
  float dmax1 = dmax_g;
  int n1 = n_query;
  Band B1 = B;
  const double load = (double)g->n / (double)std::max<int64_t>(g->n_cells - 1, 1);
  if (load > 0.0) {
    const double want = k + 2.0 * std::sqrt((double)k) + 4.0;
    const double r1 = std::cbrt(3.0 * want / (4.0 * M_PI * load)) / (double)lat.inv_s;   // world units
    if (r1 < 0.9 * (double)r_max_query) {
      B1 = make_band(lat, (float)r1);
      dmax1 = (float)r1 * lat.inv_s + (float)lat.eps;
      n1 = std::min((int)std::floor(dmax1 * dmax1), g->tables.n_max);
    }
  }
  // a warp per query; the queries it hands back go to the per-thread kernel
  SI_CUDA_TRY(cudaMemsetAsync(fallq, 0, sizeof(int), st));
  const unsigned wblocks = (unsigned)((m + kKnnWarps - 1) / kKnnWarps);
  SI_KLAUNCH("k_knn_warp", st, k_knn_warp<<<wblocks, kKnnWarps * 32, 0, st>>>(dv, k, dmax_g, n_query, B, dmax1,
                                                                              n1, B1, pb, flags, d_ids, d_d2,
                                                                              d_counts, fallq, list));
  // sized for every query; blocks past the queue's length exit at once
  const unsigned fblocks = (unsigned)((m + kKnnThreads - 1) / kKnnThreads);
  SI_KLAUNCH("k_knn", st, k_knn<<<fblocks, kKnnThreads, smem, st>>>(dv, k, dmax_g, n_query, B, pb, flags,
                                                                   d_ids, d_d2, d_counts, fallq));
  return SI_OK;
}
