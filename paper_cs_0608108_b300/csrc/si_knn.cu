// All-agents K-nearest query (Sec. II.A, last paragraph; Sec. IV.B): walk the
// sorted offset table from the center outwards and, once K neighbors are
// held, shrink the search radius to the K-th distance; the walk stops at the
// first table entry whose minimum bound b exceeds it (early cut-off).
//
// Order is (canonical FP64 D2, index).  Candidates are compared in FP32; two
// FP32 values closer than the proven FP32 error bound are compared again in
// FP64 (values cached per held entry), so the kept set and its order are
// exact while almost every comparison stays in FP32.
#include <cmath>

#include "si_host.h"
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

__global__ void __launch_bounds__(kKnnThreads) k_knn(GridDev g, int K, float dmax_g, int n_query,
                                                     Band B, PairBand pb, unsigned flags,
                                                     int *__restrict__ out_ids,
                                                     float *__restrict__ out_d2,
                                                     int *__restrict__ out_counts) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int T = blockDim.x;
  KnnList L;
  L.d = (float *)smem;
  L.j = (int *)(L.d + (size_t)K * T);
  L.T = T;
  L.t = threadIdx.x;
  const int s = blockIdx.x * T + threadIdx.x;
  if (s >= g.n) return;
  const QueryGeom Q = make_geom(g.spos[s], g);
  const int self = (flags & SI_INCLUDE_SELF) ? -1 : s;
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

  const int orig = __ldg(g.perm + s);
  int *oi = out_ids + (size_t)orig * K;
  for (int k = 0; k < K; ++k) oi[k] = k < cnt ? __ldg(g.perm + L.j[L.at(k)]) : -1;
  if (out_d2) {
    float *od = out_d2 + (size_t)orig * K;
    for (int k = 0; k < K; ++k) od[k] = k < cnt ? L.d[L.at(k)] : __int_as_float(0x7f800000);
  }
  out_counts[orig] = cnt;
}

}  // namespace si

using namespace si;

extern "C" si_status si_query_knn(si_grid *g, const float *d_centers, int64_t m, int k,
                                  float r_max_query, uint32_t flags, int32_t *d_ids, float *d_d2,
                                  int32_t *d_counts, void *stream) {
  if (!g) return fail(SI_ERR_INVALID, "null grid");
  if (d_centers) return fail(SI_ERR_INVALID, "only the all-agents mode is supported (centers must be NULL)");
  if (m != g->n) return fail(SI_ERR_INVALID, "all-agents mode: m must equal the grid's point count");
  if (k < 1 || k > 64) return fail(SI_ERR_INVALID, "k must be in [1, 64]");
  if (!d_ids || !d_counts) return fail(SI_ERR_INVALID, "null output");
  if (flags & ~(SI_INCLUDE_SELF)) return fail(SI_ERR_INVALID, "unknown flags");
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
  const unsigned blocks = (unsigned)((m + kKnnThreads - 1) / kKnnThreads);
  SI_KLAUNCH("k_knn", st, k_knn<<<blocks, kKnnThreads, smem, st>>>(g->dev(), k, dmax_g, n_query, B, pb, flags, d_ids, d_d2,
                                           d_counts));
  return SI_OK;
}
