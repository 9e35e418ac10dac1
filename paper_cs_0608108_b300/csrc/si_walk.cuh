// The cell walks of one query, as device templates shared by the radius,
// reduction and batched kernels.
#pragma once

#include "si_internal.cuh"

namespace si {

// Per-call culling parameters (cell units).
struct WalkParams {
  float dg;        // query distance d = r / s, grown by the margin eps
  int rt_b2;       // run-time exact cell test for entries with b2 >= rt_b2
  int incl_b2;     // unconditional-inclusion test for entries with b2 <= incl_b2 (-1: off)
  float incl_d2;   // (d - eps)^2: far corner below this => whole cell inside
};

// Spherical-index walk (Sec. II.A, Sec. III.A).  The main table is read from
// the center up to the shell floor(d); the rest comes from the specialized
// table chosen by the 6 direction bits f < zeta (Eq. 2); a cell whose b2 is
// at or above rt_b2 gets the exact test t^2 > d^2 (Eq. 1).  Offsets that
// leave the region on a non-cyclic axis all map to the one outside cell,
// which is visited at most once.  visit(Target, bool whole_cell_inside).
template <class V>
__device__ __forceinline__ void walk_sphere(const GridDev &g, const QueryGeom &Q, const WalkParams &P,
                                            V &visit) {
  const float dg2 = P.dg * P.dg;
  const int n = min((int)dg2, g.n_max);
  const int fl = isqrt_small(n);
  const float f = P.dg - (float)fl;
  unsigned mask = 0;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    mask |= (f < Q.zp[a]) ? (1u << (2 * a)) : 0u;
    mask |= (f < Q.zn[a]) ? (1u << (2 * a + 1)) : 0u;
  }
  bool out_seen = false;
  auto entry = [&](const TabEntry &e) {
    if (e.b2 >= P.rt_b2 && cell_t2(e, Q) > dg2) return;
    const Target t = translate(e, Q, g);
    if (t.outside) {
      if (out_seen) return;
      out_seen = true;
    }
    const bool full = !t.outside && e.b2 <= P.incl_b2 && cell_far2(e, Q, g.eps) <= P.incl_d2;
    visit(t, full);
  };
  const int main_end = fl > 0 ? __ldg(g.tab_end + fl * fl - 1) : 0;
  for (int i = 0; i < main_end; ++i) entry(g.tab[i]);
  if (fl < g.spec_shells) {
    const int sb = __ldg(g.spec_begin + fl * 64 + (int)mask);
    const int se = __ldg(g.spec_end + 64 * fl * fl + (int)mask * (2 * fl + 1) + (n - fl * fl));
    for (int i = sb; i < se; ++i) entry(g.spec[i]);
  } else {
    const int te = __ldg(g.tab_end + n);
    for (int i = main_end; i < te; ++i) entry(g.tab[i]);
  }
}

// Sub-cell class walk: the query's sub-cell position selects one of q^3
// precomputed lists holding exactly the cells within d of that sub-cell box,
// center to edge; no run-time cell test is needed.  This refines the 64
// direction-bit tables of Sec. III.A (which select by f < zeta only).
// cls / begin may point to global or to shared memory (plain loads).  Each
// entry is an x-row run of cells; consecutive x cells are consecutive packed
// indices (Sec. II.B), so a run's points are one contiguous range of the
// sorted array: two cell-start loads per run.  The visitor is called as
// visit(target, whole_run_inside, first_point, end_point).
template <class V>
__device__ __forceinline__ void walk_classes_in(const GridDev &g, const QueryGeom &Q,
                                                const unsigned long long *cls, const int *begin, int q,
                                                V &visit) {
  const int i = min((int)(Q.phi[0] * (float)q), q - 1);
  const int j = min((int)(Q.phi[1] * (float)q), q - 1);
  const int k = min((int)(Q.phi[2] * (float)q), q - 1);
  const int c = (k * q + j) * q + i;
  const int b = begin[c], e = begin[c + 1];
  const int Gx = 1 << g.wx;
  const bool cyc_x = g.cyc & 1u;
  bool out_seen = false;
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
    visit(t, false, __ldg(g.cell_start + g.outside), __ldg(g.cell_start + g.outside + 1));
  };
  for (int t = b; t < e; ++t) {
    const unsigned long long E = cls[t];
    const int lo = (int)(signed char)((E >> 48) & 0xffull);
    const int len = (int)((E >> 56) & 127ull);
    const bool full = (E >> 63) != 0ull;
    // the row's y and z by the SWAR add (x field stays the query's own)
    Target tg = translate_raw(E & ((1ull << 48) - 1ull), Q, g);
    if (tg.outside) {
      outside();
      continue;
    }
    const unsigned row = tg.key - (unsigned)Q.c[0];   // packed index of x = 0 in that row
    int x0 = Q.c[0] + lo, x1 = x0 + len - 1;
    if (!cyc_x) {
      if (x0 < 0 || x1 >= Gx) outside();
      x0 = max(x0, 0);
      x1 = min(x1, Gx - 1);
      if (x0 > x1) continue;
    } else if (x0 < 0 || x1 >= Gx) {
      // the run crosses the cyclic x boundary: the wrapped part first
      const int wa = x0 < 0 ? x0 + Gx : 0;
      const int wb = x0 < 0 ? Gx - 1 : x1 - Gx;
      Target tw = tg;
      tw.qx = Q.q.x + (x0 < 0 ? g.Lx : -g.Lx);
      tw.wrapped = true;
      visit(tw, full, __ldg(g.cell_start + row + wa), __ldg(g.cell_start + row + wb + 1));
      x0 = max(x0, 0);
      x1 = min(x1, Gx - 1);
    }
    visit(tg, full, __ldg(g.cell_start + row + x0), __ldg(g.cell_start + row + x1 + 1));
  }
}

// Adapter: a visitor that loads its cell range itself, for the prefetching walk.
template <class V>
struct RangeAdapter {
  V &v;
  __device__ __forceinline__ void operator()(const Target &t, bool full, int, int) { v(t, full); }
};

template <class V>
__device__ __forceinline__ void walk_classes(const GridDev &g, const QueryGeom &Q, V &visit) {
  walk_classes_in(g, Q, g.cls, g.cls_begin, g.cls_q, visit);
}

// Bin-lattice walk (Sec. I; Sec. III.C parallelepiped): every cell of the
// sphere's bounding cube, clipped to the region on non-cyclic axes (the
// outside cell visited once if the cube leaves the region), wrapped with an
// image shift on cyclic axes.  Also serves query centers outside the region.
template <class V>
__device__ __forceinline__ void walk_cube(const GridDev &g, const QueryGeom &Q, float dg, V &visit) {
  int lo[3], hi[3];
  bool leaves = false;
  const int w[3] = {g.wx, g.wy, g.wz};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int G = 1 << w[a];
    float fl = floorf(Q.u[a] - dg), fh = floorf(Q.u[a] + dg);
    fl = fmaxf(fminf(fl, 4096.f), -4096.f);
    fh = fmaxf(fminf(fh, 4096.f), -4096.f);
    lo[a] = (int)fl;
    hi[a] = (int)fh;
    if (!((g.cyc >> a) & 1u)) {
      if (lo[a] < 0 || hi[a] >= G) leaves = true;
      lo[a] = max(lo[a], 0);
      hi[a] = min(hi[a], G - 1);
    }
  }
  const float Ls[3] = {g.Lx, g.Ly, g.Lz};
  for (int tz = lo[2]; tz <= hi[2]; ++tz) {
    const int Gz = 1 << g.wz;
    const int cz = tz & (Gz - 1);
    const float sz = tz < 0 ? -Ls[2] : (tz >= Gz ? Ls[2] : 0.f);
    for (int ty = lo[1]; ty <= hi[1]; ++ty) {
      const int Gy = 1 << g.wy;
      const int cy = ty & (Gy - 1);
      const float sy = ty < 0 ? -Ls[1] : (ty >= Gy ? Ls[1] : 0.f);
      for (int tx = lo[0]; tx <= hi[0]; ++tx) {
        const int Gx = 1 << g.wx;
        const int cx = tx & (Gx - 1);
        const float sx = tx < 0 ? -Ls[0] : (tx >= Gx ? Ls[0] : 0.f);
        Target t;
        t.key = pack3(cx, cy, cz, g);
        t.outside = false;
        t.wrapped = (sx != 0.f) | (sy != 0.f) | (sz != 0.f);
        t.qx = Q.q.x - sx;
        t.qy = Q.q.y - sy;
        t.qz = Q.q.z - sz;
        visit(t, false);
      }
    }
  }
  if (leaves) {
    Target t;
    t.key = g.outside;
    t.outside = true;
    t.wrapped = false;
    t.qx = Q.q.x;
    t.qy = Q.q.y;
    t.qz = Q.q.z;
    visit(t, false);
  }
}

// Stacked planes (Sec. V: circle-indexed planes stacked to make the sphere,
// each plane choosing between its circle and its non-empty list).  For each
// z-plane the sphere reaches (its minimum z-distance from the query, with the
// shrunk zetas, within d), the plane's points are one contiguous range of
// the sorted array (consecutive packed indices): an empty plane costs its two
// bounds; a plane holding fewer points than half its circle's x-rows is
// visited as that one range, every pair tested in FP64 (any image may be
// nearest, as for the outside cell); otherwise the circle of radius
// sqrt(d^2 - gz^2) is walked row by row, each row's x-interval from the
// query's exact y-distance to it, one contiguous range per row (two where it
// crosses the cyclic x boundary).  Points agents concentrate on a few planes
// skip the empty ones wholesale.  Query centers outside the region take the
// bounding-cube walk (walk_one).
template <class V>
__device__ __forceinline__ void walk_planes(const GridDev &g, const QueryGeom &Q, float dg, V &visit) {
  const int Gx = 1 << g.wx, Gy = 1 << g.wy, Gz = 1 << g.wz;
  const bool cyc_x = g.cyc & 1u, cyc_y = (g.cyc >> 1) & 1u, cyc_z = (g.cyc >> 2) & 1u;
  const int pshift = g.wx + g.wy;
  bool out_seen = false;
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
    visit(t, false, __ldg(g.cell_start + g.outside), __ldg(g.cell_start + g.outside + 1));
  };
  const int R = (int)dg + 1;
  for (int dz = -R; dz <= R; ++dz) {
    const float gz = dz > 0 ? (float)(dz - 1) + Q.zp[2] : (dz < 0 ? (float)(-dz - 1) + Q.zn[2] : 0.f);
    if (gz > dg) continue;
    int z = Q.c[2] + dz;
    float sz = 0.f;
    if (z < 0 || z >= Gz) {
      if (!cyc_z) {
        outside();
        continue;
      }
      sz = z < 0 ? -g.Lz : g.Lz;   // the plane's image: compare against q - sz
      z = z < 0 ? z + Gz : z - Gz;
    }
    const int ps = __ldg(g.cell_start + ((unsigned)z << pshift));
    const int pe = __ldg(g.cell_start + ((unsigned)(z + 1) << pshift));
    if (pe == ps) continue;
    const float rc2 = fmaxf(dg * dg - gz * gz, 0.f);
    const float rc = sqrtf(rc2);
    if (2 * (pe - ps) <= 2 * (int)rc + 1) {   // fewer points than half the circle's rows
      Target t;
      t.key = 0u;
      t.outside = true;
      t.wrapped = false;
      t.qx = Q.q.x;
      t.qy = Q.q.y;
      t.qz = Q.q.z;
      visit(t, false, ps, pe);
      continue;
    }
    const int Ry = (int)rc + 1;
    for (int dy = -Ry; dy <= Ry; ++dy) {
      const float gy = dy > 0 ? (float)(dy - 1) + Q.zp[1] : (dy < 0 ? (float)(-dy - 1) + Q.zn[1] : 0.f);
      if (gy > rc) continue;
      int y = Q.c[1] + dy;
      float sy = 0.f;
      if (y < 0 || y >= Gy) {
        if (!cyc_y) {
          outside();
          continue;
        }
        sy = y < 0 ? -g.Ly : g.Ly;
        y = y < 0 ? y + Gy : y - Gy;
      }
      const float h = sqrtf(fmaxf(rc2 - gy * gy, 0.f)) + g.eps;
      int x0 = (int)floorf(Q.u[0] - h), x1 = (int)floorf(Q.u[0] + h);
      const unsigned row = ((unsigned)z << pshift) | ((unsigned)y << g.wx);
      Target tg;
      tg.key = row;
      tg.outside = false;
      tg.wrapped = (sy != 0.f) || (sz != 0.f);
      tg.qx = Q.q.x;
      tg.qy = Q.q.y - sy;
      tg.qz = Q.q.z - sz;
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
        visit(tw, false, __ldg(g.cell_start + row + wa), __ldg(g.cell_start + row + wb + 1));
        x0 = max(x0, 0);
        x1 = min(x1, Gx - 1);
      }
      visit(tg, false, __ldg(g.cell_start + row + x0), __ldg(g.cell_start + row + x1 + 1));
    }
  }
}

// FP32 candidate test with FP64 recheck inside the guard band.  The outside
// cell holds arbitrary positions (any image may be nearest), so its
// candidates always take the FP64 path.
__device__ __forceinline__ bool pair_hit(const GridDev &g, const QueryGeom &Q, const Target &t,
                                         const Band &B, const float4 &p) {
  if (t.outside) return canon_d2(Q.q, p, g) <= B.r2;
  const float dx = p.x - t.qx, dy = p.y - t.qy, dz = p.z - t.qz;
  const float d2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
  const float lo = t.wrapped ? B.lo_w : B.lo;
  const float hi = t.wrapped ? B.hi_w : B.hi;
  if (d2 <= lo) return true;
  if (d2 > hi) return false;
  return canon_d2(Q.q, p, g) <= B.r2;
}

}  // namespace si
