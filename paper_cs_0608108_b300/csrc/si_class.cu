// Sub-cell class tables for the per-query radius walk.
//
// Sec. III.A selects one of 64 specialized offset tables from 6 bits that
// compare frac(d) with the query's distances zeta to its own cell faces, and
// tests the remaining cells at run time (Eq. 1).  On the GPU every run-time
// test costs each lane of a warp, so the selection is refined: the query's
// sub-cell position (phi_x, phi_y, phi_z) in [0,1)^3 is cut into q^3 classes,
// and class (i, j, k) lists, center to edge (by b^2, Sec. II.A), exactly the
// offsets whose cell lies within d of the class's sub-box -- a superset of the
// cells any query of the class needs, and no cell the walk could skip for
// every query of the class.  Entries carry bit 63 when the whole target cell
// lies within d of every point of the sub-box (unconditional inclusion).
// The tables depend on d, so they are rebuilt when the radius changes; their
// device storage is sized for r_max when the grid is created.
#include <algorithm>
#include <cmath>

#include "si_host.h"

namespace si {

int class_q_for(double dmax) { return dmax <= 4.5 ? 8 : 4; }

int64_t class_capacity(const Lattice &lat, int64_t table_entries) {
  const int q = class_q_for(std::sqrt((double)lat.n_max + 1.0));
  const int64_t cap = table_entries * (int64_t)q * q * q;
  return cap <= (int64_t)kClassCapMax ? cap : 0;
}

// Entry layout (one per x-row run of cells):
//   bits  0..47  the run's (0, oy, oz) offset in unpacked form ((w+1)-bit fields)
//   bits 48..55  ox_lo, the run's first x offset (int8)
//   bits 56..62  run length in cells (1..127)
//   bit  63      every cell of the run lies wholly within d of the sub-box
void build_class_tables(const Lattice &lat, double dg, int q, std::vector<unsigned long long> &ent,
                        std::vector<int> &begin) {
  const int W = lat.W;
  const int pos[3] = {0, W + lat.w[0], lat.w[0] + lat.w[1]};
  const int reach = (int)std::floor(dg) + 1;
  int lim[3];
  for (int a = 0; a < 3; ++a)
    lim[a] = ((lat.cyc >> a) & 1u) ? reach : std::min(reach, (1 << lat.w[a]) - 1);
  const double m = lat.eps;                 // sub-box grown by the binning margin
  const double d_in = dg - 2.0 * lat.eps;   // inclusion uses d shrunk by the margin
  struct Run {
    int b2;                                 // smallest b^2 of the run's cells (center-to-edge order)
    int oy, oz, lo, len;
    bool full;
  };
  ent.clear();
  begin.assign((size_t)q * q * q + 1, 0);
  std::vector<Run> runs;
  for (int k = 0; k < q; ++k)
    for (int j = 0; j < q; ++j)
      for (int i = 0; i < q; ++i) {
        const int c = (k * q + j) * q + i;
        begin[c] = (int)ent.size();
        const int idx[3] = {i, j, k};
        double lo[3], hi[3];
        for (int a = 0; a < 3; ++a) {
          lo[a] = (double)idx[a] / q - m;
          hi[a] = (double)(idx[a] + 1) / q + m;
        }
        runs.clear();
        for (int oz = -lim[2]; oz <= lim[2]; ++oz)
          for (int oy = -lim[1]; oy <= lim[1]; ++oy) {
            // cells of this row within dg of the sub-box form one x-interval
            Run r{1 << 30, oy, oz, 0, 0, true};
            for (int ox = -lim[0]; ox <= lim[0]; ++ox) {
              const int o[3] = {ox, oy, oz};
              double g2 = 0.0, far2 = 0.0;
              int b2 = 0;
              for (int a = 0; a < 3; ++a) {
                const double gap =
                    std::max(std::max((double)o[a] - hi[a], lo[a] - (double)(o[a] + 1)), 0.0);
                g2 += gap * gap;
                const double far = std::max((double)(o[a] + 1) - lo[a], hi[a] - (double)o[a]);
                far2 += far * far;
                const int bb = std::max(std::abs(o[a]) - 1, 0);
                b2 += bb * bb;
              }
              if (g2 > dg * dg) continue;
              if (r.len == 0) r.lo = ox;
              r.len = ox - r.lo + 1;          // convex region: the kept ox are contiguous
              r.b2 = std::min(r.b2, b2);
              r.full = r.full && d_in > 0.0 && far2 <= d_in * d_in;
            }
            if (r.len > 0) runs.push_back(r);
          }
        std::stable_sort(runs.begin(), runs.end(), [](const Run &x, const Run &y) { return x.b2 < y.b2; });
        for (const Run &r : runs) {
          unsigned long long u = 0;
          const int o[3] = {0, r.oy, r.oz};
          for (int a = 1; a < 3; ++a) {
            const unsigned long long fieldmask = (1ull << (lat.w[a] + 1)) - 1ull;
            u |= ((unsigned long long)(long long)o[a] & fieldmask) << pos[a];
          }
          u |= (unsigned long long)(unsigned char)(signed char)r.lo << 48;
          u |= (unsigned long long)(r.len & 127) << 56;
          if (r.full) u |= 1ull << 63;
          ent.push_back(u);
        }
      }
  begin[(size_t)q * q * q] = (int)ent.size();
}

// x-row runs of the cells within d of a box of B x B x B cells (offsets
// relative to the box's lowest cell, box [0, B)^3 grown by the binning
// margin), in the same entry format; B = 1 gives the cell-level rows.
void build_box_rows(const Lattice &lat, double dg, int B, std::vector<unsigned long long> &ent) {
  const int W = lat.W;
  const int pos[3] = {0, W + lat.w[0], lat.w[0] + lat.w[1]};
  const int reach = (int)std::floor(dg) + 1;
  const double m = lat.eps;
  struct Run {
    int b2, oy, oz, lo, len;
  };
  std::vector<Run> runs;
  for (int oz = -reach; oz <= B - 1 + reach; ++oz)
    for (int oy = -reach; oy <= B - 1 + reach; ++oy) {
      Run r{1 << 30, oy, oz, 0, 0};
      for (int ox = -reach; ox <= B - 1 + reach; ++ox) {
        const int o[3] = {ox, oy, oz};
        double g2 = 0.0;
        int b2 = 0;
        for (int a = 0; a < 3; ++a) {
          const double gap = std::max(std::max((double)o[a] - ((double)B + m), -m - (double)(o[a] + 1)), 0.0);
          g2 += gap * gap;
          const int bb = std::max(std::max(o[a] - B, -o[a] - 1), 0);
          b2 += bb * bb;
        }
        if (g2 > dg * dg) continue;
        if (r.len == 0) r.lo = ox;
        r.len = ox - r.lo + 1;   // convex region: the kept ox are contiguous
        r.b2 = std::min(r.b2, b2);
      }
      if (r.len > 0) runs.push_back(r);
    }
  std::stable_sort(runs.begin(), runs.end(), [](const Run &x, const Run &y) { return x.b2 < y.b2; });
  ent.clear();
  for (const Run &r : runs) {
    unsigned long long u = 0;
    const int o[3] = {0, r.oy, r.oz};
    for (int a = 1; a < 3; ++a) {
      const unsigned long long fieldmask = (1ull << (lat.w[a] + 1)) - 1ull;
      u |= ((unsigned long long)(long long)o[a] & fieldmask) << pos[a];
    }
    u |= (unsigned long long)(unsigned char)(signed char)r.lo << 48;
    u |= (unsigned long long)(r.len & 127) << 56;
    ent.push_back(u);
  }
}

}  // namespace si

using namespace si;

// Cell-level rows for the heavy-cell kernel: the class table of the whole
// cell (q = 1), i.e. the x-row runs of every cell within d of the query
// cell, which are the cells with b^2 <= floor(d^2) (Sec. II.A).
bool si_grid::ensure_cell_rows(float dg, cudaStream_t st) {
  if (crow_dg == dg) return true;
  std::vector<int> begin;
  build_class_tables(lat, (double)dg, 1, crow_host, begin);
  if ((int64_t)crow_host.size() > crow_cap) return false;
  if (cudaMemcpyAsync(crow, crow_host.data(), crow_host.size() * sizeof(unsigned long long),
                      cudaMemcpyHostToDevice, st) != cudaSuccess)
    return false;
  if (cudaStreamSynchronize(st) != cudaSuccess) return false;
  n_crow = (int)crow_host.size();
  crow_dg = dg;
  return true;
}

// Rows of the 2 x 2 x 2 cell groups of the heavy-cell kernel (si_group.cu);
// false when the lattice is too small for a group's rows to stay distinct
// (then every heavy cell is served on its own).
bool si_grid::ensure_group_rows(float dg, cudaStream_t st) {
  if (grow_dg == dg) return n_grow > 0;
  grow_dg = dg;
  n_grow = 0;
  const int reach = (int)std::floor((double)dg) + 1;
  for (int a = 0; a < 3; ++a)
    if (lat.w[a] < 1 || (1 << lat.w[a]) < 2 * reach + 2) return false;
  build_box_rows(lat, (double)dg, 2, grow_host);
  if ((int64_t)grow_host.size() > grow_cap || 2 * (int64_t)grow_host.size() + 1 > kGroupTCap) return false;
  if (cudaMemcpyAsync(grow, grow_host.data(), grow_host.size() * sizeof(unsigned long long),
                      cudaMemcpyHostToDevice, st) != cudaSuccess)
    return false;
  if (cudaStreamSynchronize(st) != cudaSuccess) return false;
  n_grow = (int)grow_host.size();
  return true;
}

// Make the grid's class tables match grown distance dg (cell units); returns
// false when they cannot (capacity), in which case the Eq. 2 walk is used.
bool si_grid::ensure_classes(float dg, cudaStream_t st) {
  if (cls_cap <= 0) return false;
  if (cls_dg == dg) return true;
  // q = 4 when the whole table fits a block's shared memory (the per-query
  // kernels stage it there); otherwise the finer q of the grid, read from L2
  int q = 4;
  build_class_tables(lat, (double)dg, q, cls_host, cls_begin_host);
  cls_smem_bytes = cls_host.size() * sizeof(unsigned long long) + cls_begin_host.size() * sizeof(int);
  if (cls_smem_bytes > kClassSmemMax) {
    q = class_q_for(std::sqrt((double)lat.n_max + 1.0));
    build_class_tables(lat, (double)dg, q, cls_host, cls_begin_host);
    cls_smem_bytes = 0;
  }
  if ((int64_t)cls_host.size() > cls_cap) return false;
  if (cudaMemcpyAsync(cls, cls_host.data(), cls_host.size() * sizeof(unsigned long long),
                      cudaMemcpyHostToDevice, st) != cudaSuccess)
    return false;
  if (cudaMemcpyAsync(cls_begin, cls_begin_host.data(), cls_begin_host.size() * sizeof(int),
                      cudaMemcpyHostToDevice, st) != cudaSuccess)
    return false;
  // the host vectors are reused only after the copies have been consumed
  if (cudaStreamSynchronize(st) != cudaSuccess) return false;
  cls_dg = dg;
  cls_q = q;
  return true;
}
