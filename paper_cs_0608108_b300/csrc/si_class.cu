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

void build_class_tables(const Lattice &lat, double dg, int q, std::vector<unsigned long long> &ent,
                        std::vector<int> &begin) {
  const int W = lat.W;
  const int pos[3] = {0, W + lat.w[0], lat.w[0] + lat.w[1]};
  const int reach = (int)std::floor(dg) + 1;
  int lim[3];
  for (int a = 0; a < 3; ++a)
    lim[a] = ((lat.cyc >> a) & 1u) ? reach : std::min(reach, (1 << lat.w[a]) - 1);
  struct Off {
    int b2, o[3];
  };
  std::vector<Off> offs;
  for (int oz = -lim[2]; oz <= lim[2]; ++oz)
    for (int oy = -lim[1]; oy <= lim[1]; ++oy)
      for (int ox = -lim[0]; ox <= lim[0]; ++ox) {
        const int o[3] = {ox, oy, oz};
        int b2 = 0;
        for (int a = 0; a < 3; ++a) {
          const int b = std::max(std::abs(o[a]) - 1, 0);
          b2 += b * b;
        }
        if ((double)b2 <= dg * dg) offs.push_back({b2, {ox, oy, oz}});
      }
  std::stable_sort(offs.begin(), offs.end(), [](const Off &x, const Off &y) { return x.b2 < y.b2; });
  const double m = lat.eps;                 // sub-box grown by the binning margin
  const double d_in = dg - 2.0 * lat.eps;   // inclusion uses d shrunk by the margin
  ent.clear();
  begin.assign((size_t)q * q * q + 1, 0);
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
        for (const Off &f : offs) {
          double g2 = 0.0, far2 = 0.0;
          for (int a = 0; a < 3; ++a) {
            const double gap = std::max(std::max((double)f.o[a] - hi[a], lo[a] - (double)(f.o[a] + 1)), 0.0);
            g2 += gap * gap;
            const double far = std::max((double)(f.o[a] + 1) - lo[a], hi[a] - (double)f.o[a]);
            far2 += far * far;
          }
          if (g2 > dg * dg) continue;
          unsigned long long u = 0;
          for (int a = 0; a < 3; ++a) {
            const unsigned long long fieldmask = (1ull << (lat.w[a] + 1)) - 1ull;
            u |= ((unsigned long long)(long long)f.o[a] & fieldmask) << pos[a];
          }
          if (d_in > 0.0 && far2 <= d_in * d_in) u |= 1ull << 63;
          ent.push_back(u);
        }
      }
  begin[(size_t)q * q * q] = (int)ent.size();
}

}  // namespace si

using namespace si;

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
