// Grid object: lattice validation, the offset tables (Sec. II.A, Sec. III.A),
// binning of points into cells (Sec. I, Sec. II.B), status handling.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <new>

#include "si_host.h"
#include "si_sort.cuh"

namespace si {

// ---------------------------------------------------------------------------
// Errors, launch counting
// ---------------------------------------------------------------------------
static thread_local std::string t_last_error;
static std::atomic<long long> g_launches{0};

si_status fail(si_status s, const std::string &msg) {
  t_last_error = msg;
  return s;
}

si_status cuda_fail(cudaError_t e, const char *what) {
  t_last_error = std::string(what) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? SI_ERR_OOM : SI_ERR_CUDA;
}

void count_launch(int k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

// ---------------------------------------------------------------------------
// Optional per-kernel event timing
// ---------------------------------------------------------------------------
namespace {
struct ProfRec {
  const char *name;
  cudaEvent_t a, b;
};
std::mutex g_prof_mu;
bool g_prof_on = false;
std::vector<ProfRec> g_prof_recs;
std::vector<cudaEvent_t> g_prof_pool;
cudaEvent_t g_prof_pending = nullptr;

cudaEvent_t prof_event() {
  if (!g_prof_pool.empty()) {
    cudaEvent_t e = g_prof_pool.back();
    g_prof_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}
}  // namespace

void prof_begin(cudaStream_t st) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (!g_prof_on) return;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;
  cudaEvent_t e = prof_event();
  if (e && cudaEventRecord(e, st) == cudaSuccess) g_prof_pending = e;
}

void prof_end(cudaStream_t st, const char *name) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (!g_prof_on || !g_prof_pending) return;
  cudaEvent_t e = prof_event();
  if (e && cudaEventRecord(e, st) == cudaSuccess) g_prof_recs.push_back({name, g_prof_pending, e});
  g_prof_pending = nullptr;
}

// ---------------------------------------------------------------------------
// Lattice
// ---------------------------------------------------------------------------
static constexpr double kU = 5.9604644775390625e-08;   // 2^-24, float32 unit roundoff

si_status make_lattice(const si_grid_desc &d, double r_for_tables, Lattice &lat) {
  int W = 0;
  for (int a = 0; a < 3; ++a) {
    const int w = d.log2_cells[a];
    if (w < 2 || w > 10) return fail(SI_ERR_INVALID, "log2_cells must be in [2, 10] on every axis");
    lat.w[a] = w;
    W += w;
  }
  if (W > 27) return fail(SI_ERR_INVALID, "lattice too large: sum of log2_cells must be <= 27");
  if (d.cyclic_mask > 7u) return fail(SI_ERR_INVALID, "cyclic_mask has bits beyond x, y, z");
  if (!(d.cell_size > 0.f) || !std::isfinite(d.cell_size))
    return fail(SI_ERR_INVALID, "cell_size must be positive and finite");
  for (int a = 0; a < 3; ++a)
    if (!std::isfinite(d.origin[a])) return fail(SI_ERR_INVALID, "origin must be finite");
  lat.W = W;
  lat.cyc = d.cyclic_mask;
  lat.s = d.cell_size;
  lat.inv_s = (float)(1.0 / (double)d.cell_size);
  int gmax = 0;
  for (int a = 0; a < 3; ++a) {
    lat.origin[a] = d.origin[a];
    lat.L[a] = d.cell_size * (float)(1 << lat.w[a]);   // power-of-two scaling: exact
    if (!std::isfinite(lat.L[a])) return fail(SI_ERR_INVALID, "box side overflows float32");
    gmax = std::max(gmax, 1 << lat.w[a]);
  }
  // Margin (cell units) covering float32 binning and cell arithmetic: a
  // coordinate in cell units (<= G) carries <= ~3 u G error from the
  // subtraction, the rounded 1/s and the product; the query's sub-cell
  // position the same; t^2, d^2 and d = r/s add a few u G more.  64 u G is a
  // comfortable bound, and 1e-6 covers tiny lattices.
  lat.eps = 64.0 * kU * gmax + 1e-6;
  const bool unbounded = !(r_for_tables > 0.0) || std::isinf(r_for_tables);
  lat.unbounded = unbounded;
  if (unbounded) {
    if (lat.cyc) return fail(SI_ERR_INVALID, "unbounded r_max needs every axis non-cyclic");
    int n = 0;
    for (int a = 0; a < 3; ++a) n += ((1 << lat.w[a]) - 2) * ((1 << lat.w[a]) - 2);
    lat.n_max = n;
  } else {
    const double dmax = r_for_tables * (double)lat.inv_s * (1.0 + 1e-6) + 2.0 * lat.eps + 1e-6;
    if (dmax > 4096.0) return fail(SI_ERR_INVALID, "radius too large for the lattice tables");
    lat.n_max = (int)std::floor(dmax * dmax);
    const int reach = (int)std::floor(std::sqrt((double)lat.n_max)) + 1;
    for (int a = 0; a < 3; ++a)
      if (((lat.cyc >> a) & 1u) && 2 * reach + 1 > (1 << lat.w[a]))
        return fail(SI_ERR_INVALID,
                    "radius wraps a cyclic axis onto itself (needs 2*(floor(r/s)+1)+1 <= cells)");
    // on non-cyclic axes offsets beyond G-1 always leave the region
    int nlim = 0;
    for (int a = 0; a < 3; ++a) {
      const int lim = std::min(reach, (1 << lat.w[a]) - 1);
      const int b = std::max(lim - 1, 0);
      nlim += b * b;
    }
    lat.n_max = std::min(lat.n_max, nlim);
  }
  return SI_OK;
}

// ---------------------------------------------------------------------------
// Tables (Sec. II.A; Sec. III.A Eq. 1-2)
// ---------------------------------------------------------------------------
static int isqrt_i(int n) {
  int r = (int)std::sqrt((double)n);
  while (r * r > n) --r;
  while ((r + 1) * (r + 1) <= n) ++r;
  return r;
}

bool build_tables(const int w[3], unsigned cyc, int n_max, HostTables &out, std::string &err) {
  const int W = w[0] + w[1] + w[2];
  const int pos[3] = {0, W + w[0], w[0] + w[1]};   // x, y, z fields in unpacked form
  const int reach = isqrt_i(n_max) + 1;
  int lim[3];
  for (int a = 0; a < 3; ++a) {
    const int G = 1 << w[a];
    if ((cyc >> a) & 1u) {
      if (2 * reach + 1 > G) {
        err = "table would wrap a cyclic axis onto itself";
        return false;
      }
      lim[a] = reach;
    } else {
      lim[a] = std::min(reach, G - 1);
    }
  }
  struct Raw {
    int b2, ox, oy, oz;
  };
  std::vector<Raw> raw;
  for (int oz = -lim[2]; oz <= lim[2]; ++oz)
    for (int oy = -lim[1]; oy <= lim[1]; ++oy)
      for (int ox = -lim[0]; ox <= lim[0]; ++ox) {
        const int bx = std::max(std::abs(ox) - 1, 0), by = std::max(std::abs(oy) - 1, 0),
                  bz = std::max(std::abs(oz) - 1, 0);
        const int b2 = bx * bx + by * by + bz * bz;
        if (b2 <= n_max) raw.push_back({b2, ox, oy, oz});
      }
  // center to edge: by b2, then (z, y, x) for a fixed order
  std::stable_sort(raw.begin(), raw.end(), [](const Raw &a, const Raw &b) { return a.b2 < b.b2; });
  auto encode = [&](const Raw &r) {
    TabEntry e;
    const int o[3] = {r.ox, r.oy, r.oz};
    unsigned long long u = 0;
    unsigned dirs = 0;
    for (int a = 0; a < 3; ++a) {
      const unsigned long long fieldmask = (1ull << (w[a] + 1)) - 1ull;   // w+1 bits
      u |= ((unsigned long long)(long long)o[a] & fieldmask) << pos[a];
      if (o[a] > 0) dirs |= 1u << (2 * a);
      if (o[a] < 0) dirs |= 1u << (2 * a + 1);
    }
    e.unp = u;
    e.ox = (signed char)std::max(-127, std::min(127, r.ox));
    e.oy = (signed char)std::max(-127, std::min(127, r.oy));
    e.oz = (signed char)std::max(-127, std::min(127, r.oz));
    e.dirs = (unsigned char)dirs;
    e.b2 = r.b2;
    return e;
  };
  for (int a = 0; a < 3; ++a)
    if (lim[a] > 127) {
      err = "offset beyond 127 cells is not representable";
      return false;
    }
  out.tab.clear();
  out.tab.reserve(raw.size());
  for (const Raw &r : raw) out.tab.push_back(encode(r));
  out.n_max = n_max;
  out.tab_end.assign(n_max + 1, 0);
  {
    size_t i = 0;
    for (int n = 0; n <= n_max; ++n) {
      while (i < out.tab.size() && out.tab[i].b2 <= n) ++i;
      out.tab_end[n] = (int)i;
    }
  }
  // x-rows of the sphere for the K-nearest walk: every (oy, oz) whose y-z
  // minimum bound is within n_max, center to edge
  {
    struct RowRaw {
      int b2, oy, oz;
    };
    std::vector<RowRaw> rr;
    for (int oz = -lim[2]; oz <= lim[2]; ++oz)
      for (int oy = -lim[1]; oy <= lim[1]; ++oy) {
        const int by = std::max(std::abs(oy) - 1, 0), bz = std::max(std::abs(oz) - 1, 0);
        if (by * by + bz * bz <= n_max) rr.push_back({by * by + bz * bz, oy, oz});
      }
    std::stable_sort(rr.begin(), rr.end(), [](const RowRaw &a, const RowRaw &b) { return a.b2 < b.b2; });
    out.rows.clear();
    for (const RowRaw &r : rr) {
      RowEntry e;
      unsigned long long u = 0;
      const int o[3] = {0, r.oy, r.oz};
      for (int a = 1; a < 3; ++a) {
        const unsigned long long fieldmask = (1ull << (w[a] + 1)) - 1ull;
        u |= ((unsigned long long)(long long)o[a] & fieldmask) << pos[a];
      }
      e.unp = u;
      e.oy = (short)r.oy;
      e.oz = (short)r.oz;
      e.b2 = r.b2;
      out.rows.push_back(e);
    }
    out.row_end.assign((size_t)n_max + 1, 0);
    for (const RowRaw &r : rr) ++out.row_end[(size_t)r.b2];
    for (int n = 1; n <= n_max; ++n) out.row_end[(size_t)n] += out.row_end[(size_t)n - 1];
    out.row_lim_x = lim[0];
  }
  // Specialized tables: for shell fl (fl^2 <= b2 < (fl+1)^2) and the 6-bit
  // mask of directions where f < zeta, drop every non-center offset whose
  // directions all have their bit set (Eq. 2: then t > d).
  const int shells = std::min(isqrt_i(n_max) + 1, kSpecShellsMax);
  out.spec_shells = shells;
  out.spec.clear();
  out.spec_begin.assign((size_t)shells * 64, 0);
  out.spec_end.assign((size_t)64 * shells * shells, 0);
  for (int fl = 0; fl < shells; ++fl) {
    const int lo = fl * fl;
    const int hi = std::min((fl + 1) * (fl + 1) - 1, n_max);
    const int b0 = lo > 0 ? out.tab_end[lo - 1] : 0;
    const int b1 = out.tab_end[hi];
    for (int mask = 0; mask < 64; ++mask) {
      out.spec_begin[fl * 64 + mask] = (int)out.spec.size();
      int n = lo;
      const size_t endbase = (size_t)64 * fl * fl + (size_t)mask * (2 * fl + 1);
      for (int i = b0; i < b1; ++i) {
        const TabEntry &e = out.tab[i];
        while (n < e.b2) {
          out.spec_end[endbase + (n - lo)] = (int)out.spec.size();
          ++n;
        }
        const bool center = e.dirs == 0;
        const bool rejected = !center && ((e.dirs & ~(unsigned)mask) == 0);
        if (!rejected) out.spec.push_back(e);
      }
      for (; n <= lo + 2 * fl; ++n) out.spec_end[endbase + (n - lo)] = (int)out.spec.size();
    }
  }
  return true;
}

template <typename T>
static si_status upload(const std::vector<T> &h, T *&d) {
  const size_t bytes = std::max<size_t>(h.size(), 1) * sizeof(T);
  SI_CUDA_TRY(cudaMalloc((void **)&d, bytes));
  if (!h.empty()) SI_CUDA_TRY(cudaMemcpy(d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
  return SI_OK;
}

si_status upload_tables(const HostTables &h, DevTables &d) {
  si_status s;
  if ((s = upload(h.tab, d.tab)) != SI_OK) return s;
  if ((s = upload(h.tab_end, d.tab_end)) != SI_OK) return s;
  if ((s = upload(h.spec, d.spec)) != SI_OK) return s;
  if ((s = upload(h.spec_begin, d.spec_begin)) != SI_OK) return s;
  if ((s = upload(h.spec_end, d.spec_end)) != SI_OK) return s;
  if ((s = upload(h.rows, d.rows)) != SI_OK) return s;
  d.n_rows = (int)h.rows.size();
  d.row_end = h.row_end;
  d.row_lim_x = h.row_lim_x;
  d.n_max = h.n_max;
  d.spec_shells = h.spec_shells;
  d.entries = (int64_t)h.tab.size();
  return SI_OK;
}

void free_tables(DevTables &d) {
  cudaFree(d.tab);
  cudaFree(d.tab_end);
  cudaFree(d.spec);
  cudaFree(d.spec_begin);
  cudaFree(d.spec_end);
  cudaFree(d.rows);
  d = DevTables();
}

void fill_griddev(const Lattice &lat, const DevTables &t, GridDev &g) {
  g.ox = lat.origin[0];
  g.oy = lat.origin[1];
  g.oz = lat.origin[2];
  g.inv_s = lat.inv_s;
  g.Lx = lat.L[0];
  g.Ly = lat.L[1];
  g.Lz = lat.L[2];
  g.wx = lat.w[0];
  g.wy = lat.w[1];
  g.wz = lat.w[2];
  g.W = lat.W;
  g.cyc = lat.cyc;
  g.outside = 1u << lat.W;
  g.qpos = nullptr;   // set with the arrays (si_grid::dev, or the query-center path)
  g.qid = nullptr;
  g.q_agents = 1;
  const int pos[3] = {0, lat.W + lat.w[0], lat.w[0] + lat.w[1]};
  unsigned long long valid = 0, guard[3], non = 0;
  for (int a = 0; a < 3; ++a) {
    valid |= ((1ull << lat.w[a]) - 1ull) << pos[a];
    guard[a] = 1ull << (pos[a] + lat.w[a]);
    if (!((lat.cyc >> a) & 1u)) non |= guard[a];
  }
  g.valid = valid;
  g.gx = guard[0];
  g.gy = guard[1];
  g.gz = guard[2];
  g.guard_non = non;
  g.tab = t.tab;
  g.tab_end = t.tab_end;
  g.n_max = t.n_max;
  g.spec = t.spec;
  g.spec_begin = t.spec_begin;
  g.spec_end = t.spec_end;
  g.spec_shells = t.spec_shells;
  g.eps = (float)lat.eps;
  g.cls = nullptr;
  g.cls_begin = nullptr;
  g.cls_q = 0;
  g.crow = nullptr;
  g.n_crow = 0;
  g.rows = t.rows;
  g.n_rows = t.n_rows;
  g.row_lim_x = t.row_lim_x;
}

// ---------------------------------------------------------------------------
// FP32 guard bands.
// A pair compared directly: dx = fl(xj - xi) has relative error <= u; three
// squares and two sums add <= ~5u more, so |d2f - D2| <= 8u D2.  A pair
// compared through a wrapped image uses q' = fl(q -/+ L) (absolute error
// <= u (|q| + L)) then dx = fl(xj - q'): |dx err| <= u (Qmax + L) + u |dx|,
// giving |d2f - D2| <= 2 sqrt(3) u (Qmax + L) D + 8u D2.  Bands use 1.5x these
// bounds and never less than the stated relative band 1e-6.
// ---------------------------------------------------------------------------
static double qmax_of(const Lattice &lat) {
  double q = 0.0;
  for (int a = 0; a < 3; ++a)
    if ((lat.cyc >> a) & 1u)
      q = std::max(q, std::max(std::fabs((double)lat.origin[a]),
                               std::fabs((double)lat.origin[a] + (double)lat.L[a])) +
                          (double)lat.L[a]);
  return q;
}

static float round_down(double v) {
  float f = (float)v;
  if ((double)f > v) f = std::nextafter(f, -INFINITY);
  return f;
}
static float round_up(double v) {
  float f = (float)v;
  if ((double)f < v) f = std::nextafter(f, INFINITY);
  return f;
}

Band make_band(const Lattice &lat, float r) {
  Band b;
  const double r2 = (double)r * (double)r;
  b.r2 = r2;
  const double g = std::max(1e-6, 1.5 * 8.0 * kU);
  const double gw = g + 1.5 * (2.0 * std::sqrt(3.0) * kU * qmax_of(lat) / std::max((double)r, 1e-300) +
                               8.0 * kU);
  if (r2 < 1e-30) {
    // tiny radius: squares may underflow in float32; send everything near to FP64
    b.lo = b.lo_w = -1.f;
    b.hi = b.hi_w = round_up(std::max(r2 * (1.0 + gw), 1e-30));
    return b;
  }
  b.lo = round_down(r2 * (1.0 - g));
  b.hi = round_up(r2 * (1.0 + g));
  b.lo_w = round_down(r2 * (1.0 - std::min(gw, 0.5)));
  b.hi_w = round_up(r2 * (1.0 + gw));
  return b;
}

PairBand make_pair_band(const Lattice &lat) {
  PairBand p;
  p.c2 = (float)(2.0 * 1.5 * 8.0 * kU);
  p.c1 = (float)(2.0 * 1.5 * 2.0 * std::sqrt(3.0) * kU * qmax_of(lat));
  return p;
}

// ---------------------------------------------------------------------------
// Binning kernels (Sec. I: one cell per object; Sec. II.B: packed index)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_bin_key(const float4 *__restrict__ pos, int n, GridDev g,
                                                 uint2 *__restrict__ key_slot,
                                                 int *__restrict__ count) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float4 p = __ldg(pos + i);
  bool out = false, bad = false;
  const int cx = axis_cell(p.x, g.ox, g.Lx, g.inv_s, g.wx, g.cyc & 1u, out, bad);
  const int cy = axis_cell(p.y, g.oy, g.Ly, g.inv_s, g.wy, (g.cyc >> 1) & 1u, out, bad);
  const int cz = axis_cell(p.z, g.oz, g.Lz, g.inv_s, g.wz, (g.cyc >> 2) & 1u, out, bad);
  if (bad) atomicOr(g.status, ST_INVALID);
  const unsigned key = out ? g.outside : pack3(cx, cy, cz, g);
  const int slot = atomicAdd(count + key, 1);
  key_slot[i] = make_uint2(key, (unsigned)slot);
}

// Scatter into cell order (points of a cell in atomic arrival order).
__global__ void __launch_bounds__(256) k_bin_scatter(const float4 *__restrict__ pos, int n,
                                                     const uint2 *__restrict__ key_slot,
                                                     const int *__restrict__ start,
                                                     float4 *__restrict__ spos,
                                                     int *__restrict__ perm) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint2 ks = key_slot[i];
  const int dst = __ldg(start + ks.x) + (int)ks.y;
  spos[dst] = __ldg(pos + i);
  perm[dst] = i;
}

// ---------------------------------------------------------------------------
// Order the points of every cell by input index.  The scatter places them in
// atomic arrival order; ordered cells make every later step deterministic and
// give the cell kernel runs of candidates already sorted by id.  Only the
// permutation is sorted; positions are then gathered again from the input.
// ---------------------------------------------------------------------------
constexpr int kOrderLocal = 16;      // cells up to this size: one thread, insertion sort
constexpr int kOrderWarps = 8;
constexpr int kOrderWarpCap = 2048;  // cells up to this size: one warp, shared memory
constexpr int kOrderBlockCap = 16384;

// The same pass classifies every non-empty cell (cell_class; one thread per
// cell, so that the neighbours' cell starts are contiguous loads): heavy
// cells are listed by key, the query slots of dense cells and of light cells
// are queued (the light ones a block's worth at a time, in cell order), and
// every slot gets its cell's class byte.
__global__ void __launch_bounds__(256) k_cell_order(const int *__restrict__ start, int n_cells,
                                                    const float4 *__restrict__ pos, float4 *spos,
                                                    int *perm, int *bigq, unsigned char *__restrict__ cell_cls,
                                                    unsigned char *__restrict__ slot_cls, int *__restrict__ heavy,
                                                    int *__restrict__ heavy_big, int *__restrict__ dense,
                                                    int *__restrict__ light, int wx, int wy, int wz) {
  __shared__ int scan[8];
  __shared__ int light_base;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  int b = 0, m = 0, k = kCellLight;
  if (c < n_cells) {
    b = __ldg(start + c);
    m = __ldg(start + c + 1) - b;
  }
  if (m >= 1) {
    k = cell_class(start, (unsigned)c, (unsigned)(n_cells - 1), wx, wy, wz);
    cell_cls[c] = (unsigned char)k;
    if (m <= kOrderLocal)
      for (int i = 0; i < m; ++i) slot_cls[b + i] = (unsigned char)k;
    if (k == kCellHeavy || k == kCellHeavyBig) {
      const int slot = atomicAdd(heavy, 1);
      heavy[1 + slot] = c;
      if (k == kCellHeavyBig) {
        const int sb = atomicAdd(heavy_big, 1);
        heavy_big[1 + sb] = c;
      }
    } else if (k == kCellDense) {
      const int slot = atomicAdd(dense, m);
      for (int i = 0; i < m; ++i) dense[1 + slot + i] = b + i;
    }
  }
  const int nl = (m >= 1 && k == kCellLight) ? m : 0;
  int total;
  const int ex = block_excl_scan_i(nl, total, scan);
  if (threadIdx.x == 0) light_base = total > 0 ? atomicAdd(light, total) : 0;
  __syncthreads();
  for (int i = 0; i < nl; ++i) light[1 + light_base + ex + i] = b + i;
  if (m < 2) return;
  if (m > kOrderLocal) {
    const int slot = atomicAdd(bigq, 1);
    bigq[1 + slot] = c;
    return;
  }
  int id[kOrderLocal];
  bool moved = false;
  for (int i = 0; i < m; ++i) {
    const int v = perm[b + i];
    int p = i;
    while (p > 0 && id[p - 1] > v) {
      id[p] = id[p - 1];
      --p;
    }
    id[p] = v;
    moved |= p != i;
  }
  if (!moved) return;
  for (int i = 0; i < m; ++i) {
    perm[b + i] = id[i];
    spos[b + i] = __ldg(pos + id[i]);
  }
}

__global__ void __launch_bounds__(kOrderWarps * 32) k_cell_order_big(const int *__restrict__ start,
                                                                    const float4 *__restrict__ pos,
                                                                    float4 *spos, int *perm,
                                                                    const int *__restrict__ bigq,
                                                                    int *hugeq, const unsigned char *cell_cls,
                                                                    unsigned char *__restrict__ slot_cls) {
  extern __shared__ int obuf[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int *buf = obuf + w * kOrderWarpCap;
  const int nq = bigq[0];
  for (int item = blockIdx.x * kOrderWarps + w; item < nq; item += gridDim.x * kOrderWarps) {
    const int c = bigq[1 + item];
    const int b = __ldg(start + c), m = __ldg(start + c + 1) - b;
    const unsigned char k = cell_cls[c];   // written by k_cell_order
    for (int i = lane; i < m; i += 32) slot_cls[b + i] = k;
    if (m > kOrderWarpCap) {
      if (lane == 0) {
        const int slot = atomicAdd(hugeq, 1);
        hugeq[1 + slot] = c;
      }
      continue;
    }
    for (int i = lane; i < m; i += 32) buf[i] = perm[b + i];
    __syncwarp();
    warp_sort(buf, m, lane, 0x7fffffff);
    __syncwarp();
    for (int i = lane; i < m; i += 32) {
      perm[b + i] = buf[i];
      spos[b + i] = __ldg(pos + buf[i]);
    }
    __syncwarp();
  }
}

__global__ void __launch_bounds__(512) k_cell_order_huge(const int *__restrict__ start,
                                                        const float4 *__restrict__ pos, float4 *spos,
                                                        int *perm, const int *__restrict__ hugeq) {
  extern __shared__ int obuf[];
  const int nq = hugeq[0];
  for (int item = blockIdx.x; item < nq; item += gridDim.x) {
    const int c = hugeq[1 + item];
    const int b = __ldg(start + c), m = __ldg(start + c + 1) - b;
    int *a = perm + b;
    if (m <= kOrderBlockCap) {
      for (int i = threadIdx.x; i < m; i += blockDim.x) obuf[i] = a[i];
      __syncthreads();
      bitonic_padded(obuf, m, threadIdx.x, blockDim.x, BlockSync());
      for (int i = threadIdx.x; i < m; i += blockDim.x) a[i] = obuf[i];
    } else {
      bitonic_padded(a, m, threadIdx.x, blockDim.x, BlockSync());
    }
    __syncthreads();
    for (int i = threadIdx.x; i < m; i += blockDim.x) spos[b + i] = __ldg(pos + a[i]);
    __syncthreads();
  }
}

si_status order_cells(const int *start, int64_t n_cells, const float4 *pos, float4 *spos, int *perm,
                      int *bigq, int *hugeq, unsigned char *cell_cls, unsigned char *slot_cls, int *heavy,
                      int *heavy_big, int *dense, int *light, const int w[3], cudaStream_t st) {
  SI_CUDA_TRY(cudaMemsetAsync(bigq, 0, sizeof(int), st));
  SI_CUDA_TRY(cudaMemsetAsync(hugeq, 0, sizeof(int), st));
  SI_KLAUNCH("k_cell_order", st,
             k_cell_order<<<(unsigned)((n_cells + 255) / 256), 256, 0, st>>>(start, (int)n_cells, pos, spos,
                                                                              perm, bigq, cell_cls, slot_cls,
                                                                              heavy, heavy_big, dense, light,
                                                                              w[0], w[1], w[2]));
  const size_t wsm = (size_t)kOrderWarps * kOrderWarpCap * sizeof(int);
  SI_CUDA_TRY(cudaFuncSetAttribute(k_cell_order_big, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)wsm));
  SI_KLAUNCH("k_cell_order_big", st,
             k_cell_order_big<<<148 * 2, kOrderWarps * 32, wsm, st>>>(start, pos, spos, perm, bigq, hugeq,
                                                                     cell_cls, slot_cls));
  const size_t bsm = (size_t)kOrderBlockCap * sizeof(int);
  SI_CUDA_TRY(cudaFuncSetAttribute(k_cell_order_huge, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bsm));
  SI_KLAUNCH("k_cell_order_huge", st,
             k_cell_order_huge<<<148, 512, bsm, st>>>(start, pos, spos, perm, hugeq));
  return SI_OK;
}

}  // namespace si

using namespace si;

si::GridDev si_grid::dev() const {
  GridDev g;
  fill_griddev(lat, tables, g);
  g.spos = spos;
  g.perm = perm;
  g.cell_start = cell_start;
  g.cell_cls = cell_cls;
  g.slot_cls = slot_cls;
  g.n = (int)n;
  g.status = status;
  g.cls = cls;
  g.cls_begin = cls_begin;
  g.cls_q = cls_q;
  g.crow = crow;
  g.n_crow = n_crow;
  g.qpos = spos;
  g.qid = perm;
  g.q_agents = 1;
  return g;
}

static void grid_free(si_grid *g) {
  if (!g) return;
  cudaFree(g->key_slot);
  cudaFree(g->cell_count);
  cudaFree(g->cell_start);
  cudaFree(g->cell_cls);
  cudaFree(g->slot_cls);
  cudaFree(g->spos);
  cudaFree(g->perm);
  cudaFree(g->scan_i32);
  cudaFree(g->scan_i64);
  cudaFree(g->status);
  cudaFree(g->longq);
  cudaFree(g->hugeq);
  cudaFree(g->heavy);
  cudaFree(g->heavy_big);
  cudaFree(g->heavy_big_built);
  cudaFree(g->groups);
  cudaFree(g->hsolo);
  cudaFree(g->xblock);
  cudaFree(g->xitems);
  cudaFree(g->grow);
  cudaFree(g->over);
  cudaFree(g->denseq);
  cudaFree(g->lightq);
  cudaFree(g->lstage);
  cudaFree(g->cell_rec);
  cudaFree(g->scr_top);
  cudaFree(g->scratch);
  cudaFree(g->counters);
  cudaFree(g->partial);
  cudaFree(g->cls);
  cudaFree(g->cls_begin);
  cudaFree(g->crow);
  cudaFree(g->cpos);
  cudaFree(g->cid);
  cudaFree(g->ckey);
  cudaFree(g->cbuck);
  cudaFree(g->cscan);
  cudaFree(g->cscan64);
  cudaFree(g->clist0);
  cudaFree(g->clist1);
  cudaFree(g->clong);
  cudaFree(g->chuge);
  cudaFree(g->cstage);
  cudaFree(g->ipos);
  cudaFree(g->io_pos);
  cudaFree(g->io_off);
  cudaFree(g->io_ids);
  if (g->h_pinned) cudaFreeHost(g->h_pinned);
  if (g->side) cudaStreamDestroy(g->side);
  if (g->fork_ev) cudaEventDestroy(g->fork_ev);
  if (g->join_ev) cudaEventDestroy(g->join_ev);
  free_tables(g->tables);
  delete g;
}

extern "C" si_status si_grid_create(const si_grid_desc *desc, int64_t n_capacity, si_grid **out) {
  if (!desc || !out) return fail(SI_ERR_INVALID, "null descriptor or output pointer");
  *out = nullptr;
  if (n_capacity < 0 || n_capacity > (int64_t)0x7fffffff - 1)
    return fail(SI_ERR_INVALID, "n_capacity must be in [0, 2^31 - 2]");
  si_grid *g = new (std::nothrow) si_grid();
  if (!g) return fail(SI_ERR_OOM, "host allocation failed");
  g->desc = *desc;
  si_status s = make_lattice(*desc, (double)desc->r_max, g->lat);
  if (s != SI_OK) {
    delete g;
    return s;
  }
  HostTables ht;
  std::string err;
  if (!build_tables(g->lat.w, g->lat.cyc, g->lat.n_max, ht, err)) {
    delete g;
    return fail(SI_ERR_INVALID, err);
  }
  g->cap = n_capacity;
  g->n_cells = (1ll << g->lat.W) + 1;
  const int64_t cap1 = std::max<int64_t>(n_capacity, 1);
  auto alloc = [&](void **p, size_t bytes) -> si_status {
    cudaError_t e = cudaMalloc(p, std::max<size_t>(bytes, 16));
    return e == cudaSuccess ? SI_OK : cuda_fail(e, "cudaMalloc (grid)");
  };
#define SI_ALLOC(ptr, bytes)                     \
  if ((s = alloc((void **)&(ptr), (bytes))) != SI_OK) { \
    grid_free(g);                                \
    return s;                                    \
  }
  SI_ALLOC(g->key_slot, cap1 * sizeof(uint2));
  SI_ALLOC(g->cell_count, g->n_cells * sizeof(int));
  SI_ALLOC(g->cell_start, (g->n_cells + 1) * sizeof(int));
  SI_ALLOC(g->cell_cls, g->n_cells);
  SI_ALLOC(g->slot_cls, cap1);
  SI_ALLOC(g->spos, cap1 * sizeof(float4));
  SI_ALLOC(g->perm, cap1 * sizeof(int));
  SI_ALLOC(g->scan_i32, scan_scratch_elems(g->n_cells + 1) * sizeof(int));
  SI_ALLOC(g->scan_i64, scan_scratch_elems(cap1 + 1) * sizeof(long long));
  SI_ALLOC(g->status, sizeof(int));
  SI_ALLOC(g->longq, (cap1 + 1) * sizeof(int));
  SI_ALLOC(g->hugeq, (cap1 + 1) * sizeof(int));
  SI_ALLOC(g->heavy, (cap1 / kHeavyMinDense + 2) * sizeof(int));
  SI_ALLOC(g->heavy_big, (cap1 / kHeavyMinDense + 2) * sizeof(int));
  SI_ALLOC(g->heavy_big_built, sizeof(int));
  SI_ALLOC(g->groups, (cap1 / kHeavyMinDense + 2) * sizeof(int));
  SI_ALLOC(g->hsolo, (cap1 / kHeavyMinDense + 2) * sizeof(int));
  SI_ALLOC(g->xblock, (cap1 / kHeavyMinDense + 2) * sizeof(int));
  // items of at most 8 queries of one heavy cell (a heavy cell holds >= 3 points)
  SI_ALLOC(g->xitems, (cap1 / 8 + cap1 / kHeavyMinDense + 2) * sizeof(int4));
  SI_ALLOC(g->over, (cap1 + 1) * sizeof(int));
  SI_ALLOC(g->denseq, (cap1 + 1) * sizeof(int));
  SI_ALLOC(g->lightq, (cap1 + 1) * sizeof(int));
  SI_ALLOC(g->cell_rec, g->n_cells * sizeof(long long));
  SI_ALLOC(g->scr_top, sizeof(unsigned long long));
  g->scr_cap = 4 * cap1;
  SI_ALLOC(g->scratch, g->scr_cap * sizeof(int));
  SI_ALLOC(g->counters, kCounterInts * sizeof(int));
  g->partial_len = (cap1 + 127) / 128 + 1;
  SI_ALLOC(g->partial, g->partial_len * sizeof(double));
#undef SI_ALLOC
  cudaError_t e = cudaMallocHost((void **)&g->h_pinned, 4 * sizeof(long long));
  if (e != cudaSuccess) {
    grid_free(g);
    return cuda_fail(e, "cudaMallocHost");
  }
  if ((s = upload_tables(ht, g->tables)) != SI_OK) {
    grid_free(g);
    return s;
  }
  g->tab_end_host = ht.tab_end;
  g->cls_cap = class_capacity(g->lat, (int64_t)ht.tab.size());
  if (g->cls_cap > 0) {
    const int q = class_q_for(std::sqrt((double)g->lat.n_max + 1.0));
    e = cudaMalloc((void **)&g->cls, g->cls_cap * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMalloc((void **)&g->cls_begin, ((size_t)q * q * q + 1) * sizeof(int));
    if (e != cudaSuccess) {
      grid_free(g);
      return cuda_fail(e, "cudaMalloc (class tables)");
    }
  }
  // cell-level rows: at most (2 reach + 1)^2 for the largest distance
  {
    const int reach = (int)std::floor(std::sqrt((double)g->lat.n_max + 1.0)) + 2;
    g->crow_cap = (int64_t)(2 * reach + 1) * (2 * reach + 1);
    e = cudaMalloc((void **)&g->crow, g->crow_cap * sizeof(unsigned long long));
    g->grow_cap = (int64_t)(2 * reach + 2) * (2 * reach + 2);
    if (e == cudaSuccess) e = cudaMalloc((void **)&g->grow, g->grow_cap * sizeof(unsigned long long));
    if (e != cudaSuccess) {
      grid_free(g);
      return cuda_fail(e, "cudaMalloc (cell rows)");
    }
  }
  e = cudaMemset(g->status, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(g->heavy, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(g->over, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(g->denseq, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(g->lightq, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(g->cell_start, 0, (g->n_cells + 1) * sizeof(int));
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    grid_free(g);
    return cuda_fail(e, "grid initialisation");
  }
  *out = g;
  return SI_OK;
}

extern "C" si_status si_grid_build(si_grid *g, const float *d_pos, int64_t n, void *stream) {
  if (!g) return fail(SI_ERR_INVALID, "null grid");
  if (n < 0 || n > g->cap) return fail(SI_ERR_INVALID, "n exceeds the grid's capacity");
  if (n > 0 && (!d_pos || ((uintptr_t)d_pos & 15u)))
    return fail(SI_ERR_INVALID, "positions must be a non-null, 16-byte aligned float4 array");
  cudaStream_t st = (cudaStream_t)stream;
  g->n = n;
  GridDev dv = g->dev();
  SI_CUDA_TRY(cudaMemsetAsync(g->cell_count, 0, g->n_cells * sizeof(int), st));
  if (n > 0) {
    SI_KLAUNCH("k_bin_key", st, k_bin_key<<<(unsigned)((n + 255) / 256), 256, 0, st>>>((const float4 *)d_pos, (int)n, dv,
                                                           g->key_slot, g->cell_count));
  }
  // cell_start[0] = 0; cell_start[c + 1] = sum of counts of cells 0..c
  SI_CUDA_TRY(cudaMemsetAsync(g->cell_start, 0, sizeof(int), st));
  SI_CUDA_TRY(cudaMemsetAsync(g->heavy, 0, sizeof(int), st));
  SI_CUDA_TRY(cudaMemsetAsync(g->denseq, 0, sizeof(int), st));
  SI_CUDA_TRY(cudaMemsetAsync(g->lightq, 0, sizeof(int), st));
  SI_CUDA_TRY(cudaMemsetAsync(g->heavy_big, 0, sizeof(int), st));
  si_status s = scan_inclusive_i32(g->cell_count, g->cell_start + 1, g->n_cells, g->scan_i32, st);
  if (s != SI_OK) return s;
  if (n > 0) {
    SI_KLAUNCH("k_bin_scatter", st, k_bin_scatter<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
        (const float4 *)d_pos, (int)n, g->key_slot, g->cell_start, g->spos, g->perm));
    // the query kernels are idle during a build: their queues serve as scratch
    s = order_cells(g->cell_start, g->n_cells, (const float4 *)d_pos, g->spos, g->perm, g->longq, g->hugeq,
                    g->cell_cls, g->slot_cls, g->heavy, g->heavy_big, g->denseq, g->lightq, g->lat.w,
                    st);
    if (s != SI_OK) return s;
    // the radius query appends the cells that overflow the small cell kernel
    SI_CUDA_TRY(cudaMemcpyAsync(g->heavy_big_built, g->heavy_big, sizeof(int), cudaMemcpyDeviceToDevice, st));
  }
  return SI_OK;
}

extern "C" si_status si_build_grid(const si_grid_desc *desc, const float *d_pos, int64_t n,
                                   void *stream, si_grid **out) {
  si_status s = si_grid_create(desc, n, out);
  if (s != SI_OK) return s;
  s = si_grid_build(*out, d_pos, n, stream);
  if (s != SI_OK) {
    si_grid_destroy(*out);
    *out = nullptr;
  }
  return s;
}

extern "C" si_status si_grid_sync(si_grid *g, void *stream) {
  if (!g) return fail(SI_ERR_INVALID, "null grid");
  cudaStream_t st = (cudaStream_t)stream;
  int *h = (int *)g->h_pinned;
  SI_CUDA_TRY(cudaMemcpyAsync(h, g->status, sizeof(int), cudaMemcpyDeviceToHost, st));
  SI_CUDA_TRY(cudaMemsetAsync(g->status, 0, sizeof(int), st));
  SI_CUDA_TRY(cudaStreamSynchronize(st));
  const int v = h[0];
  if (v & ST_INVALID)
    return fail(SI_ERR_INVALID, "a point lies outside a cyclic axis' box or is not finite");
  if (v & ST_INTERNAL) return fail(SI_ERR_INTERNAL, "device-side consistency check failed");
  if (v & ST_TIMEOUT) return fail(SI_ERR_TIMEOUT, "a bounded device wait gave up");
  if (v & ST_CAPACITY) return fail(SI_ERR_CAPACITY, "neighbor id buffer too small");
  return SI_OK;
}

extern "C" si_status si_grid_get_info(const si_grid *g, si_grid_info *info) {
  if (!g || !info) return fail(SI_ERR_INVALID, "null argument");
  info->n = g->n;
  info->n_cells = g->n_cells;
  info->d_cell_start = g->cell_start;
  info->d_sorted_pos = (const float *)g->spos;
  info->d_perm = g->perm;
  info->table_entries = g->tables.entries;
  info->table_n_max = g->tables.n_max;
  info->spec_shells = g->tables.spec_shells;
  return SI_OK;
}

bool si_grid::ensure_side() {
  // per-kernel timing serialises the kernels on the caller's stream, so
  // that each launch's two events bracket that kernel alone
  {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (g_prof_on) return false;
  }
  if (side) return true;
  if (cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&fork_ev, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&join_ev, cudaEventDisableTiming) != cudaSuccess) {
    if (side) cudaStreamDestroy(side);
    if (fork_ev) cudaEventDestroy(fork_ev);
    if (join_ev) cudaEventDestroy(join_ev);
    side = nullptr;
    fork_ev = join_ev = nullptr;
    cudaGetLastError();
    return false;
  }
  return true;
}

extern "C" si_status si_grid_set_method(si_grid *g, float list_weight, float cube_below, float knn_cube_below) {
  if (!g) return fail(SI_ERR_INVALID, "null grid");
  if (!(list_weight >= 0.f) || !(cube_below >= 0.f) || !(knn_cube_below >= 0.f))
    return fail(SI_ERR_INVALID, "list_weight, cube_below and knn_cube_below must be >= 0");
  g->list_weight = (double)list_weight;
  g->cube_below = (double)cube_below;
  g->knn_cube_below = (double)knn_cube_below;
  return SI_OK;
}

extern "C" si_status si_grid_destroy(si_grid *g) {
  if (!g) return SI_OK;
  cudaDeviceSynchronize();
  grid_free(g);
  return SI_OK;
}

extern "C" int64_t si_launch_count(void) { return g_launches.load(); }

extern "C" si_status si_kernel_timing_enable(int enable) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  g_prof_on = enable != 0;
  return SI_OK;
}

extern "C" si_status si_kernel_timing_report(char *buf, size_t cap) {
  if (!buf || cap == 0) return fail(SI_ERR_INVALID, "null report buffer");
  buf[0] = 0;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  SI_CUDA_TRY(cudaDeviceSynchronize());
  std::map<std::string, std::pair<long long, double>> agg;
  for (const ProfRec &r : g_prof_recs) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
      auto &v = agg[r.name];
      v.first += 1;
      v.second += ms;
    }
    g_prof_pool.push_back(r.a);
    g_prof_pool.push_back(r.b);
  }
  g_prof_recs.clear();
  std::string out;
  char line[256];
  for (const auto &kv : agg) {
    snprintf(line, sizeof line, "%s %lld %.6f\n", kv.first.c_str(), kv.second.first, kv.second.second);
    out += line;
  }
  const size_t n = std::min(out.size(), cap - 1);
  memcpy(buf, out.data(), n);
  buf[n] = 0;
  return out.size() < cap ? SI_OK : fail(SI_ERR_CAPACITY, "report truncated");
}

extern "C" const char *si_status_string(si_status s) {
  switch (s) {
    case SI_OK: return "ok";
    case SI_ERR_INVALID: return "invalid argument or input";
    case SI_ERR_OOM: return "out of memory";
    case SI_ERR_CUDA: return "CUDA error";
    case SI_ERR_CAPACITY: return "output capacity exceeded";
    case SI_ERR_TIMEOUT: return "device wait timed out";
    case SI_ERR_INTERNAL: return "internal consistency check failed";
  }
  return "unknown status";
}

extern "C" const char *si_last_error(void) { return t_last_error.c_str(); }
