// Discretization tuning (Sec. IV.A, Fig. 9 and 10): with the region, the
// objects and the query centers fixed, the cost of a query depends on the
// cell size -- finer cells hold fewer objects out of range but make more
// cells to visit -- and the best size depends on the number of objects, the
// query distance and on K.  si_tune_lattice measures it: each candidate
// lattice is built and queried on the device, timed with CUDA events.
#include <algorithm>
#include <cmath>
#include <vector>

#include "si_host.h"

using namespace si;

namespace {

struct DevBuf {
  void *p = nullptr;
  ~DevBuf() { cudaFree(p); }
  cudaError_t alloc(size_t bytes) {
    cudaFree(p);
    p = nullptr;
    return cudaMalloc(&p, std::max<size_t>(bytes, 16));
  }
};

struct GridHolder {
  si_grid *g = nullptr;
  ~GridHolder() { si_grid_destroy(g); }
};

struct EventPair {
  cudaEvent_t a = nullptr, b = nullptr;
  ~EventPair() {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
  }
};

}  // namespace

extern "C" si_status si_tune_lattice(const si_grid_desc *desc, const float *d_pos, int64_t n,
                                     const float *d_centers, int64_t m, float r, int k, const int32_t *h_shifts,
                                     int n_cand, int reps, float *h_ms, int32_t *h_best, void *stream) {
  if (!desc || !h_shifts || !h_ms || !h_best) return fail(SI_ERR_INVALID, "null argument");
  if (n_cand < 1 || reps < 1) return fail(SI_ERR_INVALID, "need at least one candidate and one round");
  if (!(r > 0.f) || !std::isfinite(r)) return fail(SI_ERR_INVALID, "r must be finite and > 0");
  if (k < 0 || k > 64) return fail(SI_ERR_INVALID, "k must be 0 (radius) or in [1, 64]");
  if (n < 0 || (!d_centers && m != n) || m < 0) return fail(SI_ERR_INVALID, "bad point or center count");
  cudaStream_t st = (cudaStream_t)stream;
  EventPair ev;
  SI_CUDA_TRY(cudaEventCreate(&ev.a));
  SI_CUDA_TRY(cudaEventCreate(&ev.b));
  DevBuf off, ids, kids, kcnt;
  int64_t ids_cap = 0;
  SI_CUDA_TRY(off.alloc((size_t)(m + 1) * sizeof(int64_t)));
  if (k > 0) {
    SI_CUDA_TRY(kids.alloc((size_t)m * k * sizeof(int32_t)));
    SI_CUDA_TRY(kcnt.alloc((size_t)m * sizeof(int32_t)));
  }
  *h_best = -1;
  float best = INFINITY;
  for (int c = 0; c < n_cand; ++c) {
    h_ms[c] = INFINITY;
    // the same region cut into 2^shift times as many cells per axis
    si_grid_desc d = *desc;
    const int sh = h_shifts[c];
    bool ok = std::abs(sh) <= 8;
    for (int a = 0; a < 3 && ok; ++a) {
      const int w = (int)desc->log2_cells[a] + sh;
      ok = w >= 2 && w <= 10;
      d.log2_cells[a] = (uint8_t)(ok ? w : 0);
    }
    if (!ok) continue;
    d.cell_size = std::ldexp(desc->cell_size, -sh);
    d.r_max = r;
    GridHolder G;
    si_status s = si_grid_create(&d, std::max<int64_t>(n, 1), &G.g);
    if (s == SI_ERR_INVALID) continue;   // not a valid lattice for this region and radius
    if (s != SI_OK) return s;
    auto round = [&](int64_t *h_total) -> si_status {
      si_status rs = si_grid_build(G.g, d_pos, n, st);
      if (rs != SI_OK) return rs;
      if (k == 0)
        return si_query_radius(G.g, d_centers, m, r, 0u, (int64_t *)off.p, (int32_t *)ids.p, ids_cap, h_total, st);
      return si_query_knn(G.g, d_centers, m, k, r, 0u, (int32_t *)kids.p, nullptr, (int32_t *)kcnt.p, st);
    };
    // warm-up round: tables, classes and scratch sized; the id buffer grown
    int64_t total = 0;
    s = round(k == 0 ? &total : nullptr);
    if (s == SI_ERR_CAPACITY) {
      SI_CUDA_TRY(ids.alloc((size_t)total * sizeof(int32_t)));
      ids_cap = total;
      s = round(&total);
    }
    if (s != SI_OK) return s;
    if ((s = si_grid_sync(G.g, st)) != SI_OK) return s;
    std::vector<float> t(reps);
    for (int i = 0; i < reps; ++i) {
      SI_CUDA_TRY(cudaEventRecord(ev.a, st));
      if ((s = round(nullptr)) != SI_OK) return s;
      SI_CUDA_TRY(cudaEventRecord(ev.b, st));
      SI_CUDA_TRY(cudaEventSynchronize(ev.b));
      SI_CUDA_TRY(cudaEventElapsedTime(&t[i], ev.a, ev.b));
    }
    if ((s = si_grid_sync(G.g, st)) != SI_OK) return s;
    std::nth_element(t.begin(), t.begin() + reps / 2, t.end());
    h_ms[c] = t[reps / 2];
    if (h_ms[c] < best) {
      best = h_ms[c];
      *h_best = c;
    }
  }
  if (*h_best < 0) return fail(SI_ERR_INVALID, "no candidate is a valid lattice for this region and radius");
  return SI_OK;
}
