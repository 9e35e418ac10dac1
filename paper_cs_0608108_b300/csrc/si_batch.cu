// Batched scenes: many independent grids (own lattice, cyclic mask, radius,
// point set) binned and queried together.  All scenes' cells live in one
// concatenated cell array and all points in one sorted array, so binning is
// a fixed number of launches for the whole batch, and the two query passes
// are persistent kernels that pull (scene, tile of queries) items from a
// device work queue ordered heaviest first.  Nothing synchronises with the
// host, so the whole sequence can be captured in a CUDA graph and replayed.
#include <algorithm>
#include <cmath>
#include <new>
#include <numeric>
#include <vector>

#include "si_host.h"
#include "si_walk.cuh"

namespace si {

constexpr int kBinTile = 256;
constexpr int kQTile = 128;
constexpr int kBatchInlineSort = 32;
constexpr int kBatchSortThreads = 512;
constexpr int kBatchSortSmem = 8192;

struct SceneDev {
  GridDev g;               // spos/perm: batch-global arrays; cell_start: the scene's cells
  WalkParams P;
  Band B;
  long long pbase;         // first slot of the scene in the global point arrays
  long long cbase;         // first cell of the scene in the global cell arrays
  const float4 *pos;       // caller's points
  long long *offsets;      // caller's CSR offsets (n + 1)
  int *ids;                // caller's ids
  long long cap;
  int cube;                // 1: bin-lattice walk chosen by the planner
  int include_self;
};

struct Item {
  int scene;
  int first;               // first local point (binning) or first sorted slot (queries)
};

__global__ void __launch_bounds__(kBinTile) k_batch_key(const SceneDev *__restrict__ sc,
                                                        const Item *__restrict__ items,
                                                        uint2 *__restrict__ key_slot,
                                                        int *__restrict__ count,
                                                        int *__restrict__ scene_status) {
  const Item it = items[blockIdx.x];
  const SceneDev &S = sc[it.scene];
  const GridDev &g = S.g;
  const int i = it.first + threadIdx.x;
  if (i >= g.n) return;
  const float4 p = __ldg(S.pos + i);
  bool out = false, bad = false;
  const int cx = axis_cell(p.x, g.ox, g.Lx, g.inv_s, g.wx, g.cyc & 1u, out, bad);
  const int cy = axis_cell(p.y, g.oy, g.Ly, g.inv_s, g.wy, (g.cyc >> 1) & 1u, out, bad);
  const int cz = axis_cell(p.z, g.oz, g.Lz, g.inv_s, g.wz, (g.cyc >> 2) & 1u, out, bad);
  if (bad) atomicOr(scene_status + it.scene, ST_INVALID);
  const unsigned key = out ? g.outside : pack3(cx, cy, cz, g);
  const long long gk = S.cbase + key;
  const int slot = atomicAdd(count + gk, 1);
  key_slot[S.pbase + i] = make_uint2((unsigned)key, (unsigned)slot);
}

__global__ void __launch_bounds__(kBinTile) k_batch_scatter(const SceneDev *__restrict__ sc,
                                                            const Item *__restrict__ items,
                                                            const uint2 *__restrict__ key_slot,
                                                            const int *__restrict__ start,
                                                            float4 *__restrict__ spos,
                                                            int *__restrict__ perm) {
  const Item it = items[blockIdx.x];
  const SceneDev &S = sc[it.scene];
  const int i = it.first + threadIdx.x;
  if (i >= S.g.n) return;
  const uint2 ks = key_slot[S.pbase + i];
  const int dst = __ldg(start + S.cbase + ks.x) + (int)ks.y;
  spos[dst] = __ldg(S.pos + i);
  perm[dst] = i;
}

// Persistent query pass.  WRITE = false: counts into gcount (global index
// pbase + local id).  WRITE = true: lists into each scene's ids, using the
// inclusive scan gscan of gcount.
template <bool WRITE>
__global__ void __launch_bounds__(kQTile) k_batch_query(const SceneDev *__restrict__ sc,
                                                        const Item *__restrict__ items, int n_items,
                                                        int *__restrict__ queue,
                                                        long long *__restrict__ gcount,
                                                        const long long *__restrict__ gscan,
                                                        int *__restrict__ longq,
                                                        int *__restrict__ scene_status) {
  __shared__ int s_item;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(queue, 1);
    __syncthreads();
    const int item = s_item;
    __syncthreads();
    if (item >= n_items) return;           // every block leaves after at most n_items + 1 pulls
    const Item it = items[item];
    const SceneDev &S = sc[it.scene];
    const GridDev g = S.g;
    const int sl = it.first + threadIdx.x;
    if (sl >= g.n) continue;
    const int s = (int)S.pbase + sl;       // global sorted slot
    const QueryGeom Q = make_geom(g.spos[s], g);
    const int self = S.include_self ? -1 : s;
    const int orig = __ldg(g.perm + s);
    if (!WRITE) {
      long long count = 0;
      auto v = [&](const Target &t, bool full) {
        const int b = __ldg(g.cell_start + t.key), e = __ldg(g.cell_start + t.key + 1);
        if (full) {
          count += e - b - ((self >= b && self < e) ? 1 : 0);
          return;
        }
        for (int j = b; j < e; ++j)
          if (j != self && pair_hit(g, Q, t, S.B, g.spos[j])) ++count;
      };
      if (S.cube || Q.outside) walk_cube(g, Q, S.P.dg, v);
      else walk_sphere(g, Q, S.P, v);
      gcount[S.pbase + orig] = count;
    } else {
      const long long sbase = S.pbase > 0 ? gscan[S.pbase - 1] : 0ll;
      const long long beg = (orig > 0 || S.pbase > 0 ? gscan[S.pbase + orig - 1] : 0ll) - sbase;
      const long long end = gscan[S.pbase + orig] - sbase;
      const int len = (int)(end - beg);
      if (len == 0) continue;
      const long long total = gscan[S.pbase + g.n - 1] - sbase;
      if (total > S.cap) {
        atomicOr(scene_status + it.scene, ST_CAPACITY);
        continue;
      }
      int *out = S.ids + beg;
      const bool inl = len <= kBatchInlineSort;
      int k = 0;
      auto emit = [&](int id) {
        if (k >= len) return;
        if (inl) {
          int p = k;
          while (p > 0) {
            const int prev = out[p - 1];
            if (prev <= id) break;
            out[p] = prev;
            --p;
          }
          out[p] = id;
        } else {
          out[k] = id;
        }
        ++k;
      };
      auto v = [&](const Target &t, bool full) {
        const int b = __ldg(g.cell_start + t.key), e = __ldg(g.cell_start + t.key + 1);
        for (int j = b; j < e; ++j) {
          if (j == self) continue;
          if (full || pair_hit(g, Q, t, S.B, g.spos[j])) emit(__ldg(g.perm + j));
        }
      };
      if (S.cube || Q.outside) walk_cube(g, Q, S.P.dg, v);
      else walk_sphere(g, Q, S.P, v);
      if (k != len) atomicOr(scene_status + it.scene, ST_INTERNAL);
      if (!inl) {
        const int slot = atomicAdd(longq, 1);
        longq[1 + 2 * slot] = it.scene;
        longq[2 + 2 * slot] = orig;
      }
    }
  }
}

// Scene-local CSR offsets from the global inclusive scan.
__global__ void k_batch_offsets(const SceneDev *__restrict__ sc, const Item *__restrict__ items,
                                const long long *__restrict__ gscan) {
  const Item it = items[blockIdx.x];
  const SceneDev &S = sc[it.scene];
  const int i = it.first + threadIdx.x;
  const long long sbase = S.pbase > 0 ? gscan[S.pbase - 1] : 0ll;
  if (i < S.g.n) S.offsets[i + 1] = gscan[S.pbase + i] - sbase;
  if (i == 0) S.offsets[0] = 0;
}

__device__ void block_bitonic_b(int *a, int n) {
  int P = 1;
  while (P < n) P <<= 1;
  for (int k = 2; k <= P; k <<= 1) {
    for (int i = threadIdx.x; i < P / 2; i += blockDim.x) {
      const int lo = (i / (k / 2)) * k + (i % (k / 2));
      const int hi = (lo / k) * k + (k - 1 - (lo % k));
      if (hi < n && a[hi] < a[lo]) {
        const int t = a[lo];
        a[lo] = a[hi];
        a[hi] = t;
      }
    }
    __syncthreads();
    for (int h = k / 4; h >= 1; h >>= 1) {
      for (int i = threadIdx.x; i < P / 2; i += blockDim.x) {
        const int lo = (i / h) * 2 * h + (i % h);
        const int hi = lo + h;
        if (hi < n && a[hi] < a[lo]) {
          const int t = a[lo];
          a[lo] = a[hi];
          a[hi] = t;
        }
      }
      __syncthreads();
    }
  }
}

__global__ void __launch_bounds__(kBatchSortThreads) k_batch_sort(const SceneDev *__restrict__ sc,
                                                                 const int *__restrict__ longq,
                                                                 const int *__restrict__ scene_status) {
  __shared__ int buf[kBatchSortSmem];
  const int nq = longq[0];
  for (int item = blockIdx.x; item < nq; item += gridDim.x) {
    const int scene = longq[1 + 2 * item], q = longq[2 + 2 * item];
    const SceneDev &S = sc[scene];
    const long long base = S.offsets[q];
    const int len = (int)(S.offsets[q + 1] - base);
    int *list = S.ids + base;
    if (len <= kBatchSortSmem) {
      for (int i = threadIdx.x; i < len; i += blockDim.x) buf[i] = list[i];
      __syncthreads();
      block_bitonic_b(buf, len);
      for (int i = threadIdx.x; i < len; i += blockDim.x) list[i] = buf[i];
    } else {
      block_bitonic_b(list, len);
    }
    __syncthreads();
  }
}

}  // namespace si

using namespace si;

struct si_batch {
  int n_scenes = 0;
  std::vector<si_scene> scenes;
  std::vector<DevTables> tables;
  std::vector<Lattice> lats;
  int64_t n_total = 0, cells_total = 0;
  int n_bin_items = 0, n_q_items = 0;
  SceneDev *d_scenes = nullptr;
  Item *d_bin_items = nullptr, *d_q_items = nullptr;
  uint2 *key_slot = nullptr;
  int *count = nullptr, *start = nullptr, *scan_i32 = nullptr;
  float4 *spos = nullptr;
  int *perm = nullptr;
  long long *gcount = nullptr, *scan_i64 = nullptr;
  int *queues = nullptr;          // [0] count-pass queue, [1] write-pass queue
  int *longq = nullptr;           // 1 + 2 * n_total
  int *scene_status = nullptr;
  long long *h_pinned = nullptr;  // per-scene totals readback
  int *h_status = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t graph_stream = nullptr;
};

static void batch_free(si_batch *b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (auto &t : b->tables) free_tables(t);
  cudaFree(b->d_scenes);
  cudaFree(b->d_bin_items);
  cudaFree(b->d_q_items);
  cudaFree(b->key_slot);
  cudaFree(b->count);
  cudaFree(b->start);
  cudaFree(b->scan_i32);
  cudaFree(b->spos);
  cudaFree(b->perm);
  cudaFree(b->gcount);
  cudaFree(b->scan_i64);
  cudaFree(b->queues);
  cudaFree(b->longq);
  cudaFree(b->scene_status);
  if (b->h_pinned) cudaFreeHost(b->h_pinned);
  if (b->h_status) cudaFreeHost(b->h_status);
  delete b;
}

// Expected cells visited per query by the spherical walk vs the cube scan,
// and the planner's choice (Sec. III.B-C: pick the method with the smaller
// volume).  Sphere: exact per-query culling visits on average the Steiner
// volume 1 + 6d + 3 pi d^2 + 4/3 pi d^3 cells (the walk's partial culling sits
// between that and the table size); cube: (2d + 1)^3 on average.
static bool plan_cube(double d) {
  const double sphere = 1.0 + 6.0 * d + 3.0 * M_PI * d * d + 4.0 / 3.0 * M_PI * d * d * d;
  const double cube = std::pow(2.0 * d + 1.0, 3.0);
  return d < 1.0 && cube < 1.15 * sphere;
}

extern "C" si_status si_batch_create(const si_scene *scenes, int n_scenes, uint32_t flags,
                                     si_batch **out) {
  if (!scenes || !out || n_scenes <= 0) return fail(SI_ERR_INVALID, "bad batch arguments");
  if (flags & ~(SI_METHOD_CUBE | SI_INCLUDE_SELF)) return fail(SI_ERR_INVALID, "unknown flags");
  *out = nullptr;
  si_batch *b = new (std::nothrow) si_batch();
  if (!b) return fail(SI_ERR_OOM, "host allocation failed");
  b->n_scenes = n_scenes;
  b->scenes.assign(scenes, scenes + n_scenes);
  std::vector<SceneDev> hs(n_scenes);
  std::vector<Item> bin_items;
  struct QItem {
    Item it;
    double cost;
  };
  std::vector<QItem> q_items;
  si_status s = SI_OK;
  for (int k = 0; k < n_scenes; ++k) {
    const si_scene &sc = scenes[k];
    if (sc.n < 0 || sc.n > 0x7fffffff || (sc.n > 0 && (!sc.d_pos || ((uintptr_t)sc.d_pos & 15u))) ||
        !sc.d_offsets || sc.ids_capacity < 0 || (sc.ids_capacity > 0 && !sc.d_ids) ||
        !(sc.r >= 0.f) || !std::isfinite(sc.r)) {
      batch_free(b);
      return fail(SI_ERR_INVALID, "scene " + std::to_string(k) + ": bad arguments");
    }
    Lattice lat;
    if ((s = make_lattice(sc.desc, (double)sc.r, lat)) != SI_OK) {
      batch_free(b);
      return fail(s, "scene " + std::to_string(k) + ": " + si_last_error());
    }
    HostTables ht;
    std::string err;
    if (!build_tables(lat.w, lat.cyc, lat.n_max, ht, err)) {
      batch_free(b);
      return fail(SI_ERR_INVALID, "scene " + std::to_string(k) + ": " + err);
    }
    DevTables dt;
    if ((s = upload_tables(ht, dt)) != SI_OK) {
      batch_free(b);
      return s;
    }
    b->tables.push_back(dt);
    b->lats.push_back(lat);
    SceneDev &S = hs[k];
    fill_griddev(lat, dt, S.g);
    S.g.n = (int)sc.n;
    S.pbase = b->n_total;
    S.cbase = b->cells_total;
    S.pos = (const float4 *)sc.d_pos;
    S.offsets = (long long *)sc.d_offsets;
    S.ids = sc.d_ids;
    S.cap = sc.ids_capacity;
    const float d = sc.r * lat.inv_s;
    S.P.dg = d + (float)lat.eps;
    const float thr = d - 1.f;
    S.P.rt_b2 = thr <= 0.f ? 0 : (int)std::floor(thr * thr) + 1;
    const double load = (double)sc.n / (double)(1ll << lat.W);
    if (load >= 4.0 && d >= 1.f) {
      S.P.incl_b2 = (int)std::floor((d - 1.f) * (d - 1.f));
      const float dm = d - (float)lat.eps;
      S.P.incl_d2 = dm * dm;
    } else {
      S.P.incl_b2 = -1;
      S.P.incl_d2 = 0.f;
    }
    S.B = make_band(lat, sc.r);
    S.cube = (flags & SI_METHOD_CUBE) ? 1 : (plan_cube(d) ? 1 : 0);
    S.include_self = (flags & SI_INCLUDE_SELF) ? 1 : 0;
    for (int64_t f = 0; f < sc.n; f += kBinTile) bin_items.push_back({k, (int)f});
    // cost of one query tile: cells visited x (1 + load): heaviest first
    const double cells = 1.0 + 6.0 * d + 3.0 * M_PI * d * d + 4.0 / 3.0 * M_PI * d * d * d;
    for (int64_t f = 0; f < sc.n; f += kQTile) q_items.push_back({{k, (int)f}, cells * (1.0 + load)});
    b->n_total += sc.n;
    b->cells_total += (1ll << lat.W) + 1;
  }
  std::stable_sort(q_items.begin(), q_items.end(),
                   [](const QItem &a, const QItem &c) { return a.cost > c.cost; });
  std::vector<Item> qi(q_items.size());
  for (size_t i = 0; i < q_items.size(); ++i) qi[i] = q_items[i].it;
  b->n_bin_items = (int)bin_items.size();
  b->n_q_items = (int)qi.size();
  auto alloc = [&](void **p, size_t bytes) -> si_status {
    cudaError_t e = cudaMalloc(p, std::max<size_t>(bytes, 16));
    return e == cudaSuccess ? SI_OK : cuda_fail(e, "cudaMalloc (batch)");
  };
  const int64_t N = std::max<int64_t>(b->n_total, 1);
#define SI_BALLOC(ptr, bytes)                          \
  if ((s = alloc((void **)&(ptr), (bytes))) != SI_OK) { \
    batch_free(b);                                     \
    return s;                                          \
  }
  SI_BALLOC(b->d_scenes, n_scenes * sizeof(SceneDev));
  SI_BALLOC(b->d_bin_items, std::max<size_t>(bin_items.size(), 1) * sizeof(Item));
  SI_BALLOC(b->d_q_items, std::max<size_t>(qi.size(), 1) * sizeof(Item));
  SI_BALLOC(b->key_slot, N * sizeof(uint2));
  SI_BALLOC(b->count, b->cells_total * sizeof(int));
  SI_BALLOC(b->start, (b->cells_total + 1) * sizeof(int));
  SI_BALLOC(b->scan_i32, scan_scratch_elems(b->cells_total + 1) * sizeof(int));
  SI_BALLOC(b->spos, N * sizeof(float4));
  SI_BALLOC(b->perm, N * sizeof(int));
  SI_BALLOC(b->gcount, N * sizeof(long long));
  SI_BALLOC(b->scan_i64, scan_scratch_elems(N) * sizeof(long long));
  SI_BALLOC(b->queues, 2 * sizeof(int));
  SI_BALLOC(b->longq, (1 + 2 * N) * sizeof(int));
  SI_BALLOC(b->scene_status, n_scenes * sizeof(int));
#undef SI_BALLOC
  for (int k = 0; k < n_scenes; ++k) {
    hs[k].g.spos = b->spos;
    hs[k].g.perm = b->perm;
    hs[k].g.cell_start = b->start + hs[k].cbase;
    hs[k].g.status = b->scene_status + k;
  }
  cudaError_t e = cudaMemcpy(b->d_scenes, hs.data(), n_scenes * sizeof(SceneDev), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !bin_items.empty())
    e = cudaMemcpy(b->d_bin_items, bin_items.data(), bin_items.size() * sizeof(Item), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !qi.empty())
    e = cudaMemcpy(b->d_q_items, qi.data(), qi.size() * sizeof(Item), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(b->scene_status, 0, n_scenes * sizeof(int));
  if (e == cudaSuccess) e = cudaMallocHost((void **)&b->h_pinned, (n_scenes + 1) * sizeof(long long) * 2);
  if (e == cudaSuccess) e = cudaMallocHost((void **)&b->h_status, n_scenes * sizeof(int));
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    batch_free(b);
    return cuda_fail(e, "batch initialisation");
  }
  *out = b;
  return SI_OK;
}

static si_status batch_launches(si_batch *b, cudaStream_t st) {
  const int64_t N = b->n_total;
  SI_CUDA_TRY(cudaMemsetAsync(b->count, 0, b->cells_total * sizeof(int), st));
  SI_CUDA_TRY(cudaMemsetAsync(b->queues, 0, 2 * sizeof(int), st));
  SI_CUDA_TRY(cudaMemsetAsync(b->longq, 0, sizeof(int), st));
  for (const si_scene &sc : b->scenes)
    if (sc.n == 0) SI_CUDA_TRY(cudaMemsetAsync(sc.d_offsets, 0, sizeof(int64_t), st));
  if (b->n_bin_items > 0) {
    SI_KLAUNCH("k_batch_key", st, k_batch_key<<<b->n_bin_items, kBinTile, 0, st>>>(b->d_scenes, b->d_bin_items, b->key_slot, b->count,
                                                     b->scene_status));
  }
  SI_CUDA_TRY(cudaMemsetAsync(b->start, 0, sizeof(int), st));
  si_status s = scan_inclusive_i32(b->count, b->start + 1, b->cells_total, b->scan_i32, st);
  if (s != SI_OK) return s;
  if (b->n_bin_items > 0) {
    SI_KLAUNCH("k_batch_scatter", st, k_batch_scatter<<<b->n_bin_items, kBinTile, 0, st>>>(b->d_scenes, b->d_bin_items, b->key_slot,
                                                         b->start, b->spos, b->perm));
  }
  if (N == 0) return SI_OK;
  const int grid = 148 * 8;
  SI_KLAUNCH("k_batch_query count", st, k_batch_query<false><<<grid, kQTile, 0, st>>>(b->d_scenes, b->d_q_items, b->n_q_items, b->queues,
                                               b->gcount, nullptr, b->longq, b->scene_status));
  if ((s = scan_inclusive_i64(b->gcount, b->gcount, N, b->scan_i64, st)) != SI_OK) return s;
  SI_KLAUNCH("k_batch_offsets", st, k_batch_offsets<<<b->n_q_items, kQTile, 0, st>>>(b->d_scenes, b->d_q_items, b->gcount));
  SI_KLAUNCH("k_batch_query write", st, k_batch_query<true><<<grid, kQTile, 0, st>>>(b->d_scenes, b->d_q_items, b->n_q_items, b->queues + 1,
                                              nullptr, b->gcount, b->longq, b->scene_status));
  SI_KLAUNCH("k_batch_sort", st, k_batch_sort<<<2 * 148, kBatchSortThreads, 0, st>>>(b->d_scenes, b->longq, b->scene_status));
  return SI_OK;
}

extern "C" si_status si_batch_run(si_batch *b, int use_graph, void *stream) {
  if (!b) return fail(SI_ERR_INVALID, "null batch");
  cudaStream_t st = (cudaStream_t)stream;
  if (!use_graph) return batch_launches(b, st);
  if (!b->exec) {
    // capture on a private stream so the caller's stream may be the legacy one
    cudaStream_t cs;
    SI_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    SI_CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    si_status s = batch_launches(b, cs);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(cs, &graph);
    cudaStreamDestroy(cs);
    if (s != SI_OK) {
      if (graph) cudaGraphDestroy(graph);
      return s;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    b->graph = graph;
    SI_CUDA_TRY(cudaGraphInstantiate(&b->exec, graph, 0));
  }
  prof_begin(st);
  SI_CUDA_TRY(cudaGraphLaunch(b->exec, st));
  count_launch();
  prof_end(st, "batch_graph");
  return SI_OK;
}

extern "C" si_status si_batch_sync(si_batch *b, int64_t *h_totals, void *stream) {
  if (!b) return fail(SI_ERR_INVALID, "null batch");
  cudaStream_t st = (cudaStream_t)stream;
  SI_CUDA_TRY(cudaMemcpyAsync(b->h_status, b->scene_status, b->n_scenes * sizeof(int),
                              cudaMemcpyDeviceToHost, st));
  SI_CUDA_TRY(cudaMemsetAsync(b->scene_status, 0, b->n_scenes * sizeof(int), st));
  for (int k = 0; k < b->n_scenes; ++k) {
    const si_scene &sc = b->scenes[k];
    if (h_totals)
      SI_CUDA_TRY(cudaMemcpyAsync(b->h_pinned + k, sc.d_offsets + sc.n, sizeof(long long),
                                  cudaMemcpyDeviceToHost, st));
  }
  SI_CUDA_TRY(cudaStreamSynchronize(st));
  int agg = 0;
  for (int k = 0; k < b->n_scenes; ++k) agg |= b->h_status[k];
  if (h_totals)
    for (int k = 0; k < b->n_scenes; ++k) h_totals[k] = b->h_pinned[k];
  if (agg & ST_INVALID) return fail(SI_ERR_INVALID, "a scene has a point outside a cyclic box or not finite");
  if (agg & ST_INTERNAL) return fail(SI_ERR_INTERNAL, "device-side consistency check failed");
  if (agg & ST_CAPACITY) return fail(SI_ERR_CAPACITY, "a scene's id buffer is too small");
  return SI_OK;
}

extern "C" si_status si_batch_destroy(si_batch *b) {
  if (!b) return SI_OK;
  cudaDeviceSynchronize();
  batch_free(b);
  return SI_OK;
}
