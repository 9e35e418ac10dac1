// Batched scenes: many independent grids (own lattice, cyclic mask, radius,
// point set) served together, in one CUDA graph.
//
// Light scenes (short lists) are fused: all their cells live in one
// concatenated cell array and all their points in one sorted array, so
// binning is a fixed number of launches for all of them, and the two query
// passes are persistent kernels that pull (scene, tile of queries) items
// from a device work queue ordered heaviest first.
// Heavy scenes (long lists, crowded cells) each get a grid of their own and
// the single-scene pipeline (binning with cell classes, per-query, per-warp
// and per-cell kernels, slab splitting, expansion), whose work per scene is
// large enough to fill the GPU's share it gets: they run on concurrent
// branches of the same graph, heaviest first on the least-loaded branch.
// The first run is eager (it builds the heavy scenes' radius tables and
// sizes their scratch, which needs host round trips); with use_graph the
// launches are then captured once and replayed.
#include <algorithm>
#include <cmath>
#include <new>
#include <numeric>
#include <vector>

#include "si_host.h"
#include "si_walk.cuh"

namespace si {

constexpr int kBinTile = 256;
constexpr int kBatchInlineSort = 32;
constexpr int kBatchSortThreads = 512;
constexpr int kBatchSortSmem = 8192;
// Planner defaults (si_batch_params; si_batch_tune times alternatives): the
// expected list length from which a scene gets its own pipeline, the
// queries per item (threads per block) of the fused query kernels, the
// concurrent graph branches of the own pipelines, the resident blocks per
// SM of the fused persistent kernels.
constexpr float kDefHeavyHits = 24.f;
constexpr int kDefQTile = 128;
constexpr int kDefBranches = 8;
constexpr int kDefBlocksPerSm = 8;

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
template <bool WRITE, int TILE>
__global__ void __launch_bounds__(TILE) k_batch_query(const SceneDev *__restrict__ sc,
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
  si_batch_params params;         // the planner's choices
  struct Heavy {
    int scene;                    // index in `scenes`
    si_grid *grid;
    double work;                  // expected hits
    int branch;
  };
  int n_scenes = 0;               // all scenes
  std::vector<si_scene> scenes;
  uint32_t flags = 0;
  std::vector<int> fused;         // original index of each fused (light) scene
  std::vector<Heavy> heavy;
  int n_branches = 0;             // concurrent graph branches for heavy scenes
  std::vector<cudaStream_t> branch;
  std::vector<cudaEvent_t> branch_done;
  cudaEvent_t fork = nullptr;
  bool warmed = false;
  int warm_status = 0;            // SI_ERR_* of the eager first run of the heavy scenes
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
  for (auto &h : b->heavy) si_grid_destroy(h.grid);
  for (cudaStream_t s : b->branch) cudaStreamDestroy(s);
  for (cudaEvent_t e : b->branch_done) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
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

static bool params_valid(const si_batch_params &p) {
  return p.heavy_hits >= 0.f && (p.q_tile == 64 || p.q_tile == 128 || p.q_tile == 256) && p.branches >= 1 &&
         p.branches <= 32 && p.blocks_per_sm >= 1 && p.blocks_per_sm <= 2048 / p.q_tile;
}

extern "C" si_status si_batch_default_params(si_batch_params *p) {
  if (!p) return fail(SI_ERR_INVALID, "null params");
  p->heavy_hits = kDefHeavyHits;
  p->q_tile = kDefQTile;
  p->branches = kDefBranches;
  p->blocks_per_sm = kDefBlocksPerSm;
  return SI_OK;
}

extern "C" si_status si_batch_create(const si_scene *scenes, int n_scenes, uint32_t flags,
                                     si_batch **out) {
  return si_batch_create_params(scenes, n_scenes, flags, nullptr, out);
}

extern "C" si_status si_batch_create_params(const si_scene *scenes, int n_scenes, uint32_t flags,
                                            const si_batch_params *params, si_batch **out) {
  if (!scenes || !out || n_scenes <= 0) return fail(SI_ERR_INVALID, "bad batch arguments");
  if (flags & ~(SI_METHOD_CUBE | SI_INCLUDE_SELF)) return fail(SI_ERR_INVALID, "unknown flags");
  si_batch_params prm;
  si_batch_default_params(&prm);
  if (params) prm = *params;
  if (!params_valid(prm)) return fail(SI_ERR_INVALID, "batch parameters out of range");
  *out = nullptr;
  si_batch *b = new (std::nothrow) si_batch();
  if (!b) return fail(SI_ERR_OOM, "host allocation failed");
  b->params = prm;
  b->n_scenes = n_scenes;
  b->scenes.assign(scenes, scenes + n_scenes);
  b->flags = flags;
  std::vector<SceneDev> hs;
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
    // expected list length: load times the sphere's volume in cells
    const double dcell = (double)sc.r * lat.inv_s;
    const double hits = (double)sc.n / (double)(1ll << lat.W) * 4.0 / 3.0 * M_PI * dcell * dcell * dcell;
    if (!(flags & SI_METHOD_CUBE) && sc.n > 0 && hits >= (double)prm.heavy_hits) {
      si_grid_desc desc = sc.desc;
      desc.r_max = sc.r;
      si_grid *gr = nullptr;
      if ((s = si_grid_create(&desc, sc.n, &gr)) != SI_OK) {
        const std::string why = si_last_error();
        batch_free(b);
        return fail(s, "scene " + std::to_string(k) + ": " + why);
      }
      gr->fork = false;   // the scenes' pipelines already run side by side on the graph's branches
      b->heavy.push_back({k, gr, (double)sc.n * hits, 0});
      continue;
    }
    const int fi = (int)b->fused.size();
    b->fused.push_back(k);
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
    hs.emplace_back();
    SceneDev &S = hs.back();
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
    for (int64_t f = 0; f < sc.n; f += kBinTile) bin_items.push_back({fi, (int)f});
    // cost of one query tile: cells visited x (1 + load): heaviest first
    const double cells = 1.0 + 6.0 * d + 3.0 * M_PI * d * d + 4.0 / 3.0 * M_PI * d * d * d;
    for (int64_t f = 0; f < sc.n; f += prm.q_tile) q_items.push_back({{fi, (int)f}, cells * (1.0 + load)});
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
  const int n_fused = (int)hs.size();
  SI_BALLOC(b->d_scenes, std::max(n_fused, 1) * sizeof(SceneDev));
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
  SI_BALLOC(b->scene_status, std::max(n_fused, 1) * sizeof(int));
#undef SI_BALLOC
  for (int k = 0; k < n_fused; ++k) {
    hs[k].g.spos = b->spos;
    hs[k].g.perm = b->perm;
    hs[k].g.cell_start = b->start + hs[k].cbase;
    hs[k].g.status = b->scene_status + k;
  }
  cudaError_t e = n_fused > 0 ? cudaMemcpy(b->d_scenes, hs.data(), n_fused * sizeof(SceneDev), cudaMemcpyHostToDevice)
                              : cudaSuccess;
  if (e == cudaSuccess && !bin_items.empty())
    e = cudaMemcpy(b->d_bin_items, bin_items.data(), bin_items.size() * sizeof(Item), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !qi.empty())
    e = cudaMemcpy(b->d_q_items, qi.data(), qi.size() * sizeof(Item), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(b->scene_status, 0, std::max(n_fused, 1) * sizeof(int));
  if (e == cudaSuccess) e = cudaMallocHost((void **)&b->h_pinned, (n_scenes + 1) * sizeof(long long) * 2);
  if (e == cudaSuccess) e = cudaMallocHost((void **)&b->h_status, std::max(n_fused, 1) * sizeof(int));
  // heavy scenes: heaviest first on the least-loaded branch
  b->n_branches = std::min<int>(prm.branches, (int)b->heavy.size());
  {
    std::vector<size_t> order(b->heavy.size());
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(),
                     [&](size_t x, size_t y) { return b->heavy[x].work > b->heavy[y].work; });
    std::vector<double> load(b->n_branches, 0.0);
    for (size_t i : order) {
      const int br = (int)(std::min_element(load.begin(), load.end()) - load.begin());
      b->heavy[i].branch = br;
      load[br] += b->heavy[i].work;
    }
    std::vector<si_batch::Heavy> sorted;
    for (size_t i : order) sorted.push_back(b->heavy[i]);
    b->heavy.swap(sorted);
  }
  for (int i = 0; e == cudaSuccess && i < b->n_branches; ++i) {
    cudaStream_t bs;
    cudaEvent_t be;
    e = cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking);
    if (e != cudaSuccess) break;
    b->branch.push_back(bs);
    e = cudaEventCreateWithFlags(&be, cudaEventDisableTiming);
    if (e != cudaSuccess) break;
    b->branch_done.push_back(be);
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    batch_free(b);
    return cuda_fail(e, "batch initialisation");
  }
  *out = b;
  return SI_OK;
}

// The fused launches of the light scenes.
static si_status batch_launches(si_batch *b, cudaStream_t st) {
  if (b->fused.empty()) return SI_OK;
  const int64_t N = b->n_total;
  SI_CUDA_TRY(cudaMemsetAsync(b->count, 0, b->cells_total * sizeof(int), st));
  SI_CUDA_TRY(cudaMemsetAsync(b->queues, 0, 2 * sizeof(int), st));
  SI_CUDA_TRY(cudaMemsetAsync(b->longq, 0, sizeof(int), st));
  for (int k : b->fused) {
    const si_scene &sc = b->scenes[k];
    if (sc.n == 0) SI_CUDA_TRY(cudaMemsetAsync(sc.d_offsets, 0, sizeof(int64_t), st));
  }
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
  const int tile = b->params.q_tile;
  const int grid = 148 * b->params.blocks_per_sm;
  auto query = [&](bool write) -> si_status {
    const char *name = write ? "k_batch_query write" : "k_batch_query count";
    int *q = b->queues + (write ? 1 : 0);
    long long *cnt = write ? nullptr : b->gcount;
    const long long *scn = write ? b->gcount : nullptr;
#define SI_BATCH_Q(W, T)                                                                                      \
  SI_KLAUNCH(name, st, k_batch_query<W, T><<<grid, T, 0, st>>>(b->d_scenes, b->d_q_items, b->n_q_items, q, cnt, \
                                                                scn, b->longq, b->scene_status))
    if (write) {
      if (tile == 64) SI_BATCH_Q(true, 64);
      else if (tile == 256) SI_BATCH_Q(true, 256);
      else SI_BATCH_Q(true, 128);
    } else {
      if (tile == 64) SI_BATCH_Q(false, 64);
      else if (tile == 256) SI_BATCH_Q(false, 256);
      else SI_BATCH_Q(false, 128);
    }
#undef SI_BATCH_Q
    return SI_OK;
  };
  if ((s = query(false)) != SI_OK) return s;
  if ((s = scan_inclusive_i64(b->gcount, b->gcount, N, b->scan_i64, st)) != SI_OK) return s;
  SI_KLAUNCH("k_batch_offsets", st, k_batch_offsets<<<b->n_q_items, tile, 0, st>>>(b->d_scenes, b->d_q_items, b->gcount));
  if ((s = query(true)) != SI_OK) return s;
  SI_KLAUNCH("k_batch_sort", st, k_batch_sort<<<2 * 148, kBatchSortThreads, 0, st>>>(b->d_scenes, b->longq, b->scene_status));
  return SI_OK;
}

// One heavy scene through the single-scene pipeline.  total (nullable): the
// list total, read back (a host round trip that lets the query size its
// scratch); without it the call is asynchronous.
static si_status heavy_run(si_batch *b, const si_batch::Heavy &h, cudaStream_t st, int64_t *total) {
  const si_scene &sc = b->scenes[h.scene];
  si_status s = si_grid_build(h.grid, sc.d_pos, sc.n, st);
  if (s != SI_OK) return s;
  return si_query_radius(h.grid, nullptr, sc.n, sc.r, b->flags & SI_INCLUDE_SELF, sc.d_offsets, sc.d_ids,
                         sc.ids_capacity, total, st);
}

// Capture: the fused launches on the origin stream, each heavy scene on its
// branch, branches forked from and joined back to the origin.
static si_status batch_capture(si_batch *b) {
  cudaStream_t cs;
  SI_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    cudaStreamDestroy(cs);
    return cuda_fail(e, "cudaStreamBeginCapture");
  }
  si_status s = SI_OK;
  if (b->n_branches > 0) {
    e = cudaEventRecord(b->fork, cs);
    for (int i = 0; e == cudaSuccess && i < b->n_branches; ++i) e = cudaStreamWaitEvent(b->branch[i], b->fork, 0);
    if (e != cudaSuccess) s = cuda_fail(e, "graph fork");
  }
  if (s == SI_OK) s = batch_launches(b, cs);
  for (size_t i = 0; s == SI_OK && i < b->heavy.size(); ++i)
    s = heavy_run(b, b->heavy[i], b->branch[b->heavy[i].branch], nullptr);
  for (int i = 0; i < b->n_branches; ++i) {   // joined even after an error, so that the capture can end
    cudaEventRecord(b->branch_done[i], b->branch[i]);
    cudaStreamWaitEvent(cs, b->branch_done[i], 0);
  }
  cudaGraph_t graph = nullptr;
  e = cudaStreamEndCapture(cs, &graph);
  cudaStreamDestroy(cs);
  if (s != SI_OK) {
    if (graph) cudaGraphDestroy(graph);
    return s;
  }
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
  b->graph = graph;
  SI_CUDA_TRY(cudaGraphInstantiate(&b->exec, graph, 0));
  return SI_OK;
}

extern "C" si_status si_batch_run(si_batch *b, int use_graph, void *stream) {
  if (!b) return fail(SI_ERR_INVALID, "null batch");
  cudaStream_t st = (cudaStream_t)stream;
  si_status s;
  if (!b->warmed) {
    // eager first run: the heavy scenes build their radius tables and size
    // their scratch from the list totals (host round trips); a capacity
    // shortfall is reported by si_batch_sync
    if ((s = batch_launches(b, st)) != SI_OK) return s;
    for (const auto &h : b->heavy) {
      int64_t total = 0;
      s = heavy_run(b, h, st, &total);
      if (s == SI_ERR_CAPACITY) b->warm_status = SI_ERR_CAPACITY;
      else if (s != SI_OK) return s;
    }
    b->warmed = true;
    return use_graph ? batch_capture(b) : SI_OK;
  }
  if (!use_graph) {
    if ((s = batch_launches(b, st)) != SI_OK) return s;
    for (const auto &h : b->heavy)
      if ((s = heavy_run(b, h, st, nullptr)) != SI_OK) return s;
    return SI_OK;
  }
  if (!b->exec && (s = batch_capture(b)) != SI_OK) return s;
  prof_begin(st);
  SI_CUDA_TRY(cudaGraphLaunch(b->exec, st));
  count_launch();
  prof_end(st, "batch_graph");
  return SI_OK;
}

extern "C" si_status si_batch_sync(si_batch *b, int64_t *h_totals, void *stream) {
  if (!b) return fail(SI_ERR_INVALID, "null batch");
  cudaStream_t st = (cudaStream_t)stream;
  const int nf = (int)b->fused.size();
  if (nf > 0) {
    SI_CUDA_TRY(cudaMemcpyAsync(b->h_status, b->scene_status, nf * sizeof(int), cudaMemcpyDeviceToHost, st));
    SI_CUDA_TRY(cudaMemsetAsync(b->scene_status, 0, nf * sizeof(int), st));
  }
  for (int k = 0; k < b->n_scenes; ++k) {
    const si_scene &sc = b->scenes[k];
    if (h_totals)
      SI_CUDA_TRY(cudaMemcpyAsync(b->h_pinned + k, sc.d_offsets + sc.n, sizeof(long long),
                                  cudaMemcpyDeviceToHost, st));
  }
  SI_CUDA_TRY(cudaStreamSynchronize(st));
  int agg = 0;
  for (int k = 0; k < nf; ++k) agg |= b->h_status[k];
  if (h_totals)
    for (int k = 0; k < b->n_scenes; ++k) h_totals[k] = b->h_pinned[k];
  // heavy scenes: their grids' status words
  si_status worst = SI_OK;
  for (const auto &h : b->heavy) {
    const si_status hs = si_grid_sync(h.grid, st);
    if (hs == SI_ERR_INVALID) agg |= ST_INVALID;
    else if (hs == SI_ERR_CAPACITY) agg |= ST_CAPACITY;
    else if (hs != SI_OK) worst = hs;
  }
  if (b->warm_status == SI_ERR_CAPACITY) agg |= ST_CAPACITY;
  b->warm_status = 0;
  if (agg & ST_INVALID) return fail(SI_ERR_INVALID, "a scene has a point outside a cyclic box or not finite");
  if (agg & ST_INTERNAL) return fail(SI_ERR_INTERNAL, "device-side consistency check failed");
  if (worst != SI_OK) return worst;
  if (agg & ST_CAPACITY) return fail(SI_ERR_CAPACITY, "a scene's id buffer is too small");
  return SI_OK;
}

extern "C" si_status si_batch_destroy(si_batch *b) {
  if (!b) return SI_OK;
  cudaDeviceSynchronize();
  batch_free(b);
  return SI_OK;
}

// Planner tuning: each candidate batch is created, run once eagerly (tables,
// scratch), captured, warmed by two replays and timed over `reps` replays
// with CUDA events on a stream of its own (median); the candidates write the
// scenes' outputs in turn.
extern "C" si_status si_batch_tune(const si_scene *scenes, int n_scenes, uint32_t flags,
                                   const si_batch_params *cands, int n_cand, int reps, float *h_ms,
                                   int32_t *h_best) {
  if (!cands || n_cand <= 0 || reps <= 0 || !h_ms || !h_best) return fail(SI_ERR_INVALID, "bad tuning arguments");
  for (int i = 0; i < n_cand; ++i)
    if (!params_valid(cands[i])) return fail(SI_ERR_INVALID, "candidate " + std::to_string(i) + " out of range");
  cudaStream_t st;
  SI_CUDA_TRY(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  si_status s = e == cudaSuccess ? SI_OK : cuda_fail(e, "cudaEventCreate");
  int best = -1;
  for (int i = 0; s == SI_OK && i < n_cand; ++i) {
    si_batch *b = nullptr;
    if ((s = si_batch_create_params(scenes, n_scenes, flags, cands + i, &b)) != SI_OK) break;
    s = si_batch_run(b, 1, st);
    if (s == SI_OK) s = si_batch_sync(b, nullptr, st);
    for (int w = 0; s == SI_OK && w < 2; ++w) s = si_batch_run(b, 1, st);
    std::vector<float> ms;
    for (int r = 0; s == SI_OK && r < reps; ++r) {
      cudaEventRecord(e0, st);
      s = si_batch_run(b, 1, st);
      cudaEventRecord(e1, st);
      if (s == SI_OK && (e = cudaEventSynchronize(e1)) != cudaSuccess) s = cuda_fail(e, "batch tuning");
      float t = 0.f;
      if (s == SI_OK) cudaEventElapsedTime(&t, e0, e1);
      ms.push_back(t);
    }
    if (s == SI_OK) s = si_batch_sync(b, nullptr, st);
    si_batch_destroy(b);
    if (s != SI_OK) break;
    std::sort(ms.begin(), ms.end());
    h_ms[i] = ms[ms.size() / 2];
    if (best < 0 || h_ms[i] < h_ms[best]) best = i;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaStreamDestroy(st);
  if (s != SI_OK) return s;
  *h_best = best;
  return SI_OK;
}
