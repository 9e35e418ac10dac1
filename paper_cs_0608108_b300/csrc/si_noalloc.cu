// Neighbor energy for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at the point where they need the
// energy: code running under a framework that owns every device allocation
// (a caching allocator that must not be bypassed), plug-ins with a fixed
// device-memory budget, or a real-time simulation step that must never touch
// the allocator.  si_neighbor_energy_noalloc serves them: it bins the points
// and sums the smooth-kernel energy like si_grid_build + si_neighbor_reduce,
// but all of its scratch (cell keys and ranks, cell counts and starts, points
// in cell order, per-block partial sums, a status word) lives in one
// file-scope static device array of kNoAllocBytes, so the call allocates
// nothing.  Every GPU that loads the library holds that array until the
// process exits.
//
// The scratch is shared by all calls: it keeps the last call's contents (the
// counters that must start at zero are cleared on every call), and two calls
// whose work overlaps on the GPU race on it.
#include <cmath>
#include <mutex>

#include "si_host.h"
#include "si_walk.cuh"

namespace si {

// kernels of the binning step and the scan (defined in si_grid.cu)
__global__ void k_bin_key(const float4 *__restrict__ pos, int n, GridDev g, uint2 *__restrict__ key_slot,
                          int *__restrict__ count);
__global__ void k_bin_scatter(const float4 *__restrict__ pos, int n, const uint2 *__restrict__ key_slot,
                              const int *__restrict__ start, float4 *__restrict__ spos,
                              int *__restrict__ perm);

namespace {

constexpr int kNAMaxPoints = 1 << 16;        // points per call
constexpr int kNAMaxLog2Cells = 16;          // lattice of at most 2^16 cells
constexpr int kNAMaxCells = (1 << kNAMaxLog2Cells) + 1;
constexpr int kNAThreads = 128;
constexpr int kNAMaxBlocks = (kNAMaxPoints + kNAThreads - 1) / kNAThreads;

// byte offsets of the scratch regions (256-byte aligned)
constexpr size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t kOffKeySlot = 0;
constexpr size_t kOffCount = align256(kOffKeySlot + sizeof(uint2) * kNAMaxPoints);
constexpr size_t kOffStart = align256(kOffCount + sizeof(int) * kNAMaxCells);
constexpr size_t kOffSpos = align256(kOffStart + sizeof(int) * (kNAMaxCells + 1));
constexpr size_t kOffPerm = align256(kOffSpos + sizeof(float4) * kNAMaxPoints);
constexpr size_t kOffScan = align256(kOffPerm + sizeof(int) * kNAMaxPoints);
constexpr size_t kOffPartial = align256(kOffScan + sizeof(int) * scan_scratch_count(kNAMaxCells));
constexpr size_t kOffStatus = align256(kOffPartial + sizeof(double) * kNAMaxBlocks);
constexpr size_t kNoAllocBytes = align256(kOffStatus + sizeof(int));
// the figure the header states (2,364,416 bytes, 2.25 MiB)
static_assert(kNoAllocBytes == 2364416, "update the scratch size stated in include/si.h");

__device__ __align__(256) static unsigned char g_noalloc_scratch[kNoAllocBytes];

// Device address of the scratch array, looked up once per device with that
// device current (the host-side symbol is only a stand-in for it) and kept
// for the life of the process: a reset of that device's context would leave
// it stale, which the header states.
std::mutex g_na_mu;
unsigned char *g_na_addr[64] = {nullptr};

si_status scratch_address(unsigned char **out) {
  int dev = 0;
  SI_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail(SI_ERR_INVALID, "device index out of range");
  std::lock_guard<std::mutex> lk(g_na_mu);
  if (!g_na_addr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress (no-allocation scratch)");
    g_na_addr[dev] = (unsigned char *)p;
  }
  *out = g_na_addr[dev];
  return SI_OK;
}

struct EnergyVisitor {
  const GridDev &g;
  const QueryGeom &Q;
  float r2, inv_r2;
  int self;
  double e;   // FP32 terms, FP64 sum: the order of a cell's points varies between calls
  __device__ __forceinline__ void operator()(const Target &t, bool) {
    const int b = __ldg(g.cell_start + t.key), en = __ldg(g.cell_start + t.key + 1);
    for (int j = b; j < en; ++j) {
      if (j == self) continue;
      const float4 p = g.spos[j];
      float dx, dy, dz;
      if (t.outside) {
        dx = Q.q.x - p.x;
        dy = Q.q.y - p.y;
        dz = Q.q.z - p.z;
        if (g.cyc & 1u) dx = dx > 0.5f * g.Lx ? dx - g.Lx : (dx < -0.5f * g.Lx ? dx + g.Lx : dx);
        if (g.cyc & 2u) dy = dy > 0.5f * g.Ly ? dy - g.Ly : (dy < -0.5f * g.Ly ? dy + g.Ly : dy);
        if (g.cyc & 4u) dz = dz > 0.5f * g.Lz ? dz - g.Lz : (dz < -0.5f * g.Lz ? dz + g.Lz : dz);
      } else {
        dx = t.qx - p.x;
        dy = t.qy - p.y;
        dz = t.qz - p.z;
      }
      const float d2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
      if (d2 < r2) {
        const float w = fmaf(-d2, inv_r2, 1.f);
        e += (double)(w * w * w);
      }
    }
  }
};

// The energy-reduction kernel with its per-block partial sums in the static
// scratch; neighbors come from the bin-lattice walk, which needs no tables.
__global__ void __launch_bounds__(kNAThreads) k_energy_noalloc(GridDev g, float dg, float r2, float inv_r2,
                                                               double *__restrict__ partial) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  double e = 0.0;
  if (s < g.n) {
    const QueryGeom Q = make_geom(g.spos[s], g);
    EnergyVisitor v{g, Q, r2, inv_r2, s, 0.0};
    walk_cube(g, Q, dg, v);
    e = v.e;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) e += __shfl_down_sync(0xffffffffu, e, o);
  __shared__ double ws[kNAThreads / 32];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = e;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < kNAThreads / 32; ++w) t += ws[w];
    partial[blockIdx.x] = t;
  }
}

// Sum of the partials; NaN when the binning flagged an invalid point.
__global__ void __launch_bounds__(1024) k_energy_noalloc_final(const double *__restrict__ partial, int nb,
                                                               const int *__restrict__ status,
                                                               double *__restrict__ out) {
  double e = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) e += partial[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) e += __shfl_down_sync(0xffffffffu, e, o);
  __shared__ double ws[32];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = e;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += ws[w];
    out[0] = status[0] ? __longlong_as_double(0x7ff8000000000000ll) : t;
  }
}

}  // namespace
}  // namespace si

using namespace si;

extern "C" si_status si_neighbor_energy_noalloc(const si_grid_desc *desc, const float *d_pos, int64_t n,
                                                float r, double *d_energy, void *stream) {
  if (!desc || !d_energy) return fail(SI_ERR_INVALID, "null descriptor or energy pointer");
  if (n < 0 || n > kNAMaxPoints)
    return fail(SI_ERR_INVALID, "no-allocation energy: n must be in [0, 65536]");
  if (n > 0 && (!d_pos || ((uintptr_t)d_pos & 15u)))
    return fail(SI_ERR_INVALID, "positions must be a non-null, 16-byte aligned float4 array");
  if (!(r > 0.f) || !std::isfinite(r)) return fail(SI_ERR_INVALID, "radius must be finite and > 0");
  if ((int)desc->log2_cells[0] + desc->log2_cells[1] + desc->log2_cells[2] > kNAMaxLog2Cells)
    return fail(SI_ERR_INVALID, "no-allocation energy: the lattice may have at most 2^16 cells");
  Lattice lat;
  si_status s = make_lattice(*desc, (double)r, lat);   // r sizes nothing here; it is validated
  if (s != SI_OK) return s;
  unsigned char *base = nullptr;
  if ((s = scratch_address(&base)) != SI_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  uint2 *key_slot = (uint2 *)(base + kOffKeySlot);
  int *count = (int *)(base + kOffCount);
  int *start = (int *)(base + kOffStart);
  float4 *spos = (float4 *)(base + kOffSpos);
  int *perm = (int *)(base + kOffPerm);
  int *scan = (int *)(base + kOffScan);
  double *partial = (double *)(base + kOffPartial);
  int *status = (int *)(base + kOffStatus);
  const int64_t n_cells = (1ll << lat.W) + 1;
  GridDev g;
  DevTables none;
  fill_griddev(lat, none, g);
  g.spos = spos;
  g.perm = perm;
  g.qpos = spos;
  g.qid = perm;
  g.cell_start = start;
  g.n = (int)n;
  g.status = status;
  // what must start at zero: cell counts, the status
  SI_CUDA_TRY(cudaMemsetAsync(count, 0, n_cells * sizeof(int), st));
  SI_CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(int), st));
  SI_CUDA_TRY(cudaMemsetAsync(start, 0, sizeof(int), st));
  if (n > 0)
    SI_KLAUNCH("k_bin_key", st,
               k_bin_key<<<(unsigned)((n + 255) / 256), 256, 0, st>>>((const float4 *)d_pos, (int)n, g,
                                                                      key_slot, count));
  if ((s = scan_inclusive_i32(count, start + 1, n_cells, scan, st)) != SI_OK) return s;
  if (n > 0)
    SI_KLAUNCH("k_bin_scatter", st,
               k_bin_scatter<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
                   (const float4 *)d_pos, (int)n, key_slot, start, spos, perm));
  const unsigned blocks = n > 0 ? (unsigned)((n + kNAThreads - 1) / kNAThreads) : 0u;
  const float r2 = r * r;
  if (blocks > 0)
    SI_KLAUNCH("k_energy_noalloc", st,
               k_energy_noalloc<<<blocks, kNAThreads, 0, st>>>(g, r * lat.inv_s + (float)lat.eps, r2,
                                                               1.f / r2, partial));
  SI_KLAUNCH("k_energy_noalloc_final", st,
             k_energy_noalloc_final<<<1, 1024, 0, st>>>(partial, (int)blocks, status, d_energy));
  return SI_OK;
}
