// Device-wide inclusive prefix sum (reduce-then-scan, three launches, no
// inter-block waiting).  Used for the cell histogram -> cell start array of
// the binning step and for the per-query counts -> CSR offsets of the
// two-pass neighbor-list emission.
#include "si_host.h"

namespace si {
namespace {

constexpr int kThreads = 256;
constexpr int kItems = 16;
constexpr int kTile = kThreads * kItems;   // values per block
static_assert(kTile == kScanTile, "the scan's tile is the one scan_scratch_count assumes");

template <typename T>
__device__ __forceinline__ T warp_incl_scan(T v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

// Exclusive scan of one value per thread across the block; returns the
// block total through `total`.
template <typename T>
__device__ __forceinline__ T block_excl_scan(T v, T &total) {
  __shared__ T warp_sums[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  T inc = warp_incl_scan(v);
  if (lane == 31) warp_sums[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    T s = lane < nw ? warp_sums[lane] : T(0);
    s = warp_incl_scan(s);
    if (lane < nw) warp_sums[lane] = s;
  }
  __syncthreads();
  const T before = wid > 0 ? warp_sums[wid - 1] : T(0);
  total = warp_sums[nw - 1];
  __syncthreads();
  return before + inc - v;
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_tile_sums(const T *__restrict__ in, int64_t n,
                                                        T *__restrict__ sums) {
  const int64_t base = (int64_t)blockIdx.x * kTile;
  T acc = 0;
#pragma unroll
  for (int k = 0; k < kItems; ++k) {
    const int64_t i = base + k * kThreads + threadIdx.x;
    if (i < n) acc += in[i];
  }
  T total;
  block_excl_scan(acc, total);
  if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// One block scans the tile sums in place (exclusive), chunk by chunk.
template <typename T>
__global__ void __launch_bounds__(1024) k_scan_sums(T *sums, int64_t ntiles) {
  T carry = 0;
  for (int64_t b = 0; b < ntiles; b += blockDim.x) {
    const int64_t i = b + threadIdx.x;
    const T v = i < ntiles ? sums[i] : T(0);
    T total;
    const T ex = block_excl_scan(v, total);
    if (i < ntiles) sums[i] = carry + ex;
    carry += total;
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_scan_tiles(const T *in, T *out, int64_t n,
                                                         const T *__restrict__ sums) {
  // padded shared tile: index i stored at i + i/32 to avoid bank conflicts
  __shared__ T tile[kTile + kTile / 32];
  const int64_t base = (int64_t)blockIdx.x * kTile;
#pragma unroll
  for (int k = 0; k < kItems; ++k) {
    const int li = k * kThreads + threadIdx.x;
    const int64_t i = base + li;
    tile[li + li / 32] = i < n ? in[i] : T(0);
  }
  __syncthreads();
  T run = 0;
  const int t0 = threadIdx.x * kItems;
#pragma unroll
  for (int k = 0; k < kItems; ++k) {
    const int li = t0 + k;
    run += tile[li + li / 32];
  }
  T total;
  T prefix = block_excl_scan(run, total) + sums[blockIdx.x];
#pragma unroll
  for (int k = 0; k < kItems; ++k) {
    const int li = t0 + k;
    prefix += tile[li + li / 32];
    tile[li + li / 32] = prefix;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < kItems; ++k) {
    const int li = k * kThreads + threadIdx.x;
    const int64_t i = base + li;
    if (i < n) out[i] = tile[li + li / 32];
  }
}

template <typename T>
si_status scan_inclusive(const T *in, T *out, int64_t n, T *scratch, cudaStream_t st) {
  if (n <= 0) return SI_OK;
  const int64_t ntiles = (n + kTile - 1) / kTile;
  SI_KLAUNCH("scan tile sums", st, k_tile_sums<T><<<(unsigned)ntiles, kThreads, 0, st>>>(in, n, scratch));
  SI_KLAUNCH("scan of tile sums", st, k_scan_sums<T><<<1, 1024, 0, st>>>(scratch, ntiles));
  SI_KLAUNCH("scan tiles", st, k_scan_tiles<T><<<(unsigned)ntiles, kThreads, 0, st>>>(in, out, n, scratch));
  return SI_OK;
}

}  // namespace

int64_t scan_scratch_elems(int64_t n) { return scan_scratch_count(n); }

si_status scan_inclusive_i32(const int *in, int *out, int64_t n, int *scratch, cudaStream_t st) {
  return scan_inclusive<int>(in, out, n, scratch, st);
}

si_status scan_inclusive_i64(const long long *in, long long *out, int64_t n, long long *scratch,
                             cudaStream_t st) {
  return scan_inclusive<long long>(in, out, n, scratch, st);
}

}  // namespace si
