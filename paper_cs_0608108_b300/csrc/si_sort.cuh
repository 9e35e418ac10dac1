// Small sorting networks shared by the binning and query kernels.
#pragma once

#include <cuda_runtime.h>

namespace si {

// Ascending bitonic sort of a[0..n) with +inf padding up to the next power
// of two, by `lanes` cooperating threads (rank = thread's index among them);
// sync() separates the stages.  Every compare-exchange puts the smaller value
// at the lower index (first step of each merge compares mirrored pairs), so
// a pair whose upper index is past n never moves anything.
template <class T, class Sync>
__device__ __forceinline__ void bitonic_padded(T *a, int n, int rank, int lanes, Sync sync) {
  int lg = 0;
  while ((1 << lg) < n) ++lg;
  const int half = (1 << lg) >> 1;
  // merge width k = 2^ks; pair i of a stage: block of k, then offset inside
  for (int ks = 1; ks <= lg; ++ks) {
    const int k = 1 << ks;
    for (int i = rank; i < half; i += lanes) {
      const int lo = ((i >> (ks - 1)) << ks) + (i & ((k >> 1) - 1));
      const int hi = (lo & ~(k - 1)) + (k - 1 - (lo & (k - 1)));
      if (hi < n && a[hi] < a[lo]) {
        const T t = a[lo];
        a[lo] = a[hi];
        a[hi] = t;
      }
    }
    sync();
    for (int hs = ks - 2; hs >= 0; --hs) {
      const int h = 1 << hs;
      for (int i = rank; i < half; i += lanes) {
        const int lo = ((i >> hs) << (hs + 1)) + (i & (h - 1));
        const int hi = lo + h;
        if (hi < n && a[hi] < a[lo]) {
          const T t = a[lo];
          a[lo] = a[hi];
          a[hi] = t;
        }
      }
      sync();
    }
  }
}

// Ascending sort of a[0..n), n <= 32 L, by one warp with the keys in
// registers: element e = r * 32 + lane sits in lane `lane`, slot r; keys past
// n are padded with the largest value.  Every merge of the bitonic network
// is ascending and opens with a mirrored step (e against e ^ (k - 1) in each
// block of k); a compare-exchange always puts the smaller key at the lower
// index, so the padding at the end never moves, and the slots r >= L of a
// network of 32 E elements (E a power of two, L <= E) hold padding only and
// take no part: with L = 3 of E = 4, 96 keys cost three quarters of a
// 128-key sort.  The network is unrolled at compile time: a partner in
// another slot of the same lane is exchanged in registers, one in another
// lane by shuffle, so no index arithmetic, shared-memory round trip or
// barrier sits between steps.  All 32 lanes must call it; a[] is read before
// and written after (callers order those accesses with __syncwarp).
template <int E, int L, class T>
__device__ __forceinline__ void warp_sort_regs(T *a, int n, int lane, T pad) {
  static_assert(L >= 1 && L <= E && (E & (E - 1)) == 0, "E a power of two, 1 <= L <= E");
  constexpr int N = 32 * E;
  T v[E];
#pragma unroll
  for (int r = 0; r < E; ++r) v[r] = (r < L && r * 32 + lane < n) ? a[r * 32 + lane] : pad;
#pragma unroll
  for (int k = 2; k <= N; k <<= 1) {
    if (k <= 32) {   // mirrored step inside a lane group: partner lane ^ (k - 1)
      const bool lower = (lane & (k >> 1)) == 0;
#pragma unroll
      for (int r = 0; r < L; ++r) {
        const T o = __shfl_xor_sync(0xffffffffu, v[r], k - 1);
        const T x = v[r];
        v[r] = lower ? (o < x ? o : x) : (x < o ? o : x);
      }
    } else {         // mirrored step across slots: (r, lane) against (rp, lane ^ 31)
      const int kr = k >> 5;   // slots per block
#pragma unroll
      for (int r = 0; r < E; ++r) {
        const int ri = r & (kr - 1);
        const int rp = (r & ~(kr - 1)) + (kr - 1 - ri);
        if (ri >= (kr >> 1) || rp >= L) continue;   // upper half, or a padding partner (no move)
        const T ou = __shfl_xor_sync(0xffffffffu, v[rp], 31);
        const T ol = __shfl_xor_sync(0xffffffffu, v[r], 31);
        const T x = v[r], y = v[rp];
        v[r] = ou < x ? ou : x;
        v[rp] = y < ol ? ol : y;
      }
    }
#pragma unroll
    for (int j = k >> 2; j > 0; j >>= 1) {   // half-cleaners, ascending
      if (j >= 32) {
        const int rj = j >> 5;
#pragma unroll
        for (int r = 0; r < E; ++r) {
          if ((r & rj) || (r | rj) >= L) continue;
          const T x = v[r], y = v[r | rj];
          const bool sw = y < x;
          v[r] = sw ? y : x;
          v[r | rj] = sw ? x : y;
        }
      } else {
        const bool lower = (lane & j) == 0;
#pragma unroll
        for (int r = 0; r < L; ++r) {
          // a block of several slots whose upper half is padding only was
          // left sorted by the previous stage: its merge moves nothing
          if (k >= 64 && (r & ~((k >> 5) - 1)) + (k >> 6) >= L) continue;
          const T o = __shfl_xor_sync(0xffffffffu, v[r], j);
          const T x = v[r];
          v[r] = lower ? (o < x ? o : x) : (x < o ? o : x);
        }
      }
    }
  }
#pragma unroll
  for (int r = 0; r < L; ++r)
    if (r * 32 + lane < n) a[r * 32 + lane] = v[r];
}

struct WarpSync {
  __device__ __forceinline__ void operator()() const { __syncwarp(); }
};

// One warp sorts a[0..n) ascending: up to 128 keys in registers, more with
// the shared-memory network.  pad must exceed every key.  Callers order the
// accesses to a[] around it with __syncwarp.
template <class T>
__device__ __forceinline__ void warp_sort(T *a, int n, int lane, T pad) {
  if (n <= 1) return;
  if (n <= 32) warp_sort_regs<1, 1>(a, n, lane, pad);
  else if (n <= 64) warp_sort_regs<2, 2>(a, n, lane, pad);
  else if (n <= 96) warp_sort_regs<4, 3>(a, n, lane, pad);
  else if (n <= 128) warp_sort_regs<4, 4>(a, n, lane, pad);
  else bitonic_padded(a, n, lane, 32, WarpSync());
}
struct BlockSync {
  __device__ __forceinline__ void operator()() const { __syncthreads(); }
};

}  // namespace si
