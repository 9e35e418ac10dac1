// Small sorting networks shared by the binning and query kernels.
#pragma once

#include <cuda_runtime.h>

namespace si {

// Ascending bitonic sort of a[0..n) with +inf padding up to the next power
// of two, by `lanes` cooperating threads (rank = thread's index among them);
// sync() separates the stages.  Every compare-exchange puts the smaller value
// at the lower index (first step of each merge compares mirrored pairs), so
// a pair whose upper index is past n never moves anything.
template <class Sync>
__device__ __forceinline__ void bitonic_padded(int *a, int n, int rank, int lanes, Sync sync) {
  int P = 1;
  while (P < n) P <<= 1;
  for (int k = 2; k <= P; k <<= 1) {
    for (int i = rank; i < P / 2; i += lanes) {
      const int lo = (i / (k / 2)) * k + (i % (k / 2));
      const int hi = (lo / k) * k + (k - 1 - (lo % k));
      if (hi < n && a[hi] < a[lo]) {
        const int t = a[lo];
        a[lo] = a[hi];
        a[hi] = t;
      }
    }
    sync();
    for (int h = k / 4; h >= 1; h >>= 1) {
      for (int i = rank; i < P / 2; i += lanes) {
        const int lo = (i / h) * 2 * h + (i % h);
        const int hi = lo + h;
        if (hi < n && a[hi] < a[lo]) {
          const int t = a[lo];
          a[lo] = a[hi];
          a[hi] = t;
        }
      }
      sync();
    }
  }
}

struct WarpSync {
  __device__ __forceinline__ void operator()() const { __syncwarp(); }
};
struct BlockSync {
  __device__ __forceinline__ void operator()() const { __syncthreads(); }
};

}  // namespace si
