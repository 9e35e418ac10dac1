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

struct WarpSync {
  __device__ __forceinline__ void operator()() const { __syncwarp(); }
};
struct BlockSync {
  __device__ __forceinline__ void operator()() const { __syncthreads(); }
};

}  // namespace si
