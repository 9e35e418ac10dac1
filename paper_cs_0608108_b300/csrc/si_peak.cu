// Measured pair-test rate of this GPU: the denominator of the arithmetic
// roofline of the radius kernels.  A pair test is the FP32 filter of the
// canonical predicate (per-axis difference, square, two fused multiply-adds)
// and the sign of d^2 - t moved into a hit mask, exactly the operations of
// the heavy-cell test phase, with the candidates read from shared memory by
// broadcast as there; nothing else (no loads from global memory, no
// stores but one word per thread).  Timed with CUDA events on a stream of
// its own, best of several launches after a warm-up.
#include <cmath>

#include "si_cell.cuh"

namespace si {

constexpr int kPeakThreads = 256;
constexpr int kPeakCands = 1024;   // candidates in shared memory (a whole number of chunks of 32)

// variant 0: scalar FP32 operations, one candidate per step;
// variant 1: packed f32x2 operations, two candidates per step (the form the
// test phase uses).
template <int VARIANT>
__global__ void __launch_bounds__(kPeakThreads) k_pair_rate(int reps, float t, unsigned *sink) {
  __shared__ float4 xy[kPeakCands / 2];
  __shared__ float2 zz[kPeakCands / 2];
  for (int i = threadIdx.x; i < kPeakCands / 2; i += blockDim.x) {
    const float a = 0.001f * (float)i, b = 0.0007f * (float)(i ^ 5);
    xy[i] = make_float4(a, b, b, a);
    zz[i] = make_float2(a * 0.5f, b * 0.5f);
  }
  __syncthreads();
  const float qx = 0.0003f * (float)(threadIdx.x + blockIdx.x), qy = 0.2f, qz = 0.1f;
  const float tn = nextafterf(t, INFINITY);
  unsigned acc = 0u;
  for (int r = 0; r < reps; ++r) {
    for (int c = 0; c < kPeakCands / 2; c += 16) {
      unsigned m = 0u;
      if (VARIANT == 0) {
#pragma unroll
        for (int p = 0; p < 16; ++p) {
          const float4 a = xy[c + p];
          const float2 b = zz[c + p];
          const float dx0 = a.x - qx, dy0 = a.z - qy, dz0 = b.x - qz;
          const float dx1 = a.y - qx, dy1 = a.w - qy, dz1 = b.y - qz;
          const float d0 = fmaf(dz0, dz0, fmaf(dy0, dy0, dx0 * dx0));
          const float d1 = fmaf(dz1, dz1, fmaf(dy1, dy1, dx1 * dx1));
          m = __funnelshift_l(__float_as_uint(d1 - tn), m, 1);
          m = __funnelshift_l(__float_as_uint(d0 - tn), m, 1);
        }
      } else {
        const unsigned long long QX = pack2(qx, qx), QY = pack2(qy, qy), QZ = pack2(qz, qz), T = pack2(tn, tn);
#pragma unroll
        for (int p = 0; p < 16; ++p) {
          const float4 a = xy[c + p];
          const float2 b = zz[c + p];
          unsigned long long dx, dy, dz, D2, x;
          asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(dx) : "l"(pack2(a.x, a.y)), "l"(QX));
          asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(dy) : "l"(pack2(a.z, a.w)), "l"(QY));
          asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(dz) : "l"(pack2(b.x, b.y)), "l"(QZ));
          asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(D2) : "l"(dx), "l"(dx));
          asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(D2) : "l"(dy), "l"(dy), "l"(D2));
          asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(D2) : "l"(dz), "l"(dz), "l"(D2));
          asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(x) : "l"(D2), "l"(T));
          m = __funnelshift_l((unsigned)(x >> 32), m, 1);
          m = __funnelshift_l((unsigned)x, m, 1);
        }
      }
      acc += __popc(m);
    }
  }
  sink[blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

}  // namespace si

using namespace si;

extern "C" si_status si_measure_pair_rate(uint32_t variant, double *pairs_per_second) {
  if (!pairs_per_second) return fail(SI_ERR_INVALID, "null output");
  if (variant > 1u) return fail(SI_ERR_INVALID, "variant must be 0 (scalar FP32) or 1 (packed f32x2)");
  int dev = 0, sms = 0;
  SI_CUDA_TRY(cudaGetDevice(&dev));
  SI_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  int per_sm = 0;
  SI_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      &per_sm, variant ? (const void *)k_pair_rate<1> : (const void *)k_pair_rate<0>, kPeakThreads, 0));
  const int blocks = sms * std::max(per_sm, 1);
  const int reps = 64;
  unsigned *sink = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  si_status s = SI_OK;
  auto cleanup = [&]() {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    if (sink) cudaFree(sink);
  };
  cudaError_t e = cudaMalloc((void **)&sink, (size_t)blocks * kPeakThreads * sizeof(unsigned));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e != cudaSuccess) {
    cleanup();
    return cuda_fail(e, "pair-rate set-up");
  }
  float best = INFINITY;
  for (int it = 0; it < 6 && s == SI_OK; ++it) {   // the first launch warms up
    cudaEventRecord(e0, st);
    if (variant) k_pair_rate<1><<<blocks, kPeakThreads, 0, st>>>(reps, 2.25f, sink);
    else k_pair_rate<0><<<blocks, kPeakThreads, 0, st>>>(reps, 2.25f, sink);
    count_launch();
    cudaEventRecord(e1, st);
    e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
      s = cuda_fail(e, "k_pair_rate");
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (it > 0) best = std::min(best, ms);
  }
  cleanup();
  if (s != SI_OK) return s;
  const double pairs = (double)blocks * kPeakThreads * reps * kPeakCands;
  *pairs_per_second = pairs / ((double)best * 1e-3);
  return SI_OK;
}
