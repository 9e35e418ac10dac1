// Smooth neighbor reduction: the user functor applied to each neighbor of
// every agent (Sec. IV.A, "the functor applied to each neighbor"), made a
// differentiable energy
//   E = sum_i sum_{j != i, D_ij < r} (1 - D_ij^2 / r^2)^3
// with its hand-written adjoint
//   dE/dx_i = -(12 / r^2) sum_{j != i, D_ij < r} (1 - D_ij^2 / r^2)^2 (x_i - x_j)
// (every unordered pair appears twice in E, hence 2 * 3 * 2 = 12).  One walk
// computes both; no neighbor list is materialised.
#include <algorithm>
#include <cmath>

#include "si_host.h"
#include "si_walk.cuh"

namespace si {

constexpr int kReduceThreads = 128;

struct ReduceVisitor {
  const GridDev &g;
  const QueryGeom &Q;
  float r2, inv_r2;
  int self;
  bool want_grad;
  float e, gx, gy, gz;
  __device__ __forceinline__ void operator()(const Target &t, bool f) {
    (*this)(t, f, __ldg(g.cell_start + t.key), __ldg(g.cell_start + t.key + 1));
  }
  __device__ __forceinline__ void operator()(const Target &t, bool, int b, int en) {
    for (int j = b; j < en; ++j) {
      if (j == self) continue;
      const float4 p = g.spos[j];
      float dx, dy, dz;
      if (t.outside) {
        // arbitrary position: shortest displacement per cyclic axis
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
        const float w2 = w * w;
        e = fmaf(w2, w, e);
        if (want_grad) {
          gx = fmaf(w2, dx, gx);
          gy = fmaf(w2, dy, gy);
          gz = fmaf(w2, dz, gz);
        }
      }
    }
  }
};

// One query per thread.  CLASSES: the sub-cell class tables are staged in
// shared memory once per block and the grid is persistent (grid-stride over
// the queries); otherwise the walk of Sec. III.A reads the global tables.
template <bool GRAD, bool CLASSES>
__global__ void __launch_bounds__(kReduceThreads) k_reduce(GridDev g, WalkParams P, float r2,
                                                           float inv_r2, int n_entries,
                                                           const float *__restrict__ scale,
                                                           float4 *__restrict__ grad,
                                                           double *__restrict__ partial) {
  extern __shared__ __align__(16) unsigned long long cls_smem[];
  if (CLASSES) {
    const int nbeg = g.cls_q * g.cls_q * g.cls_q + 1;
    int *beg_smem = reinterpret_cast<int *>(cls_smem + n_entries);
    for (int i = threadIdx.x; i < n_entries; i += blockDim.x) cls_smem[i] = __ldg(g.cls + i);
    for (int i = threadIdx.x; i < nbeg; i += blockDim.x) beg_smem[i] = __ldg(g.cls_begin + i);
    __syncthreads();
    g.cls = cls_smem;
    g.cls_begin = beg_smem;
  }
  double e = 0.0;
  const float c = -12.f * inv_r2 * ((GRAD && scale) ? __ldg(scale) : 1.f);
  const int stride = CLASSES ? gridDim.x * blockDim.x : g.n;
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < g.n; s += stride) {
    const QueryGeom Q = make_geom(g.spos[s], g);
    ReduceVisitor v{g, Q, r2, inv_r2, s, GRAD, 0.f, 0.f, 0.f, 0.f};
    if (Q.outside) walk_cube(g, Q, P.dg, v);
    else if (CLASSES) walk_classes_in(g, Q, g.cls, g.cls_begin, g.cls_q, v);
    else walk_sphere(g, Q, P, v);
    e += (double)v.e;
    if (GRAD) grad[__ldg(g.perm + s)] = make_float4(c * v.gx, c * v.gy, c * v.gz, 0.f);
  }
  // block sum of the energy in FP64, one partial per block (deterministic)
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) e += __shfl_down_sync(0xffffffffu, e, o);
  __shared__ double ws[kReduceThreads / 32];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = e;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < kReduceThreads / 32; ++w) t += ws[w];
    partial[blockIdx.x] = t;
  }
}

__global__ void __launch_bounds__(1024) k_reduce_final(const double *__restrict__ partial, int nb,
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
    out[0] = t;
  }
}

}  // namespace si

using namespace si;

extern "C" si_status si_neighbor_reduce(si_grid *g, float r, int kernel, double *d_energy,
                                        float *d_grad, const float *d_grad_scale, void *stream) {
  if (!g) return fail(SI_ERR_INVALID, "null grid");
  if (kernel != SI_KERNEL_POLY6_CUBED) return fail(SI_ERR_INVALID, "unknown reduction kernel");
  if (!(r > 0.f) || !std::isfinite(r)) return fail(SI_ERR_INVALID, "radius must be finite and > 0");
  if (!g->lat.unbounded && (double)r > (double)g->desc.r_max)
    return fail(SI_ERR_INVALID, "radius exceeds the grid's r_max");
  if (d_grad && ((uintptr_t)d_grad & 15u)) return fail(SI_ERR_INVALID, "gradient must be 16-byte aligned");
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t n = g->n;
  if (n == 0) {
    if (d_energy) SI_CUDA_TRY(cudaMemsetAsync(d_energy, 0, sizeof(double), st));
    return SI_OK;
  }
  WalkParams P;
  const float d = r * g->lat.inv_s;
  P.dg = d + (float)g->lat.eps;
  const float thr = d - 1.f;
  P.rt_b2 = thr <= 0.f ? 0 : (int)floorf(thr * thr) + 1;
  P.incl_b2 = -1;
  P.incl_d2 = 0.f;
  const float r2 = r * r;
  const float inv_r2 = 1.f / r2;
  const bool classes = g->ensure_classes(P.dg, st) && g->cls_smem_bytes > 0;
  const GridDev dv = g->dev();
  unsigned blocks = (unsigned)((n + kReduceThreads - 1) / kReduceThreads);
  const size_t smem = classes ? g->cls_smem_bytes : 0;
  const int n_entries = classes ? (int)g->cls_host.size() : 0;
  if (classes) {
    auto kern = d_grad ? k_reduce<true, true> : k_reduce<false, true>;
    SI_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    SI_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kReduceThreads, smem));
    blocks = std::min<unsigned>(blocks, (unsigned)std::max(1, std::min(per_sm, 16)) * 148u);
  }
  if ((int64_t)blocks > g->partial_len) return fail(SI_ERR_INTERNAL, "partial buffer too small");
  if (d_grad && classes)
    SI_KLAUNCH("k_reduce_grad", st,
               k_reduce<true, true><<<blocks, kReduceThreads, smem, st>>>(
                   dv, P, r2, inv_r2, n_entries, d_grad_scale, (float4 *)d_grad, g->partial));
  else if (d_grad)
    SI_KLAUNCH("k_reduce_grad_eq2", st,
               k_reduce<true, false><<<blocks, kReduceThreads, 0, st>>>(
                   dv, P, r2, inv_r2, 0, d_grad_scale, (float4 *)d_grad, g->partial));
  else if (classes)
    SI_KLAUNCH("k_reduce", st,
               k_reduce<false, true><<<blocks, kReduceThreads, smem, st>>>(dv, P, r2, inv_r2, n_entries,
                                                                          nullptr, nullptr, g->partial));
  else
    SI_KLAUNCH("k_reduce_eq2", st,
               k_reduce<false, false><<<blocks, kReduceThreads, 0, st>>>(dv, P, r2, inv_r2, 0, nullptr,
                                                                        nullptr, g->partial));
  if (d_energy) {
    SI_KLAUNCH("k_reduce_final", st, k_reduce_final<<<1, 1024, 0, st>>>(g->partial, (int)blocks, d_energy));
  }
  return SI_OK;
}
