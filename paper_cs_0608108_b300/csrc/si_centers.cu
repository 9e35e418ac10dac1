// Query centers given by the caller (Sec. I, Sec. II.A: a query is a center
// and a radius; the all-agents mode is the special case where the centers
// are the objects themselves).
//
// The centers are put in coarse cell order before the query kernels run, so
// that neighbouring threads and warps walk neighbouring cells: a counting
// sort on a bucket key made of the top (at most 5) bits of each cell
// coordinate, with one more bucket for centers outside the region.  With
// `split`, the key also holds the class of the center's cell in the point
// lattice (cell_class: the points in and around it), which picks the kernel:
// light cells one thread per center, the others one warp per center.  A
// center with a non-finite coordinate, or one outside its box on a cyclic
// axis, is not queried: its result is empty and the grid's status records
// SI_ERR_INVALID (reported by si_grid_sync).
#include <algorithm>

#include "si_host.h"
#include "si_radius.cuh"

namespace si {

struct CenterBuckets {
  int cb[3];      // coarse bits per axis
  int nb;         // cell buckets per group (2^(cbx+cby+cbz)); bucket nb is the outside one
};

static CenterBuckets center_buckets(const Lattice &lat) {
  CenterBuckets B;
  int bits = 0;
  for (int a = 0; a < 3; ++a) {
    B.cb[a] = std::min(lat.w[a], 5);
    bits += B.cb[a];
  }
  B.nb = 1 << bits;
  return B;
}

// Bucket of every center: group (0: light or every valid center, 1: the
// rest) times (nb + 1) plus its coarse cell; invalid centers take the last
// bucket, 2 (nb + 1).  count[1 + bucket] gets the histogram.
__global__ void __launch_bounds__(256) k_center_key(const float4 *__restrict__ c, int m, GridDev g, int split,
                                                    int cbx, int cby, int cbz, int nb,
                                                    uint2 *__restrict__ key_slot, int *__restrict__ count) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  const float4 p = __ldg(c + i);
  bool out = false, bad = false;
  const int cx = axis_cell(p.x, g.ox, g.Lx, g.inv_s, g.wx, g.cyc & 1u, out, bad);
  const int cy = axis_cell(p.y, g.oy, g.Ly, g.inv_s, g.wy, (g.cyc >> 1) & 1u, out, bad);
  const int cz = axis_cell(p.z, g.oz, g.Lz, g.inv_s, g.wz, (g.cyc >> 2) & 1u, out, bad);
  int bucket;
  if (bad) {
    atomicOr(g.status, ST_INVALID);
    bucket = 2 * (nb + 1);
  } else {
    const unsigned key = out ? g.outside : pack3(cx, cy, cz, g);
    const int grp = split ? (cell_class(g.cell_start, key, g.outside, g.wx, g.wy, g.wz) == kCellLight ? 0 : 1) : 0;
    const int coarse = out ? nb
                           : (((cz >> (g.wz - cbz)) << (cbx + cby)) | ((cy >> (g.wy - cby)) << cbx) |
                              (cx >> (g.wx - cbx)));
    bucket = grp * (nb + 1) + coarse;
  }
  const int rank = atomicAdd(count + 1 + bucket, 1);
  key_slot[i] = make_uint2((unsigned)bucket, (unsigned)rank);
}

// Scatter into bucket order and list the two groups by slot.  start[b] is
// the first slot of bucket b (start[0] = 0).
__global__ void __launch_bounds__(256) k_center_scatter(const float4 *__restrict__ c, int m, int nb,
                                                        const uint2 *__restrict__ key_slot,
                                                        const int *__restrict__ start, float4 *__restrict__ cpos,
                                                        int *__restrict__ cid, int *__restrict__ l0,
                                                        int *__restrict__ l1, CenterOut out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  const int n0 = __ldg(start + nb + 1), n01 = __ldg(start + 2 * (nb + 1));
  if (i == 0) {
    l0[0] = n0;
    l1[0] = n01 - n0;
  }
  const uint2 ks = key_slot[i];
  const int dst = __ldg(start + ks.x) + (int)ks.y;
  cpos[dst] = __ldg(c + i);
  cid[dst] = i;
  if (dst < n0) {
    l0[1 + dst] = dst;
  } else if (dst < n01) {
    l1[1 + dst - n0] = dst;
  } else {   // invalid center: empty result
    if (out.rad_counts) out.rad_counts[i] = 0;
    if (out.counts) {
      out.counts[i] = 0;
      for (int k = 0; k < out.K; ++k) {
        out.ids[(size_t)i * out.K + k] = -1;
        if (out.d2) out.d2[(size_t)i * out.K + k] = __int_as_float(0x7f800000);
      }
    }
  }
}

}  // namespace si

using namespace si;

si_status si_grid::ensure_centers(int64_t m, bool stage) {
  const int64_t want = std::max<int64_t>(m, 1);
  if (want > ccap) {
    const int64_t c = std::max<int64_t>(want, ccap + ccap / 2);
    cudaFree(cpos);
    cudaFree(cid);
    cudaFree(ckey);
    cudaFree(clist0);
    cudaFree(clist1);
    cudaFree(clong);
    cudaFree(chuge);
    cudaFree(cstage);
    cudaFree(cscan64);
    cscan64 = nullptr;
    cpos = nullptr;
    cid = clist0 = clist1 = clong = chuge = cstage = nullptr;
    ckey = nullptr;
    ccap = 0;
    cstage_cap = 0;
    cudaError_t e = cudaMalloc((void **)&cpos, c * sizeof(float4));
    if (e == cudaSuccess) e = cudaMalloc((void **)&cid, c * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc((void **)&ckey, c * sizeof(uint2));
    if (e == cudaSuccess) e = cudaMalloc((void **)&clist0, (c + 1) * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc((void **)&clist1, (c + 1) * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc((void **)&clong, (c + 1) * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc((void **)&chuge, (c + 1) * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc((void **)&cscan64, scan_scratch_elems(c + 1) * sizeof(long long));
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(SI_ERR_OOM, "query-center buffers");
    }
    ccap = c;
  }
  if (!cbuck) {
    const int64_t nbt = 2 * ((int64_t)center_buckets(lat).nb + 1) + 1;
    cudaError_t e = cudaMalloc((void **)&cbuck, (nbt + 1) * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc((void **)&cscan, scan_scratch_elems(nbt) * sizeof(int));
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(SI_ERR_OOM, "query-center buckets");
    }
  }
  // the short-list staging area is optional: without it the write pass
  // walks the cells again
  if (stage && cstage_cap < ccap) {
    cudaFree(cstage);
    cstage = nullptr;
    cstage_cap = 0;
    if (cudaMalloc((void **)&cstage, (size_t)kInlineSort * (size_t)ccap * sizeof(int)) == cudaSuccess)
      cstage_cap = ccap;
    else
      cudaGetLastError();
  }
  return SI_OK;
}

namespace si {

si_status prepare_centers(si_grid *g, const float *d_centers, int64_t m, bool split, bool stage,
                          const CenterOut &out, GridDev &dv, cudaStream_t st) {
  si_status s = g->ensure_centers(m, stage);
  if (s != SI_OK) return s;
  const CenterBuckets CB = center_buckets(g->lat);
  const int64_t nbt = 2 * ((int64_t)CB.nb + 1) + 1;
  dv = g->dev();
  dv.qpos = g->cpos;
  dv.qid = g->cid;
  dv.q_agents = 0;
  SI_CUDA_TRY(cudaMemsetAsync(g->cbuck, 0, (nbt + 1) * sizeof(int), st));
  if (m == 0) {
    SI_CUDA_TRY(cudaMemsetAsync(g->clist0, 0, sizeof(int), st));
    SI_CUDA_TRY(cudaMemsetAsync(g->clist1, 0, sizeof(int), st));
    return SI_OK;
  }
  const unsigned blocks = (unsigned)((m + 255) / 256);
  SI_KLAUNCH("k_center_key", st,
             k_center_key<<<blocks, 256, 0, st>>>((const float4 *)d_centers, (int)m, dv, split ? 1 : 0, CB.cb[0],
                                                  CB.cb[1], CB.cb[2], CB.nb, g->ckey, g->cbuck));
  if ((s = scan_inclusive_i32(g->cbuck + 1, g->cbuck + 1, nbt, g->cscan, st)) != SI_OK) return s;
  SI_KLAUNCH("k_center_scatter", st,
             k_center_scatter<<<blocks, 256, 0, st>>>((const float4 *)d_centers, (int)m, CB.nb, g->ckey, g->cbuck,
                                                      g->cpos, g->cid, g->clist0, g->clist1, out));
  return SI_OK;
}

}  // namespace si
