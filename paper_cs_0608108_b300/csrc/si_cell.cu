// Radius query for heavily loaded cells (Sec. I: with many objects per cell
// the cost of processing cells dominates, so it pays to share that work).
//
// One block per query cell holding at least kHeavyMin points:
//  1. the cell-level sphere: every table entry whose minimum cell-to-cell
//     bound satisfies b^2 <= floor(d^2) (Sec. II.A) is translated to the query
//     cell (SWAR add/mask/pack, Sec. II.B); non-empty target cells are listed;
//  2. their points are moved into the query cell's frame (image shift on
//     wrapped cyclic axes) and kept when they lie within d of the query cell
//     box -- the union of the spheres of every point of the cell -- and are
//     staged in shared memory;
//  3. write pass only: the staged candidates are sorted by input index;
//  4. lanes take 32 candidates at a time, warps take the cell's queries: each
//     (query, 32 candidates) test is one ballot; the count pass adds popc, the
//     write pass appends the hits at the query's running position, so every
//     list comes out ascending without a separate sort and with coalesced
//     stores.
// A cell whose candidates or queries do not fit is handed to the per-query
// path (overflow list).
#include <cmath>

#include "si_host.h"
#include "si_radius.cuh"
#include "si_walk.cuh"

namespace si {

struct CellSmem {
  float4 c[kCellCap];                  // candidate in the query frame; x = NaN: outside cell; w = slot bits
  unsigned long long key[kCellKeyCap]; // write pass: (input index << 32) | staging slot
  float4 q[kCellMaxQ];                 // the cell's query points
  long long pos[kCellMaxQ];            // count (count pass) / running write position (write pass)
  int qid[kCellMaxQ];                  // input index of each query
  unsigned tkey[kCellTCap];
  int tbeg[kCellTCap];
  int tcnt[kCellTCap];
  int tpre[kCellTCap + 1];
  unsigned char tcode[kCellTCap];
  int nt, nc, out_seen, item;
};

size_t cell_smem_bytes() { return sizeof(CellSmem); }

__device__ __forceinline__ int warp_incl_scan_i(int v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

// Ascending bitonic sort of P (a power of two) 64-bit keys by the whole block.
__device__ void block_sort_u64(unsigned long long *a, int P) {
  for (int k = 2; k <= P; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < P; i += blockDim.x) {
        const int l = i ^ j;
        if (l > i) {
          const unsigned long long x = a[i], y = a[l];
          const bool up = (i & k) == 0;
          if ((x > y) == up) {
            a[i] = y;
            a[l] = x;
          }
        }
      }
      __syncthreads();
    }
  }
}

template <bool WRITE>
__global__ void __launch_bounds__(kCellThreads) k_cell(GridDev g, WalkParams P, Band B, unsigned flags,
                                                       const int *__restrict__ heavy, int *work,
                                                       int *__restrict__ over,
                                                       long long *__restrict__ counts,
                                                       const long long *__restrict__ offsets,
                                                       int *__restrict__ ids, long long cap) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  CellSmem &S = *reinterpret_cast<CellSmem *>(smem_raw);
  const int nheavy = heavy[0];
  const int n = min((int)(P.dg * P.dg), g.n_max);
  const int n_tab = __ldg(g.tab_end + n);
  const bool incl_self = flags & SI_INCLUDE_SELF;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  const unsigned lt_mask = (1u << lane) - 1u;
  const float box2 = (P.dg + g.eps) * (P.dg + g.eps);
  if (WRITE && offsets[g.n] > cap) {
    if (tid == 0 && blockIdx.x == 0) atomicOr(g.status, ST_CAPACITY);
    return;
  }
  for (;;) {
    if (tid == 0) S.item = atomicAdd(work, 1);
    __syncthreads();
    const int item = S.item;
    if (item >= nheavy) return;
    const unsigned key = (unsigned)heavy[1 + item];
    const int qs = g.cell_start[key], nq = g.cell_start[key + 1] - qs;
    const int cx = (int)(key & ((1u << g.wx) - 1u));
    const int cy = (int)((key >> g.wx) & ((1u << g.wy) - 1u));
    const int cz = (int)(key >> (g.wx + g.wy));
    const unsigned long long cu = unpack3(cx, cy, cz, g);
    if (tid == 0) {
      S.nt = 0;
      S.nc = 0;
      S.out_seen = 0;
    }
    __syncthreads();
    bool fits = nq <= kCellMaxQ && n_tab <= kCellTCap;
    if (fits) {
      // 1. non-empty target cells of the cell-level sphere
      for (int e = tid; e < n_tab; e += blockDim.x) {
        const TabEntry E = g.tab[e];
        const unsigned long long s = cu + E.unp;
        unsigned tk, code = 0;
        if (s & g.guard_non) {
          if (atomicExch(&S.out_seen, 1)) continue;   // the outside cell is listed once
          tk = g.outside;
          code = 64u;
        } else {
          tk = repack(s & g.valid, g);
          if (s & g.gx) code |= E.ox > 0 ? 1u : 2u;
          if (s & g.gy) code |= (E.oy > 0 ? 1u : 2u) << 2;
          if (s & g.gz) code |= (E.oz > 0 ? 1u : 2u) << 4;
        }
        const int b = __ldg(g.cell_start + tk), c = __ldg(g.cell_start + tk + 1) - b;
        if (c == 0) continue;
        const int t = atomicAdd(&S.nt, 1);
        S.tkey[t] = tk;
        S.tbeg[t] = b;
        S.tcnt[t] = c;
        S.tcode[t] = (unsigned char)code;
      }
      __syncthreads();
      const int nt = S.nt;
      // 2. prefix of target sizes (one warp)
      if (wid == 0) {
        int run = 0;
        for (int b0 = 0; b0 < nt; b0 += 32) {
          const int t = b0 + lane;
          const int v = t < nt ? S.tcnt[t] : 0;
          const int inc = warp_incl_scan_i(v);
          if (t < nt) S.tpre[t] = run + inc - v;
          run += __shfl_sync(0xffffffffu, inc, 31);
        }
        if (lane == 0) S.tpre[nt] = run;
      }
      __syncthreads();
      const int ntot = S.tpre[nt];
      // 3. gather candidates within d of the query cell box, in the query frame
      for (int base = 0; base < ntot; base += blockDim.x) {
        const int f = base + tid;
        bool keep = false;
        float4 cp = make_float4(0.f, 0.f, 0.f, 0.f);
        int cj = 0;
        if (f < ntot) {
          int lo = 0, hi = nt - 1;
          while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (S.tpre[mid] <= f) lo = mid;
            else hi = mid - 1;
          }
          cj = S.tbeg[lo] + (f - S.tpre[lo]);
          const float4 p = g.spos[cj];
          const unsigned code = S.tcode[lo];
          if (code & 64u) {
            cp = make_float4(__int_as_float(0x7fc00000), p.y, p.z, 0.f);   // FP64 test for every pair
            keep = true;
          } else {
            cp = p;
            if (code & 3u) cp.x += (code & 1u) ? g.Lx : -g.Lx;
            if (code & 12u) cp.y += (code & 4u) ? g.Ly : -g.Ly;
            if (code & 48u) cp.z += (code & 16u) ? g.Lz : -g.Lz;
            const float ux = (cp.x - g.ox) * g.inv_s - (float)cx;
            const float uy = (cp.y - g.oy) * g.inv_s - (float)cy;
            const float uz = (cp.z - g.oz) * g.inv_s - (float)cz;
            const float gx = fmaxf(fmaxf(-ux, ux - 1.f), 0.f);
            const float gy = fmaxf(fmaxf(-uy, uy - 1.f), 0.f);
            const float gz = fmaxf(fmaxf(-uz, uz - 1.f), 0.f);
            keep = fmaf(gz, gz, fmaf(gy, gy, gx * gx)) <= box2;
          }
        }
        const unsigned m = __ballot_sync(0xffffffffu, keep);
        int wbase = 0;
        if (lane == 0 && m) wbase = atomicAdd(&S.nc, __popc(m));
        wbase = __shfl_sync(0xffffffffu, wbase, 0);
        if (keep) {
          const int idx = wbase + __popc(m & lt_mask);
          if (idx < kCellCap) {
            cp.w = __int_as_float(cj);
            S.c[idx] = cp;
            if (WRITE) S.key[idx] = ((unsigned long long)(unsigned)__ldg(g.perm + cj) << 32) | (unsigned)idx;
          }
        }
      }
      __syncthreads();
      fits = S.nc <= kCellCap;
    }
    if (!fits) {
      if (!WRITE && tid == 0) {
        const int o = atomicAdd(over, 1);
        over[1 + o] = (int)key;
      }
      __syncthreads();
      continue;
    }
    const int nc = S.nc;
    for (int i = tid; i < nq; i += blockDim.x) {
      S.q[i] = g.spos[qs + i];
      if (WRITE) {
        const int id = __ldg(g.perm + qs + i);
        S.qid[i] = id;
        S.pos[i] = offsets[id];
      } else {
        S.pos[i] = 0;
      }
    }
    if (WRITE) {
      int P2 = 32;
      while (P2 < nc) P2 <<= 1;
      for (int i = nc + tid; i < P2; i += blockDim.x) S.key[i] = ~0ull;
      __syncthreads();
      block_sort_u64(S.key, P2);
    }
    __syncthreads();
    // 4. lanes = candidates (ascending input index in the write pass), warps = queries
    const int nchunk = (nc + 31) >> 5;
    for (int ch = 0; ch < nchunk; ++ch) {
      const int k = ch * 32 + lane;
      float4 c = make_float4(INFINITY, INFINITY, INFINITY, 0.f);
      int cid = -1;
      if (k < nc) {
        if (WRITE) {
          const unsigned long long kk = S.key[k];
          c = S.c[(int)(kk & 0xffffffffull)];
          cid = (int)(kk >> 32);
        } else {
          c = S.c[k];
        }
      }
      for (int qi = wid; qi < nq; qi += nw) {
        const float4 q = S.q[qi];
        const float dx = c.x - q.x, dy = c.y - q.y, dz = c.z - q.z;
        const float d2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
        bool hit = d2 <= B.lo_w;
        if (!hit && !(d2 > B.hi_w) && k < nc)
          hit = canon_d2(q, g.spos[__float_as_int(c.w)], g) <= B.r2;
        if (WRITE) {
          if (!incl_self) hit = hit && cid != S.qid[qi];
          const unsigned m = __ballot_sync(0xffffffffu, hit);
          if (m) {
            const long long base = S.pos[qi];
            if (hit) ids[base + __popc(m & lt_mask)] = cid;
            __syncwarp();
            if (lane == 0) S.pos[qi] = base + __popc(m);
            __syncwarp();
          }
        } else {
          const unsigned m = __ballot_sync(0xffffffffu, hit);
          if (lane == 0) S.pos[qi] += __popc(m);
        }
      }
    }
    __syncthreads();
    for (int i = tid; i < nq; i += blockDim.x) {
      if (WRITE) {
        if (S.pos[i] != offsets[S.qid[i] + 1]) atomicOr(g.status, ST_INTERNAL);
      } else {
        counts[__ldg(g.perm + qs + i)] = S.pos[i] - (incl_self ? 0 : 1);
      }
    }
    __syncthreads();
  }
}

si_status launch_cell_pass(bool write, const GridDev &g, const WalkParams &P, const Band &B,
                           unsigned flags, const int *heavy, int *work, int *over, long long *counts,
                           const long long *offsets, int *ids, long long cap, cudaStream_t st) {
  const size_t smem = sizeof(CellSmem);
  const int grid = 148 * 2;
  if (write) {
    SI_CUDA_TRY(cudaFuncSetAttribute(k_cell<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    SI_KLAUNCH("k_cell_write", st,
               k_cell<true><<<grid, kCellThreads, smem, st>>>(g, P, B, flags, heavy, work, over, counts,
                                                              offsets, ids, cap));
  } else {
    SI_CUDA_TRY(cudaFuncSetAttribute(k_cell<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    SI_KLAUNCH("k_cell_count", st,
               k_cell<false><<<grid, kCellThreads, smem, st>>>(g, P, B, flags, heavy, work, over, counts,
                                                               offsets, ids, cap));
  }
  return SI_OK;
}

}  // namespace si
