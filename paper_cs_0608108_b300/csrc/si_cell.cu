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

template <bool WRITE>
struct CellSmem {
  float4 c[kCellCap];                  // candidate in the query frame; x = NaN: outside cell; w = slot bits
  // write pass: sort keys (input index << 32 | staging slot); after the
  // permutation into id order the first kCellCap ints hold the ids
  unsigned long long key[WRITE ? kCellKeyCap : 1];
  union {
    struct {                           // gather phase: the cell-level sphere's target cells
      unsigned tkey[kCellTCap];
      int tbeg[kCellTCap];
      int tcnt[kCellTCap];
      int tpre[kCellTCap + 1];
      unsigned char tcode[kCellTCap];
    } t;
    unsigned mask[kCellMaskCap];       // test phase: ballot of each (query, 32 candidates) item
  } u;
  long long pos[kCellMaxQ];            // count (count pass) / write position (write pass)
  int nt, nc, out_seen, item;
};

size_t cell_smem_bytes() { return sizeof(CellSmem<true>); }

__device__ __forceinline__ int warp_incl_scan_i(int v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

// Ascending bitonic sort of P 64-bit keys (P a power of two, >= 32) by the
// whole block.  Element i sits in row i/32, lane i%32.  Stages whose partner
// distance j is below 32 stay inside a row and run in registers with warp
// shuffles; wider stages go through shared memory.  Standard network:
// at merge size k, element i sorts ascending when (i & k) == 0.
__device__ __forceinline__ unsigned long long bitonic_row_stage(unsigned long long x, int i, int lane,
                                                                int k, int j) {
  const unsigned long long y = __shfl_xor_sync(0xffffffffu, x, j);
  const bool up = (i & k) == 0;
  const bool lower = (lane & j) == 0;
  const unsigned long long lo = x < y ? x : y, hi = x < y ? y : x;
  return (lower == up) ? lo : hi;
}

__device__ void block_sort_u64(unsigned long long *a, int P) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int rows = P >> 5;
  // merge sizes 2..32: every row on its own, in registers
  for (int r = wid; r < rows; r += nw) {
    const int i = r * 32 + lane;
    unsigned long long x = a[i];
    for (int k = 2; k <= 32; k <<= 1)
      for (int j = k >> 1; j > 0; j >>= 1) x = bitonic_row_stage(x, i, lane, k, j);
    a[i] = x;
  }
  __syncthreads();
  for (int k = 64; k <= P; k <<= 1) {
    for (int j = k >> 1; j >= 32; j >>= 1) {
      for (int i = threadIdx.x; i < P; i += blockDim.x) {
        const int l = i ^ j;
        if (l > i) {
          const unsigned long long x = a[i], y = a[l];
          if ((x > y) == ((i & k) == 0)) {
            a[i] = y;
            a[l] = x;
          }
        }
      }
      __syncthreads();
    }
    for (int r = wid; r < rows; r += nw) {
      const int i = r * 32 + lane;
      unsigned long long x = a[i];
      for (int j = 16; j > 0; j >>= 1) x = bitonic_row_stage(x, i, lane, k, j);
      a[i] = x;
    }
    __syncthreads();
  }
}

template <bool WRITE>
__global__ void __launch_bounds__(kCellThreads, 2) k_cell(GridDev g, WalkParams P, Band B, unsigned flags,
                                                       const int *__restrict__ heavy, int *work,
                                                       int *__restrict__ over,
                                                       long long *__restrict__ counts,
                                                       const long long *__restrict__ offsets,
                                                       int *__restrict__ ids, long long cap) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  CellSmem<WRITE> &S = *reinterpret_cast<CellSmem<WRITE> *>(smem_raw);
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
        S.u.t.tkey[t] = tk;
        S.u.t.tbeg[t] = b;
        S.u.t.tcnt[t] = c;
        S.u.t.tcode[t] = (unsigned char)code;
      }
      __syncthreads();
      const int nt = S.nt;
      // 2. prefix of target sizes (one warp)
      if (wid == 0) {
        int run = 0;
        for (int b0 = 0; b0 < nt; b0 += 32) {
          const int t = b0 + lane;
          const int v = t < nt ? S.u.t.tcnt[t] : 0;
          const int inc = warp_incl_scan_i(v);
          if (t < nt) S.u.t.tpre[t] = run + inc - v;
          run += __shfl_sync(0xffffffffu, inc, 31);
        }
        if (lane == 0) S.u.t.tpre[nt] = run;
      }
      __syncthreads();
      const int ntot = S.u.t.tpre[nt];
      // 3. gather candidates within d of the query cell box, in the query
      //    frame; each thread keeps kGather loads in flight
      constexpr int kGather = 4;
      for (int base = 0; base < ntot; base += kGather * blockDim.x) {
        int cj[kGather];
        unsigned code[kGather];
        float4 p[kGather];
#pragma unroll
        for (int r = 0; r < kGather; ++r) {
          const int f = base + r * blockDim.x + tid;
          cj[r] = -1;
          code[r] = 0;
          if (f < ntot) {
            int lo = 0, hi = nt - 1;
            while (lo < hi) {
              const int mid = (lo + hi + 1) >> 1;
              if (S.u.t.tpre[mid] <= f) lo = mid;
              else hi = mid - 1;
            }
            cj[r] = S.u.t.tbeg[lo] + (f - S.u.t.tpre[lo]);
            code[r] = S.u.t.tcode[lo];
          }
        }
#pragma unroll
        for (int r = 0; r < kGather; ++r) p[r] = cj[r] >= 0 ? g.spos[cj[r]] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int r = 0; r < kGather; ++r) {
          bool keep = false;
          float4 cp = p[r];
          if (cj[r] >= 0) {
            if (code[r] & 64u) {
              cp.x = __int_as_float(0x7fc00000);   // outside cell: FP64 test for every pair
              keep = true;
            } else {
              if (code[r] & 3u) cp.x += (code[r] & 1u) ? g.Lx : -g.Lx;
              if (code[r] & 12u) cp.y += (code[r] & 4u) ? g.Ly : -g.Ly;
              if (code[r] & 48u) cp.z += (code[r] & 16u) ? g.Lz : -g.Lz;
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
              cp.w = __int_as_float(cj[r]);
              S.c[idx] = cp;
              if (WRITE) S.key[idx] = ((unsigned long long)(unsigned)__ldg(g.perm + cj[r]) << 32) | (unsigned)idx;
            }
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
    for (int i = tid; i < nq; i += blockDim.x) S.pos[i] = 0;
    int *cid = reinterpret_cast<int *>(S.key);    // ids in candidate order (write pass)
    if (WRITE) {
      // candidates into ascending input-index order: sort the keys, then
      // permute positions and ids through registers
      int P2 = 32;
      while (P2 < nc) P2 <<= 1;
      for (int i = nc + tid; i < P2; i += blockDim.x) S.key[i] = ~0ull;
      __syncthreads();
      block_sort_u64(S.key, P2);
      constexpr int kPer = (kCellCap + kCellThreads - 1) / kCellThreads;
      float4 rc[kPer];
      int rid[kPer];
#pragma unroll
      for (int r = 0; r < kPer; ++r) {
        const int k = tid + r * kCellThreads;
        if (k < nc) {
          const unsigned long long kk = S.key[k];
          rc[r] = S.c[(int)(kk & 0xffffffffull)];
          rid[r] = (int)(kk >> 32);
        }
      }
      __syncthreads();
#pragma unroll
      for (int r = 0; r < kPer; ++r) {
        const int k = tid + r * kCellThreads;
        if (k < nc) {
          S.c[k] = rc[r];
          cid[k] = rid[r];
        }
      }
    }
    __syncthreads();
    // 4. (query, 32 candidates) items spread evenly over all warps; each
    //    item is one ballot: lanes test their candidate against the query
    const int nchunk = (nc + 31) >> 5;
    const int qbatch = WRITE ? max(1, min(nq, kCellMaskCap / nchunk)) : nq;
    for (int qb = 0; qb < nq; qb += qbatch) {
      const int nqb = min(qbatch, nq - qb);
      const int nitems = nqb * nchunk;
      for (int it = wid; it < nitems; it += nw) {
        const int ql = it / nchunk;
        const int k = (it - ql * nchunk) * 32 + lane;
        const int sq = qs + qb + ql;               // the query's sorted slot
        const float4 q = g.spos[sq];
        bool hit = false;
        if (k < nc) {
          const float4 c = S.c[k];
          const float dx = c.x - q.x, dy = c.y - q.y, dz = c.z - q.z;
          const float d2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
          const int j = __float_as_int(c.w);
          hit = d2 <= B.lo_w;
          if (!hit && !(d2 > B.hi_w)) hit = canon_d2(q, g.spos[j], g) <= B.r2;
          if (!incl_self) hit = hit && j != sq;
        }
        const unsigned m = __ballot_sync(0xffffffffu, hit);
        if (lane == 0) {
          if (WRITE) S.u.mask[it] = m;
          else if (m) atomicAdd(reinterpret_cast<unsigned long long *>(&S.pos[qb + ql]),
                                (unsigned long long)__popc(m));
        }
      }
      if (WRITE) {
        __syncthreads();
        // 5. emission: one warp per query, chunks in ascending id order
        for (int ql = wid; ql < nqb; ql += nw) {
          const int id = __ldg(g.perm + qs + qb + ql);
          long long base = offsets[id];
          for (int ch = 0; ch < nchunk; ++ch) {
            const unsigned m = S.u.mask[ql * nchunk + ch];
            if (m) {
              if ((m >> lane) & 1u) ids[base + __popc(m & lt_mask)] = cid[ch * 32 + lane];
              base += __popc(m);
            }
          }
          if (lane == 0 && base != offsets[id + 1]) atomicOr(g.status, ST_INTERNAL);
        }
        __syncthreads();
      }
    }
    if (!WRITE) {
      __syncthreads();
      for (int i = tid; i < nq; i += blockDim.x) counts[__ldg(g.perm + qs + i)] = S.pos[i];
    }
    __syncthreads();
  }
}

si_status launch_cell_pass(bool write, const GridDev &g, const WalkParams &P, const Band &B,
                           unsigned flags, const int *heavy, int *work, int *over, long long *counts,
                           const long long *offsets, int *ids, long long cap, cudaStream_t st) {
  if (write) {
    const size_t smem = sizeof(CellSmem<true>);
    const int grid = 148 * 2;
    SI_CUDA_TRY(cudaFuncSetAttribute(k_cell<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    SI_KLAUNCH("k_cell_write", st,
               k_cell<true><<<grid, kCellThreads, smem, st>>>(g, P, B, flags, heavy, work, over, counts,
                                                              offsets, ids, cap));
  } else {
    const size_t smem = sizeof(CellSmem<false>);
    const int grid = 148 * 2;   // 2 blocks of 512 threads fit the register file
    SI_CUDA_TRY(cudaFuncSetAttribute(k_cell<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    SI_KLAUNCH("k_cell_count", st,
               k_cell<false><<<grid, kCellThreads, smem, st>>>(g, P, B, flags, heavy, work, over, counts,
                                                               offsets, ids, cap));
  }
  return SI_OK;
}

}  // namespace si
