// Radius query for heavily loaded cells (Sec. I: with many objects per cell
// the cost of processing cells dominates, so it pays to share that work).
//
// One block per heavy query cell (heavy_cell), in a single
// pass that runs before the prefix sum of the list lengths:
//  1. the cell-level sphere: every table entry whose minimum cell-to-cell
//     bound satisfies b^2 <= floor(d^2) (Sec. II.A) is translated to the query
//     cell (SWAR add/mask/pack, Sec. II.B); non-empty target cells are listed;
//  2. their points are moved into the query cell's frame (image shift on
//     wrapped cyclic axes), kept when they lie within d of the query cell box
//     (the union of the spheres of every point of the cell) and staged in
//     shared memory;
//  3. the staged candidates are put in ascending input-index order: one
//     counting pass into 1024 buckets by the index's top bits, then an
//     insertion sort inside each (small) bucket;
//  4. warps take chunks of 32 candidates (lane = candidate) and test them
//     against every query of the cell: one ballot per (query, chunk);
//  5. each query's hits are counted, the cell reserves a region of a scratch
//     buffer with one atomic, and a warp per query stores its hits there,
//     ascending.  After the prefix sum, k_cell_copy moves every list to its
//     place in the output.
// A cell whose candidates or queries do not fit shared memory, or whose lists
// do not fit the scratch buffer, hands its queries to the per-query path.
#include <cmath>

#include "si_host.h"
#include "si_radius.cuh"
#include "si_walk.cuh"

namespace si {

constexpr int kBuckets = 1024;

struct CellSmem {
  float4 c[kCellCap];                      // candidate in the query frame; x = NaN: outside cell; w = slot bits
  unsigned long long key[2 * kCellCap];    // sort buffers: (input index << 32) | staging slot
  union {
    struct {                               // gather: the cell-level sphere's target cells
      unsigned tkey[kCellTCap];
      int tbeg[kCellTCap];
      int tcnt[kCellTCap];
      int tpre[kCellTCap + 1];
      unsigned char tcode[kCellTCap];
    } t;
    struct {                               // bucket sort
      int start[kBuckets];
      int cur[kBuckets];
    } b;
    unsigned mask[kCellMaskCap];           // tests: ballot of each (query, chunk)
  } u;
  float4 q[kCellMaxQ];                     // the cell's query points
  int qcnt[kCellMaxQ];                     // hits per query of the current batch
  int qoff[kCellMaxQ];                     // their offsets inside the batch's scratch region
  int scan[kCellThreads / 32];
  long long base;                          // the batch's scratch region
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

// Exclusive block scan of one int per thread; returns the block total.
__device__ __forceinline__ int block_excl_scan_i(int v, int &total, int *scan) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int inc = warp_incl_scan_i(v);
  if (lane == 31) scan[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    const int x = lane < nw ? scan[lane] : 0;
    const int y = warp_incl_scan_i(x);
    if (lane < nw) scan[lane] = y;
  }
  __syncthreads();
  total = scan[nw - 1];
  const int before = wid > 0 ? scan[wid - 1] : 0;
  __syncthreads();
  return before + inc - v;
}

// Packed FP32 pairs (low half = first value) and the squared distance of
// two candidates to one query with f32x2 instructions.
__device__ __forceinline__ unsigned long long pack2(float a, float b) {
  return ((unsigned long long)__float_as_uint(b) << 32) | (unsigned long long)__float_as_uint(a);
}
__device__ __forceinline__ float lo_half(unsigned long long v) { return __uint_as_float((unsigned)v); }
__device__ __forceinline__ float hi_half(unsigned long long v) { return __uint_as_float((unsigned)(v >> 32)); }

__device__ __forceinline__ unsigned long long dist2_x2(unsigned long long X, unsigned long long Y,
                                                       unsigned long long Z, const float4 &q) {
  const unsigned long long qx = pack2(q.x, q.x), qy = pack2(q.y, q.y), qz = pack2(q.z, q.z);
  unsigned long long dx, dy, dz, d2;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(dx) : "l"(X), "l"(qx));
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(dy) : "l"(Y), "l"(qy));
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(dz) : "l"(Z), "l"(qz));
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d2) : "l"(dx), "l"(dx));
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d2) : "l"(dy), "l"(dy), "l"(d2));
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d2) : "l"(dz), "l"(dz), "l"(d2));
  return d2;
}

__global__ void __launch_bounds__(kCellThreads, 2) k_cell(GridDev g, WalkParams P, Band B, unsigned flags,
                                                          const int *__restrict__ heavy, int *work,
                                                          int *__restrict__ over,
                                                          long long *__restrict__ counts,
                                                          long long *__restrict__ scr_off,
                                                          int *__restrict__ scratch, long long scr_cap,
                                                          unsigned long long *scr_top) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  CellSmem &S = *reinterpret_cast<CellSmem *>(smem_raw);
  const int nheavy = heavy[0];
  const int n = min((int)(P.dg * P.dg), g.n_max);
  const int n_tab = __ldg(g.tab_end + n);
  const bool incl_self = flags & SI_INCLUDE_SELF;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  const unsigned lt_mask = (1u << lane) - 1u;
  const float box2 = (P.dg + g.eps) * (P.dg + g.eps);
  // bucket of an input index: its top 10 bits within [0, n)
  int idbits = 1;
  while (idbits < 31 && (1 << idbits) < g.n) ++idbits;
  const int bshift = max(idbits - 10, 0);
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
      // 2a. prefix of target sizes (one warp)
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
      // 2b. gather: candidates within d of the query cell box, in the query frame
      constexpr int kGather = 4;
      for (int base = 0; base < ntot; base += kGather * blockDim.x) {
        int cj[kGather], tt[kGather];
        float4 p[kGather];
#pragma unroll
        for (int r = 0; r < kGather; ++r) {
          const int f = base + r * blockDim.x + tid;
          cj[r] = -1;
          tt[r] = 0;
          if (f < ntot) {
            int lo = 0, hi = nt - 1;
            while (lo < hi) {
              const int mid = (lo + hi + 1) >> 1;
              if (S.u.t.tpre[mid] <= f) lo = mid;
              else hi = mid - 1;
            }
            tt[r] = lo;
            cj[r] = S.u.t.tbeg[lo] + (f - S.u.t.tpre[lo]);
          }
        }
#pragma unroll
        for (int r = 0; r < kGather; ++r) p[r] = cj[r] >= 0 ? g.spos[cj[r]] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int r = 0; r < kGather; ++r) {
          bool keep = false;
          if (cj[r] >= 0) {
            const unsigned code = S.u.t.tcode[tt[r]];
            if (code & 64u) {
              p[r].x = __int_as_float(0x7fc00000);   // outside cell: FP64 test for every pair
              keep = true;
            } else {
              if (code & 3u) p[r].x += (code & 1u) ? g.Lx : -g.Lx;
              if (code & 12u) p[r].y += (code & 4u) ? g.Ly : -g.Ly;
              if (code & 48u) p[r].z += (code & 16u) ? g.Lz : -g.Lz;
              const float ux = (p[r].x - g.ox) * g.inv_s - (float)cx;
              const float uy = (p[r].y - g.oy) * g.inv_s - (float)cy;
              const float uz = (p[r].z - g.oz) * g.inv_s - (float)cz;
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
            const int at = wbase + __popc(m & lt_mask);
            if (at < kCellCap) {
              float4 cp = p[r];
              cp.w = __int_as_float(cj[r]);
              S.c[at] = cp;
              S.key[at] = ((unsigned long long)(unsigned)__ldg(g.perm + cj[r]) << 32) | (unsigned)at;
            }
          }
        }
      }
      __syncthreads();
      fits = S.nc <= kCellCap;
    }
    if (!fits) {
      // the per-query path takes every query of this cell
      for (int i = tid; i < nq; i += blockDim.x) {
        const int o = atomicAdd(over, 1);
        over[1 + o] = qs + i;
        scr_off[__ldg(g.perm + qs + i)] = -1;
      }
      __syncthreads();
      continue;
    }
    const int nc = S.nc;
    for (int i = tid; i < nq; i += blockDim.x) S.q[i] = g.spos[qs + i];
    // 3. ascending input index: counting pass into buckets, then each bucket
    //    (a handful of keys) sorted by insertion
    unsigned long long *src = S.key, *dst = S.key + kCellCap;
    for (int b = tid; b < kBuckets; b += blockDim.x) S.u.b.start[b] = 0;
    __syncthreads();
    for (int p = tid; p < nc; p += blockDim.x) atomicAdd(&S.u.b.start[(int)(src[p] >> 32) >> bshift], 1);
    __syncthreads();
    {
      constexpr int kPerB = kBuckets / kCellThreads;
      int v[kPerB], sum = 0;
#pragma unroll
      for (int r = 0; r < kPerB; ++r) {
        v[r] = S.u.b.start[tid * kPerB + r];
        sum += v[r];
      }
      int total;
      int run = block_excl_scan_i(sum, total, S.scan);
#pragma unroll
      for (int r = 0; r < kPerB; ++r) {
        S.u.b.start[tid * kPerB + r] = run;
        S.u.b.cur[tid * kPerB + r] = run;
        run += v[r];
      }
    }
    __syncthreads();
    for (int p = tid; p < nc; p += blockDim.x) {
      const unsigned long long x = src[p];
      dst[atomicAdd(&S.u.b.cur[(int)(x >> 32) >> bshift], 1)] = x;
    }
    __syncthreads();
    for (int b = tid; b < kBuckets; b += blockDim.x) {
      const int lo = S.u.b.start[b], hi = S.u.b.cur[b];
      for (int i = lo + 1; i < hi; ++i) {
        const unsigned long long x = dst[i];
        int p = i;
        while (p > lo && dst[p - 1] > x) {
          dst[p] = dst[p - 1];
          --p;
        }
        dst[p] = x;
      }
    }
    __syncthreads();
    // permute the candidates into id order; ids go to the spare buffer
    constexpr int kPer = (kCellCap + kCellThreads - 1) / kCellThreads;
    float4 rc[kPer];
    int rid[kPer];
#pragma unroll
    for (int r = 0; r < kPer; ++r) {
      const int k = tid + r * kCellThreads;
      if (k < nc) {
        const unsigned long long kk = dst[k];
        rc[r] = S.c[(int)(kk & 0xffffffffull)];
        rid[r] = (int)(kk >> 32);
      }
    }
    __syncthreads();
    int *cid = reinterpret_cast<int *>(src);
#pragma unroll
    for (int r = 0; r < kPer; ++r) {
      const int k = tid + r * kCellThreads;
      if (k < nc) {
        S.c[k] = rc[r];
        cid[k] = rid[r];
      }
    }
    __syncthreads();
    // 4. tests.  Items (two chunks of 32 candidates, group of queries) are
    //    spread over all warps; a lane holds candidates k and k + 32 and runs
    //    both distances at once with packed FP32x2 arithmetic (the same
    //    round-to-nearest operations, in the same order, as the scalar path).
    const int nchunk = (nc + 31) >> 5;
    const int npair = (nchunk + 1) >> 1;
    const int qbatch = max(1, min(nq, kCellMaskCap / max(nchunk, 1)));
    for (int qb = 0; qb < nq; qb += qbatch) {
      const int nqb = min(qbatch, nq - qb);
      const int qsz = max(1, min(nqb, (nqb * npair + 2 * nw - 1) / (2 * nw)));
      const int ngrp = (nqb + qsz - 1) / qsz;
      const int nitems = npair * ngrp;
      for (int it = wid; it < nitems; it += nw) {
        const int grp = it / npair;
        const int cp = it - grp * npair;
        const int k0 = cp * 64 + lane, k1 = k0 + 32;
        const float4 c0 = k0 < nc ? S.c[k0] : make_float4(INFINITY, INFINITY, INFINITY, 0.f);
        const float4 c1 = k1 < nc ? S.c[k1] : make_float4(INFINITY, INFINITY, INFINITY, 0.f);
        const unsigned long long X = pack2(c0.x, c1.x), Y = pack2(c0.y, c1.y), Z = pack2(c0.z, c1.z);
        const int ch0 = 2 * cp, ch1 = 2 * cp + 1;
        const int q_end = min(nqb, (grp + 1) * qsz);
        for (int ql = grp * qsz; ql < q_end; ++ql) {
          const float4 q = S.q[qb + ql];
          const unsigned long long D2 = dist2_x2(X, Y, Z, q);
          const float d0 = lo_half(D2), d1 = hi_half(D2);
          bool h0 = d0 <= B.lo_w, h1 = d1 <= B.lo_w;
          if (!h0 && !(d0 > B.hi_w) && k0 < nc) h0 = canon_d2(q, g.spos[__float_as_int(c0.w)], g) <= B.r2;
          if (!h1 && !(d1 > B.hi_w) && k1 < nc) h1 = canon_d2(q, g.spos[__float_as_int(c1.w)], g) <= B.r2;
          const unsigned m0 = __ballot_sync(0xffffffffu, h0);
          const unsigned m1 = __ballot_sync(0xffffffffu, h1);
          if (lane == 0) {
            S.u.mask[ql * nchunk + ch0] = m0;
            if (ch1 < nchunk) S.u.mask[ql * nchunk + ch1] = m1;
          }
        }
      }
      __syncthreads();
      // 5. the query's own bit cleared (it is always a candidate and a hit),
      //    counts, one scratch region for the batch, lists stored ascending
      for (int ql = wid; ql < nqb; ql += nw) {
        if (!incl_self && lane == 0) {
          const int id = __ldg(g.perm + qs + qb + ql);
          int lo = 0, hi = nc - 1;
          while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (cid[mid] < id) lo = mid + 1;
            else hi = mid;
          }
          S.u.mask[ql * nchunk + (lo >> 5)] &= ~(1u << (lo & 31));
        }
        __syncwarp();
        int cnt = 0;
        for (int c0 = 0; c0 < nchunk; c0 += 32) {
          const int ch = c0 + lane;
          cnt += ch < nchunk ? __popc(S.u.mask[ql * nchunk + ch]) : 0;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
        if (lane == 0) S.qcnt[ql] = cnt;
      }
      __syncthreads();
      {
        const int v = tid < nqb ? S.qcnt[tid] : 0;   // nqb <= kCellMaxQ == blockDim
        int total;
        const int ex = block_excl_scan_i(v, total, S.scan);
        if (tid < nqb) S.qoff[tid] = ex;
        if (tid == 0) {
          const unsigned long long b = atomicAdd(scr_top, (unsigned long long)total);
          S.base = (b + (unsigned long long)total <= (unsigned long long)scr_cap) ? (long long)b : -1ll;
        }
      }
      __syncthreads();
      const long long sbase = S.base;
      for (int ql = wid; ql < nqb; ql += nw) {
        const int s = qs + qb + ql;
        const int id = __ldg(g.perm + s);
        if (sbase < 0) {
          // scratch full: this query goes to the per-query path
          if (lane == 0) {
            const int o = atomicAdd(over, 1);
            over[1 + o] = s;
            scr_off[id] = -1;
          }
          continue;
        }
        const long long qbase = sbase + S.qoff[ql];
        if (lane == 0) {
          counts[id] = S.qcnt[ql];
          scr_off[id] = qbase;
        }
        long long wpos = qbase;
        for (int c0 = 0; c0 < nchunk; c0 += 32) {
          const int ch = c0 + lane;
          const unsigned mm = ch < nchunk ? S.u.mask[ql * nchunk + ch] : 0u;
          const int cnt = __popc(mm);
          const int inc = warp_incl_scan_i(cnt);
          const int lim = min(32, nchunk - c0);
          for (int i = 0; i < lim; ++i) {
            const unsigned mi = __shfl_sync(0xffffffffu, mm, i);
            const int oi = __shfl_sync(0xffffffffu, inc - cnt, i);
            if ((mi >> lane) & 1u) scratch[wpos + oi + __popc(mi & lt_mask)] = cid[(c0 + i) * 32 + lane];
          }
          wpos += __shfl_sync(0xffffffffu, inc, 31);
        }
      }
      __syncthreads();
    }
  }
}

// After the prefix sum: every heavy query's list from the scratch buffer to
// its place in the output (a warp per query, coalesced both ways).
__global__ void __launch_bounds__(256) k_cell_copy(GridDev g, const int *__restrict__ heavy,
                                                   const long long *__restrict__ scr_off,
                                                   const int *__restrict__ scratch,
                                                   const long long *__restrict__ offsets, int *ids,
                                                   long long cap) {
  if (offsets[g.n] > cap) {
    if (threadIdx.x == 0 && blockIdx.x == 0) atomicOr(g.status, ST_CAPACITY);
    return;
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nwb = blockDim.x >> 5;
  const int nheavy = heavy[0];
  for (int item = blockIdx.x; item < nheavy; item += gridDim.x) {
    const unsigned key = (unsigned)heavy[1 + item];
    const int qs = __ldg(g.cell_start + key), qe = __ldg(g.cell_start + key + 1);
    for (int s = qs + w; s < qe; s += nwb) {
      const int id = __ldg(g.perm + s);
      const long long src = scr_off[id];
      if (src < 0) continue;
      const long long dst = offsets[id];
      const int len = (int)(offsets[id + 1] - dst);
      for (int i = lane; i < len; i += 32) ids[dst + i] = scratch[src + i];
    }
  }
}

si_status launch_cell_pass(const GridDev &g, const WalkParams &P, const Band &B, unsigned flags,
                           const int *heavy, int *work, int *over, long long *counts, long long *scr_off,
                           int *scratch, long long scr_cap, unsigned long long *scr_top, cudaStream_t st) {
  const size_t smem = sizeof(CellSmem);
  SI_CUDA_TRY(cudaFuncSetAttribute(k_cell, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  SI_KLAUNCH("k_cell", st,
             k_cell<<<148 * 2, kCellThreads, smem, st>>>(g, P, B, flags, heavy, work, over, counts, scr_off,
                                                        scratch, scr_cap, scr_top));
  return SI_OK;
}

si_status launch_cell_copy(const GridDev &g, const int *heavy, const long long *scr_off, const int *scratch,
                           const long long *offsets, int *ids, long long cap, cudaStream_t st) {
  SI_KLAUNCH("k_cell_copy", st,
             k_cell_copy<<<148 * 8, 256, 0, st>>>(g, heavy, scr_off, scratch, offsets, ids, cap));
  return SI_OK;
}

}  // namespace si
