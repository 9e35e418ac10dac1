// Radius query for heavily loaded cells (Sec. I: with many objects per cell
// the cost of processing cells dominates, so it pays to share that work).
//
// One block per heavy query cell (heavy_cell), in a single pass that runs
// before the prefix sum of the list lengths:
//  1. the cell-level sphere: every table entry whose minimum cell-to-cell
//     bound satisfies b^2 <= floor(d^2) (Sec. II.A) is translated to the query
//     cell (SWAR add/mask/pack, Sec. II.B); non-empty target cells are listed;
//  2. their points are moved into the query cell's frame (image shift on
//     wrapped cyclic axes), kept when they lie within d of the query cell box
//     (the union of the spheres of every point of the cell) and staged in
//     shared memory; each kept candidate's input index is counted into one of
//     1024 buckets by its top bits;
//  3. the staged candidates are put in ascending input-index order (bucket
//     scatter, then insertion inside each small bucket) and the ordered ids
//     are stored to the cell's record in a scratch buffer, reserved with one
//     atomic as soon as the number of candidates is known;
//  4. the test phase (cell_test_phase, si_cell.cuh): a lane owns one query
//     and builds its hit mask over each chunk of 32 candidates, which the
//     lanes read as packed FP32 pairs; the masks go to the record and their
//     population counts to the query's count.
// Record of a cell in the scratch buffer: nc, the nc ordered ids, then one
// 32-bit mask per (query, 32 candidates), query-major.  After the prefix sum,
// k_expand_items (a warp per few queries of one record) and k_cell_expand
// (a block per split cell) turn every query's masks into its ids at their
// place in the output.
// Two configurations: most heavy cells fit a small block (8 warps, 1280
// candidates, 128 queries, four blocks per SM); a cell that does not is
// listed for the large one (16 warps, 2560 candidates, 512 queries), launched
// after it.  The large one splits a cell whose candidates exceed its capacity
// into slabs of input indices [lo, lo + span): each slab is gathered, sorted
// and tested on its own, and since every index of a slab is below every
// index of the next, a query's hits slab after slab are already its sorted
// list.  A split cell's record is a header (the slab count and each slab
// record's offset) and one record per slab.  A cell that fits neither, or
// whose records do not fit the scratch buffer, hands its queries to the
// per-query path.
#include "si_cell.cuh"

namespace si {

using CellSmall = CellCfg<256, 1280, 128, 512, 4>;
using CellLarge = CellCfg<kCellThreads, kCellCap, kCellMaxQ, 1024, 2>;

template <class C>
struct CellSmem {
  static constexpr int kChunks = (C::kCap + 31) / 32;
  float4 c[C::kCap];                       // staged candidate in the query frame; x = NaN: outside cell; w = spos slot
  union {
    struct {                               // sort phase
      unsigned long long key[C::kCap];     // (input index << 32) | staging slot, in bucket order
      int sid[C::kCap];                    // input index of each staged candidate
    } s;
    struct {                               // test phase, candidates in id order
      float4 xy[kChunks * kPairRow];       // (x_2p, x_2p+1, y_2p, y_2p+1)
      float2 z[kChunks * kPairRow];        // (z_2p, z_2p+1)
    } t;
  } u;
  unsigned outb[kChunks];                  // per chunk: candidates of the outside cell (FP64 for every pair)
  unsigned short sslot[C::kCap];           // staging slot (in c) of each candidate in id order
  int bstart[C::kBuckets];                 // bucket counts, then starts
  int bcur[C::kBuckets];                   // bucket fill pointers
  struct {                                 // gather: runs of points of the cell-level sphere
    int tbeg[kCellTCap];
    int tcnt[kCellTCap];
    int tpre[kCellTCap + 1];
    int tsh[kCellTCap];                    // bytes 0-2: image shift per axis (-1, 0, +1 box sides); byte 3: outside cell
  } t;
  float4 qa[C::kMaxQ];                     // the cell's query points as FP32x2 pairs: (x, x, y, y)
  float4 qb[C::kMaxQ];                     // (z, z, own position among the candidates, -)
  int qcnt[C::kMaxQ];                      // hits per query
  int scan[C::kThreads / 32];
  long long base;                          // the slab's record in the scratch buffer (-1: no room)
  long long hdr;                           // the split cell's header (-1: no room)
  int nt, nc, out_seen, item, qs, nq, cls;
  unsigned key;
};

size_t cell_smem_bytes() { return sizeof(CellSmem<CellLarge>); }

// cells: [0] = count, then cell keys; next (nullable): where cells that do
// not fit go (else they are split into slabs, or the per-query path takes
// them).  cell_rec[key]: the record (>= 0), the header of a split cell
// (-2 - header), or -1 (per-query path).
constexpr int kMaxSlabs = 256;

template <class C>
__global__ void __launch_bounds__(C::kThreads, C::kMinBlocks) k_cell(GridDev g, WalkParams P, Band B,
                                                                    unsigned flags, const int *__restrict__ cells,
                                                                    int *work, int *next, int *__restrict__ over,
                                                                    long long *__restrict__ counts,
                                                                    long long *__restrict__ cell_rec,
                                                                    int *__restrict__ scratch, long long scr_cap,
                                                                    unsigned long long *scr_top) {
  constexpr int kBuckets = C::kBuckets;
  constexpr int kCap = C::kCap;
  constexpr int kSlabFill = kCap * 3 / 4;   // target candidates per slab (the rest is margin)
  extern __shared__ __align__(16) unsigned char smem_raw[];
  CellSmem<C> &S = *reinterpret_cast<CellSmem<C> *>(smem_raw);
  const int nheavy = cells[0];
  const bool incl_self = flags & SI_INCLUDE_SELF;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  const unsigned lt_mask = (1u << lane) - 1u;
  const float box2 = (P.dg + g.eps) * (P.dg + g.eps);
  const int Gx = 1 << g.wx;
  const bool cyc_x = g.cyc & 1u;
  // bucket of an input index: its top bits within the slab's range
  auto bucket_shift = [&](int range) {
    int idbits = 1;
    while (idbits < 31 && (1 << idbits) < range) ++idbits;
    return max(idbits - C::kBucketBits, 0);
  };
  const int bshift_all = bucket_shift(g.n);
  // reservations are kept even so that headers hold aligned 64-bit offsets
  // (scr_top also tells the host how much scratch a call needs: a cell whose
  // reservation fails adds a bound for the slabs it did not reach)
  auto slab_bound = [&](int nq) { return 2ll + kCap + (long long)nq * ((kCap + 31) / 32); };
  auto reserve = [&](long long need) -> long long {
    need = (need + 1) & ~1ll;
    const unsigned long long b = atomicAdd(scr_top, (unsigned long long)need);
    return (b + (unsigned long long)need <= (unsigned long long)scr_cap) ? (long long)b : -1ll;
  };
  // the next cell is fetched while this one is processed (thread 0): its
  // item number at the start, its key after the gather, its bounds after
  // the sort, so that no dependent global load waits at the loop head
  int n_item = 0, n_qs = 0, n_qe = 0, n_cls = 0;
  unsigned n_key = 0u;
  bool keyed = false, bounded = false;   // this iteration's fetches done
  auto fetch_key = [&]() {
    if (keyed) return;
    keyed = true;
    if (tid == 0 && n_item < nheavy) n_key = (unsigned)cells[1 + n_item];
  };
  auto fetch_bounds = [&]() {
    if (bounded) return;
    fetch_key();
    bounded = true;
    if (tid == 0 && n_item < nheavy) {
      n_qs = __ldg(g.cell_start + n_key);
      n_qe = __ldg(g.cell_start + n_key + 1);
      n_cls = g.cell_cls[n_key];
    }
  };
  if (tid == 0) n_item = atomicAdd(work, 1);
  fetch_key();
  fetch_bounds();
  for (;;) {
    if (tid == 0) {
      S.item = n_item;
      S.key = n_key;
      S.qs = n_qs;
      S.nq = n_qe - n_qs;
      S.cls = n_cls;
      if (n_item < nheavy) n_item = atomicAdd(work, 1);
    }
    keyed = bounded = false;
    __syncthreads();
    const int item = S.item;
    if (item >= nheavy) return;
    const unsigned key = S.key;
    if (next && S.cls == kCellHeavyBig) {   // listed for the large configuration
      fetch_key();
      fetch_bounds();
      __syncthreads();   // every thread has read S before it is rewritten
      continue;
    }
    const int qs = S.qs, nq = S.nq;
    const int cx = (int)(key & ((1u << g.wx) - 1u));
    const int cy = (int)((key >> g.wx) & ((1u << g.wy) - 1u));
    const int cz = (int)(key >> (g.wx + g.wy));
    const unsigned long long cu = unpack3(cx, cy, cz, g);
    if (tid == 0) {
      S.nt = 0;
      S.nc = 0;
      S.out_seen = 0;
    }
    for (int b = tid; b < kBuckets; b += blockDim.x) S.bstart[b] = 0;
    const bool qfit = nq <= C::kMaxQ;
    __syncthreads();
    int nt = 0, ntot = 0;
    if (qfit) {
      // 1. runs of the cell-level sphere: each x-row of cells within d of the
      //    query cell (b^2 <= floor(d^2)) is one run of points, or two where
      //    it crosses the cyclic x boundary; rows leaving the region on a
      //    non-cyclic axis stand for the outside cell, listed once
      auto add_run = [&](unsigned ka, unsigned kb, unsigned code) {
        const int b = __ldg(g.cell_start + ka), c = __ldg(g.cell_start + kb + 1) - b;
        if (c == 0) return;
        const int t = atomicAdd(&S.nt, 1);
        S.t.tbeg[t] = b;
        S.t.tcnt[t] = c;
        // code: bits 2a, 2a + 1 = +L, -L on axis a; bit 6 = the outside cell
        unsigned sh = (code & 64u) ? (1u << 24) : 0u;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          const unsigned c2 = (code >> (2 * a)) & 3u;
          sh |= (c2 == 1u ? 0x01u : (c2 == 2u ? 0xffu : 0u)) << (8 * a);
        }
        S.t.tsh[t] = (int)sh;
      };
      for (int e = tid; e < g.n_crow; e += blockDim.x) {
        const unsigned long long E = g.crow[e];
        const int lo = (int)(signed char)((E >> 48) & 0xffull);
        const int len = (int)((E >> 56) & 127ull);
        const unsigned long long off = E & ((1ull << 48) - 1ull);
        const unsigned long long sum = cu + off;   // the row's y and z; x stays the cell's own
        bool out = (sum & g.guard_non) != 0ull;
        if (!out) {
          // image shift of the row's candidates on wrapped y / z (1: +L, 2: -L)
          unsigned code = 0;
          if (sum & g.gy) code |= ((off & g.gy) ? 2u : 1u) << 2;
          if (sum & g.gz) code |= ((off & g.gz) ? 2u : 1u) << 4;
          const unsigned row = repack(sum & g.valid, g) - (unsigned)cx;   // packed index of x = 0
          int x0 = cx + lo, x1 = x0 + len - 1;
          if (!cyc_x) {
            if (x0 < 0 || x1 >= Gx) out = true;
            x0 = max(x0, 0);
            x1 = min(x1, Gx - 1);
          } else if (x0 < 0 || x1 >= Gx) {
            const int wa = x0 < 0 ? x0 + Gx : 0, wb = x0 < 0 ? Gx - 1 : x1 - Gx;
            add_run(row + (unsigned)wa, row + (unsigned)wb, code | (x0 < 0 ? 2u : 1u));
            x0 = max(x0, 0);
            x1 = min(x1, Gx - 1);
          }
          if (x0 <= x1) add_run(row + (unsigned)x0, row + (unsigned)x1, code);
        }
        if (out && !atomicExch(&S.out_seen, 1)) add_run(g.outside, g.outside, 64u);
      }
      // the cell's queries as FP32x2 pairs (their loads overlap the runs')
      for (int i = tid; i < nq; i += blockDim.x) {
        const float4 q = g.spos[qs + i];
        S.qa[i] = make_float4(q.x, q.x, q.y, q.y);
        S.qb[i] = make_float4(q.z, q.z, __int_as_float(-1), 0.f);
        S.qcnt[i] = 0;
      }
      __syncthreads();
      nt = S.nt;
      // 2a. prefix of run sizes (one warp)
      if (wid == 0) {
        int run = 0;
        for (int b0 = 0; b0 < nt; b0 += 32) {
          const int t = b0 + lane;
          const int v = t < nt ? S.t.tcnt[t] : 0;
          const int inc = warp_incl_scan_i(v);
          if (t < nt) S.t.tpre[t] = run + inc - v;
          run += __shfl_sync(0xffffffffu, inc, 31);
        }
        if (lane == 0) S.t.tpre[nt] = run;
      }
      __syncthreads();
      ntot = S.t.tpre[nt];
    }
    // 2b-4, slab by slab of input indices [lo, hi)
    int nslab = 1, span = g.n;
    bool ok = qfit, room = true, split = false;
    for (int sl = 0; ok && sl < nslab;) {
      const int lo = sl * span, hi = min(g.n, lo + span);
      const int bshift = split ? bucket_shift(hi - lo) : bshift_all;
      // 2b. gather: candidates of the slab within d of the query cell box, in
      //     the query frame, their indices counted into buckets.  A warp
      //     takes 32 * kGather consecutive candidates: the first one's run by
      //     binary search, the others' by stepping forward.
      constexpr int kGather = 4;
      for (int f0 = wid * 32 * kGather; f0 < ntot; f0 += nw * 32 * kGather) {
        int rr = 0;
        {
          int top = nt - 1;
          while (rr < top) {
            const int mid = (rr + top + 1) >> 1;
            if (S.t.tpre[mid] <= f0) rr = mid;
            else top = mid - 1;
          }
        }
        int cj[kGather], tt[kGather], pid[kGather];
        float4 p[kGather];
#pragma unroll
        for (int u = 0; u < kGather; ++u) {
          const int f = f0 + u * 32 + lane;
          cj[u] = -1;
          tt[u] = 0;
          if (f < ntot) {
            while (S.t.tpre[rr + 1] <= f) ++rr;
            tt[u] = rr;
            cj[u] = S.t.tbeg[rr] + (f - S.t.tpre[rr]);
          }
        }
#pragma unroll
        for (int u = 0; u < kGather; ++u) {
          p[u] = cj[u] >= 0 ? g.spos[cj[u]] : make_float4(0.f, 0.f, 0.f, 0.f);
          pid[u] = cj[u] >= 0 ? __ldg(g.perm + cj[u]) : 0;
        }
#pragma unroll
        for (int u = 0; u < kGather; ++u) {
          bool keep = false;
          if (cj[u] >= 0 && pid[u] >= lo && pid[u] < hi) {
            const int sh = S.t.tsh[tt[u]];
            if (sh >> 24) {
              p[u].x = __int_as_float(0x7fc00000);   // outside cell: FP64 test for every pair
              keep = true;
            } else {
              // image shift: x + k L with k in {-1, 0, 1} (the product is exact)
              p[u].x = fmaf((float)(signed char)(sh & 0xff), g.Lx, p[u].x);
              p[u].y = fmaf((float)(signed char)((sh >> 8) & 0xff), g.Ly, p[u].y);
              p[u].z = fmaf((float)(signed char)((sh >> 16) & 0xff), g.Lz, p[u].z);
              const float ux = (p[u].x - g.ox) * g.inv_s - (float)cx;
              const float uy = (p[u].y - g.oy) * g.inv_s - (float)cy;
              const float uz = (p[u].z - g.oz) * g.inv_s - (float)cz;
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
            if (at < kCap) {
              float4 cp = p[u];
              cp.w = __int_as_float(cj[u]);
              S.c[at] = cp;
              S.u.s.sid[at] = pid[u] - lo;
              atomicAdd(&S.bstart[(pid[u] - lo) >> bshift], 1);
            }
          }
        }
      }
      __syncthreads();
      fetch_key();
      const int nc = S.nc;
      if (nc > kCap) {
        if (!next && !split) {
          // the large configuration splits the cell into slabs of indices
          nslab = (nc + kSlabFill - 1) / kSlabFill;
          split = true;
          if (nslab > kMaxSlabs) {
            ok = false;
            room = false;
            break;
          }
          span = (g.n + nslab - 1) / nslab;
          __syncthreads();   // every thread has read S.nc before it is reset
          if (tid == 0) {
            S.hdr = reserve(2 + 2ll * nslab);
            if (S.hdr >= 0) scratch[S.hdr] = nslab;
            else atomicAdd(scr_top, (unsigned long long)(nslab * slab_bound(nq)));
            S.nc = 0;
          }
          for (int b = tid; b < kBuckets; b += blockDim.x) S.bstart[b] = 0;
          __syncthreads();
          if (S.hdr < 0) {
            ok = false;
            room = false;
          }
          continue;   // slab 0 again, under the new span
        }
        ok = false;   // small configuration: the large one takes it; a slab that overflows: per-query path
        room = !split;
        break;
      }
      const int nchunk = (nc + 31) >> 5;
      // the slab's record: nc, ids, masks
      if (tid == 0) {
        S.base = reserve(1 + (long long)nc + (long long)nq * nchunk);
        if (split && S.base >= 0) reinterpret_cast<long long *>(scratch + S.hdr + 2)[sl] = S.base;
      }
      // 3. ascending input index: scan of the bucket counts, scatter, then
      //    each bucket (a handful of keys) sorted by insertion
      constexpr int kPerB = kBuckets / C::kThreads;
      int v[kPerB], bsum = 0;
#pragma unroll
      for (int r = 0; r < kPerB; ++r) {
        v[r] = S.bstart[tid * kPerB + r];
        bsum += v[r];
      }
      int total;
      int run = block_excl_scan_i(bsum, total, S.scan);   // its barriers also publish S.base
#pragma unroll
      for (int r = 0; r < kPerB; ++r) {
        S.bstart[tid * kPerB + r] = run;
        S.bcur[tid * kPerB + r] = run;
        run += v[r];
      }
      if (S.base < 0) {
        if (split && tid == 0 && sl + 1 < nslab)
          atomicAdd(scr_top, (unsigned long long)((nslab - sl - 1) * slab_bound(nq)));
        ok = false;
        room = false;
        break;
      }
      __syncthreads();
      for (int p = tid; p < nc; p += blockDim.x) {
        const int id = S.u.s.sid[p];
        S.u.s.key[atomicAdd(&S.bcur[id >> bshift], 1)] = ((unsigned long long)(unsigned)id << 32) | (unsigned)p;
      }
      __syncthreads();
      for (int b = tid; b < kBuckets; b += blockDim.x) {
        const int blo = S.bstart[b], bhi = S.bcur[b];
        for (int i = blo + 1; i < bhi; ++i) {
          const unsigned long long x = S.u.s.key[i];
          int p = i;
          while (p > blo && S.u.s.key[p - 1] > x) {
            S.u.s.key[p] = S.u.s.key[p - 1];
            --p;
          }
          S.u.s.key[p] = x;
        }
      }
      fetch_bounds();
      __syncthreads();
      // id order: the ordered ids go to the record and each sorted position
      // notes its staging slot (the sort's keys are read here for the last
      // time; the staged candidates in S.c stay where the gather put them)
      const long long rec = S.base;
      int *rec_ids = scratch + rec + 1;
      unsigned *rec_masks = reinterpret_cast<unsigned *>(rec_ids + nc);
      if (tid == 0) scratch[rec] = nc;
      for (int k = tid; k < nc; k += blockDim.x) {
        const unsigned long long kk = S.u.s.key[k];
        S.sslot[k] = (unsigned short)(kk & 0xffffu);
        rec_ids[k] = (int)(kk >> 32) + lo;
      }
      if (split)   // own positions of this slab only
        for (int i = tid; i < nq; i += blockDim.x) S.qb[i].z = __int_as_float(-1);
      __syncthreads();
      // the candidates in id order as the packed pairs of the test phase
      // (over the sort's arrays, free now); chunk k >> 5 is one warp's row of
      // this loop, so a ballot gives its outside-cell candidates; the padding
      // up to whole chunks is +inf (never a hit, never in the band); each
      // query notes its own position
      for (int k = tid; k < nchunk * 32; k += blockDim.x) {
        const bool in = k < nc;
        const float4 v = in ? S.c[S.sslot[k]] : make_float4(INFINITY, INFINITY, INFINITY, 0.f);
        if (in) {
          const int ql = __float_as_int(v.w) - qs;
          if (!incl_self && ql >= 0 && ql < nq) S.qb[ql].z = __int_as_float(k);
        }
        const unsigned ob = __ballot_sync(0xffffffffu, in && isnan(v.x));
        put_pair(S.u.t.xy, S.u.t.z, k, v);
        if (lane == 0) S.outb[k >> 5] = ob;
      }
      __syncthreads();
      // 4. tests: one hit mask per (query, chunk of 32 candidates)
      cell_test_phase(g, B, nq, nchunk, S.u.t.xy, S.u.t.z, S.outb, S.c, S.sslot, S.qa, S.qb, S.qcnt, rec_masks,
                      lane, wid, nw);
      __syncthreads();
      if (++sl < nslab) {   // the next slab starts from empty buckets
        if (tid == 0) S.nc = 0;
        for (int b = tid; b < kBuckets; b += blockDim.x) S.bstart[b] = 0;
        __syncthreads();
      }
    }
    fetch_bounds();
    if (!ok) {
      if (next && room) {
        // the larger configuration takes this cell
        if (tid == 0) {
          const int o = atomicAdd(next, 1);
          next[1 + o] = (int)key;
        }
      } else {
        // the per-query path takes every query of this cell
        for (int i = tid; i < nq; i += blockDim.x) {
          const int o = atomicAdd(over, 1);
          over[1 + o] = qs + i;
        }
        if (tid == 0) cell_rec[key] = -1;
      }
      __syncthreads();
      continue;
    }
    for (int i = tid; i < nq; i += blockDim.x) counts[__ldg(g.perm + qs + i)] = S.qcnt[i];
    if (tid == 0) cell_rec[key] = split ? -2 - S.hdr : S.base;
  }
}

// After the prefix sum: every heavy query's masks expanded into its ids at
// their place in the output.  A block per heavy cell, slab after slab (one
// for an unsplit cell): the slab's ordered ids are staged in shared memory
// (32 per row, rows padded to kRowW words); each warp takes every
// kExpWarps-th query of the cell (a query's masks are row `slot - first slot`
// of the slab record).  The warp keeps its queries' write positions in
// registers (its t-th query in lane t % 32, slot t / 32), fetched at once and
// carried from slab to slab.  For 32 masks at a time, lane j takes the j-th
// and, over its 32 bit positions in turn (reading its row's ids four at a
// time), appends the ids of the set bits to the warp's shared buffer after
// the hits of the masks before it; the warp
// then stores the buffer contiguously.  The next masks are loaded while the
// current ones are expanded.
// words per staged row: 32 ids and padding to a 16-byte multiple, so that a
// lane reads four ids of its row at once (rows of 36 words: the eight lanes
// of each quarter-warp phase of a 16-byte read hit distinct banks)
constexpr int kRowW = 36;
constexpr int kExpWarps = 4;
constexpr int kExpRows = (kCellCap + 31) / 32;
constexpr int kExpSlots = (kCellMaxQ + 32 * kExpWarps - 1) / (32 * kExpWarps);   // positions per lane

__global__ void __launch_bounds__(kExpWarps * 32, 8) k_cell_expand(GridDev g, const int *__restrict__ heavy,
                                                                   const long long *__restrict__ cell_rec,
                                                                   const int *__restrict__ scratch,
                                                                   const long long *__restrict__ offsets,
                                                                   int *__restrict__ ids, long long cap) {
  __shared__ __align__(16) int sids[kExpRows * kRowW];
  __shared__ int sbuf[kExpWarps][1024];
  if (offsets[g.n] > cap) {
    if (threadIdx.x == 0 && blockIdx.x == 0) atomicOr(g.status, ST_CAPACITY);
    return;
  }
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  int *buf = sbuf[wid];
  const int nheavy = heavy[0];
  for (int item = blockIdx.x; item < nheavy; item += gridDim.x) {
    const unsigned key = (unsigned)heavy[1 + item];
    const long long ref = cell_rec[key];
    if (ref == -1) continue;   // served by the per-query path (the same for the whole block)
    const int qs = __ldg(g.cell_start + key), nq = __ldg(g.cell_start + key + 1) - qs;
    int nslab = 1;
    const long long *slabs = nullptr;
    if (ref < -1) {
      const long long hdr = -2 - ref;
      nslab = __ldg(scratch + hdr);
      slabs = reinterpret_cast<const long long *>(scratch + hdr + 2);
    }
    const int nmine = (nq - wid + kExpWarps - 1) / kExpWarps;   // this warp's queries: wid + kExpWarps t
    long long wpos_of[kExpSlots];
#pragma unroll
    for (int k = 0; k < kExpSlots; ++k) {
      const int t = k * 32 + lane;
      wpos_of[k] = t < nmine ? offsets[__ldg(g.perm + qs + wid + kExpWarps * t)] : 0ll;
    }
    for (int sl = 0; sl < nslab; ++sl) {
      const long long rec = slabs ? slabs[sl] : ref;
      const int nc = __ldg(scratch + rec);
      const int nchunk = (nc + 31) >> 5;
      const int *rec_ids = scratch + rec + 1;
      const unsigned *rec_masks = reinterpret_cast<const unsigned *>(rec_ids + nc);
      __syncthreads();   // the previous slab's (or cell's) ids are no longer read
      for (int k = tid; k < nc; k += blockDim.x) sids[(k >> 5) * kRowW + (k & 31)] = __ldg(rec_ids + k);
      __syncthreads();
      unsigned mnext = (nmine > 0 && lane < nchunk) ? __ldg(rec_masks + (long long)wid * nchunk + lane) : 0u;
      for (int t = 0; t < nmine; ++t) {
        const int ql = wid + kExpWarps * t, qn = ql + kExpWarps;
        long long mine = wpos_of[0];
#pragma unroll
        for (int k = 1; k < kExpSlots; ++k)
          if ((t >> 5) == k) mine = wpos_of[k];
        long long wpos = __shfl_sync(0xffffffffu, mine, t & 31);
        const unsigned *mk = rec_masks + (long long)ql * nchunk;
        for (int c0 = 0; c0 < nchunk; c0 += 32) {
          const unsigned mm = mnext;
          // prefetch: the rest of this query's masks, else the next query's first 32
          if (c0 + 32 < nchunk) {
            const int ch = c0 + 32 + lane;
            mnext = ch < nchunk ? __ldg(mk + ch) : 0u;
          } else if (qn < nq) {
            mnext = lane < nchunk ? __ldg(rec_masks + (long long)qn * nchunk + lane) : 0u;
          }
          const int cnt = __popc(mm);
          const int inc = warp_incl_scan_i(cnt);
          int o = inc - cnt;
          const int4 *row4 = reinterpret_cast<const int4 *>(sids + (c0 + lane) * kRowW);
#pragma unroll
          for (int b4 = 0; b4 < 8; ++b4) {
            const int4 v = row4[b4];   // ids 4 b4 .. 4 b4 + 3 of the lane's chunk
            const unsigned nb = mm >> (4 * b4);
            if (nb & 1u) buf[o] = v.x;
            o += (int)(nb & 1u);
            if (nb & 2u) buf[o] = v.y;
            o += (int)((nb >> 1) & 1u);
            if (nb & 4u) buf[o] = v.z;
            o += (int)((nb >> 2) & 1u);
            if (nb & 8u) buf[o] = v.w;
            o += (int)((nb >> 3) & 1u);
          }
          __syncwarp();
          const int tot = __shfl_sync(0xffffffffu, inc, 31);
          for (int i = lane; i < tot; i += 32) ids[wpos + i] = buf[i];
          __syncwarp();
          wpos += tot;
        }
        if (lane == (t & 31)) {
#pragma unroll
          for (int k = 0; k < kExpSlots; ++k)
            if ((t >> 5) == k) wpos_of[k] = wpos;
        }
      }
    }
  }
}

template <class C>
static si_status launch_cell_cfg(const char *name, const GridDev &g, const WalkParams &P, const Band &B,
                                 unsigned flags, const int *cells, int *work, int *next, int *over,
                                 long long *counts, long long *cell_rec, int *scratch, long long scr_cap,
                                 unsigned long long *scr_top, cudaStream_t st) {
  const size_t smem = sizeof(CellSmem<C>);
  SI_CUDA_TRY(cudaFuncSetAttribute(k_cell<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  SI_KLAUNCH(name, st,
             k_cell<C><<<148 * C::kMinBlocks, C::kThreads, smem, st>>>(g, P, B, flags, cells, work, next, over,
                                                                      counts, cell_rec, scratch, scr_cap, scr_top));
  return SI_OK;
}

si_status launch_cell_pass(const GridDev &g, const WalkParams &P, const Band &B, unsigned flags,
                           const int *heavy, int *big, int *work, int *over, long long *counts,
                           long long *cell_rec, int *scratch, long long scr_cap, unsigned long long *scr_top,
                           cudaStream_t st) {
  si_status s = launch_cell_cfg<CellSmall>("k_cell", g, P, B, flags, heavy, work, big, over, counts, cell_rec,
                                           scratch, scr_cap, scr_top, st);
  if (s != SI_OK) return s;
  return launch_cell_cfg<CellLarge>("k_cell_large", g, P, B, flags, big, work + 1, nullptr, over, counts,
                                    cell_rec, scratch, scr_cap, scr_top, st);
}

// The expansion of most cells runs a warp per item of at most kItemQ
// queries of one cell, with no block-wide barrier, so that the latency of
// each item's loads (its record, its queries' output positions) is hidden
// by the other warps of the SM.  k_expand_plan lists the items: a cell
// served by one record gives ceil(nq / kItemQ) of them; split cells go to
// k_cell_expand (a block per cell).  A warp goes through its item's
// candidates a round of 32 chunks (1024 candidates) at a time: it stages
// the round's ordered ids in its own shared rows (32 ids per row, rows
// padded to 36 words), then expands that round's masks of each query as
// k_cell_expand does, but reading a lane's ids four at a time, carrying
// each query's write position from round to round in the register of lane
// t (query q0 + t).
constexpr int kItemQ = 8;
constexpr int kItemWarps = 8;
constexpr int kItemRows = 32;

__global__ void __launch_bounds__(256) k_expand_plan(GridDev g, const int *__restrict__ heavy,
                                                     const long long *__restrict__ cell_rec,
                                                     const int *__restrict__ scratch, int4 *items, int *blocks) {
  const int n = heavy[0];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const unsigned key = (unsigned)heavy[1 + i];
    const long long ref = cell_rec[key];
    if (ref == -1) continue;   // served by the per-query path
    const int qs = __ldg(g.cell_start + key), nq = __ldg(g.cell_start + key + 1) - qs;
    if (ref < -1) {
      blocks[1 + atomicAdd(blocks, 1)] = (int)key;
      continue;
    }
    const int nit = (nq + kItemQ - 1) / kItemQ;
    const int at = atomicAdd(reinterpret_cast<int *>(items), nit);
    for (int t = 0; t < nit; ++t) {
      const int q0 = t * kItemQ;
      items[1 + at + t] = make_int4((int)(ref & 0xffffffffll), (int)(ref >> 32), qs, q0 | (min(kItemQ, nq - q0) << 16));
    }
  }
}

__global__ void __launch_bounds__(kItemWarps * 32) k_expand_items(GridDev g, const int4 *__restrict__ items,
                                                                 const int *__restrict__ scratch,
                                                                 const long long *__restrict__ offsets,
                                                                 int *__restrict__ ids, long long cap) {
  extern __shared__ __align__(16) int item_smem[];   // per warp: kItemRows * kRowW id slots, then a 1024-id buffer
  if (offsets[g.n] > cap) {
    if (threadIdx.x == 0 && blockIdx.x == 0) atomicOr(g.status, ST_CAPACITY);
    return;
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int *rows = item_smem + wid * (kItemRows * kRowW + 1024), *buf = rows + kItemRows * kRowW;
  const int nitems = items[0].x;
  for (int it = blockIdx.x * kItemWarps + wid; it < nitems; it += gridDim.x * kItemWarps) {
    const int4 d = items[1 + it];
    const long long rec = (long long)(unsigned)d.x | ((long long)d.y << 32);
    const int qs = d.z, q0 = d.w & 0xffff, cnt = d.w >> 16;
    const int nc = __ldg(scratch + rec);
    const int nchunk = (nc + 31) >> 5;
    const int *rec_ids = scratch + rec + 1;
    const unsigned *rec_masks = reinterpret_cast<const unsigned *>(rec_ids + nc);
    // output positions of the item's queries (lane t: query q0 + t)
    long long wp = lane < cnt ? offsets[__ldg(g.perm + qs + q0 + lane)] : 0ll;
    unsigned mnext = lane < nchunk ? __ldg(rec_masks + (long long)q0 * nchunk + lane) : 0u;
    for (int c0 = 0; c0 < nchunk; c0 += 32) {
      __syncwarp();   // the previous round's (or item's) rows are no longer read
      const int kend = min(nc, (c0 + 32) * 32);
      for (int k = c0 * 32 + lane; k < kend; k += 32) rows[((k >> 5) - c0) * kRowW + (k & 31)] = __ldg(rec_ids + k);
      __syncwarp();
      for (int t = 0; t < cnt; ++t) {
        const unsigned mm = mnext;
        // prefetch: the next query's masks of this round, else the first
        // query's masks of the next round
        if (t + 1 < cnt) {
          const int ch = c0 + lane;
          mnext = ch < nchunk ? __ldg(rec_masks + (long long)(q0 + t + 1) * nchunk + ch) : 0u;
        } else if (c0 + 32 < nchunk) {
          const int ch = c0 + 32 + lane;
          mnext = ch < nchunk ? __ldg(rec_masks + (long long)q0 * nchunk + ch) : 0u;
        }
        const long long wpos = __shfl_sync(0xffffffffu, wp, t);
        const int c = __popc(mm);
        const int inc = warp_incl_scan_i(c);
        int o = inc - c;
        const int4 *row4 = reinterpret_cast<const int4 *>(rows + lane * kRowW);
#pragma unroll
        for (int b4 = 0; b4 < 8; ++b4) {
          const int4 v = row4[b4];   // ids 4 b4 .. 4 b4 + 3 of the lane's chunk
          const unsigned nb = mm >> (4 * b4);
          if (nb & 1u) buf[o] = v.x;
          o += (int)(nb & 1u);
          if (nb & 2u) buf[o] = v.y;
          o += (int)((nb >> 1) & 1u);
          if (nb & 4u) buf[o] = v.z;
          o += (int)((nb >> 2) & 1u);
          if (nb & 8u) buf[o] = v.w;
          o += (int)((nb >> 3) & 1u);
        }
        __syncwarp();
        const int tot = __shfl_sync(0xffffffffu, inc, 31);
        for (int i = lane; i < tot; i += 32) ids[wpos + i] = buf[i];
        __syncwarp();
        if (lane == t) wp += tot;
      }
    }
  }
}

si_status launch_cell_expand(const GridDev &g, const int *heavy, const long long *cell_rec, const int *scratch,
                             int4 *items, int *blocks, const long long *offsets, int *ids, long long cap,
                             cudaStream_t st) {
  SI_CUDA_TRY(cudaMemsetAsync(items, 0, sizeof(int4), st));
  SI_CUDA_TRY(cudaMemsetAsync(blocks, 0, sizeof(int), st));
  SI_KLAUNCH("k_expand_plan", st,
             k_expand_plan<<<148 * 4, 256, 0, st>>>(g, heavy, cell_rec, scratch, items, blocks));
  const size_t ism = (size_t)kItemWarps * (kItemRows * kRowW + 1024) * sizeof(int);
  SI_CUDA_TRY(cudaFuncSetAttribute(k_expand_items, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ism));
  SI_KLAUNCH("k_expand_items", st,
             k_expand_items<<<148 * 3, kItemWarps * 32, ism, st>>>(g, items, scratch, offsets, ids, cap));
  SI_KLAUNCH("k_cell_expand", st,
             k_cell_expand<<<148 * 8, kExpWarps * 32, 0, st>>>(g, blocks, cell_rec, scratch, offsets, ids, cap));
  return SI_OK;
}

}  // namespace si
