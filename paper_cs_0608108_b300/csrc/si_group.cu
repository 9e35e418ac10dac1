// Radius query for groups of heavy cells: one block per aligned 2 x 2 x 2
// group of lattice cells holding two or more heavy cells (heavy_cell, the
// small class), so that neighbouring heavy cells share one gather and one
// sort of their candidates (Sec. I: with many objects per cell the cost of
// processing cells dominates, and it pays to share that work).
//
//  1. the rows of cells within d of the group's box (x-row runs, translated
//     to the group's lowest cell by the SWAR add of Sec. II.B) give the
//     candidate points; each is moved to the group's frame (image shift on
//     wrapped cyclic axes) and kept when it lies within d of the box of at
//     least one heavy cell of the group, with one membership bit per cell;
//  2. the kept candidates (the union of the cells' candidate sets) are put
//     in ascending input-index order once (bucket counting sort, insertion
//     inside buckets);
//  3. each heavy cell in turn takes its members from the ordered union (an
//     ordered compaction, so its candidates are already sorted), writes its
//     record (ordered ids, then one hit mask per query and chunk of 32
//     candidates, the format of si_cell.cu) and runs the test phase.
// A group whose union exceeds the block's capacity, or a cell with more
// queries than a block holds, is listed for the large per-cell
// configuration; a cell whose record does not fit the scratch buffer hands
// its queries to the per-query path.  k_group_list splits the heavy list
// into the groups and the cells served one at a time.
#include "si_cell.cuh"

namespace si {

using GroupCfg = CellCfg<512, 2560, 128, 1024, 2>;

struct GroupSmem {
  static constexpr int kCap = GroupCfg::kCap;
  static constexpr int kChunks = kCap / 32;
  float4 c[kCap];                          // staged candidate in the group's frame; x = NaN: outside cell; w = spos slot
  union {
    struct {                               // sort of the union
      unsigned long long key[kCap];        // (input index << 32) | staging slot, in bucket order
      int sid[kCap];                       // input index of each staged candidate
    } s;
    struct {                               // test phase of one cell, its candidates in id order
      float4 xy[kChunks * kPairRow];
      float2 z[kChunks * kPairRow];
    } t;
  } u;
  int uid[kCap];                           // input index of the union's k-th candidate in id order
  unsigned short uslot[kCap];              // its staging slot
  unsigned short cslot[kCap];              // staging slot of the current cell's k-th candidate
  unsigned char mem[kCap];                 // per staging slot: bit i + 2 j + 4 k = within d of cell (i, j, k)
  unsigned outb[kChunks];                  // current cell: candidates of the outside cell, per chunk
  int bstart[GroupCfg::kBuckets];
  int bcur[GroupCfg::kBuckets];
  int tbeg[kGroupTCap];
  int tcnt[kGroupTCap];
  int tpre[kGroupTCap + 1];
  int tsh[kGroupTCap];                     // bytes 0-2: image shift per axis; byte 3: outside cell
  float4 qa[GroupCfg::kMaxQ];
  float4 qb[GroupCfg::kMaxQ];
  int qcnt[GroupCfg::kMaxQ];
  int wcnt[8][GroupCfg::kThreads / 32];    // per member cell: members per warp range, then their prefix
  int scan[GroupCfg::kThreads / 32];
  int cq_s[8], cq_n[8], cnc[8];            // per cell of the group: first slot, queries, candidates
  long long coff[8];                       // its record's offset from the group's reservation
  unsigned ckey[8];
  long long base;                          // the group's records in the scratch buffer (-1: no room)
  int nt, nc, out_seen, item, hm;
  unsigned nck;                            // the next group's lowest cell
};

size_t group_smem_bytes() { return sizeof(GroupSmem); }

// Heavy cells (small class) split into groups: a heavy cell whose aligned
// 2 x 2 x 2 group holds another non-empty heavy cell is served by its group
// (listed once, by its lowest heavy cell); the others go to solo.  Cells of
// the large class are already listed for the large per-cell configuration.
__global__ void __launch_bounds__(256) k_group_list(GridDev g, const int *__restrict__ heavy, int *groups,
                                                    int *solo) {
  const int n = heavy[0];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const unsigned key = (unsigned)heavy[1 + i];
    if (g.cell_cls[key] != kCellHeavy) continue;
    const int cx = (int)(key & ((1u << g.wx) - 1u));
    const int cy = (int)((key >> g.wx) & ((1u << g.wy) - 1u));
    const int cz = (int)(key >> (g.wx + g.wy));
    const int x0 = cx & ~1, y0 = cy & ~1, z0 = cz & ~1;
    int cnt = 0;
    unsigned first = 0xffffffffu;
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const unsigned k0 = pack3(x0, y0 + (t & 1), z0 + (t >> 1), g);
      const int s0 = __ldg(g.cell_start + k0), s1 = __ldg(g.cell_start + k0 + 1), s2 = __ldg(g.cell_start + k0 + 2);
      if (s1 > s0 && g.cell_cls[k0] == kCellHeavy) {
        ++cnt;
        first = min(first, k0);
      }
      if (s2 > s1 && g.cell_cls[k0 + 1] == kCellHeavy) {
        ++cnt;
        first = min(first, k0 + 1);
      }
    }
    if (cnt >= 2) {
      if (key == first) groups[1 + atomicAdd(groups, 1)] = (int)pack3(x0, y0, z0, g);
    } else {
      solo[1 + atomicAdd(solo, 1)] = (int)key;
    }
  }
}

__global__ void __launch_bounds__(GroupCfg::kThreads, GroupCfg::kMinBlocks)
    k_cell_group(GridDev g, WalkParams P, Band B, unsigned flags, const int *__restrict__ groups, int *work,
                 int *big, int *__restrict__ over, long long *__restrict__ counts, long long *__restrict__ cell_rec,
                 int *__restrict__ scratch, long long scr_cap, unsigned long long *scr_top,
                 const unsigned long long *__restrict__ grow, int n_grow) {
  constexpr int kCap = GroupCfg::kCap;
  constexpr int kBuckets = GroupCfg::kBuckets;
  constexpr int kMaxQ = GroupCfg::kMaxQ;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  GroupSmem &S = *reinterpret_cast<GroupSmem *>(smem_raw);
  const int ngroups = groups[0];
  const bool incl_self = flags & SI_INCLUDE_SELF;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  const unsigned lt_mask = (1u << lane) - 1u;
  const float box2 = (P.dg + g.eps) * (P.dg + g.eps);
  const int Gx = 1 << g.wx;
  const bool cyc_x = g.cyc & 1u;
  int bshift = 0;   // bucket of an input index: its top bits
  {
    int idbits = 1;
    while (idbits < 31 && (1 << idbits) < g.n) ++idbits;
    bshift = max(idbits - GroupCfg::kBucketBits, 0);
  }
  auto reserve = [&](long long need) -> long long {
    need = (need + 1) & ~1ll;
    const unsigned long long b = atomicAdd(scr_top, (unsigned long long)need);
    return (b + (unsigned long long)need <= (unsigned long long)scr_cap) ? (long long)b : -1ll;
  };
  // the next group is fetched while this one is processed: its item number
  // at the start (thread 0), its key after the gather, its cells' bounds
  // (threads 0-7, one cell each) after the counts of the member cells, so
  // that no dependent global load waits at the loop head
  int n_item = 0, n_qs = 0, n_qe = 0, n_cls = 0, stage = 0;
  unsigned n_ck = 0u;
  auto advance = [&](int target) {   // called by every thread at the same points
    if (stage < 1 && target >= 1) {
      if (tid == 0 && n_item < ngroups) n_ck = (unsigned)groups[1 + n_item];
      stage = 1;
    }
    if (stage < 2 && target >= 2) {
      if (tid == 0) S.nck = n_ck;
      stage = 2;
    }
    if (stage < 3 && target >= 3) {
      __syncthreads();
      // n_item is thread 0's; lanes 0-7 of warp 0 take its verdict
      const bool more = tid < 8 && __shfl_sync(0xffu, n_item < ngroups, 0);
      if (more) {
        const unsigned nk = S.nck;
        const unsigned key = pack3((int)(nk & ((1u << g.wx) - 1u)) + (tid & 1),
                                   (int)((nk >> g.wx) & ((1u << g.wy) - 1u)) + ((tid >> 1) & 1),
                                   (int)(nk >> (g.wx + g.wy)) + (tid >> 2), g);
        n_qs = __ldg(g.cell_start + key);
        n_qe = __ldg(g.cell_start + key + 1);
        n_cls = g.cell_cls[key];
      }
      stage = 3;
    }
  };
  if (tid == 0) n_item = atomicAdd(work, 1);
  advance(3);
  for (;;) {
    // the group's cells (bit i + 2 j + 4 k); the heavy ones are its members
    if (tid < 8) {
      const unsigned ck = S.nck;
      const unsigned key = pack3((int)(ck & ((1u << g.wx) - 1u)) + (tid & 1),
                                 (int)((ck >> g.wx) & ((1u << g.wy) - 1u)) + ((tid >> 1) & 1),
                                 (int)(ck >> (g.wx + g.wy)) + (tid >> 2), g);
      const int nq = n_qe - n_qs;
      const bool valid = __shfl_sync(0xffu, n_item < ngroups, 0);
      bool mine = valid && nq > 0 && n_cls == kCellHeavy;
      if (mine && nq > kMaxQ) {   // more queries than a block holds: the large configuration
        big[1 + atomicAdd(big, 1)] = (int)key;
        mine = false;
      }
      S.ckey[tid] = key;
      S.cq_s[tid] = n_qs;
      S.cq_n[tid] = nq;
      const unsigned b = __ballot_sync(0xffu, mine);
      if (tid == 0) {
        S.hm = (int)b;
        S.item = n_item;
        S.nt = 0;
        S.nc = 0;
        S.out_seen = 0;
        if (n_item < ngroups) n_item = atomicAdd(work, 1);
      }
    }
    for (int b = tid; b < kBuckets; b += blockDim.x) S.bstart[b] = 0;
    for (int i = tid; i < GroupSmem::kChunks; i += blockDim.x) S.outb[i] = 0u;
    stage = 0;
    __syncthreads();
    if (S.item >= ngroups) return;
    const unsigned ck = S.ckey[0];
    const int c0x = (int)(ck & ((1u << g.wx) - 1u));
    const int c0y = (int)((ck >> g.wx) & ((1u << g.wy) - 1u));
    const int c0z = (int)(ck >> (g.wx + g.wy));
    const int hm = S.hm;
    if (hm == 0) {
      advance(3);
      __syncthreads();
      continue;
    }
    // 1. runs of the group's rows: each x-row of cells within d of the
    //    group's box is one run of points, or two where it crosses the
    //    cyclic x boundary; rows leaving the region on a non-cyclic axis
    //    stand for the outside cell, listed once
    const unsigned long long cu = unpack3(c0x, c0y, c0z, g);
    auto add_run = [&](unsigned ka, unsigned kb, unsigned code) {
      const int b = __ldg(g.cell_start + ka), c = __ldg(g.cell_start + kb + 1) - b;
      if (c == 0) return;
      const int t = atomicAdd(&S.nt, 1);
      S.tbeg[t] = b;
      S.tcnt[t] = c;
      unsigned sh = (code & 64u) ? (1u << 24) : 0u;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const unsigned c2 = (code >> (2 * a)) & 3u;
        sh |= (c2 == 1u ? 0x01u : (c2 == 2u ? 0xffu : 0u)) << (8 * a);
      }
      S.tsh[t] = (int)sh;
    };
    for (int e = tid; e < n_grow; e += blockDim.x) {
      const unsigned long long E = grow[e];
      const int lo = (int)(signed char)((E >> 48) & 0xffull);
      const int len = (int)((E >> 56) & 127ull);
      const unsigned long long off = E & ((1ull << 48) - 1ull);
      const unsigned long long sum = cu + off;
      bool out = (sum & g.guard_non) != 0ull;
      if (!out) {
        unsigned code = 0;
        if (sum & g.gy) code |= ((off & g.gy) ? 2u : 1u) << 2;
        if (sum & g.gz) code |= ((off & g.gz) ? 2u : 1u) << 4;
        const unsigned row = repack(sum & g.valid, g) - (unsigned)c0x;   // packed index of x = 0
        int x0 = c0x + lo, x1 = x0 + len - 1;
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
    __syncthreads();
    const int nt = S.nt;
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
    // 2. gather: every point of the runs, moved to the group's frame; its
    //    member bits are the heavy cells whose box it lies within d of
    const float fx = (float)c0x, fy = (float)c0y, fz = (float)c0z;
    constexpr int kGather = 4;
    for (int f0 = wid * 32 * kGather; f0 < ntot; f0 += nw * 32 * kGather) {
      int rr = 0;
      {
        int top = nt - 1;
        while (rr < top) {
          const int mid = (rr + top + 1) >> 1;
          if (S.tpre[mid] <= f0) rr = mid;
          else top = mid - 1;
        }
      }
      int cj[kGather], tt[kGather];
#pragma unroll
      for (int u = 0; u < kGather; ++u) {
        const int f = f0 + u * 32 + lane;
        cj[u] = -1;
        tt[u] = 0;
        if (f < ntot) {
          while (S.tpre[rr + 1] <= f) ++rr;
          tt[u] = rr;
          cj[u] = S.tbeg[rr] + (f - S.tpre[rr]);
        }
      }
      float4 p[kGather];
      int pid[kGather];
#pragma unroll
      for (int u = 0; u < kGather; ++u) {
        p[u] = cj[u] >= 0 ? g.spos[cj[u]] : make_float4(0.f, 0.f, 0.f, 0.f);
        pid[u] = cj[u] >= 0 ? __ldg(g.perm + cj[u]) : 0;
      }
#pragma unroll
      for (int u = 0; u < kGather; ++u) {
        unsigned mem = 0u;
        if (cj[u] >= 0) {
          const int sh = S.tsh[tt[u]];
          if (sh >> 24) {
            p[u].x = __int_as_float(0x7fc00000);   // outside cell: FP64 test for every pair, for every cell
            mem = (unsigned)hm;
          } else {
            p[u].x = fmaf((float)(signed char)(sh & 0xff), g.Lx, p[u].x);
            p[u].y = fmaf((float)(signed char)((sh >> 8) & 0xff), g.Ly, p[u].y);
            p[u].z = fmaf((float)(signed char)((sh >> 16) & 0xff), g.Lz, p[u].z);
            // cell units from the group's lowest cell, for its lower and
            // upper cell along each axis (the cell kernel's box test)
            const float tx = (p[u].x - g.ox) * g.inv_s, ty = (p[u].y - g.oy) * g.inv_s,
                        tz = (p[u].z - g.oz) * g.inv_s;
            const float ux0 = tx - fx, ux1 = tx - (fx + 1.f);
            const float uy0 = ty - fy, uy1 = ty - (fy + 1.f);
            const float uz0 = tz - fz, uz1 = tz - (fz + 1.f);
            const float gx0 = fmaxf(fmaxf(-ux0, ux0 - 1.f), 0.f), gx1 = fmaxf(fmaxf(-ux1, ux1 - 1.f), 0.f);
            const float gy0 = fmaxf(fmaxf(-uy0, uy0 - 1.f), 0.f), gy1 = fmaxf(fmaxf(-uy1, uy1 - 1.f), 0.f);
            const float gz0 = fmaxf(fmaxf(-uz0, uz0 - 1.f), 0.f), gz1 = fmaxf(fmaxf(-uz1, uz1 - 1.f), 0.f);
            const float x2[2] = {gx0 * gx0, gx1 * gx1};
            const float yz[4] = {fmaf(gz0, gz0, gy0 * gy0), fmaf(gz0, gz0, gy1 * gy1), fmaf(gz1, gz1, gy0 * gy0),
                                 fmaf(gz1, gz1, gy1 * gy1)};
#pragma unroll
            for (int b = 0; b < 8; ++b)
              if (x2[b & 1] + yz[b >> 1] <= box2) mem |= 1u << b;
            mem &= (unsigned)hm;
          }
        }
        const bool keep = mem != 0u;
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
            S.mem[at] = (unsigned char)mem;
            S.u.s.sid[at] = pid[u];
            atomicAdd(&S.bstart[pid[u] >> bshift], 1);
          }
        }
      }
    }
    __syncthreads();
    advance(1);
    const int nu = S.nc;
    if (nu > kCap) {   // the union does not fit: every member cell to the large configuration
      if (tid < 8 && ((hm >> tid) & 1)) big[1 + atomicAdd(big, 1)] = (int)S.ckey[tid];
      advance(3);
      __syncthreads();
      continue;
    }
    // 3. the union in ascending input index
    {
      constexpr int kPerB = kBuckets / GroupCfg::kThreads;
      int v[kPerB], bsum = 0;
#pragma unroll
      for (int r = 0; r < kPerB; ++r) {
        v[r] = S.bstart[tid * kPerB + r];
        bsum += v[r];
      }
      int total;
      int run = block_excl_scan_i(bsum, total, S.scan);
#pragma unroll
      for (int r = 0; r < kPerB; ++r) {
        S.bstart[tid * kPerB + r] = run;
        S.bcur[tid * kPerB + r] = run;
        run += v[r];
      }
      __syncthreads();
      for (int p = tid; p < nu; p += blockDim.x) {
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
      __syncthreads();
      for (int k = tid; k < nu; k += blockDim.x) {
        const unsigned long long kk = S.u.s.key[k];
        S.uslot[k] = (unsigned short)(kk & 0xffffu);
        S.uid[k] = (int)(kk >> 32);
      }
      advance(2);
      __syncthreads();
    }
    // 4. the member cells' candidates, each in id order: warp w compacts the
    //    union positions [w per, (w + 1) per).  First every member cell's
    //    count per warp range, then one reservation for all their records
    //    (the cell's ordered ids, then its hit masks), then each cell in turn.
    const int per = ((nu + nw * 32 - 1) / (nw * 32)) * 32;
    const int kb = min(nu, wid * per), ke = min(nu, kb + per);
    {
      int cntw[8] = {0, 0, 0, 0, 0, 0, 0, 0};
      for (int k0 = kb; k0 < ke; k0 += 32) {
        const int k = k0 + lane;
        const unsigned mb = k < ke ? (unsigned)S.mem[S.uslot[k]] : 0u;
#pragma unroll
        for (int h = 0; h < 8; ++h)
          if ((hm >> h) & 1) cntw[h] += __popc(__ballot_sync(0xffffffffu, (mb >> h) & 1u));
      }
      if (lane == 0)
#pragma unroll
        for (int h = 0; h < 8; ++h) S.wcnt[h][wid] = cntw[h];
    }
    __syncthreads();
    if (wid == 0) {
      long long need = 0;
      for (int h = 0; h < 8; ++h) {
        if (!((hm >> h) & 1)) continue;
        const int x = lane < nw ? S.wcnt[h][lane] : 0;
        const int inc = warp_incl_scan_i(x);
        if (lane < nw) S.wcnt[h][lane] = inc - x;
        const int nc = __shfl_sync(0xffffffffu, inc, 31);
        if (lane == 0) {
          S.cnc[h] = nc;
          S.coff[h] = need;
        }
        need += (2ll + nc + (long long)S.cq_n[h] * ((nc + 31) >> 5)) & ~1ll;
      }
      if (lane == 0) S.base = reserve(need);
    }
    advance(3);   // its barrier also publishes the counts and the reservation
    if (S.base < 0) {   // no room in the scratch buffer: the per-query path serves the group's cells
      for (int h = 0; h < 8; ++h) {
        if (!((hm >> h) & 1)) continue;
        const int qs = S.cq_s[h], nq = S.cq_n[h];
        for (int i = tid; i < nq; i += blockDim.x) over[1 + atomicAdd(over, 1)] = qs + i;
        if (tid == 0) cell_rec[S.ckey[h]] = -1;
      }
      __syncthreads();
      continue;
    }
    for (int h = 0; h < 8; ++h) {
      if (!((hm >> h) & 1)) continue;
      const int qs = S.cq_s[h], nq = S.cq_n[h], nc = S.cnc[h];
      const int nchunk = (nc + 31) >> 5;
      const long long rec = S.base + S.coff[h];
      int *rec_ids = scratch + rec + 1;
      unsigned *rec_masks = reinterpret_cast<unsigned *>(rec_ids + nc);
      if (tid == 0) scratch[rec] = nc;
      // the cell's candidates in id order into the packed pairs; its own
      // points (unshifted: the group's own rows never wrap) are its queries
      int pos = S.wcnt[h][wid];
      for (int k0 = kb; k0 < ke; k0 += 32) {
        const int k = k0 + lane;
        const int sl = k < ke ? (int)S.uslot[k] : 0;
        const bool m = k < ke && ((S.mem[sl] >> h) & 1u);
        const unsigned bal = __ballot_sync(0xffffffffu, m);
        if (m) {
          const int kc = pos + __popc(bal & lt_mask);
          const float4 v = S.c[sl];
          put_pair(S.u.t.xy, S.u.t.z, kc, v);
          S.cslot[kc] = (unsigned short)sl;
          rec_ids[kc] = S.uid[k];
          const int ql = __float_as_int(v.w) - qs;
          if (ql >= 0 && ql < nq) {
            S.qa[ql] = make_float4(v.x, v.x, v.y, v.y);
            S.qb[ql] = make_float4(v.z, v.z, __int_as_float(incl_self ? -1 : kc), 0.f);
            S.qcnt[ql] = 0;
          }
          if (isnan(v.x)) atomicOr(&S.outb[kc >> 5], 1u << (kc & 31));
        }
        pos += __popc(bal);
      }
      for (int kc = nc + tid; kc < nchunk * 32; kc += blockDim.x)
        put_pair(S.u.t.xy, S.u.t.z, kc, make_float4(INFINITY, INFINITY, INFINITY, 0.f));
      __syncthreads();
      cell_test_phase(g, B, nq, nchunk, S.u.t.xy, S.u.t.z, S.outb, S.c, S.cslot, S.qa, S.qb, S.qcnt, rec_masks,
                      lane, wid, nw);
      __syncthreads();
      for (int i = tid; i < nq; i += blockDim.x) counts[__ldg(g.perm + qs + i)] = S.qcnt[i];
      if (tid == 0) cell_rec[S.ckey[h]] = rec;
      for (int i = tid; i < nchunk; i += blockDim.x) S.outb[i] = 0u;
      __syncthreads();   // the next cell rewrites the query and candidate arrays
    }
  }
}

si_status launch_cell_group(const GridDev &g, const WalkParams &P, const Band &B, unsigned flags,
                            const int *heavy, int *groups, int *solo, int *work, int *big, int *over,
                            long long *counts, long long *cell_rec, int *scratch, long long scr_cap,
                            unsigned long long *scr_top, const unsigned long long *grow, int n_grow,
                            cudaStream_t st) {
  SI_KLAUNCH("k_group_list", st, k_group_list<<<148 * 4, 256, 0, st>>>(g, heavy, groups, solo));
  const size_t smem = sizeof(GroupSmem);
  SI_CUDA_TRY(cudaFuncSetAttribute(k_cell_group, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  SI_KLAUNCH("k_cell_group", st,
             k_cell_group<<<148 * GroupCfg::kMinBlocks, GroupCfg::kThreads, smem, st>>>(
                 g, P, B, flags, groups, work, big, over, counts, cell_rec, scratch, scr_cap, scr_top, grow,
                 n_grow));
  return SI_OK;
}

}  // namespace si
