// Shared pieces of the heavy-cell kernels (si_cell.cu: one block per
// heavy cell; si_group.cu: one block per 2x2x2 group of heavy cells): the
// block configurations, the packed-pair layout of the staged candidates and
// the test phase that turns them into per-query hit masks.
#pragma once

#include <cmath>

#include "si_host.h"
#include "si_radius.cuh"
#include "si_walk.cuh"

namespace si {

template <int THREADS, int CAP, int MAXQ, int BUCKETS, int MINB>
struct CellCfg {
  static constexpr int kThreads = THREADS;   // block size
  static constexpr int kCap = CAP;           // staged candidates
  static constexpr int kMaxQ = MAXQ;         // queries of the cell
  static constexpr int kBuckets = BUCKETS;   // id buckets of the sort
  static constexpr int kMinBlocks = MINB;    // resident blocks per SM
  static constexpr int kBucketBits = BUCKETS == 1024 ? 10 : (BUCKETS == 512 ? 9 : 8);
  static_assert((1 << kBucketBits) == BUCKETS, "bucket count must be 256, 512 or 1024");
  static_assert(CAP % 32 == 0 && CAP <= 65536, "candidate capacity: whole chunks, 16-bit slots");
};

// Candidates of the test phase: packed FP32 pairs, 16 per chunk of 32
// candidates, each chunk padded to kPairRow entries so that the streams of a
// warp (which read different chunks at once) fall in different banks.
constexpr int kPairRow = 17;

// Packed FP32 pairs (low half = first value) for f32x2 instructions.
__device__ __forceinline__ unsigned long long pack2(float a, float b) {
  return ((unsigned long long)__float_as_uint(b) << 32) | (unsigned long long)__float_as_uint(a);
}

// Write candidate k (in the query frame; +inf for the padding of the last
// chunk) into the packed pairs.
__device__ __forceinline__ void put_pair(float4 *xy, float2 *z, int k, const float4 &v) {
  const int at = (k >> 5) * kPairRow + ((k & 31) >> 1);
  float *pxy = reinterpret_cast<float *>(xy + at);
  float *pz = reinterpret_cast<float *>(z + at);
  pxy[k & 1] = v.x;
  pxy[2 + (k & 1)] = v.y;
  pz[k & 1] = v.z;
}

// The test phase of a heavy cell: nq queries (qa: (x, x, y, y), qb: (z, z,
// own position among the candidates or -1, -)) against nc candidates in id
// order (packed pairs xy / z; outb: per chunk, the candidates of the outside
// cell; candidate k is staged at c[slot[k]], whose w is its sorted slot).
// Writes one 32-bit hit mask per (query, chunk) to masks (query-major, bit b
// of chunk ch = candidate 32 ch + b) and adds each query's hits to qcnt.
//
// A lane owns one query and builds that query's mask over a chunk, reading
// the candidates as packed FP32 pairs that every lane of its stream reads at
// once (broadcast).  The queries go in tiles of 32 lanes; what remains
// (r < 32 queries) goes in a tile of 32 (r > 24), of 16 and one of 8
// (16 < r <= 24), of 16 (8 < r <= 16) or of 8, and a warp reads a tile of
// 16 (8) lanes as 2 (4) streams, each on its own chunk; warps take
// (tile, chunk row) items round-robin.  Both distances of a pair are
// computed with the f32x2 operations of the scalar path (the same
// round-to-nearest operations, in the same order).  For the sign test,
// d2 <= t holds exactly when d2 - next_up(t) is negative (a float
// difference has the sign of the exact one), so a funnel shift moves the
// sign bit into the mask: one instruction per candidate.  Two masks, against
// the two ends of the guard band, give the pairs inside it, which are
// decided with the FP64 predicate; so are the candidates of the outside
// cell.  A query's own position is never a hit.
__device__ __forceinline__ void cell_test_phase(const GridDev &g, const Band &B, int nq, int nchunk,
                                                const float4 *__restrict__ pxy, const float2 *__restrict__ pz,
                                                const unsigned *__restrict__ outb, const float4 *__restrict__ c,
                                                const unsigned short *__restrict__ slot, const float4 *qa_s,
                                                const float4 *qb_s, int *qcnt, unsigned *__restrict__ rec_masks,
                                                int lane, int wid, int nw) {
  const float tlo = nextafterf(B.lo_w, INFINITY), thi = nextafterf(B.hi_w, INFINITY);
  const unsigned long long TL = pack2(tlo, tlo), TH = pack2(thi, thi);
  const int nfull = nq >> 5, rem = nq & 31;
  const int ntile = nfull + (rem == 0 ? 0 : ((rem > 16 && rem <= 24) ? 2 : 1));
  int ibase = 0;   // items of the tiles before this one (warps take items round-robin)
  for (int tile = 0; tile < ntile; ++tile) {
    int q0 = tile << 5, lgG = 5, nqt = 32;
    if (tile == nfull) {
      lgG = rem > 24 ? 5 : (rem > 8 ? 4 : 3);
      nqt = (rem > 16 && rem <= 24) ? 16 : rem;
    } else if (tile > nfull) {
      q0 = (nfull << 5) + 16;
      lgG = 3;
      nqt = rem - 16;
    }
    const int lgS = 5 - lgG;   // log2 of the streams per warp
    const int items = (nchunk + (1 << lgS) - 1) >> lgS;
    const int st = lane >> lgG, qi = lane & ((1 << lgG) - 1);
    const int q = q0 + qi;
    const bool qok = qi < nqt;
    const float4 qa = qa_s[qok ? q : 0], qb = qb_s[qok ? q : 0];
    const unsigned long long QX = pack2(qa.x, qa.y), QY = pack2(qa.z, qa.w), QZ = pack2(qb.x, qb.y);
    const int own = __float_as_int(qb.z);
    int cnt = 0;
    for (int j = (wid - ibase) & (nw - 1); j < items; j += nw) {
      const int ch = (j << lgS) + st;
      if (ch >= nchunk) continue;
      const float4 *xy = pxy + ch * kPairRow;
      const float2 *zz = pz + ch * kPairRow;
      unsigned mlo = 0u, mhi = 0u;
#pragma unroll
      for (int p = 15; p >= 0; --p) {
        const float4 a = xy[p];
        const float2 b = zz[p];
        unsigned long long dx, dy, dz, D2, xl, xh;
        asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(dx) : "l"(pack2(a.x, a.y)), "l"(QX));
        asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(dy) : "l"(pack2(a.z, a.w)), "l"(QY));
        asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(dz) : "l"(pack2(b.x, b.y)), "l"(QZ));
        asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(D2) : "l"(dx), "l"(dx));
        asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(D2) : "l"(dy), "l"(dy), "l"(D2));
        asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(D2) : "l"(dz), "l"(dz), "l"(D2));
        asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(xl) : "l"(D2), "l"(TL));
        asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(xh) : "l"(D2), "l"(TH));
        // candidate 2p + 1 (high half), then 2p: after the 32 shifts
        // candidate k of the chunk sits at bit k
        mlo = __funnelshift_l((unsigned)(xl >> 32), mlo, 1);
        mlo = __funnelshift_l((unsigned)xl, mlo, 1);
        mhi = __funnelshift_l((unsigned)(xh >> 32), mhi, 1);
        mhi = __funnelshift_l((unsigned)xh, mhi, 1);
      }
      unsigned band = (mhi & ~mlo) | outb[ch];
      if (band && qok) {
        const float4 qp = make_float4(qa.x, qa.z, qb.x, 0.f);
        do {
          const int bit = __ffs(band) - 1;
          band &= band - 1u;
          const float4 cand = c[slot[(ch << 5) + bit]];
          const bool h = canon_d2(qp, g.spos[__float_as_int(cand.w)], g) <= B.r2;
          mlo = h ? (mlo | (1u << bit)) : (mlo & ~(1u << bit));
        } while (band);
      }
      if ((own >> 5) == ch) mlo &= ~(1u << (own & 31));
      if (qok) {
        rec_masks[q * nchunk + ch] = mlo;
        cnt += __popc(mlo);
      }
    }
    if (qok && cnt) atomicAdd(&qcnt[q], cnt);
    ibase += items;
  }
}

}  // namespace si
