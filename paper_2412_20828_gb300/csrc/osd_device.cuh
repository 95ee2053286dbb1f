// Order-p OSD of one frame by one warp (arXiv 2412.20828, Sec. II-B): the device code
// shared by the batch OSD kernel and the serving kernel.
//
// One warp decodes one failed frame:
//  * reliabilities |L| (FP32) are ranked by counting against 64-bit keys
//    (|L| bits, index) -- a total order equal to a stable ascending sort;
//  * Gaussian elimination over GF(2) runs on the standard H in its original column
//    order, visiting columns from least to most reliable: lane l holds rows l and
//    l + 32 as 128-bit words, the pivot row is found by ballot and broadcast by
//    shuffles;
//  * with the reduced rows, the disagreement pattern of a test pattern e on the
//    most reliable basis is D(e) = D0 xor (xor of the basis columns in e) restricted
//    to the n-k pivot positions, so a candidate costs a few XORs plus a weighted
//    popcount done with 16-entry tables of pivot weights, one per 4 pivot rows (built
//    by doubling: entry v = entry v - 2^b + weight b for the top bit b of v);
//  * scores are exact 64-bit integers (weights floor(|L| 2^24)), and the warp keeps
//    the lexicographic minimum of (score, enumeration index): the result equals a
//    sequential scan that keeps the first minimum.
#pragma once
#include "nms_device.cuh"

namespace bchlib {


// About 4.9 KB per warp, so that many warps share an SM (the elimination is a chain of
// dependent ballots and shuffles that needs other warps to hide its latency).
struct OsdSmem {
  union {
    unsigned long long key[128];      // sort keys (ranking phase only)
    unsigned long long colbits[128];  // basis columns on the pivot rows (after elimination)
  };
  unsigned long long wm[128];  // weights of the MRB positions, by basis index
  unsigned long long wp[64];   // weights of the pivot positions, by row
  unsigned long long tab[16][16];  // weighted popcount of each 4-row chunk
  uint8_t perm[128];           // sorted position -> original index
  uint8_t mrb[128];            // basis index -> original index
  uint8_t ispiv[128];          // by original index
};

__device__ __forceinline__ bool bit128(uint4 r, uint32_t c) {
  const uint32_t w = c < 32 ? r.x : (c < 64 ? r.y : (c < 96 ? r.z : r.w));
  return (w >> (c & 31)) & 1u;
}
__device__ __forceinline__ uint4 xor4(uint4 a, uint4 b) {
  return make_uint4(a.x ^ b.x, a.y ^ b.y, a.z ^ b.z, a.w ^ b.w);
}
__device__ __forceinline__ uint4 and4(uint4 a, uint4 b) {
  return make_uint4(a.x & b.x, a.y & b.y, a.z & b.z, a.w & b.w);
}
__device__ __forceinline__ uint32_t parity4(uint4 a) { return __popc(a.x ^ a.y ^ a.z ^ a.w) & 1u; }
__device__ __forceinline__ uint4 shfl4(uint4 v, int src) {
  return make_uint4(__shfl_sync(kFull, v.x, src), __shfl_sync(kFull, v.y, src),
                    __shfl_sync(kFull, v.z, src), __shfl_sync(kFull, v.w, src));
}

__device__ __forceinline__ unsigned long long wsum(const OsdSmem &S, unsigned long long D, int nch) {
  unsigned long long s = 0;
  for (int c = 0; c < nch; c++) s += S.tab[c][(D >> (4 * c)) & 0xfu];
  return s;
}

struct Best {
  unsigned long long s;
  uint32_t idx;
  uint32_t ab;  // (a + 1) | (b + 1) << 8, 0 = no flip
};

__device__ __forceinline__ void consider(Best &b, unsigned long long s, uint32_t idx, uint32_t ab) {
  if (s < b.s || (s == b.s && idx < b.idx)) {
    b.s = s;
    b.idx = idx;
    b.ab = ab;
  }
}

// Order-p OSD of one frame by one warp (all 32 lanes call it with the same
// arguments).  L: the frame's FP32 channel LLRs; rows: the M standard-H rows;
// hard: the frame's ceil(n/64) output words; flag: its flag byte (nullable).
__device__ __forceinline__ void osd_one_frame(OsdSmem &S, int n, int K, int M, const uint4 *rows,
                                              const float *L, int order, uint64_t *hard,
                                              uint8_t *flag) {
  const int lane = int(lane_id());
  // ---- reliabilities, hard decision, weights
  float lv[4];
  unsigned long long wv[4];
  uint4 h = make_uint4(0, 0, 0, 0);
#pragma unroll
  for (int r = 0; r < 4; r++) {
    const int i = lane + 32 * r;
    lv[r] = i < n ? L[i] : 0.0f;
    const float al = fabsf(lv[r]);
    const float fw = fminf(floorf(al * 16777216.0f), 1099511627776.0f);
    wv[r] = __float2ull_rz(fw);
    const unsigned hb = __ballot_sync(kFull, i < n && lv[r] < 0.0f);
    if (r == 0) h.x = hb;
    if (r == 1) h.y = hb;
    if (r == 2) h.z = hb;
    if (r == 3) h.w = hb;
    if (i < 128)
      S.key[i] = i < n ? ((unsigned long long)__float_as_uint(al) << 7) | unsigned(i)
                       : ~0ull;
    if (i < 128) S.ispiv[i] = 0;
  }
  __syncwarp();
  // rank by counting (keys are distinct)
#pragma unroll
  for (int r = 0; r < 4; r++) {
    const int i = lane + 32 * r;
    if (i < n) {
      const unsigned long long ki = S.key[i];
      int rank = 0;
      for (int q = 0; q < n; q++) rank += S.key[q] < ki;
      S.perm[rank] = uint8_t(i);
    }
  }
  __syncwarp();
  // ---- elimination in reliability order
  uint4 row0 = make_uint4(0, 0, 0, 0), row1 = make_uint4(0, 0, 0, 0);
  if (lane < M) row0 = rows[lane];
  if (lane + 32 < M) row1 = rows[lane + 32];
  bool piv0 = lane >= M, piv1 = lane + 32 >= M;
  int pc0 = 0, pc1 = 0;
  int npiv = 0;
  for (int q = 0; q < n && npiv < M; q++) {
    const uint32_t c = S.perm[q];
    const unsigned m0 = __ballot_sync(kFull, !piv0 && bit128(row0, c));
    const unsigned m1 = __ballot_sync(kFull, !piv1 && bit128(row1, c));
    if ((m0 | m1) == 0) continue;
    const int pr = m0 ? (__ffs(m0) - 1) : (32 + __ffs(m1) - 1);
    const int src = pr & 31;
    const uint4 pv = shfl4(pr < 32 ? row0 : row1, src);
    if (bit128(row0, c) && lane != pr) row0 = xor4(row0, pv);
    if (bit128(row1, c) && lane + 32 != pr) row1 = xor4(row1, pv);
    if (lane == pr) {
      piv0 = true;
      pc0 = int(c);
    }
    if (lane + 32 == pr) {
      piv1 = true;
      pc1 = int(c);
    }
    if (lane == 0) S.ispiv[c] = 1;
    npiv++;
  }
  __syncwarp();
  // ---- most reliable basis in sorted order
  int kk = 0;
  for (int base = 0; base < n; base += 32) {
    const int q = base + lane;
    const bool isb = q < n && !S.ispiv[S.perm[q < n ? q : 0]];
    const unsigned bm = __ballot_sync(kFull, isb);
    if (isb) S.mrb[kk + __popc(bm & ((1u << lane) - 1u))] = S.perm[q];
    kk += __popc(bm);
  }
  __syncwarp();
  // weights by original index are held per lane (wv); gather the needed ones
  for (int a2 = lane; a2 < K; a2 += 32) {
    const int ci = S.mrb[a2];
    const float al = fabsf(L[ci]);
    S.wm[a2] = __float2ull_rz(fminf(floorf(al * 16777216.0f), 1099511627776.0f));
  }
  {
    const float al0 = lane < M ? fabsf(L[pc0]) : 0.f;
    const float al1 = lane + 32 < M ? fabsf(L[pc1]) : 0.f;
    S.wp[lane] = lane < M ? __float2ull_rz(fminf(floorf(al0 * 16777216.0f), 1099511627776.0f)) : 0ull;
    S.wp[lane + 32] =
        lane + 32 < M ? __float2ull_rz(fminf(floorf(al1 * 16777216.0f), 1099511627776.0f)) : 0ull;
  }
  // basis columns restricted to the pivot rows
  for (int a2 = 0; a2 < K; a2++) {
    const uint32_t c = S.mrb[a2];
    const unsigned b0 = __ballot_sync(kFull, lane < M && bit128(row0, c));
    const unsigned b1 = __ballot_sync(kFull, lane + 32 < M && bit128(row1, c));
    if (lane == 0) S.colbits[a2] = (unsigned long long)b0 | ((unsigned long long)b1 << 32);
  }
  // D0: disagreement of the re-encoded hard decision on the pivot positions
  const unsigned d0a = __ballot_sync(kFull, lane < M && parity4(and4(row0, h)));
  const unsigned d0b = __ballot_sync(kFull, lane + 32 < M && parity4(and4(row1, h)));
  const unsigned long long D0 = (unsigned long long)d0a | ((unsigned long long)d0b << 32);
  __syncwarp();
  const int nch = (M + 3) / 4;
  if (lane < nch) S.tab[lane][0] = 0ull;
  __syncwarp();
  for (int b = 0; b < 4; b++) {
    const int per = 1 << b;
    for (int e = lane; e < nch * per; e += 32) {
      const int c = e >> b, v = e & (per - 1);
      S.tab[c][per + v] = S.tab[c][v] + S.wp[4 * c + b];
    }
    __syncwarp();
  }
  // ---- enumerate test patterns
  Best best;
  best.s = ~0ull;
  best.idx = 0xffffffffu;
  best.ab = 0;
  if (lane == 0) consider(best, wsum(S, D0, nch), 0u, 0u);
  if (order >= 1) {
    for (int x = lane; x < K; x += 32)
      consider(best, S.wm[x] + wsum(S, D0 ^ S.colbits[x], nch), uint32_t(1 + x), uint32_t(x + 1));
  }
  if (order >= 2) {
    // Exact pruning.  A candidate's score is at least wm[x] + wm[y] (all weights are
    // non-negative) and wm ascends with the basis index (reliability order).  Every
    // weight-2 candidate comes after the weight <= 1 ones in the enumeration, and a
    // lane's earlier candidates come before its later ones, so a candidate whose bound
    // reaches either best can at most tie it with a larger index: it cannot be chosen.
    unsigned long long bound1 = best.s;
    for (int off = 16; off > 0; off >>= 1) bound1 = min(bound1, __shfl_xor_sync(kFull, bound1, off));
    for (int x = 0; x + 1 < K; x++) {
      const unsigned long long wa = S.wm[x];
      if (wa + S.wm[x + 1] >= bound1) break;  // no pair (x' >= x, y > x') can win
      const unsigned long long Da = D0 ^ S.colbits[x];
      const uint32_t base = uint32_t(1 + K) + uint32_t(x * K - x * (x + 1) / 2);
      for (int y = x + 1 + lane; y < K; y += 32) {
        const unsigned long long lb = wa + S.wm[y];
        if (lb >= bound1 || lb >= best.s) break;  // later y only raise the bound
        const unsigned long long s = lb + wsum(S, Da ^ S.colbits[y], nch);
        consider(best, s, base + uint32_t(y - x - 1), uint32_t(x + 1) | (uint32_t(y + 1) << 8));
      }
    }
  }
  for (int off = 16; off > 0; off >>= 1) {
    Best o;
    o.s = __shfl_xor_sync(kFull, best.s, off);
    o.idx = __shfl_xor_sync(kFull, best.idx, off);
    o.ab = __shfl_xor_sync(kFull, best.ab, off);
    consider(best, o.s, o.idx, o.ab);
  }
  // ---- rebuild the winner
  const int fa = int(best.ab & 0xffu) - 1, fb = int((best.ab >> 8) & 0xffu) - 1;
  unsigned long long D = D0;
  if (fa >= 0) D ^= S.colbits[fa];
  if (fb >= 0) D ^= S.colbits[fb];
  uint4 flip = make_uint4(0, 0, 0, 0);
  auto setb = [](uint4 &v, int c) {
    const uint32_t m = 1u << (c & 31);
    if (c < 32) v.x ^= m;
    else if (c < 64) v.y ^= m;
    else if (c < 96) v.z ^= m;
    else v.w ^= m;
  };
  if (lane < M && ((D >> lane) & 1ull)) setb(flip, pc0);
  if (lane + 32 < M && ((D >> (lane + 32)) & 1ull)) setb(flip, pc1);
  for (int off = 16; off > 0; off >>= 1) {
    flip.x ^= __shfl_xor_sync(kFull, flip.x, off);
    flip.y ^= __shfl_xor_sync(kFull, flip.y, off);
    flip.z ^= __shfl_xor_sync(kFull, flip.z, off);
    flip.w ^= __shfl_xor_sync(kFull, flip.w, off);
  }
  if (lane == 0) {
    if (fa >= 0) setb(flip, S.mrb[fa]);
    if (fb >= 0) setb(flip, S.mrb[fb]);
    const uint4 c = xor4(h, flip);
    const int W64 = (n + 63) / 64;
    hard[0] = (unsigned long long)c.x | ((unsigned long long)c.y << 32);
    if (W64 > 1) hard[1] = (unsigned long long)c.z | ((unsigned long long)c.w << 32);
    if (flag) *flag |= uint8_t(kFlagOsd);
  }
  __syncwarp();
}

}  // namespace bchlib
