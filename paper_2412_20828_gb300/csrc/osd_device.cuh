// Order-p OSD of one frame by one warp (arXiv 2412.20828, Sec. II-B): the device code
// shared by the batch OSD kernel and the serving kernel.
//
// One warp decodes one failed frame:
//  * reliabilities |L| (FP32) are ranked by counting against 64-bit keys
//    (|L| bits, index) -- a total order equal to a stable ascending sort;
//  * Gauss-Jordan elimination over GF(2) on the standard H visits columns from least
//    to most reliable in column-major form: lane l holds the row masks of columns l,
//    l + 32, l + 64, l + 96; a pivot step fetches the column's mask by one shuffle,
//    takes its lowest unpivoted row and xors the column (minus that row) into every
//    column having the row;
//  * with the reduced rows, the disagreement pattern of a test pattern e on the
//    most reliable basis is D(e) = D0 xor (xor of the basis columns in e) restricted
//    to the n-k pivot positions, so a candidate costs a few XORs plus a weighted
//    popcount done with 16-entry tables of pivot weights, one per 4 pivot rows (built
//    by doubling: entry v = entry v - 2^b + weight b for the top bit b of v);
//  * scores are exact 64-bit integers (weights floor(|L| 2^24)), and the warp keeps
//    the lexicographic minimum of (score, enumeration index): the result equals a
//    sequential scan that keeps the first minimum.
#pragma once
#ifndef __CUDACC_RTC__
#include "nms_device.cuh"
#endif

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
  unsigned long long colm[128];    // reduced column masks, by original index
  uint8_t perm[128];           // sorted position -> original index
  uint8_t mrb[128];            // basis index -> original index
  uint8_t ispiv[128];          // by original index
  uint8_t pivcol[64];          // pivot column of each row
};

__device__ __forceinline__ uint4 xor4(uint4 a, uint4 b) {
  return make_uint4(a.x ^ b.x, a.y ^ b.y, a.z ^ b.z, a.w ^ b.w);
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

// Mask of the M <= 64 rows: 32 bits when M <= 32.
template <typename MT>
__device__ __forceinline__ MT shfl_mask(MT v, int src) {
  if constexpr (sizeof(MT) == 4) {
    return __shfl_sync(kFull, v, src);
  } else {
    const uint32_t lo = __shfl_sync(kFull, uint32_t(v), src);
    const uint32_t hi = __shfl_sync(kFull, uint32_t(v >> 32), src);
    return (MT(hi) << 32) | lo;
  }
}
template <typename MT>
__device__ __forceinline__ int ffs_mask(MT v) {
  if constexpr (sizeof(MT) == 4) return __ffs(v) - 1;
  else return __ffsll((long long)v) - 1;
}

// Order-p OSD of one frame by one warp (all 32 lanes call it with the same
// arguments).  L: the frame's FP32 channel LLRs; cols: the n column masks of the
// standard H over its M rows; hard: the frame's ceil(n/64) output words; flag: its
// flag byte (nullable).  MT: the row-mask type (uint32_t when M <= 32).
//
// The elimination is column-major: lane l keeps the masks of columns l, l + 32, l + 64
// and l + 96.  Pivoting on column c (least reliable first) takes its current mask v,
// the lowest not-yet-pivoted row r in v, and adds row r to every other row of v -- in
// column form, every column whose mask has bit r gets v without bit r xored in
// (Gauss-Jordan over all rows, the same steps as a row-major elimination).
template <typename MT>
__device__ __forceinline__ void osd_one_frame_t(OsdSmem &S, int n, int K, int M, const uint64_t *cols,
                                                const float *L, int order, uint64_t *hard,
                                                uint8_t *flag, int sexp) {
  const int lane = int(lane_id());
  // ---- reliabilities, hard decision, sort keys
  uint4 h = make_uint4(0, 0, 0, 0);
  MT colm[4];
#pragma unroll
  for (int r = 0; r < 4; r++) {
    const int i = lane + 32 * r;
    const float lv = i < n ? ldexpf(L[i], sexp) : 0.0f;
    const float al = fabsf(lv);
    const unsigned hb = __ballot_sync(kFull, i < n && lv < 0.0f);
    if (r == 0) h.x = hb;
    if (r == 1) h.y = hb;
    if (r == 2) h.z = hb;
    if (r == 3) h.w = hb;
    S.key[i] = i < n ? ((unsigned long long)__float_as_uint(al) << 7) | unsigned(i) : ~0ull;
    S.ispiv[i] = 0;
    colm[r] = i < n ? MT(__ldg(cols + i)) : MT(0);
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
  // ---- elimination in reliability order (column-major)
  MT pivoted = 0;
  int npiv = 0;
  for (int q = 0; q < n && npiv < M; q++) {
    const int c = S.perm[q];
    const int cw = c >> 5;
    const MT mine = cw == 0 ? colm[0] : cw == 1 ? colm[1] : cw == 2 ? colm[2] : colm[3];
    const MT v = shfl_mask(mine, c & 31);
    const MT cand = v & ~pivoted;
    if (cand == 0) continue;
    const int r = ffs_mask(cand);
    const MT rbit = MT(1) << r;
    const MT vm = v & ~rbit;
    pivoted |= rbit;
    if (lane == 0) {
      S.pivcol[r] = uint8_t(c);
      S.ispiv[c] = 1;
    }
#pragma unroll
    for (int w = 0; w < 4; w++)
      if (colm[w] & rbit) colm[w] ^= vm;
    npiv++;
  }
  // reduced columns by original index
#pragma unroll
  for (int w = 0; w < 4; w++) {
    const int i = lane + 32 * w;
    if (i < n) S.colm[i] = (unsigned long long)colm[w];
  }
  // D0: disagreement of the re-encoded hard decision on the pivot rows = xor of the
  // columns the hard decision has set
  MT d0 = 0;
  {
    const uint32_t hw[4] = {h.x, h.y, h.z, h.w};
#pragma unroll
    for (int w = 0; w < 4; w++)
      if ((hw[w] >> lane) & 1u) d0 ^= colm[w];
    for (int off = 16; off > 0; off >>= 1) d0 ^= shfl_mask(d0, (lane ^ off));
  }
  const unsigned long long D0 = (unsigned long long)d0;
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
    const float al = fabsf(ldexpf(L[ci], sexp));
    S.wm[a2] = __float2ull_rz(fminf(floorf(al * 16777216.0f), 1099511627776.0f));
  }
  // weights of the pivot positions, by row
  for (int r = lane; r < 64; r += 32) {
    const float al = r < M ? fabsf(ldexpf(L[S.pivcol[r]], sexp)) : 0.f;
    S.wp[r] = r < M ? __float2ull_rz(fminf(floorf(al * 16777216.0f), 1099511627776.0f)) : 0ull;
  }
  // basis columns restricted to the pivot rows
  for (int a2 = lane; a2 < K; a2 += 32) S.colbits[a2] = S.colm[S.mrb[a2]];
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
    // The pairs (x < y) in enumeration order form one flat sequence; lane l takes pairs
    // l, l + 32, l + 64, ... so every lane stays busy across the short rows of the
    // triangle.  p is the pair's position, (x, y) the pair.
    uint32_t p = uint32_t(lane);
    int x = 0, y = 1 + lane;
    while (x + 1 < K && y >= K) {  // row x holds y = x + 1 .. K - 1
      y = y - K + x + 2;
      x++;
    }
    unsigned long long wa = 0, ca = 0;
    int xa = -1;
    while (x + 1 < K) {
      if (x != xa) {
        wa = S.wm[x];
        ca = D0 ^ S.colbits[x];
        xa = x;
      }
      const unsigned long long cap = min(bound1, best.s);
      // every later pair of this lane has x' >= x, so its bound is >= wm[x] + wm[x + 1]
      if (wa + S.wm[x + 1] >= cap) break;
      const unsigned long long lb = wa + S.wm[y];
      if (lb < cap) {
        const unsigned long long s = lb + wsum(S, ca ^ S.colbits[y], nch);
        consider(best, s, uint32_t(1 + K) + p, uint32_t(x + 1) | (uint32_t(y + 1) << 8));
      }
      p += 32;
      y += 32;
      while (x + 1 < K && y >= K) {
        y = y - K + x + 2;
        x++;
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
  if (lane < M && ((D >> lane) & 1ull)) setb(flip, S.pivcol[lane]);
  if (lane + 32 < M && ((D >> (lane + 32)) & 1ull)) setb(flip, S.pivcol[lane + 32]);
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

// Dispatch on the row count: 32-bit row masks when M <= 32.  The frame's input values
// are L[i] 2^sexp (ldexpf: exact while the result stays in the normal range).
__device__ __forceinline__ void osd_one_frame(OsdSmem &S, int n, int K, int M, const uint64_t *cols,
                                              const float *L, int order, uint64_t *hard, uint8_t *flag,
                                              int sexp = 0) {
  if (M <= 32)
    osd_one_frame_t<uint32_t>(S, n, K, M, cols, L, order, hard, flag, sexp);
  else
    osd_one_frame_t<unsigned long long>(S, n, K, M, cols, L, order, hard, flag, sexp);
}

// Exponent e that puts max_i |L_i| 2^e in [2^15, 2^16) (e = 16 - frexp exponent of the
// maximum; 16 when every value is zero), computed by the whole warp.
__device__ __forceinline__ int osd_input_exponent(const float *L, int n) {
  float mx = 0.0f;
  for (int i = int(lane_id()); i < n; i += 32) mx = fmaxf(mx, fabsf(L[i]));
  for (int off = 16; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(kFull, mx, off));
  int ex = 0;
  frexpf(mx, &ex);
  return 16 - ex;
}

}  // namespace bchlib
