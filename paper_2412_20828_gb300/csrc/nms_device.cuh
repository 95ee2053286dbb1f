// Device code of the normalized min-sum decoders, shared by the precompiled kernels
// (nvcc) and the kernels compiled at run time for one code (NVRTC).
//
// Enhanced NMS (arXiv 2412.20828, Algorithm 1, reading A).  Design:
//  * one thread owns one frame; a frame's state lives in shared memory laid out
//    [variable][thread], so every access of a warp hits 32 distinct banks whatever the
//    per-frame permutation is;
//  * the automorphism pi(i) = 2^j i + s is applied on the fly: pi^-1(u) =
//    rotr_m(u, j) + s' mod n, and rotr_m(u, j) is one bfe on the column code
//    d(u) = u | u << m;
//  * check rows keep min1 / min2 / sign product in registers and add their
//    check-to-variable values straight into an accumulator (reading A keeps no
//    per-edge messages);
//  * persistent warps: a lane whose frame stops (zero syndrome or I_m) writes its
//    outputs and pulls the next frame from a global queue (warp-aggregated atomic), so
//    early stopping turns into throughput instead of idle lanes.
#pragma once
#ifndef __CUDACC_RTC__
#include <cuda_fp16.h>
#include <stdint.h>

#include <cfloat>

#include "bch_devtypes.h"
#endif

namespace bchlib {

constexpr uint32_t kSign = 0x80000000u;
constexpr unsigned kFull = 0xffffffffu;

// m-bit field of x starting at bit `pos` (PTX bfe).
__device__ __forceinline__ uint32_t bfe32(uint32_t x, uint32_t pos, uint32_t len) {
  uint32_t r;
  asm("bfe.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(x), "r"(pos), "r"(len));
  return r;
}

// A packed automorphism s | j << 8 of frame f as the kernels take it.  Checked builds
// accept only the group's elements (s < n, j < m: pi(i) = 2^j i + s mod n, Sec. III-B)
// and replace any other value by the identity after recording it in the check word
// (flag, count, smallest frame), so that no index derived from it leaves [0, n).
__device__ __forceinline__ uint32_t checked_auto(uint32_t v, uint32_t n, uint32_t m,
                                                 unsigned *check, int f) {
#ifdef BCH_CHECKED
  if ((v & 0xffu) >= n || (v >> 8) >= m) {
    if (check) {
      atomicOr(check, kCheckAutomorphism);
      atomicAdd(check + 1, 1u);
      atomicMin(check + 2, unsigned(f));
    }
    return 0u;
  }
#endif
  return v;
}

// (a + b) mod n for a, b in [0, n): min(a + b, a + b - n) in unsigned arithmetic.
__device__ __forceinline__ uint32_t addmod(uint32_t a, uint32_t b, uint32_t n) {
  uint32_t x = a + b;
  return __viaddmin_u32(x, 0u - n, x);
}

__device__ __forceinline__ float flip_sign(float mag, uint32_t sign_src) {
  return __uint_as_float(__float_as_uint(mag) ^ (sign_src & kSign));
}

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

// Storage formats of y.  Accumulators are FP32 (FP32 / FP16) or int32 (INT8).
enum : int { kFP32 = 0, kFP16 = 1, kINT8 = 2 };

template <int MSG>
struct StoreT;
template <>
struct StoreT<kFP32> {
  using Y = float;
  using A = float;
};
template <>
struct StoreT<kFP16> {
  using Y = __half;
  using A = float;
};
template <>
struct StoreT<kINT8> {
  using Y = int8_t;
  using A = int32_t;
};

__device__ __forceinline__ float ld_y(const float *p) { return *p; }
__device__ __forceinline__ float ld_y(const __half *p) { return __half2float(*p); }
__device__ __forceinline__ int ld_y(const int8_t *p) { return int(*p); }

// A binary16 zero is stored as +0, so that the sign-bit tests of the decoder read it
// as non-negative (sgn(0) = +1), also when a tiny negative value rounded to zero.
__device__ __forceinline__ __half half_pz(__half h) {
  return __half2float(h) == 0.0f ? __float2half_rn(0.0f) : h;
}
// FP16 store: round to nearest even, saturating at +-65504.
__device__ __forceinline__ __half to_half_sat(float x) {
  x = fminf(fmaxf(x, -65504.0f), 65504.0f);
  return half_pz(__float2half_rn(x));
}
// FP16 merge: the binary16 value nearest to num / P (num = P y + sum of c2v), ties
// to even, saturating at +-65504, with num exact.  The correctly rounded FP32 quotient
// q leaves an exactly representable remainder r = num - q P (one FMA), whose sign says
// on which side of q the exact quotient lies; q rounded to odd on that information and
// then rounded once to binary16 is the exact quotient's binary16 rounding (the
// round-to-odd rule of the check-to-variable roundings below: FP32 keeps at least 13
// bits beyond binary16's 11).  One conversion.
__device__ __forceinline__ __half half_of_quotient(float num, float P) {
  const float q = __fdiv_rn(num, P);
  const float r = __fmaf_rn(-q, P, num);
  uint32_t b = __float_as_uint(q);
  if (r != 0.0f) {
    // the exact quotient q + r / P is nearer zero than q iff r and q differ in sign
    if ((__float_as_uint(r) ^ b) & kSign) b -= 1u;
    b |= 1u;
  }
  const float ro = fminf(fmaxf(__uint_as_float(b), -65504.0f), 65504.0f);
  return half_pz(__float2half_rn(ro));
}

// Check-to-variable magnitudes of the reduced formats, rounded once from the exact
// product alpha * m without FP64 arithmetic (which runs at a small fraction of the FP32
// rate): hi = fl(alpha m) and lo = fma(alpha, m, -hi) = alpha m - hi exactly (the
// error-free product).  The product rounded to odd in FP32 -- an inexact hi (lo != 0)
// replaced by its FP32 neighbour toward zero with the last bit set; hi is on the far
// side of the exact product iff lo has the opposite sign -- rounded once more to the
// target format equals the exact product rounded to that format, as long as FP32 keeps
// at least two bits beyond the target's precision (Boldo and Melquiond, "Emulation of
// FMA and correctly rounded sums: proved algorithms using rounding to odd", IEEE
// Trans. Computers 57(4), 2008).  One conversion does the final rounding.
// INT8: rne(alpha m) for an integer m, as an int; exact while |alpha m| < 2^22 (two
// bits below the integer point; the 8-bit forms' products stay below 2^15).
__device__ __forceinline__ int rne_product(float alpha, int m) {
  const float b = float(m);
  const float hi = alpha * b, lo = __fmaf_rn(alpha, b, -hi);
  uint32_t u = __float_as_uint(hi);
  if (lo != 0.0f) {
    if ((__float_as_uint(lo) ^ u) & kSign) u -= 1u;
    u |= 1u;
  }
  return __float2int_rn(__uint_as_float(u));
}
// FP16: the binary16 value nearest to alpha m (ties to even, saturating at +-65504),
// returned as a float; FP32 keeps at least 13 bits beyond binary16's 11 (more in
// binary16's subnormal range).  One conversion instead of three keeps the per-row code
// of the row-specialised kernels short.
__device__ __forceinline__ float half_product(float alpha, float m) {
  const float hi = alpha * m, lo = __fmaf_rn(alpha, m, -hi);
  uint32_t b = __float_as_uint(hi);
  if (lo != 0.0f) {
    // hi is on the far side of the exact product iff lo has the opposite sign; hi is
    // not zero here (a product that rounds to zero leaves lo = 0 too: the FMA rounds
    // the same product)
    if ((__float_as_uint(lo) ^ b) & kSign) b -= 1u;
    b |= 1u;
  }
  const float ro = fminf(fmaxf(__uint_as_float(b), -65504.0f), 65504.0f);
  return __half2float(__float2half_rn(ro));
}

// INT8 store: rne, saturating at +-31 (LSB = 1/4 of an LLR unit).
__device__ __forceinline__ int8_t to_q(float x) {
  int q = __float2int_rn(x);
  q = max(-31, min(31, q));
  return int8_t(q);
}

// 8-bit form with qfrac fractional c2v bits: the merged value of a position is the
// exact numerator N = P 2^qfrac q + sum (an integer below 2^24, so exact in FP32); the
// stored value is clamp(rne(N / (d 2^k)), +-31), d = P 2^qfrac, after k rescale halvings.
// The fractional bits in force: a compile-time constant in kernels compiled for one
// value (the run-time specialised ones define BCH_JIT_QFRAC), else the argument.
#ifdef BCH_JIT_QFRAC
#define BCH_QFRAC(a) (BCH_JIT_QFRAC)
#else
#define BCH_QFRAC(a) ((a).qfrac)
#endif
__device__ __forceinline__ float int8_numerator(int q, int sum, int d) { return float(q * d + sum); }
// ... and with the rescale on, its input is quantised after the power of two 2^-k0 that
// keeps max |4x| <= 31 (k0 starts the frame's exponent), so that strong inputs are not
// clipped at the 8-bit range.
__device__ __forceinline__ int int8_input_shift(const float *src, int n) {
  float mx = 0.0f;
  for (int i = 0; i < n; i++) mx = fmaxf(mx, fabsf(4.0f * src[i]));
  int k = 0;
  float lim = 31.0f;
  while (mx > lim && k < 60) {
    lim *= 2.0f;
    k++;
  }
  return k;
}
// exact integer form (large k only), kept out of line
static __device__ __noinline__ int int8_quotient_exact(float N, int k, int d) {
  if (k >= 40) return 0;
  const long long D = (long long)d << k, n = (long long)N;
  long long q = n / D, r = n % D;
  if (r < 0) {
    r += D;
    q -= 1;
  }
  if (2 * r > D || (2 * r == D && (q & 1))) q += 1;
  return int(q > 31 ? 31 : (q < -31 ? -31 : q));
}
__device__ __forceinline__ int8_t int8_store_quotient(float N, int k, int d) {
  // A quotient that is not a half-integer lies at least 1 / (2 d 2^k) from one, and the
  // correctly rounded FP32 quotient errs by at most 2^-20 below 32 (larger ones clamp
  // to +-31 either way): while d 2^k < 2^19 rounding it gives the exact quotient's rne.
  if (k < 12 && (d << k) < (1 << 19)) return to_q(__fdiv_rn(N, float(d << k)));
  return int8_t(int8_quotient_exact(N, k, d));
}

// Shared-memory carve-up common to the NMS kernels.
struct GroupDesc {
  int w, rows, off, pad;
};
struct SmemTables {
  uint16_t *codes;
  uint4 *rowmask;
  float *alpha;
  GroupDesc *grp;
  unsigned char *state;
};

// ---------------------------------------------------------------- row processing
// Processes `nrows` check rows of weight w (w <= WB) for one automorphism.
template <int MSG, int WB>
__device__ __forceinline__ void enh_rows(const uint16_t *__restrict__ codes, int nrows, int w,
                                      int w4, typename StoreT<MSG>::Y *__restrict__ y,
                                      typename StoreT<MSG>::A *__restrict__ acc, uint32_t jr,
                                      uint32_t sp, uint32_t n, uint32_t m, uint32_t stride,
                                      float alpha) {
  using A = typename StoreT<MSG>::A;
  for (int r = 0; r < nrows; r++) {
    const uint16_t *c = codes + r * w4;
    uint32_t ix[WB];
    if constexpr (MSG == kINT8) {
      int z[WB];
      int m1 = 1 << 20, m2 = 1 << 20;
      uint32_t sg = 0;
#pragma unroll
      for (int e = 0; e < WB; e += 4) {
        if (e < w) {
          const uint2 q = *reinterpret_cast<const uint2 *>(c + e);
#pragma unroll
          for (int h = 0; h < 4; h++) {
            if (e + h < w) {
              const uint32_t word = h < 2 ? q.x : q.y;
              const uint32_t rr = bfe32(word, jr + ((h & 1) ? 16u : 0u), m);
              const uint32_t i = addmod(rr, sp, n);
              ix[e + h] = i * stride;
              const int v = ld_y(y + ix[e + h]);
              z[e + h] = v;
              const int av = abs(v);
              m2 = min(m2, max(m1, av));
              m1 = min(m1, av);
              sg ^= uint32_t(v);
            }
          }
        }
      }
      // c2v magnitudes are integers: rne(alpha * min) of the exact product
      const int c1 = rne_product(alpha, m1);
      const int c2 = rne_product(alpha, m2);
      const int s1 = (sg & kSign) ? -c1 : c1;
      const int s2 = (sg & kSign) ? -c2 : c2;
      A o[WB];
#pragma unroll
      for (int e = 0; e < WB; e++)
        if (e < w) o[e] = acc[ix[e]];
#pragma unroll
      for (int e = 0; e < WB; e++)
        if (e < w) {
          const int mag = (abs(z[e]) == m1) ? s2 : s1;
          o[e] += (z[e] < 0) ? -mag : mag;
        }
#pragma unroll
      for (int e = 0; e < WB; e++)
        if (e < w) acc[ix[e]] = o[e];
    } else {
      float z[WB];
      float m1 = FLT_MAX, m2 = FLT_MAX;
      uint32_t sg = 0;
#pragma unroll
      for (int e = 0; e < WB; e += 4) {
        if (e < w) {
          const uint2 q = *reinterpret_cast<const uint2 *>(c + e);
#pragma unroll
          for (int h = 0; h < 4; h++) {
            if (e + h < w) {
              const uint32_t word = h < 2 ? q.x : q.y;
              const uint32_t rr = bfe32(word, jr + ((h & 1) ? 16u : 0u), m);
              const uint32_t i = addmod(rr, sp, n);
              ix[e + h] = i * stride;
              const float v = ld_y(y + ix[e + h]);
              z[e + h] = v;
              const float av = fabsf(v);
              m2 = fminf(m2, fmaxf(m1, av));
              m1 = fminf(m1, av);
              sg ^= __float_as_uint(v);
            }
          }
        }
      }
      float v1, v2;
      if constexpr (MSG == kFP16) {
        // messages are stored in binary16: alpha * min rounded once from the exact
        // product
        v1 = flip_sign(half_product(alpha, m1), sg);
        v2 = flip_sign(half_product(alpha, m2), sg);
      } else {
        v1 = flip_sign(alpha * m1, sg);
        v2 = flip_sign(alpha * m2, sg);
      }
      float o[WB];
#pragma unroll
      for (int e = 0; e < WB; e++)
        if (e < w) o[e] = acc[ix[e]];
#pragma unroll
      for (int e = 0; e < WB; e++)
        if (e < w) {
          const float mag = (fabsf(z[e]) == m1) ? v2 : v1;
          o[e] += flip_sign(mag, __float_as_uint(z[e]));
        }
#pragma unroll
      for (int e = 0; e < WB; e++)
        if (e < w) acc[ix[e]] = o[e];
    }
  }
}

template <int MSG, int WB>
__device__ __forceinline__ void enh_copy(const SmemTables &tb, int n_groups, uint32_t n, uint32_t m,
                                         typename StoreT<MSG>::Y *y, typename StoreT<MSG>::A *acc,
                                         uint32_t jr, uint32_t sp, uint32_t stride, float alpha) {
  for (int g = 0; g < n_groups; g++) {
    const GroupDesc gd = tb.grp[g];
    const int w = gd.w;
    enh_rows<MSG, WB>(tb.codes + gd.off, gd.rows, w, (w + 3) & ~3, y, acc, jr, sp, n, m, stride, alpha);
  }
}

__device__ __forceinline__ SmemTables load_tables(const NmsArgs &a, unsigned char *smem,
                                                  int code_words) {
  SmemTables t;
  t.codes = reinterpret_cast<uint16_t *>(smem);
  unsigned char *p = smem + ((size_t(code_words) * 2 + 15) & ~size_t(15));
  t.rowmask = reinterpret_cast<uint4 *>(p);
  p += size_t(a.dc.rows) * 16;
  t.alpha = reinterpret_cast<float *>(p);
  p += 32 * 4;
  t.grp = reinterpret_cast<GroupDesc *>(p);
  p += kMaxGroups * sizeof(GroupDesc);
  t.state = p;
  const uint32_t *src = reinterpret_cast<const uint32_t *>(a.dc.codes);
  uint32_t *dst = reinterpret_cast<uint32_t *>(t.codes);
  for (int i = threadIdx.x; i < code_words / 2; i += blockDim.x) dst[i] = src[i];
  const uint4 *rm = reinterpret_cast<const uint4 *>(a.dc.rowmask);
  for (int i = threadIdx.x; i < a.dc.rows; i += blockDim.x) t.rowmask[i] = rm[i];
  if (threadIdx.x == 0) {
#pragma unroll
    for (int i = 0; i < 32; i++) t.alpha[i] = a.alpha[i];
#pragma unroll
    for (int g = 0; g < kMaxGroups; g++) {
      GroupDesc d;
      d.w = a.dc.group_w[g];
      d.rows = a.dc.group_rows[g];
      d.off = a.dc.group_off[g];
      d.pad = 0;
      t.grp[g] = d;
    }
  }
  __syncthreads();
  return t;
}

// Syndrome of the hard decision cb (bit i = [y_i < 0]) against the packed rows:
// nonzero iff some row has odd overlap.
template <int NW>
__device__ __forceinline__ uint32_t syndrome_nonzero(const uint4 *rowmask, int rows,
                                                     const uint32_t (&cb)[NW]) {
  uint32_t nz = 0;
  for (int r = 0; r < rows; r++) {
    const uint4 rm = rowmask[r];
    uint32_t x = rm.x & cb[0];
    if constexpr (NW > 1) x ^= rm.y & cb[1];
    if constexpr (NW > 2) x ^= (rm.z & cb[2]) ^ (rm.w & cb[3]);
    nz |= __popc(x) & 1u;
  }
  return nz;
}

template <int NW>
__device__ __forceinline__ void write_hard(uint64_t *hard, int f, const uint32_t (&cb)[NW]) {
  constexpr int W64 = (NW + 1) / 2;
  uint64_t *h = hard + size_t(f) * W64;
  h[0] = uint64_t(cb[0]) | (NW > 1 ? uint64_t(cb[NW > 1 ? 1 : 0]) << 32 : 0);
  if constexpr (NW > 2) h[1] = uint64_t(cb[2]) | (uint64_t(cb[3]) << 32);
}

// Warp-aggregated pull from the frame queue: lanes with `need` get consecutive
// frame indices (or -1 once the queue is exhausted).
__device__ __forceinline__ int pull_frame(unsigned *queue, bool need, int F) {
  const unsigned want = __ballot_sync(kFull, need);
  if (!want) return -1;
  const unsigned lane = lane_id();
  const unsigned leader = __ffs(want) - 1;
  unsigned base = 0;
  if (lane == leader) base = atomicAdd(queue, unsigned(__popc(want)));
  base = __shfl_sync(kFull, base, leader);
  if (!need) return -1;
  const unsigned my = base + unsigned(__popc(want & ((1u << lane) - 1u)));
  return my < unsigned(F) ? int(my) : -1;
}

// ---------------------------------------------------------------- persistent loop
// The persistent frame loop shared by the precompiled and the run-time compiled
// kernels; `copy` processes one automorphism of one frame (check pass + accumulate).
// Per-thread shared columns (stride = block size): ctx[P], acc[n], y[n], then
// Copy::kScratch words of scratch for the functor.  TPBC: compile-time block size (0 =
// blockDim.x).  LOCKSTEP: the block's warps start every iteration together (a barrier
// per iteration, and one per automorphism copy unless the run-time specialised kernel
// defines BCH_JIT_NO_COPY_BARRIER) and lanes without a frame run the copies on their
// stale columns, so all warps of the block stream through the same code -- for long
// straight-line copy code this keeps the instruction cache warm.
template <int MSG, int NW, bool LOCKSTEP, int TPBC, class Copy>
__device__ __forceinline__ void nms_persistent(const NmsArgs &a, unsigned char *smem, const Copy &copy) {
  using Y = typename StoreT<MSG>::Y;
  using A = typename StoreT<MSG>::A;
  const int TPB = TPBC ? TPBC : int(blockDim.x);
  const int kShift = TPB;  // column stride (elements)
  const int code_words = a.dc.group_off[a.dc.n_groups];
  SmemTables tb = load_tables(a, smem, code_words);
  const int n = a.dc.n;
  const uint32_t m = uint32_t(a.dc.m);
  const int n_groups = a.dc.n_groups;
  const int tid = threadIdx.x;
  // per-thread columns: ctx[P], y[n], acc[n]
  uint32_t *ctx_s = reinterpret_cast<uint32_t *>(tb.state);
  A *acc_s = reinterpret_cast<A *>(tb.state + size_t(a.P) * TPB * 4);
  Y *y_s = reinterpret_cast<Y *>(tb.state + size_t(a.P) * TPB * 4 + size_t(n) * TPB * sizeof(A));
  Y *y = y_s + tid;
  unsigned char *scr_s = tb.state + size_t(a.P) * TPB * 4 + size_t(n) * TPB * (sizeof(A) + sizeof(Y));
  scr_s = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(scr_s) + 15) & ~uintptr_t(15));
  A *scratch = reinterpret_cast<A *>(scr_s) + tid;
  A *acc = acc_s + tid;
  uint32_t *ctx = ctx_s + tid;
  const float invP = 1.0f / float(a.P);
  const bool vec = ((a.ld & 3) == 0) && ((reinterpret_cast<uintptr_t>(a.llr) & 15) == 0);

  int f = -1, t = 0, escale = 0;
  bool need = true;
  for (;;) {
    const int got = pull_frame(a.queue, need, a.F);
    if (need) {
      need = false;
      f = got;
      if (f >= 0) {
        t = 0;
        escale = 0;
        const float *src = a.llr + size_t(f) * a.ld;
        float s4 = 4.0f;  // INT8 input scale: 4 (LSB 1/4), times 2^-k0 (see int8_input_shift)
        if constexpr (MSG == kINT8)
          if (BCH_QFRAC(a) && a.rescale) {
            escale = int8_input_shift(src, n);
            s4 = ldexpf(4.0f, -escale);
          }
        for (int i = 0; i < n; i += 4) {
          float4 v;
          if (vec) {
            v = __ldg(reinterpret_cast<const float4 *>(src + i));
          } else {
            v.x = src[i];
            v.y = i + 1 < n ? src[i + 1] : 0.f;
            v.z = i + 2 < n ? src[i + 2] : 0.f;
            v.w = i + 3 < n ? src[i + 3] : 0.f;
          }
          const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
          for (int h = 0; h < 4; h++) {
            if (i + h < n) {
              const float x = vv[h] + 0.0f;  // -0 -> +0: sgn(0) = +1
              if constexpr (MSG == kFP32) y[(i + h) * kShift] = x;
              if constexpr (MSG == kFP16) y[(i + h) * kShift] = to_half_sat(x);
              if constexpr (MSG == kINT8) y[(i + h) * kShift] = to_q(s4 * x);
              acc[(i + h) * kShift] = A(0);
              if (a.ckpt) a.ckpt[size_t(f) * a.ld + i + h] = x;
            }
          }
        }
        for (int p = 0; p < a.P; p++) {
          const uint32_t v = checked_auto(a.autos[size_t(f) * a.P + p], uint32_t(n), uint32_t(m), a.check, f);
          const uint32_t s = v & 0xffu, j = v >> 8;
          // pi^-1(u) = rotr_m(u, j) + s' with s' = -rotr_m(s, j) mod n
          const uint32_t rs = j ? (((s >> j) | (s << (m - j))) & uint32_t(n)) : s;
          const uint32_t sp = rs ? uint32_t(n) - rs : 0u;
          ctx[p * kShift] = j | (sp << 8);
        }
      }
    }
    if constexpr (LOCKSTEP) {
      if (!__syncthreads_or(f >= 0)) break;
    } else {
      if (!__any_sync(kFull, f >= 0)) break;
      if (f < 0) continue;
    }

    const float alpha = tb.alpha[f >= 0 ? t : 0];
    for (int p = 0; p < a.P; p++) {
#ifndef BCH_JIT_NO_COPY_BARRIER
      if constexpr (LOCKSTEP) __syncthreads();
#endif
      const uint32_t cx = f >= 0 ? ctx[p * kShift] : 0u;
      copy(tb, n_groups, uint32_t(n), m, y, acc, scratch, cx & 0xffu, cx >> 8, uint32_t(kShift), alpha);
    }
    // merge (FP32), hard decision, re-store
    uint32_t cb[NW];
#pragma unroll
    for (int w = 0; w < NW; w++) cb[w] = 0;
    if constexpr (MSG == kFP32) {
      float mx = 0.0f;
#pragma unroll
      for (int i = 0; i < NW * 32; i++) {
        if (i < n) {
          const float yn = __fmaf_rn(acc[i * kShift], invP, y[i * kShift]);
          y[i * kShift] = yn;
          acc[i * kShift] = 0.0f;
          cb[i >> 5] |= (__float_as_uint(yn) >> 31) << (i & 31);
          mx = fmaxf(mx, fabsf(yn));
        }
      }
      // y grows about tenfold per iteration; past 2^100 the frame is scaled by 2^-64
      // (exact, and min-sum is scale invariant) so that long decodes of high-degree
      // codes cannot overflow FP32.  Not in training, whose checkpoints are in LLR units.
      if (mx > 0x1p100f && !a.ckpt && f >= 0) {
#pragma unroll
        for (int i = 0; i < NW * 32; i++)
          if (i < n) y[i * kShift] *= 0x1p-64f;
        escale += 64;
      }
    } else {
      // pass 1: the merged value into the accumulator slot, track the magnitude.
      // INT8: q + (integer sum) / P with a correctly rounded division (a .5 tie stays
      // a tie).  FP16: the numerator num = P y + sum of c2v, exact whenever the FP32
      // accumulation of binary16 values was; y_new = num / P is rounded once, below.
      const float fP = float(a.P);
      float mx = 0.0f;
#pragma unroll
      for (int i = 0; i < NW * 32; i++) {
        if (i < n) {
          float yn;
          if constexpr (MSG == kINT8)
            yn = BCH_QFRAC(a) ? int8_numerator(ld_y(y + (i * kShift)), acc[i * kShift], a.P << BCH_QFRAC(a))
                         : float(ld_y(y + (i * kShift))) + __fdiv_rn(float(acc[i * kShift]), fP);
          else
            yn = __fmaf_rn(ld_y(y + (i * kShift)), fP, acc[i * kShift]);
          cb[i >> 5] |= (__float_as_uint(yn) >> 31) << (i & 31);
          mx = fmaxf(mx, fabsf(yn));
          reinterpret_cast<float *>(acc)[i * kShift] = yn;
        }
      }
      // optional power-of-two renormalisation (exact; min-sum is scale invariant):
      // halve while max |y_new| > lim (FP16 and fractional INT8: compared on the
      // numerators, exactly)
      float sc = 1.0f;
      int kr = 0;
      if (a.rescale) {
        const float lim = (MSG == kINT8) ? (BCH_QFRAC(a) ? 31.0f * float(a.P << BCH_QFRAC(a)) : 31.0f) : 16384.0f * fP;
        while (mx * sc > lim && kr < 126) {
          sc *= 0.5f;
          kr++;
        }
        escale += kr;
      }
#pragma unroll
      for (int i = 0; i < NW * 32; i++) {
        if (i < n) {
          const float yn = reinterpret_cast<float *>(acc)[i * kShift] * sc;
          if constexpr (MSG == kINT8)
            y[i * kShift] = BCH_QFRAC(a) ? int8_store_quotient(reinterpret_cast<float *>(acc)[i * kShift], kr,
                                                          a.P << BCH_QFRAC(a))
                                    : to_q(yn);
          else
            y[i * kShift] = half_of_quotient(yn, fP);
          acc[i * kShift] = A(0);
        }
      }
    }
    if (LOCKSTEP && f < 0) continue;
    t++;
    if (a.ckpt) {
      float *dst = a.ckpt + (size_t(t) * a.F + f) * a.ld;
      for (int i = 0; i < n; i++) dst[i] = float(ld_y(y + (i * kShift)));
    }
    const uint32_t nz = syndrome_nonzero<NW>(tb.rowmask, a.dc.rows, cb);
    if (t >= a.I || (a.early_stop && nz == 0)) {
      if (a.hard) write_hard<NW>(a.hard, f, cb);
      if (a.iters) a.iters[f] = uint8_t(t);
      if (a.flags) a.flags[f] = nz ? 0 : uint8_t(kFlagConverged);
      if (a.llr_out) {
        float *dst = a.llr_out + size_t(f) * a.ld;
        const float unit = MSG == kINT8 ? 0.25f : 1.0f;
        for (int i = 0; i < n; i++) dst[i] = ldexpf(float(ld_y(y + (i * kShift))) * unit, escale);
      }
      need = true;
    }
  }
}


// ---------------------------------------------------------------- split mapping (n = 127)
// Two warps share 32 frames: warp half h owns the variables [64h, 64h + 64) of every
// automorphism copy (its 64 values of z and of the row sums S stay in registers, as in
// the n <= 63 kernel), and of the frame's own positions for the merge.  A check row
// spans both halves: each half reduces its own columns to (min1, min2, sign parity),
// publishes that partial in shared memory, and after a block barrier combines it with
// the other half's -- min1 = min(a1, b1), min2 = min(max(a1, b1), a2, b2), parity
// a ^ b -- before its output pass.  Rows go in chunks of R with one barrier per
// chunk; partials alternate between two buffers, so the first pass of chunk c + 1 can
// run before the other half has read chunk c.  Row order and every addition are those
// of the one-thread-per-frame kernel, so the results are bit-identical to it.
//
// The barrier inside a copy is a named barrier over the whole block, reached by the two
// halves at different code locations (each half runs its own straight-line copy); both
// copies are emitted from one chunk list, so they pass the same number of barriers.
__device__ __forceinline__ void bar_block(unsigned nthreads) {
  asm volatile("bar.sync 1, %0;" ::"r"(nthreads) : "memory");
}

// Per-block shared-memory layout of the split kernel: tables, then (per frame slot,
// Fs = 32 G slots, element [x][slot] at x * Fs + slot) ctx[2][P], acc[n], y[n],
// partials[2 buffers][R rows][2 halves] (float2), the merge exchange and the frame
// hand-off aliasing the partial buffers (unused between the copies).
template <int MSG>
struct SplitSmem {
  static __host__ __device__ size_t state_bytes(int n, int P, int G, int R) {
    const size_t Fs = size_t(32) * G;
    const size_t ya = sizeof(typename StoreT<MSG>::Y);
    size_t b = Fs * 4 * 2 * size_t(P);                    // ctx, one copy per half
    b += Fs * 4 * size_t(n);                              // acc (FP32 / int32)
    b += (Fs * ya * size_t(n) + 15) & ~size_t(15);        // y
    b += Fs * 8 * 2 * 2 * size_t(R);                      // partials
    return b;
  }
};

template <int MSG, int G, class Copy>
__device__ __forceinline__ void nms_split_persistent(const NmsArgs &a, unsigned char *smem, const Copy &copy,
                                                     int nchunk, int R) {
  using Y = typename StoreT<MSG>::Y;
  using A = typename StoreT<MSG>::A;
  constexpr int Fs = 32 * G, TPB = 64 * G;
  const int code_words = a.dc.group_off[a.dc.n_groups];
  SmemTables tb = load_tables(a, smem, code_words);
  const int n = a.dc.n;
  const uint32_t m = uint32_t(a.dc.m);
  const int warp = int(threadIdx.x >> 5), lane = int(lane_id());
  // Warp w issues from scheduler w % 4.  Half 0 takes the warps with (w >> 1) even,
  // half 1 the others, so each scheduler runs warps of one half only -- one stream of
  // straight-line copy code per scheduler, shared by its lockstep warps.
  const int h = (warp >> 1) & 1;                               // half of the variables
  const int s = ((warp & 1) + ((warp >> 2) << 1)) * 32 + lane;  // frame slot (G = 4)
  static_assert(G == 4, "the warp-to-half map assumes 8 warps per block");
  const int i0 = h * 64, i1 = h ? n : (n < 64 ? n : 64);
  uint32_t *ctx = reinterpret_cast<uint32_t *>(tb.state) + size_t(h) * a.P * Fs + s;
  A *acc_s = reinterpret_cast<A *>(tb.state + size_t(Fs) * 4 * 2 * a.P);
  Y *y_s = reinterpret_cast<Y *>(reinterpret_cast<unsigned char *>(acc_s) + size_t(Fs) * 4 * n);
  unsigned char *pbase = reinterpret_cast<unsigned char *>(y_s) +
                         ((size_t(Fs) * sizeof(Y) * n + 15) & ~size_t(15));
  float2 *part = reinterpret_cast<float2 *>(pbase);
  uint4 *xch = reinterpret_cast<uint4 *>(pbase);                       // [2][Fs], merge exchange
  int *fslot = reinterpret_cast<int *>(pbase + size_t(Fs) * 16 * 2);   // [Fs], frame hand-off
  A *acc = acc_s + s;
  Y *y = y_s + s;
  const float invP = 1.0f / float(a.P);
  const bool vec = ((a.ld & 3) == 0) && ((reinterpret_cast<uintptr_t>(a.llr) & 15) == 0);
  for (int p = 0; p < a.P; p++) ctx[p * Fs] = 0u;  // idle slots run copies on valid maps

  int f = -1, t = 0, escale = 0;
  bool need = true;
  for (;;) {
    // half 0 pulls the slot's next frame and hands it to half 1
    if (h == 0) {
      const int got = pull_frame(a.queue, need, a.F);
      if (need) fslot[s] = got;
    }
    bar_block(TPB);
    if (need) {
      need = false;
      f = fslot[s];
      if (f >= 0) {
        t = 0;
        escale = 0;
        const float *src = a.llr + size_t(f) * a.ld;
        float s4 = 4.0f;  // as in the one-thread kernel; both halves scan all n inputs
        if constexpr (MSG == kINT8)
          if (BCH_QFRAC(a) && a.rescale) {
            escale = int8_input_shift(src, n);
            s4 = ldexpf(4.0f, -escale);
          }
        for (int i = i0; i < i1; i += 4) {
          float4 v;
          if (vec) {
            v = __ldg(reinterpret_cast<const float4 *>(src + i));
          } else {
            v.x = src[i];
            v.y = i + 1 < n ? src[i + 1] : 0.f;
            v.z = i + 2 < n ? src[i + 2] : 0.f;
            v.w = i + 3 < n ? src[i + 3] : 0.f;
          }
          const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
          for (int q = 0; q < 4; q++) {
            if (i + q < i1) {
              const float x = vv[q] + 0.0f;  // -0 -> +0: sgn(0) = +1
              if constexpr (MSG == kFP32) y[(i + q) * Fs] = x;
              if constexpr (MSG == kFP16) y[(i + q) * Fs] = to_half_sat(x);
              if constexpr (MSG == kINT8) y[(i + q) * Fs] = to_q(s4 * x);
              acc[(i + q) * Fs] = A(0);
              if (a.ckpt) a.ckpt[size_t(f) * a.ld + i + q] = x;
            }
          }
        }
        for (int p = 0; p < a.P; p++) {
          const uint32_t v = checked_auto(a.autos[size_t(f) * a.P + p], uint32_t(n), uint32_t(m), a.check, f);
          const uint32_t sh = v & 0xffu, j = v >> 8;
          const uint32_t rs = j ? (((sh >> j) | (sh << (m - j))) & uint32_t(n)) : sh;
          ctx[p * Fs] = j | ((rs ? uint32_t(n) - rs : 0u) << 8);
        }
      }
    }
    if (!__syncthreads_or(f >= 0)) break;

    const float alpha = tb.alpha[f >= 0 ? t : 0];
    for (int p = 0; p < a.P; p++) {
      const uint32_t cx = f >= 0 ? ctx[p * Fs] : 0u;
      // the partial buffers alternate across the copies' chunks too
      float2 *pa = part + (((p * nchunk) & 1) ? size_t(2) * R * Fs : 0) + s;
      float2 *pb = part + (((p * nchunk) & 1) ? 0 : size_t(2) * R * Fs) + s;
      copy(h, y, acc, pa, pb, cx & 0xffu, cx >> 8, alpha);
    }
    __syncthreads();  // every copy's accumulation is in acc

    // merge of this half's positions (FP32), its hard-decision bits and magnitude
    uint32_t cw0 = 0, cw1 = 0;
    float mx = 0.0f;
    const float fP = float(a.P);
    for (int i = i0; i < i1; i++) {
      float yn;
      if constexpr (MSG == kFP32) {
        yn = __fmaf_rn(acc[i * Fs], invP, y[i * Fs]);
        y[i * Fs] = yn;
      } else if constexpr (MSG == kINT8) {
        yn = BCH_QFRAC(a) ? int8_numerator(ld_y(y + i * Fs), acc[i * Fs], a.P << BCH_QFRAC(a))
                     : float(ld_y(y + i * Fs)) + __fdiv_rn(float(acc[i * Fs]), fP);
        reinterpret_cast<float *>(acc)[i * Fs] = yn;
      } else {
        yn = __fmaf_rn(ld_y(y + i * Fs), fP, acc[i * Fs]);
        reinterpret_cast<float *>(acc)[i * Fs] = yn;
      }
      if constexpr (MSG == kFP32) acc[i * Fs] = 0.0f;
      const uint32_t b = (__float_as_uint(yn) >> 31) << ((i - i0) & 31);
      if (i - i0 < 32) cw0 |= b; else cw1 |= b;
      mx = fmaxf(mx, fabsf(yn));
    }
    xch[h * Fs + s] = make_uint4(cw0, cw1, __float_as_uint(mx), 0u);
    __syncthreads();
    const uint4 o = xch[(1 - h) * Fs + s];
    uint32_t cb[4];
    cb[h * 2] = cw0;
    cb[h * 2 + 1] = cw1;
    cb[(1 - h) * 2] = o.x;
    cb[(1 - h) * 2 + 1] = o.y;
    mx = fmaxf(mx, __uint_as_float(o.z));
    if constexpr (MSG == kFP32) {
      // exact power-of-two renormalisation past 2^100 (as in the one-thread kernel)
      if (mx > 0x1p100f && !a.ckpt && f >= 0) {
        for (int i = i0; i < i1; i++) y[i * Fs] *= 0x1p-64f;
        escale += 64;
      }
    } else {
      float sc = 1.0f;
      int kr = 0;
      if (a.rescale) {
        const float lim = (MSG == kINT8) ? (BCH_QFRAC(a) ? 31.0f * float(a.P << BCH_QFRAC(a)) : 31.0f) : 16384.0f * fP;
        while (mx * sc > lim && kr < 126) {
          sc *= 0.5f;
          kr++;
        }
        escale += kr;
      }
      for (int i = i0; i < i1; i++) {
        const float yn = reinterpret_cast<float *>(acc)[i * Fs] * sc;
        if constexpr (MSG == kINT8)
          y[i * Fs] = BCH_QFRAC(a) ? int8_store_quotient(reinterpret_cast<float *>(acc)[i * Fs], kr, a.P << BCH_QFRAC(a))
                              : to_q(yn);
        else
          y[i * Fs] = half_of_quotient(yn, fP);
        acc[i * Fs] = A(0);
      }
    }
    if (f < 0) continue;
    t++;
    if (a.ckpt) {
      float *dst = a.ckpt + (size_t(t) * a.F + f) * a.ld;
      for (int i = i0; i < i1; i++) dst[i] = float(ld_y(y + i * Fs));
    }
    const uint32_t nz = syndrome_nonzero<4>(tb.rowmask, a.dc.rows, cb);
    if (t >= a.I || (a.early_stop && nz == 0)) {
      if (h == 0) {
        if (a.hard) write_hard<4>(a.hard, f, cb);
        if (a.iters) a.iters[f] = uint8_t(t);
        if (a.flags) a.flags[f] = nz ? 0 : uint8_t(kFlagConverged);
      }
      if (a.llr_out) {
        float *dst = a.llr_out + size_t(f) * a.ld;
        const float unit = MSG == kINT8 ? 0.25f : 1.0f;
        for (int i = i0; i < i1; i++) dst[i] = ldexpf(float(ld_y(y + i * Fs)) * unit, escale);
      }
      need = true;
    }
  }
}

// Precompiled path: rows read their column codes from shared memory.
template <int MSG, int WB>
struct GenericCopy {
  static constexpr int kScratch = 0;
  __device__ __forceinline__ void operator()(const SmemTables &tb, int n_groups, uint32_t n, uint32_t m,
                                             typename StoreT<MSG>::Y *y, typename StoreT<MSG>::A *acc,
                                             typename StoreT<MSG>::A *, uint32_t jr, uint32_t sp,
                                             uint32_t stride, float alpha) const {
    enh_copy<MSG, WB>(tb, n_groups, n, m, y, acc, jr, sp, stride, alpha);
  }
};

}  // namespace bchlib
