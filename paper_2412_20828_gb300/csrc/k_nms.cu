// Normalized min-sum decoding kernels for sm_103a.
//
// Enhanced NMS (arXiv 2412.20828, Algorithm 1, reading A) and plain flooding NMS
// (Eqs. 2-5).  Design:
//  * one thread owns one frame; a frame's state lives in shared memory laid out
//    [variable][thread], so every access of a warp hits 32 distinct banks whatever the
//    per-frame permutation is;
//  * the automorphism pi(i) = 2^j i + s is applied on the fly: pi^-1(u) =
//    rotr_m(u, j) + s' mod n, and rotr_m(u, j) is one bfe on the column code
//    d(u) = u | u << m kept in shared memory;
//  * check nodes are processed row by row with min1 / min2 / sign product in
//    registers; the check-to-variable values are added straight into the frame's
//    accumulator (no per-edge message storage: reading A keeps only y);
//  * persistent warps: a lane whose frame stops (zero syndrome or I_m) writes its
//    outputs and pulls the next frame from a global queue (warp-aggregated atomic), so
//    early stopping turns into throughput instead of idle lanes.
#include <cfloat>

#include "bch_kernels.cuh"

namespace bchlib {

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

// FP16 store: round to nearest even, saturating at +-65504.
__device__ __forceinline__ __half to_half_sat(float x) {
  x = fminf(fmaxf(x, -65504.0f), 65504.0f);
  return __float2half_rn(x);
}
// INT8 store: rne, saturating at +-31 (LSB = 1/4 of an LLR unit).
__device__ __forceinline__ int8_t to_q(float x) {
  int q = __float2int_rn(x);
  q = max(-31, min(31, q));
  return int8_t(q);
}

// ---------------------------------------------------------------- row processing
// Processes `nrows` check rows of weight w (w <= WB) for one automorphism.
template <int MSG, int WB>
__device__ __noinline__ void enh_rows(const uint16_t *__restrict__ codes, int nrows, int w,
                                      int w4, typename StoreT<MSG>::Y *__restrict__ y,
                                      typename StoreT<MSG>::A *__restrict__ acc, uint32_t jr,
                                      uint32_t sp, uint32_t n, uint32_t m, uint32_t sh,
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
              ix[e + h] = i << sh;
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
      // c2v magnitudes are integers: rne(alpha * min)
      const int c1 = __float2int_rn(alpha * float(m1));
      const int c2 = __float2int_rn(alpha * float(m2));
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
              ix[e + h] = i << sh;
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
      float v1 = flip_sign(alpha * m1, sg);
      float v2 = flip_sign(alpha * m2, sg);
      if constexpr (MSG == kFP16) {
        // messages are stored in binary16: round each c2v magnitude once
        v1 = __half2float(to_half_sat(v1));
        v2 = __half2float(to_half_sat(v2));
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

template <int MSG>
__device__ __forceinline__ void enh_copy(const NmsArgs &a, const uint16_t *codes_s,
                                         typename StoreT<MSG>::Y *y, typename StoreT<MSG>::A *acc,
                                         uint32_t jr, uint32_t sp, uint32_t sh, float alpha) {
  const uint32_t n = uint32_t(a.dc.n), m = uint32_t(a.dc.m);
  for (int g = 0; g < a.dc.n_groups; g++) {
    const int w = a.dc.group_w[g];
    const int w4 = (w + 3) & ~3;
    const uint16_t *c = codes_s + a.dc.group_off[g];
    const int nr = a.dc.group_rows[g];
    switch (w4 >> 2) {
#define BCH_CASE(K)                                                         \
  case K:                                                                   \
    enh_rows<MSG, 4 * K>(c, nr, w, w4, y, acc, jr, sp, n, m, sh, alpha);  \
    break;
      BCH_CASE(1)
      BCH_CASE(2)
      BCH_CASE(3)
      BCH_CASE(4)
      BCH_CASE(5)
      BCH_CASE(6)
      BCH_CASE(7)
      BCH_CASE(8)
      BCH_CASE(9)
      BCH_CASE(10)
      BCH_CASE(11)
      BCH_CASE(12)
#undef BCH_CASE
      default:
        break;
    }
  }
}

// Shared-memory carve-up common to the NMS kernels.
struct SmemTables {
  uint16_t *codes;
  uint4 *rowmask;
  float *alpha;
  unsigned char *state;
};

__device__ __forceinline__ SmemTables load_tables(const NmsArgs &a, unsigned char *smem,
                                                  int code_words) {
  SmemTables t;
  t.codes = reinterpret_cast<uint16_t *>(smem);
  unsigned char *p = smem + ((size_t(code_words) * 2 + 15) & ~size_t(15));
  t.rowmask = reinterpret_cast<uint4 *>(p);
  p += size_t(a.dc.rows) * 16;
  t.alpha = reinterpret_cast<float *>(p);
  p += 32 * 4;
  t.state = p;
  const uint32_t *src = reinterpret_cast<const uint32_t *>(a.dc.codes);
  uint32_t *dst = reinterpret_cast<uint32_t *>(t.codes);
  for (int i = threadIdx.x; i < code_words / 2; i += blockDim.x) dst[i] = src[i];
  const uint4 *rm = reinterpret_cast<const uint4 *>(a.dc.rowmask);
  for (int i = threadIdx.x; i < a.dc.rows; i += blockDim.x) t.rowmask[i] = rm[i];
  if (threadIdx.x < 32) t.alpha[threadIdx.x] = a.alpha[threadIdx.x];
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

// ---------------------------------------------------------------- enhanced NMS
template <int MSG, int NW, int TPB>
__global__ void __launch_bounds__(TPB) nms_enhanced_kernel(const NmsArgs a) {
  using Y = typename StoreT<MSG>::Y;
  using A = typename StoreT<MSG>::A;
  constexpr uint32_t kShift = TPB == 128 ? 7u : (TPB == 64 ? 6u : 5u);
  extern __shared__ __align__(16) unsigned char smem[];
  const int code_words = a.dc.group_off[a.dc.n_groups];
  SmemTables tb = load_tables(a, smem, code_words);
  const int n = a.dc.n;
  const uint32_t m = uint32_t(a.dc.m);
  const int tid = threadIdx.x;
  // per-thread columns: ctx[P], y[n], acc[n]
  uint32_t *ctx_s = reinterpret_cast<uint32_t *>(tb.state);
  A *acc_s = reinterpret_cast<A *>(tb.state + size_t(a.P) * TPB * 4);
  Y *y_s = reinterpret_cast<Y *>(tb.state + size_t(a.P) * TPB * 4 + size_t(n) * TPB * sizeof(A));
  Y *y = y_s + tid;
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
              if constexpr (MSG == kFP32) y[(i + h) * TPB] = x;
              if constexpr (MSG == kFP16) y[(i + h) * TPB] = to_half_sat(x);
              if constexpr (MSG == kINT8) y[(i + h) * TPB] = to_q(4.0f * x);
              acc[(i + h) * TPB] = A(0);
              if (a.ckpt) a.ckpt[size_t(f) * a.ld + i + h] = x;
            }
          }
        }
        for (int p = 0; p < a.P; p++) {
          const uint32_t v = a.autos[size_t(f) * a.P + p];
          const uint32_t s = v & 0xffu, j = v >> 8;
          // pi^-1(u) = rotr_m(u, j) + s' with s' = -rotr_m(s, j) mod n
          const uint32_t rs = j ? (((s >> j) | (s << (m - j))) & uint32_t(n)) : s;
          const uint32_t sp = rs ? uint32_t(n) - rs : 0u;
          ctx[p * TPB] = j | (sp << 8);
        }
      }
    }
    if (!__any_sync(kFull, f >= 0)) break;
    if (f < 0) continue;

    const float alpha = tb.alpha[t];
    for (int p = 0; p < a.P; p++) {
      const uint32_t cx = ctx[p * TPB];
      enh_copy<MSG>(a, tb.codes, y, acc, cx & 0xffu, cx >> 8, kShift, alpha);
    }
    // merge (FP32), hard decision, re-store
    uint32_t cb[NW];
#pragma unroll
    for (int w = 0; w < NW; w++) cb[w] = 0;
    if constexpr (MSG == kFP32) {
#pragma unroll
      for (int i = 0; i < NW * 32; i++) {
        if (i < n) {
          const float yn = __fmaf_rn(acc[i * TPB], invP, y[i * TPB]);
          y[i * TPB] = yn;
          acc[i * TPB] = 0.0f;
          cb[i >> 5] |= (__float_as_uint(yn) >> 31) << (i & 31);
        }
      }
    } else {
      // pass 1: FP32 merge into the accumulator slot, track the magnitude
      float mx = 0.0f;
#pragma unroll
      for (int i = 0; i < NW * 32; i++) {
        if (i < n) {
          float yn;
          if constexpr (MSG == kINT8)
            yn = __fmaf_rn(float(acc[i * TPB]), invP, float(ld_y(y + i * TPB)));
          else
            yn = __fmaf_rn(acc[i * TPB], invP, ld_y(y + i * TPB));
          cb[i >> 5] |= (__float_as_uint(yn) >> 31) << (i & 31);
          mx = fmaxf(mx, fabsf(yn));
          reinterpret_cast<float *>(acc)[i * TPB] = yn;
        }
      }
      // optional power-of-two renormalisation (exact; min-sum is scale invariant)
      float sc = 1.0f;
      if (a.rescale) {
        const float lim = (MSG == kINT8) ? 31.0f : 16384.0f;
        int k = 0;
        while (mx * sc > lim && k < 126) {
          sc *= 0.5f;
          k++;
        }
        escale += k;
      }
#pragma unroll
      for (int i = 0; i < NW * 32; i++) {
        if (i < n) {
          const float yn = reinterpret_cast<float *>(acc)[i * TPB] * sc;
          if constexpr (MSG == kINT8)
            y[i * TPB] = to_q(yn);
          else
            y[i * TPB] = to_half_sat(yn);
          acc[i * TPB] = A(0);
        }
      }
    }
    t++;
    if (a.ckpt) {
      float *dst = a.ckpt + (size_t(t) * a.F + f) * a.ld;
      for (int i = 0; i < n; i++) dst[i] = float(ld_y(y + i * TPB));
    }
    const uint32_t nz = syndrome_nonzero<NW>(tb.rowmask, a.dc.rows, cb);
    if (t >= a.I || (a.early_stop && nz == 0)) {
      if (a.hard) write_hard<NW>(a.hard, f, cb);
      if (a.iters) a.iters[f] = uint8_t(t);
      if (a.flags) a.flags[f] = nz ? 0 : uint8_t(BCH_FLAG_CONVERGED);
      if (a.llr_out) {
        float *dst = a.llr_out + size_t(f) * a.ld;
        float unscale = 1.0f;
        if constexpr (MSG == kINT8) unscale = 0.25f;
        for (int k = 0; k < escale; k++) unscale *= 2.0f;
        for (int i = 0; i < n; i++) dst[i] = float(ld_y(y + i * TPB)) * unscale;
      }
      need = true;
    }
  }
}

// ---------------------------------------------------------------- plain NMS
// Eqs. (2)-(5) with per-edge messages kept as a compact per-row state: alpha*min1 and
// alpha*min2 carrying the sign product, the argmin edge, and the v2c sign bits.
template <int WB>
__device__ __noinline__ void plain_rows(const uint16_t *__restrict__ codes, int row0, int nrows,
                                        int w, int w4, const float *xt, float *xn, float *rs_m1,
                                        float *rs_m2, uint32_t *rs_am, uint32_t *rs_lo,
                                        uint32_t *rs_hi, uint32_t n, uint32_t sh, float alpha) {
  for (int r = 0; r < nrows; r++) {
    const int row = row0 + r;
    const uint16_t *c = codes + r * w4;
    const int ro = row << sh;
    const float om1 = rs_m1[ro], om2 = rs_m2[ro];
    const uint32_t oam = rs_am[ro], olo = rs_lo[ro], ohi = rs_hi[ro];
    uint32_t ix[WB];
    float v[WB];
    float m1 = FLT_MAX, m2 = FLT_MAX;
    uint32_t am = 0, sg = 0, nlo = 0, nhi = 0;
#pragma unroll
    for (int e = 0; e < WB; e++) {
      if (e < w) {
        const uint32_t u = uint32_t(c[e]) & n;
        ix[e] = u << sh;
        const uint32_t sb = (e < 32) ? (olo >> e) : (ohi >> (e - 32));
        const float cold = flip_sign(uint32_t(e) == oam ? om2 : om1, sb << 31);
        const float x = xt[ix[e]] - cold;  // Eq. (2): total minus own message
        v[e] = x;
        const float ax = fabsf(x);
        if (ax < m1) am = uint32_t(e);
        m2 = fminf(m2, fmaxf(m1, ax));
        m1 = fminf(m1, ax);
        const uint32_t xs = __float_as_uint(x) >> 31;
        sg ^= xs;
        if (e < 32)
          nlo |= xs << e;
        else
          nhi |= xs << (e - 32);
      }
    }
    const float v1 = flip_sign(alpha * m1, sg << 31);
    const float v2 = flip_sign(alpha * m2, sg << 31);
    float o[WB];
#pragma unroll
    for (int e = 0; e < WB; e++)
      if (e < w) o[e] = xn[ix[e]];
#pragma unroll
    for (int e = 0; e < WB; e++)
      if (e < w) o[e] += flip_sign(uint32_t(e) == am ? v2 : v1, __float_as_uint(v[e]));
#pragma unroll
    for (int e = 0; e < WB; e++)
      if (e < w) xn[ix[e]] = o[e];
    rs_m1[ro] = v1;
    rs_m2[ro] = v2;
    rs_am[ro] = am;
    rs_lo[ro] = nlo;
    rs_hi[ro] = nhi;
  }
}

template <int NW, int TPB>
__global__ void __launch_bounds__(TPB) nms_plain_kernel(const NmsArgs a) {
  constexpr uint32_t kShift = TPB == 128 ? 7u : (TPB == 64 ? 6u : 5u);
  extern __shared__ __align__(16) unsigned char smem[];
  const int code_words = a.dc.group_off[a.dc.n_groups];
  SmemTables tb = load_tables(a, smem, code_words);
  const int n = a.dc.n, R = a.dc.rows;
  const int tid = threadIdx.x;
  float *L = reinterpret_cast<float *>(tb.state) + tid;
  float *xt = L + size_t(n) * TPB;
  float *xn = xt + size_t(n) * TPB;
  float *rs_m1 = xn + size_t(n) * TPB;
  float *rs_m2 = rs_m1 + size_t(R) * TPB;
  uint32_t *rs_am = reinterpret_cast<uint32_t *>(rs_m2 + size_t(R) * TPB);
  uint32_t *rs_lo = rs_am + size_t(R) * TPB;
  uint32_t *rs_hi = rs_lo + size_t(R) * TPB;
  int f = -1, t = 0;
  bool need = true;
  for (;;) {
    const int got = pull_frame(a.queue, need, a.F);
    if (need) {
      need = false;
      f = got;
      if (f >= 0) {
        t = 0;
        const float *src = a.llr + size_t(f) * a.ld;
        for (int i = 0; i < n; i++) {
          const float x = src[i] + 0.0f;
          L[i * TPB] = x;
          xt[i * TPB] = x;
        }
        for (int r = 0; r < R; r++) {
          rs_m1[r * TPB] = 0.f;
          rs_m2[r * TPB] = 0.f;
          rs_am[r * TPB] = 0;
          rs_lo[r * TPB] = 0;
          rs_hi[r * TPB] = 0;
        }
      }
    }
    if (!__any_sync(kFull, f >= 0)) break;
    if (f < 0) continue;
    const float alpha = tb.alpha[t];
    for (int i = 0; i < n; i++) xn[i * TPB] = L[i * TPB];
    int row0 = 0;
    for (int g = 0; g < a.dc.n_groups; g++) {
      const int w = a.dc.group_w[g];
      const int w4 = (w + 3) & ~3;
      const uint16_t *c = tb.codes + a.dc.group_off[g];
      const int nr = a.dc.group_rows[g];
      switch (w4 >> 2) {
#define BCH_PCASE(K)                                                                             \
  case K:                                                                                        \
    plain_rows<4 * K>(c, row0, nr, w, w4, xt, xn, rs_m1, rs_m2, rs_am, rs_lo, rs_hi,            \
                      uint32_t((1u << a.dc.m) - 1u), kShift, alpha);                            \
    break;
        BCH_PCASE(1)
        BCH_PCASE(2)
        BCH_PCASE(3)
        BCH_PCASE(4)
        BCH_PCASE(5)
        BCH_PCASE(6)
        BCH_PCASE(7)
        BCH_PCASE(8)
        BCH_PCASE(9)
        BCH_PCASE(10)
        BCH_PCASE(11)
        BCH_PCASE(12)
#undef BCH_PCASE
        default:
          break;
      }
      row0 += nr;
    }
    uint32_t cb[NW];
#pragma unroll
    for (int w = 0; w < NW; w++) cb[w] = 0;
#pragma unroll
    for (int i = 0; i < NW * 32; i++) {
      if (i < n) {
        const float x = xn[i * TPB];
        xt[i * TPB] = x;  // Eq. (4) output is next iteration's total
        cb[i >> 5] |= (__float_as_uint(x) >> 31) << (i & 31);
      }
    }
    t++;
    const uint32_t nz = syndrome_nonzero<NW>(tb.rowmask, R, cb);
    if (t >= a.I || (a.early_stop && nz == 0)) {
      if (a.hard) write_hard<NW>(a.hard, f, cb);
      if (a.iters) a.iters[f] = uint8_t(t);
      if (a.flags) a.flags[f] = nz ? 0 : uint8_t(BCH_FLAG_CONVERGED);
      if (a.llr_out) {
        float *dst = a.llr_out + size_t(f) * a.ld;
        for (int i = 0; i < n; i++) dst[i] = xt[i * TPB];
      }
      need = true;
    }
  }
}

// ---------------------------------------------------------------- launchers
size_t nms_table_bytes(const DevCode &dc) {
  const int code_words = dc.group_off[dc.n_groups];
  return ((size_t(code_words) * 2 + 15) & ~size_t(15)) + size_t(dc.rows) * 16 + 32 * 4;
}

static size_t state_bytes_per_thread(const DevCode &dc, int P, int msg) {
  if (P == 0) return size_t(3 * dc.n + 5 * dc.rows) * 4;
  const size_t ys = msg == kFP32 ? 4 : (msg == kFP16 ? 2 : 1);
  return size_t(P) * 4 + size_t(dc.n) * 4 + size_t(dc.n) * ys;
}

template <typename K>
static cudaError_t launch_persistent(K kernel, int tpb, size_t smem, const NmsArgs &a,
                                     cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       int(smem));
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, tpb, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  long long blocks = (long long)sms * per_sm;
  const long long need = (a.F + tpb - 1) / tpb;
  if (blocks > need) blocks = need;
  if (blocks < 1) blocks = 1;
  kernel<<<unsigned(blocks), tpb, smem, st>>>(a);
  return cudaGetLastError();
}

template <int MSG, int NW>
static cudaError_t launch_enh_tpb(const NmsArgs &a, cudaStream_t st) {
  const size_t per_thread = state_bytes_per_thread(a.dc, a.P, MSG);
  const size_t tables = nms_table_bytes(a.dc);
  // pick the block size with the most resident threads per SM under 227 KB
  const size_t limit = 227 * 1024;
  int best_tpb = 0;
  long long best_threads = -1;
  for (int tpb : {64, 128}) {
    const size_t smem = tables + per_thread * tpb;
    if (smem > limit) continue;
    const long long blocks = (long long)((228 * 1024) / (smem + 1024));
    const long long th = blocks * tpb;
    if (th > best_threads || (th == best_threads && tpb > best_tpb)) {
      best_threads = th;
      best_tpb = tpb;
    }
  }
  if (best_tpb == 0) return cudaErrorInvalidConfiguration;
  const size_t smem = tables + per_thread * best_tpb;
  if (best_tpb == 64) return launch_persistent(nms_enhanced_kernel<MSG, NW, 64>, 64, smem, a, st);
  return launch_persistent(nms_enhanced_kernel<MSG, NW, 128>, 128, smem, a, st);
}

template <int NW>
static cudaError_t launch_plain_tpb(const NmsArgs &a, cudaStream_t st) {
  const size_t per_thread = state_bytes_per_thread(a.dc, 0, kFP32);
  const size_t tables = nms_table_bytes(a.dc);
  for (int tpb : {64, 32}) {
    const size_t smem = tables + per_thread * tpb;
    if (smem > 227 * 1024) continue;
    if (tpb == 64) return launch_persistent(nms_plain_kernel<NW, 64>, 64, smem, a, st);
    return launch_persistent(nms_plain_kernel<NW, 32>, 32, smem, a, st);
  }
  return cudaErrorInvalidConfiguration;
}

cudaError_t launch_nms(const NmsArgs &a, cudaStream_t st) {
  const int NWr = (a.dc.n + 31) / 32;
  if (a.P == 0) {
    if (NWr == 1) return launch_plain_tpb<1>(a, st);
    if (NWr == 2) return launch_plain_tpb<2>(a, st);
    return launch_plain_tpb<4>(a, st);
  }
#define BCH_DISPATCH(MSG)                                     \
  if (NWr == 1) return launch_enh_tpb<MSG, 1>(a, st);         \
  if (NWr == 2) return launch_enh_tpb<MSG, 2>(a, st);         \
  return launch_enh_tpb<MSG, 4>(a, st);
  if (a.msg == kFP32) {
    BCH_DISPATCH(kFP32)
  } else if (a.msg == kFP16) {
    BCH_DISPATCH(kFP16)
  } else {
    BCH_DISPATCH(kINT8)
  }
#undef BCH_DISPATCH
}

}  // namespace bchlib
