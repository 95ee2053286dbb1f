// Precompiled min-sum kernels (generic over the code's Tanner graph) and their
// launchers; the device code lives in nms_device.cuh.
#pragma once
#include "bch_kernels.cuh"
#include "nms_device.cuh"

namespace bchlib {

template <int MSG, int NW, int WB>
__global__ void __launch_bounds__(128) nms_enhanced_kernel(const NmsArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  nms_persistent<MSG, NW, false, 0>(a, smem, GenericCopy<MSG, WB>());
}

// ---------------------------------------------------------------- plain NMS
// Eqs. (2)-(5) with per-edge messages kept as a compact per-row state: alpha*min1 and
// alpha*min2 carrying the sign product, the argmin edge, and the v2c sign bits.
template <int WB>
__device__ __forceinline__ void plain_rows(const uint16_t *__restrict__ codes, int row0, int nrows,
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

template <int NW, int WB>
__global__ void __launch_bounds__(128) nms_plain_kernel(const NmsArgs a) {
  const int TPB = blockDim.x;
  const uint32_t kShift = TPB == 128 ? 7u : 6u;
  extern __shared__ __align__(16) unsigned char smem[];
  const int code_words = a.dc.group_off[a.dc.n_groups];
  SmemTables tb = load_tables(a, smem, code_words);
  const int n = a.dc.n, R = a.dc.rows;
  const int n_groups = a.dc.n_groups;
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
          L[i << kShift] = x;
          xt[i << kShift] = x;
        }
        for (int r = 0; r < R; r++) {
          rs_m1[r << kShift] = 0.f;
          rs_m2[r << kShift] = 0.f;
          rs_am[r << kShift] = 0;
          rs_lo[r << kShift] = 0;
          rs_hi[r << kShift] = 0;
        }
      }
    }
    if (!__any_sync(kFull, f >= 0)) break;
    if (f < 0) continue;
    const float alpha = tb.alpha[t];
    for (int i = 0; i < n; i++) xn[i << kShift] = L[i << kShift];
    int row0 = 0;
    for (int g = 0; g < n_groups; g++) {
      const GroupDesc gd = tb.grp[g];
      const int w = gd.w;
      plain_rows<WB>(tb.codes + gd.off, row0, gd.rows, w, (w + 3) & ~3, xt, xn, rs_m1, rs_m2, rs_am,
                     rs_lo, rs_hi, uint32_t((1u << a.dc.m) - 1u), kShift, alpha);
      row0 += gd.rows;
    }
    uint32_t cb[NW];
#pragma unroll
    for (int w = 0; w < NW; w++) cb[w] = 0;
#pragma unroll
    for (int i = 0; i < NW * 32; i++) {
      if (i < n) {
        const float x = xn[i << kShift];
        xt[i << kShift] = x;  // Eq. (4) output is next iteration's total
        cb[i >> 5] |= (__float_as_uint(x) >> 31) << (i & 31);
      }
    }
    t++;
    const uint32_t nz = syndrome_nonzero<NW>(tb.rowmask, R, cb);
    if (t >= a.I || (a.early_stop && nz == 0)) {
      if (a.hard) write_hard<NW>(a.hard, f, cb);
      if (a.iters) a.iters[f] = uint8_t(t);
      if (a.flags) a.flags[f] = nz ? 0 : uint8_t(kFlagConverged);
      if (a.llr_out) {
        float *dst = a.llr_out + size_t(f) * a.ld;
        for (int i = 0; i < n; i++) dst[i] = xt[i << kShift];
      }
      need = true;
    }
  }
}

// ---------------------------------------------------------------- launchers
inline size_t nms_table_bytes(const DevCode &dc) {
  const int code_words = dc.group_off[dc.n_groups];
  return ((size_t(code_words) * 2 + 15) & ~size_t(15)) + size_t(dc.rows) * 16 + 32 * 4 +
         kMaxGroups * 16 + 16;
}

inline size_t state_bytes_per_thread(const DevCode &dc, int P, int msg) {
  if (P == 0) return size_t(3 * dc.n + 5 * dc.rows) * 4;
  const size_t ys = msg == kFP32 ? 4 : (msg == kFP16 ? 2 : 1);
  return size_t(P) * 4 + size_t(dc.n) * 4 + size_t(dc.n) * ys;
}

template <typename K>
static cudaError_t launch_persistent(K kernel, int tpb, size_t smem, const NmsArgs &a,
                                     cudaStream_t st) {
  int sms = 0, per_sm = 0;
  cudaError_t e = launch_geometry(reinterpret_cast<const void *>(kernel), tpb, smem, &sms, &per_sm);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  long long blocks = (long long)sms * per_sm;
  const long long need = (a.F + tpb - 1) / tpb;
  if (blocks > need) blocks = need;
  if (blocks < 1) blocks = 1;
  note_launch();
  kernel<<<unsigned(blocks), tpb, smem, st>>>(a);
  return cudaGetLastError();
}

template <int MSG, int NW, int WB>
cudaError_t launch_enh_tpb(const NmsArgs &a, cudaStream_t st) {
  const size_t per_thread = state_bytes_per_thread(a.dc, a.P, MSG);
  const size_t tables = nms_table_bytes(a.dc);
  // the block size with the most resident threads per SM under 227 KB
  int best_tpb = 0;
  long long best_threads = -1;
  for (int tpb : {64, 128}) {
    const size_t smem = tables + per_thread * tpb;
    if (smem > 227 * 1024) continue;
    const long long blocks = (long long)((228 * 1024) / (smem + 1024));
    const long long th = blocks * tpb;
    if (th > best_threads || (th == best_threads && tpb > best_tpb)) {
      best_threads = th;
      best_tpb = tpb;
    }
  }
  if (best_tpb == 0) return cudaErrorInvalidConfiguration;
  return launch_persistent(nms_enhanced_kernel<MSG, NW, WB>, best_tpb, tables + per_thread * best_tpb, a, st);
}

// Weight bucket: the smallest of 8, 16, 24, 32, 48 holding the code's heaviest row.
inline int weight_bucket(int max_w) {
  for (int b : {8, 16, 24, 32, 48})
    if (max_w <= b) return b;
  return 0;
}

template <int MSG>
cudaError_t launch_enh_msg(const NmsArgs &a, cudaStream_t st) {
  const int wb = weight_bucket(a.dc.max_w);
  if (a.dc.n <= 32) {
    if (wb == 8) return launch_enh_tpb<MSG, 1, 8>(a, st);
  } else if (a.dc.n <= 64) {
    if (wb <= 16) return launch_enh_tpb<MSG, 2, 16>(a, st);
    if (wb == 24) return launch_enh_tpb<MSG, 2, 24>(a, st);
    if (wb == 32) return launch_enh_tpb<MSG, 2, 32>(a, st);
  } else {
    if (wb <= 24) return launch_enh_tpb<MSG, 4, 24>(a, st);
    if (wb == 32) return launch_enh_tpb<MSG, 4, 32>(a, st);
    if (wb == 48) return launch_enh_tpb<MSG, 4, 48>(a, st);
  }
  return cudaErrorNotSupported;
}

template <int NW, int WB>
cudaError_t launch_plain_wb(const NmsArgs &a, cudaStream_t st) {
  const size_t per_thread = state_bytes_per_thread(a.dc, 0, kFP32);
  const size_t smem = nms_table_bytes(a.dc) + per_thread * 64;
  if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
  return launch_persistent(nms_plain_kernel<NW, WB>, 64, smem, a, st);
}

}  // namespace bchlib
