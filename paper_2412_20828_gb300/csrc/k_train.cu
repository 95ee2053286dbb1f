// Backward pass of the enhanced NMS decoder for training the per-iteration
// normalization factors (the paper tunes alpha by treating NMS as a neural network,
// arXiv 2412.20828, Sec. II-A and Sec. IV).
//
// Subgradient of reading A of Algorithm 1, one thread per frame, recomputing each
// iteration from its FP32 checkpoint y^(t-1):
//   dL/dc2v_p(j,u) = g[pi_p^-1(u)] / P                     (merge is linear)
//   dL/dalpha_t   += dL/dc2v * c2v / alpha_t
//   dL/dz_a1      += alpha_t sgn(z_a1) sum_{e != a1} dL/dc2v_e * sgn_excl(e)
//   dL/dz_a2      += alpha_t sgn(z_a2) dL/dc2v_a1 * sgn_excl(a1)
// with a1 / a2 the first / second minimum of |z| on the row (lowest column on ties)
// and sgn_excl(e) the sign product of the row without edge e; the identity path of the
// merge carries g unchanged.
#include <cfloat>

#include "bch_kernels.cuh"

namespace bchlib {

template <int WB>
__device__ __forceinline__ void bwd_rows(const uint16_t *__restrict__ codes, int nrows, int w, int w4,
                                      const float *__restrict__ y, const float *__restrict__ g,
                                      float *__restrict__ gp, uint32_t jr, uint32_t sp, uint32_t n,
                                      uint32_t m, uint32_t sh, float alpha, float invP,
                                      float &dalpha) {
  for (int r = 0; r < nrows; r++) {
    const uint16_t *c = codes + r * w4;
    uint32_t ix[WB];
    float z[WB];
    float m1 = FLT_MAX, m2 = FLT_MAX;
    int a1 = 0, a2 = 0;
    uint32_t sg = 0;
#pragma unroll
    for (int e = 0; e < WB; e++) {
      if (e < w) {
        const uint32_t d = c[e];
        const uint32_t rr = bfe32(d, jr, m);
        const uint32_t i = addmod(rr, sp, n);
        ix[e] = i << sh;
        const float v = y[ix[e]];
        z[e] = v;
        const float av = fabsf(v);
        if (av < m1) {
          m2 = m1;
          a2 = a1;
          m1 = av;
          a1 = e;
        } else if (av < m2) {
          m2 = av;
          a2 = e;
        }
        sg ^= __float_as_uint(v);
      }
    }
    float acc1 = 0.0f, acc2 = 0.0f;
#pragma unroll
    for (int e = 0; e < WB; e++) {
      if (e < w) {
        const float gz = g[ix[e]] * invP;
        const uint32_t se = sg ^ __float_as_uint(z[e]);
        const float mag = (e == a1) ? m2 : m1;
        dalpha += gz * flip_sign(mag, se);
        const float gs = flip_sign(gz, se);
        if (e == a1)
          acc2 = gs;
        else
          acc1 += gs;
      }
    }
    float za1 = 0.f, za2 = 0.f;
    uint32_t i1 = 0, i2 = 0;
#pragma unroll
    for (int e = 0; e < WB; e++) {
      if (e < w) {
        if (e == a1) {
          za1 = z[e];
          i1 = ix[e];
        }
        if (e == a2) {
          za2 = z[e];
          i2 = ix[e];
        }
      }
    }
    // sgn(0) = +1: the float sign bit of z (z is never -0)
    gp[i1] += flip_sign(alpha * acc1, __float_as_uint(za1));
    gp[i2] += flip_sign(alpha * acc2, __float_as_uint(za2));
  }
}

template <int TPB, int WB>
__global__ void __launch_bounds__(TPB) nms_backward_kernel(const BwdArgs a) {
  constexpr uint32_t kShift = TPB == 128 ? 7u : (TPB == 64 ? 6u : 5u);
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ float red[TPB / 32];
  __shared__ float alpha_s[32];
  __shared__ int gw_s[kMaxGroups], gr_s[kMaxGroups], go_s[kMaxGroups];
  const int code_words = a.dc.group_off[a.dc.n_groups];
  uint16_t *codes = reinterpret_cast<uint16_t *>(smem);
  {
    const uint32_t *src = reinterpret_cast<const uint32_t *>(a.dc.codes);
    uint32_t *dst = reinterpret_cast<uint32_t *>(codes);
    for (int i = threadIdx.x; i < code_words / 2; i += blockDim.x) dst[i] = src[i];
  }
  if (threadIdx.x == 0) {
#pragma unroll
    for (int i = 0; i < 32; i++) alpha_s[i] = a.alpha[i];
#pragma unroll
    for (int g = 0; g < kMaxGroups; g++) {
      gw_s[g] = a.dc.group_w[g];
      gr_s[g] = a.dc.group_rows[g];
      go_s[g] = a.dc.group_off[g];
    }
  }
  __syncthreads();
  const int n_groups = a.dc.n_groups;
  float *state = reinterpret_cast<float *>(smem + ((size_t(code_words) * 2 + 15) & ~size_t(15)));
  const int n = a.dc.n;
  const uint32_t m = uint32_t(a.dc.m);
  const int tid = threadIdx.x;
  float *y = state + tid;
  float *g = y + size_t(n) * TPB;
  float *gp = g + size_t(n) * TPB;
  const int f = blockIdx.x * TPB + tid;
  const bool act = f < a.F;
  const float invP = 1.0f / float(a.P);
  uint32_t ctx[9];
  if (act) {
    for (int i = 0; i < n; i++) g[i << kShift] = a.grad_out[size_t(f) * a.ld + i];
#pragma unroll
    for (int p = 0; p < 9; p++) {
      if (p < a.P) {
        const uint32_t v = checked_auto(a.autos[size_t(f) * a.P + p], uint32_t(n), uint32_t(m), a.check, f);
        const uint32_t s = v & 0xffu, j = v >> 8;
        const uint32_t rs = j ? (((s >> j) | (s << (m - j))) & uint32_t(n)) : s;
        const uint32_t spv = rs ? uint32_t(n) - rs : 0u;
        ctx[p] = j | (spv << 8);
      }
    }
  }
  for (int t = a.I; t >= 1; t--) {
    float dal = 0.0f;
    if (act) {
      const float *src = a.ckpt + (size_t(t - 1) * a.F + f) * a.ld;
      for (int i = 0; i < n; i++) {
        y[i << kShift] = src[i];
        gp[i << kShift] = g[i << kShift];
      }
      const float alpha = alpha_s[t - 1];
#pragma unroll
      for (int p = 0; p < 9; p++) {
        if (p < a.P) {
          const uint32_t jr = ctx[p] & 0xffu, spv = ctx[p] >> 8;
          for (int gi = 0; gi < n_groups; gi++) {
            const int w = gw_s[gi];
            const int w4 = (w + 3) & ~3;
            const uint16_t *c = codes + go_s[gi];
            const int nr = gr_s[gi];
            bwd_rows<WB>(c, nr, w, w4, y, g, gp, jr, spv, uint32_t(n), m, kShift, alpha, invP, dal);
          }
        }
      }
      for (int i = 0; i < n; i++) g[i << kShift] = gp[i << kShift];
    }
    // deterministic block reduction of dL/dalpha_t
    for (int off = 16; off > 0; off >>= 1) dal += __shfl_xor_sync(kFull, dal, off);
    if ((tid & 31) == 0) red[tid >> 5] = dal;
    __syncthreads();
    if (tid == 0) {
      float s = 0.0f;
      for (int w = 0; w < TPB / 32; w++) s += red[w];
      a.partial[size_t(blockIdx.x) * a.I + (t - 1)] = s;
    }
    __syncthreads();
  }
  if (act && a.grad_llr)
    for (int i = 0; i < n; i++) a.grad_llr[size_t(f) * a.ld + i] = g[i << kShift];
}

__global__ void reduce_alpha_kernel(const float *partial, int nb, int I, float *grad_alpha) {
  __shared__ float red[32];
  const int t = blockIdx.x;
  float s = 0.0f;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) s += partial[size_t(b) * I + t];
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(kFull, s, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    float v = 0.0f;
    for (int w = 0; w < int(blockDim.x >> 5); w++) v += red[w];
    grad_alpha[t] = v;
  }
}

template <int TPB, int WB>
static cudaError_t launch_bwd_wb(const BwdArgs &a, int nb, size_t smem, cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(nms_backward_kernel<TPB, WB>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  note_launch();
  nms_backward_kernel<TPB, WB><<<nb, TPB, smem, st>>>(a);
  return cudaGetLastError();
}

size_t backward_workspace(int F, int I) {
  const int nb = (F + 63) / 64;
  return size_t(nb) * size_t(I) * sizeof(float);
}

cudaError_t launch_backward(const BwdArgs &a0, float *grad_alpha, cudaStream_t st) {
  if (a0.F <= 0) return cudaMemsetAsync(grad_alpha, 0, sizeof(float) * a0.I, st);
  constexpr int TPB = 64;
  const int code_words = a0.dc.group_off[a0.dc.n_groups];
  const size_t smem = ((size_t(code_words) * 2 + 15) & ~size_t(15)) + size_t(3) * a0.dc.n * TPB * 4;
  const int nb = (a0.F + TPB - 1) / TPB;
  const int mw = a0.dc.max_w;
  cudaError_t e = cudaSuccess;
  if (mw <= 8)
    e = launch_bwd_wb<TPB, 8>(a0, nb, smem, st);
  else if (mw <= 16)
    e = launch_bwd_wb<TPB, 16>(a0, nb, smem, st);
  else if (mw <= 24)
    e = launch_bwd_wb<TPB, 24>(a0, nb, smem, st);
  else if (mw <= 32)
    e = launch_bwd_wb<TPB, 32>(a0, nb, smem, st);
  else if (mw <= 48)
    e = launch_bwd_wb<TPB, 48>(a0, nb, smem, st);
  else
    e = cudaErrorNotSupported;
  if (e != cudaSuccess) return e;
  note_launch();
  reduce_alpha_kernel<<<a0.I, 256, 0, st>>>(a0.partial, nb, a0.I, grad_alpha);
  return cudaGetLastError();
}

}  // namespace bchlib
