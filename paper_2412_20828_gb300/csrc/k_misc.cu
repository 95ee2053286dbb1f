// Frame generation, automorphism draws, error counting and the training loss
// (arXiv 2412.20828, Sec. II setting: BPSK over AWGN, LLR of Eq. 1).
#include "bch_kernels.cuh"

namespace bchlib {

// ---------------------------------------------------------------- automorphisms
__global__ void draw_autos_kernel(int n, int ord, int P, uint64_t seed, uint64_t frame0, int F,
                                  uint16_t *out) {
  const int fi = blockIdx.x * blockDim.x + threadIdx.x;
  if (fi >= F) return;
  uint32_t v[9];
  draw_frame_autos(n, ord, P, seed, frame0 + uint64_t(fi), v);
  uint16_t *o = out + size_t(fi) * P;
  for (int p = 0; p < P; p++) o[p] = uint16_t(v[p]);
}

cudaError_t launch_draw_autos(int n, int ord, int P, uint64_t seed, uint64_t frame0, int F,
                              uint16_t *out, cudaStream_t st) {
  if (F <= 0) return cudaSuccess;
  note_launch();
  draw_autos_kernel<<<(F + 255) / 256, 256, 0, st>>>(n, ord, P, seed, frame0, F, out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- frames
__global__ void gen_frames_kernel(const GenArgs a) {
  const int fi = blockIdx.x * blockDim.x + threadIdx.x;
  if (fi >= a.F) return;
  const uint64_t f = a.frame0 + uint64_t(fi);
  const uint2 key = make_uint2(uint32_t(a.seed), uint32_t(a.seed >> 32));
  const uint4 mw = philox4x32_10(make_uint4(uint32_t(f), uint32_t(f >> 32), 0u, 0u), key);
  const uint32_t msg[4] = {mw.x, mw.y, mw.z, mw.w};
  const int n = a.n, k = a.k, M = n - k;
  uint64_t par = 0;
  for (int i = 0; i < k; i++)
    if ((msg[i >> 5] >> (i & 31)) & 1u) par ^= a.par[i];
  // codeword bits: parity in 0..M-1, message i at M + i
  uint64_t cw0 = par, cw1 = 0;
  for (int i = 0; i < k; i++) {
    const uint64_t b = (msg[i >> 5] >> (i & 31)) & 1u;
    const int pos = M + i;
    if (pos < 64)
      cw0 |= b << pos;
    else
      cw1 |= b << (pos - 64);
  }
  float e = a.ebn0_lo;
  if (a.ebn0_hi > a.ebn0_lo) {
    const uint4 ew = philox4x32_10(make_uint4(uint32_t(f), uint32_t(f >> 32), 0u, 2u), key);
    e = a.ebn0_lo + (a.ebn0_hi - a.ebn0_lo) * u24(ew.x);
  }
  const float R = float(k) / float(n);
  const float s2 = 1.0f / (2.0f * R * exp10f(e / 10.0f));
  const float sg = sqrtf(s2);
  const float sc = 2.0f / s2;
  float *dst = a.llr + size_t(fi) * a.ld;
  const bool vec = ((a.ld & 3) == 0) && ((reinterpret_cast<uintptr_t>(a.llr) & 15) == 0);
  for (int b = 0; 4 * b < n; b++) {
    const uint4 w = philox4x32_10(make_uint4(uint32_t(f), uint32_t(f >> 32), uint32_t(b), 1u), key);
    float z[4];
    {
      const float r = sqrtf(-2.0f * logf(u24(w.x)));
      float sn, cs;
      sincospif(2.0f * u24(w.y), &sn, &cs);
      z[0] = r * cs;
      z[1] = r * sn;
    }
    {
      const float r = sqrtf(-2.0f * logf(u24(w.z)));
      float sn, cs;
      sincospif(2.0f * u24(w.w), &sn, &cs);
      z[2] = r * cs;
      z[3] = r * sn;
    }
    float v[4];
#pragma unroll
    for (int h = 0; h < 4; h++) {
      const int i = 4 * b + h;
      if (i < n) {
        const uint64_t bit = i < 64 ? (cw0 >> i) & 1u : (cw1 >> (i - 64)) & 1u;
        const float s = bit ? -1.0f : 1.0f;
        v[h] = sc * (s + sg * z[h]);
      } else {
        v[h] = 0.0f;
      }
    }
    if (vec && 4 * b + 3 < a.ld) {
      *reinterpret_cast<float4 *>(dst + 4 * b) = make_float4(v[0], v[1], v[2], v[3]);
    } else {
      for (int h = 0; h < 4 && 4 * b + h < a.ld; h++) dst[4 * b + h] = v[h];
    }
  }
  for (int i = ((n + 3) & ~3); i < a.ld; i++) dst[i] = 0.0f;
  if (a.codeword) {
    const int W64 = (n + 63) / 64;
    a.codeword[size_t(fi) * W64] = cw0;
    if (W64 > 1) a.codeword[size_t(fi) * W64 + 1] = cw1;
  }
}

cudaError_t launch_gen_frames(const GenArgs &a, cudaStream_t st) {
  if (a.F <= 0) return cudaSuccess;
  note_launch();
  gen_frames_kernel<<<(a.F + 127) / 128, 128, 0, st>>>(a);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- error counting
__global__ void count_errors_kernel(int n, const uint64_t *hard, const uint64_t *cw,
                                    const uint8_t *iters, const uint8_t *flags, int F,
                                    long long *counters) {
  __shared__ long long part[8][8];
  const int fi = blockIdx.x * blockDim.x + threadIdx.x;
  long long v[7] = {0, 0, 0, 0, 0, 0, 0};
  if (fi < F) {
    const int W64 = (n + 63) / 64;
    int be = 0;
    for (int w = 0; w < W64; w++) be += __popcll(hard[size_t(fi) * W64 + w] ^ cw[size_t(fi) * W64 + w]);
    const uint8_t fl = flags ? flags[fi] : 0;
    v[0] = 1;
    v[1] = be > 0;
    v[2] = be;
    v[3] = (be > 0) && (fl & BCH_FLAG_CONVERGED) && !(fl & BCH_FLAG_OSD);
    v[4] = (fl & BCH_FLAG_OSD) ? 1 : 0;
    v[5] = iters ? iters[fi] : 0;
    v[6] = (fl & BCH_FLAG_CONVERGED) ? 1 : 0;
  }
#pragma unroll
  for (int c = 0; c < 7; c++)
    for (int off = 16; off > 0; off >>= 1) v[c] += __shfl_xor_sync(kFull, v[c], off);
  const int warp = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0)
    for (int c = 0; c < 7; c++) part[warp][c] = v[c];
  __syncthreads();
  if (threadIdx.x < 7) {
    long long s = 0;
    for (int w = 0; w < int(blockDim.x >> 5); w++) s += part[w][threadIdx.x];
    atomicAdd(reinterpret_cast<unsigned long long *>(counters + threadIdx.x), (unsigned long long)s);
  }
}

cudaError_t launch_count_errors(int n, const uint64_t *hard, const uint64_t *cw, const uint8_t *iters,
                                const uint8_t *flags, int F, long long *counters, cudaStream_t st) {
  if (F <= 0) return cudaSuccess;
  note_launch();
  count_errors_kernel<<<(F + 255) / 256, 256, 0, st>>>(n, hard, cw, iters, flags, F, counters);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- training loss
// loss = mean over frames and bits of softplus(-(1 - 2c) y); grad = dloss/dy.
// Per-block partial sums, then one block adds them in a fixed order (deterministic).
__global__ void bce_kernel(int n, const float *y, int ld, const uint64_t *cw, int F, float *grad,
                           float *partial) {
  __shared__ float red[32];
  const int fi = blockIdx.x * blockDim.x + threadIdx.x;
  float s = 0.0f;
  if (fi < F) {
    const int W64 = (n + 63) / 64;
    const float inv = 1.0f / (float(F) * float(n));
    for (int i = 0; i < n; i++) {
      const uint64_t b = (cw[size_t(fi) * W64 + (i >> 6)] >> (i & 63)) & 1u;
      const float sgn = b ? -1.0f : 1.0f;
      const float x = -sgn * y[size_t(fi) * ld + i];
      s += fmaxf(x, 0.0f) + log1pf(expf(-fabsf(x)));
      const float sig = 1.0f / (1.0f + expf(-x));
      if (grad) grad[size_t(fi) * ld + i] = inv * sig * (-sgn);
    }
  }
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(kFull, s, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.0f;
    for (int w = 0; w < int(blockDim.x >> 5); w++) t += red[w];
    partial[blockIdx.x] = t;
  }
}

__global__ void sum_partials_kernel(const float *partial, int nb, float scale, float *out) {
  __shared__ float red[32];
  float s = 0.0f;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) s += partial[i];
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(kFull, s, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.0f;
    for (int w = 0; w < int(blockDim.x >> 5); w++) t += red[w];
    *out = t * scale;
  }
}

size_t bce_workspace(int F) { return size_t((F + 255) / 256) * sizeof(float); }

cudaError_t launch_bce(int n, const float *y, int ld, const uint64_t *cw, int F, float *loss,
                       float *grad, float *partial, cudaStream_t st) {
  if (F <= 0) return cudaMemsetAsync(loss, 0, sizeof(float), st);
  const int nb = (F + 255) / 256;
  note_launch();
  bce_kernel<<<nb, 256, 0, st>>>(n, y, ld, cw, F, grad, partial);
  note_launch();
  sum_partials_kernel<<<1, 256, 0, st>>>(partial, nb, 1.0f / (float(F) * float(n)), loss);
  return cudaGetLastError();
}

}  // namespace bchlib
