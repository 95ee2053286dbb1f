// Device-side helpers shared by the library's CUDA translation units.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "bch_args.h"
#include "bch_internal.h"
#include "nms_device.cuh"

namespace bchlib {


// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): two 32x32 multiplies per round,
// key bumped by the Weyl constants between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; r++) {
    if (r > 0) {
      k.x += 0x9E3779B9u;
      k.y += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

// Open-interval uniform from the top 24 bits: ((w >> 8) + 0.5) 2^-24, exact in FP32.
__device__ __forceinline__ float u24(uint32_t w) {
  return (float(w >> 8) + 0.5f) * (1.0f / 16777216.0f);
}

__device__ __forceinline__ uint64_t splitmix64_mix_d(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

// The P automorphisms (s | j << 8) of frame f: pair p takes the first of up to 16
// SplitMix64 draws at counter 1 + (f P + p) 16 + attempt that differs from the pairs
// before it; s uniform in [0, n), j uniform in [0, ord) by 32-bit multiply-shift.
__device__ __forceinline__ void draw_frame_autos(int n, int ord, int P, uint64_t seed, uint64_t f,
                                                 uint32_t *out) {
  for (int p = 0; p < P; p++) {
    uint32_t s = 0, j = 0;
    for (int att = 0; att < 16; att++) {
      const uint64_t cnt = 1 + (f * uint64_t(P) + uint64_t(p)) * 16 + uint64_t(att);
      const uint64_t x = splitmix64_mix_d(seed + 0x9E3779B97F4A7C15ULL * cnt);
      s = uint32_t(((x & 0xffffffffULL) * uint64_t(n)) >> 32);
      j = uint32_t(((x >> 32) * uint64_t(ord)) >> 32);
      bool clash = false;
      for (int q = 0; q < p; q++)
        if (out[q] == (s | (j << 8))) clash = true;
      if (!clash) break;
    }
    out[p] = s | (j << 8);
  }
}


}  // namespace bchlib
