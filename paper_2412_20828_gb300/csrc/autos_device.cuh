// Counter-based automorphism draws (the stateless SplitMix64 addressing of the
// library's draw routine), shared by the precompiled kernels and the serving kernel
// compiled at run time.
#pragma once
#ifndef __CUDACC_RTC__
#include <stdint.h>
#endif

namespace bchlib {

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
