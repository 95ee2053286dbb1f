// Device-side helpers shared by the library's CUDA translation units.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "bch_args.h"
#include "bch_internal.h"
#include "autos_device.cuh"
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

}  // namespace bchlib
