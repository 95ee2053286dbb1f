// Kernel argument blocks and launchers shared by the library's CUDA translation units.
#pragma once

#include <cuda_runtime.h>

#include "bch_internal.h"

namespace bchlib {

struct OsdArgs {
  int n, k, M;
  const uint4 *rows;  // [M] standard H rows, 4 x u32
  const uint64_t *cols;  // [n] standard H column masks over the M rows
  const float *llr;
  int ld;
  const uint32_t *list;
  const uint32_t *count;
  int max_frames;
  int order;
  uint64_t *hard;
  uint8_t *flags;
  unsigned *queue;
  int scale_input;  // 1: scale each frame's input by the power of two putting max |L| in [2^15, 2^16)
  unsigned *check;  // checked builds: the device's check word [4]; else unused
};

struct GenArgs {
  int n, k;
  const uint64_t *par;  // [k] parity words
  float ebn0_lo, ebn0_hi;
  uint64_t seed, frame0;
  int F, ld;
  float *llr;
  uint64_t *codeword;
};

struct BwdArgs {
  DevCode dc;
  const uint16_t *autos;
  int P;
  const float *ckpt;
  int ld, F, I;
  const float *grad_out;
  float *grad_llr;
  float *partial;  // [blocks][I]
  unsigned *check;  // checked builds: the device's check word [4]; else unused
  float alpha[32];
};

// Parallel annealing chains of the H_o search (one block per chain).
struct AnnealArgs {
  int n, Mo, steps, chains;
  double lam, T0, cool;            // loss weight, start temperature, cooling factor
  const ulonglong2 *rows0;         // [Mo] rows after step 5 (bits 0..63, 64..127)
  const uint64_t *state0;          // [chains] SplitMix64 states
  ulonglong2 *rows_out;            // [chains][Mo] annealed rows
};
cudaError_t launch_anneal(const AnnealArgs &a, cudaStream_t st);
size_t anneal_smem_bytes(int Mo);

// Resident blocks per SM and SM count for (fn, block size, dynamic shared memory) on the
// current device; raises the kernel's shared-memory limit when this launch needs more
// than any before.  Remembered per combination, so repeated launches cost no driver
// queries.
// Checked builds: the current device's check word (u32 [4]); nullptr otherwise or if the
// symbol cannot be resolved.
unsigned *check_word();

cudaError_t launch_geometry(const void *fn, int tpb, size_t smem, int *sms, int *per_sm);
cudaError_t launch_nms(const NmsArgs &a, cudaStream_t st);
cudaError_t launch_osd(const OsdArgs &a, cudaStream_t st);
cudaError_t launch_compact(const uint8_t *flags, int F, uint32_t *counts, uint32_t *list,
                           uint32_t *count, cudaStream_t st);
cudaError_t launch_draw_autos(int n, int ord, int P, uint64_t seed, uint64_t frame0, int F,
                              uint16_t *out, cudaStream_t st);
cudaError_t launch_gen_frames(const GenArgs &a, cudaStream_t st);
cudaError_t launch_count_errors(int n, const uint64_t *hard, const uint64_t *cw, const uint8_t *iters,
                                const uint8_t *flags, int F, long long *counters, cudaStream_t st);
cudaError_t launch_bce(int n, const float *y, int ld, const uint64_t *cw, int F, float *loss,
                       float *grad, float *partial, cudaStream_t st);
size_t bce_workspace(int F);
cudaError_t launch_backward(const BwdArgs &a, float *grad_alpha, cudaStream_t st);
size_t backward_workspace(int F, int I);

}  // namespace bchlib
