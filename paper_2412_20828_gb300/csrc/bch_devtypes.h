// Plain data types shared by the host code, the precompiled CUDA kernels and the
// kernels compiled at run time (NVRTC): the device image of a code and the argument
// block of the min-sum kernels.  No includes under NVRTC.
#pragma once
#ifndef __CUDACC_RTC__
#include <stdint.h>
#endif

namespace bchlib {

constexpr int kMaxGroups = 16;
constexpr int kMaxN = 127;
constexpr unsigned kFlagConverged = 1u;
constexpr unsigned kFlagOsd = 2u;
// Checked builds (BCH_CHECKED): bits of the check word's first entry.
constexpr unsigned kCheckAutomorphism = 1u;
constexpr unsigned kCheckOsdFrame = 2u;

// Layout of a code object on the device.  Rows are grouped by weight; each group
// stores its rows' column codes d(u) = u | u << m (so that the Frobenius power j of u,
// rotr_m(u, j), is the m-bit field of d(u) starting at bit j) contiguously, every row
// padded to a multiple of 4 entries.
struct DevCode {
  int n, k, m, rows, edges, max_w, nwords32;
  int n_groups;
  int group_w[kMaxGroups];        // row weight of the group
  int group_rows[kMaxGroups];     // number of rows
  int group_off[kMaxGroups + 1];  // offset into codes (in entries); [n_groups] = end
  const uint16_t *codes;          // column codes, group order
  const uint32_t *rowmask;        // [rows][4] bit-packed rows (syndrome test)
  const uint64_t *par;            // [k] parity words (systematic encoder)
  const uint64_t *colmask;        // [n] column masks over the rows (rows <= 64, else 0)
};

// Argument block of the enhanced / plain min-sum kernels.
struct NmsArgs {
  DevCode dc;
  const float *llr;
  int ld, F;
  const uint16_t *autos;
  int P;
  uint64_t *hard;
  uint8_t *iters;
  uint8_t *flags;
  float *llr_out;
  float *ckpt;  // training checkpoints [I+1][F][ld] or null
  unsigned *queue;
  unsigned *check;  // checked builds: the device's check word [4]; else unused
  int I, early_stop, msg, rescale, qfrac;
  float alpha[32];  // alpha_t 2^qfrac
};

}  // namespace bchlib
