// Dispatch of the normalized min-sum kernels (enhanced: by storage format; plain).
#include "bch_kernels.cuh"

namespace bchlib {

cudaError_t launch_enh_fp32(const NmsArgs &a, cudaStream_t st);
cudaError_t launch_enh_fp16(const NmsArgs &a, cudaStream_t st);
cudaError_t launch_enh_int8(const NmsArgs &a, cudaStream_t st);
cudaError_t launch_plain(const NmsArgs &a, cudaStream_t st);

size_t nms_table_bytes_host(const DevCode &dc) {
  const int code_words = dc.group_off[dc.n_groups];
  return ((size_t(code_words) * 2 + 15) & ~size_t(15)) + size_t(dc.rows) * 16 + 32 * 4 +
         kMaxGroups * 16;
}

cudaError_t launch_nms(const NmsArgs &a, cudaStream_t st) {
  if (a.P == 0) return launch_plain(a, st);
  if (a.msg == 1) return launch_enh_fp16(a, st);
  if (a.msg == 2) return launch_enh_int8(a, st);
  return launch_enh_fp32(a, st);
}

}  // namespace bchlib
