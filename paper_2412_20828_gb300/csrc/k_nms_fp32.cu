// Instantiations of the normalized min-sum kernels for FP32 message storage
// (one kernel per weight bucket; see k_nms_impl.cuh).
#include "k_nms_impl.cuh"

namespace bchlib {

cudaError_t launch_enh_fp32(const NmsArgs &a, cudaStream_t st) { return launch_enh_msg<kFP32>(a, st); }

cudaError_t launch_plain(const NmsArgs &a, cudaStream_t st) {
  const int wb = weight_bucket(a.dc.max_w);
  if (a.dc.n <= 32) {
    if (wb <= 8) return launch_plain_wb<1, 8>(a, st);
  } else if (a.dc.n <= 64) {
    if (wb <= 16) return launch_plain_wb<2, 16>(a, st);
    if (wb == 24) return launch_plain_wb<2, 24>(a, st);
    if (wb == 32) return launch_plain_wb<2, 32>(a, st);
  } else {
    if (wb <= 24) return launch_plain_wb<4, 24>(a, st);
    if (wb == 32) return launch_plain_wb<4, 32>(a, st);
    if (wb == 48) return launch_plain_wb<4, 48>(a, st);
  }
  return cudaErrorNotSupported;
}

}  // namespace bchlib
