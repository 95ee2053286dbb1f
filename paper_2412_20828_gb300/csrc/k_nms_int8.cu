// Instantiations of the normalized min-sum kernels for INT8 message storage
// (one kernel per weight bucket; see k_nms_impl.cuh).
#include "k_nms_impl.cuh"

namespace bchlib {

cudaError_t launch_enh_int8(const NmsArgs &a, cudaStream_t st) { return launch_enh_msg<kINT8>(a, st); }

}  // namespace bchlib
