// Failed-frame compaction and order-p OSD (arXiv 2412.20828, Sec. II-B and the hybrid
// decoder of Sec. IV) for sm_103a.
//
// One warp decodes one failed frame:
//  * reliabilities |L| (FP32) are ranked by counting against 64-bit keys
//    (|L| bits, index) -- a total order equal to a stable ascending sort;
//  * Gauss-Jordan elimination over GF(2) on the standard H visits columns from least
//    to most reliable in column-major form (lane l holds the row masks of columns
//    l + 32 q), one shuffle and a few xors per pivot;
//  * with the reduced rows, the disagreement pattern of a test pattern e on the
//    most reliable basis is D(e) = D0 xor (xor of the basis columns in e) restricted
//    to the n-k pivot positions, so a candidate costs a few XORs plus a weighted
//    popcount done with 16-entry tables of pivot weights (one per 4 pivot rows);
//  * scores are exact 64-bit integers (weights floor(|L| 2^24)), and the warp keeps
//    the lexicographic minimum of (score, enumeration index): the result equals a
//    sequential scan that keeps the first minimum.
#include "bch_kernels.cuh"
#include "osd_device.cuh"

namespace bchlib {

constexpr int kOsdWarps = 4;

__global__ void __launch_bounds__(32 * kOsdWarps) osd_kernel(const OsdArgs a) {
  extern __shared__ __align__(16) unsigned char osd_smem[];
  OsdSmem &S = reinterpret_cast<OsdSmem *>(osd_smem)[threadIdx.x >> 5];
  const int lane = int(lane_id());
  const uint32_t total = min(*a.count, uint32_t(a.max_frames));
  const int W64 = (a.n + 63) / 64;
  for (;;) {
    uint32_t item = 0;
    if (lane == 0) item = atomicAdd(a.queue, 1u);
    item = __shfl_sync(kFull, item, 0);
    if (item >= total) break;
    const int f = int(a.list[item]);
#ifdef BCH_CHECKED
    // a list entry outside the frames is recorded and skipped (item is warp-uniform)
    if (uint32_t(f) >= uint32_t(a.max_frames)) {
      if (lane == 0 && a.check) {
        atomicOr(a.check, kCheckOsdFrame);
        atomicAdd(a.check + 1, 1u);
        atomicMin(a.check + 3, item);
      }
      continue;
    }
#endif
    const float *L = a.llr + size_t(f) * a.ld;
    const int sexp = a.scale_input ? osd_input_exponent(L, a.n) : 0;
    osd_one_frame(S, a.n, a.k, a.M, a.cols, L, a.order, a.hard + size_t(f) * W64,
                  a.flags ? a.flags + f : nullptr, sexp);
  }
}

// ---------------------------------------------------------------- compaction
constexpr int kCompactBlock = 1024;

__global__ void __launch_bounds__(kCompactBlock)
    count_failed_kernel(const uint8_t *flags, int F, uint32_t *counts) {
  __shared__ uint32_t warp_cnt[kCompactBlock / 32];
  const int f = blockIdx.x * kCompactBlock + threadIdx.x;
  const bool fail = f < F && !(flags[f] & BCH_FLAG_CONVERGED);
  const unsigned b = __ballot_sync(kFull, fail);
  if ((threadIdx.x & 31) == 0) warp_cnt[threadIdx.x >> 5] = __popc(b);
  __syncthreads();
  if (threadIdx.x < 32) {
    uint32_t v = warp_cnt[threadIdx.x];
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(kFull, v, off);
    if (threadIdx.x == 0) counts[blockIdx.x] = v;
  }
}

__global__ void __launch_bounds__(kCompactBlock)
    write_failed_kernel(const uint8_t *flags, int F, const uint32_t *counts, uint32_t *list,
                        uint32_t *count) {
  __shared__ uint32_t warp_cnt[kCompactBlock / 32];
  __shared__ uint32_t block_off;
  // offset of this block: sum of the counts of the blocks before it
  uint32_t part = 0;
  for (int b = threadIdx.x; b < int(blockIdx.x); b += kCompactBlock) part += counts[b];
  for (int off = 16; off > 0; off >>= 1) part += __shfl_xor_sync(kFull, part, off);
  if ((threadIdx.x & 31) == 0) warp_cnt[threadIdx.x >> 5] = part;
  __syncthreads();
  if (threadIdx.x < 32) {
    uint32_t v = warp_cnt[threadIdx.x];
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(kFull, v, off);
    if (threadIdx.x == 0) block_off = v;
  }
  __syncthreads();
  const int f = blockIdx.x * kCompactBlock + threadIdx.x;
  const bool fail = f < F && !(flags[f] & BCH_FLAG_CONVERGED);
  const unsigned b = __ballot_sync(kFull, fail);
  if ((threadIdx.x & 31) == 0) warp_cnt[threadIdx.x >> 5] = __popc(b);
  __syncthreads();
  uint32_t before = block_off;
  for (int w = 0; w < int(threadIdx.x >> 5); w++) before += warp_cnt[w];
  if (fail) list[before + __popc(b & ((1u << (threadIdx.x & 31)) - 1u))] = uint32_t(f);
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) {
    uint32_t tot = block_off;
    for (int w = 0; w < kCompactBlock / 32; w++) tot += warp_cnt[w];
    *count = tot;
  }
}

cudaError_t launch_compact(const uint8_t *flags, int F, uint32_t *counts, uint32_t *list,
                           uint32_t *count, cudaStream_t st) {
  if (F <= 0) return cudaMemsetAsync(count, 0, sizeof(uint32_t), st);
  const int nb = (F + kCompactBlock - 1) / kCompactBlock;
  note_launch();
  count_failed_kernel<<<nb, kCompactBlock, 0, st>>>(flags, F, counts);
  note_launch();
  write_failed_kernel<<<nb, kCompactBlock, 0, st>>>(flags, F, counts, list, count);
  return cudaGetLastError();
}

cudaError_t launch_osd(const OsdArgs &a, cudaStream_t st) {
  int sms = 0, per_sm = 0;
  const size_t smem = sizeof(OsdSmem) * kOsdWarps;
  cudaError_t e = launch_geometry(reinterpret_cast<const void *>(osd_kernel), 32 * kOsdWarps, smem, &sms, &per_sm);
  if (e != cudaSuccess) return e;
  long long blocks = (long long)sms * (per_sm > 0 ? per_sm : 1);
  const long long need = (a.max_frames + kOsdWarps - 1) / kOsdWarps;
  if (blocks > need) blocks = need;
  if (blocks < 1) blocks = 1;
  note_launch();
  osd_kernel<<<unsigned(blocks), 32 * kOsdWarps, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace bchlib
