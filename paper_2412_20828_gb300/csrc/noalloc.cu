// bch_hybrid_decode_noalloc: the hybrid decoder for callers that cannot allocate device
// memory at decode time -- code running where cudaMalloc is forbidden or too costly
// after start-up (real-time receive loops, plug-ins handed only pre-registered
// buffers, hosts that must not grow the device heap).  The scratch that
// bch_hybrid_decode takes from a caller-provided workspace (frame-queue counters,
// per-block failure counts, the failed-frame list and its count) lives here in one
// file-scope __device__ array instead.  Only precompiled kernels are launched (no
// run-time compilation, so no module is loaded during a call).
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "bch_kernels.cuh"

using namespace bchlib;

namespace {

constexpr int kNoallocMaxFrames = 262144;
constexpr size_t kQueueOff = 0;                                          // 2 x u32 queue counters
constexpr size_t kCountsOff = 256;                                       // u32 per 1024 frames
constexpr size_t kListOff = kCountsOff + 4096;                           // u32[kNoallocMaxFrames]
constexpr size_t kCountOff = kListOff + size_t(kNoallocMaxFrames) * 4;  // u32 failed count
constexpr size_t kScratchBytes = kCountOff + 256;

// Every GPU that loads the library holds this array until the process exits.  In host
// code its name is only a host-side stand-in; the device address comes from
// cudaGetSymbolAddress, looked up once per device and context (below).
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// The address is looked up once per device and context: a context created anew on the
// same device (after cudaDeviceReset, for instance) has its own copy of the array, so
// the cache is keyed by the driver's unique context id (cuCtxGetId, reached through
// cudaGetDriverEntryPointByVersion so that the library does not link libcuda).
constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_addr[kMaxDevices] = {};
unsigned long long g_ctx_id[kMaxDevices] = {};

using CtxGetCurrentFn = int (*)(void **);
using CtxGetIdFn = int (*)(void *, unsigned long long *);

bool current_context_id(unsigned long long *id) {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<CtxGetCurrentFn>(fn);
    fn = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &fn, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<CtxGetIdFn>(fn);
  });
  void *ctx = nullptr;
  if (!get_current || !get_id || get_current(&ctx) != 0 || !ctx) return false;
  return get_id(ctx, id) == 0;
}

bch_status scratch_address(void **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(BCH_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(BCH_EINVAL, "device ordinal out of range");
  // initialises the device's primary context (a no-op once it exists) and makes it
  // current, so that its id can be read
  e = cudaSetDevice(dev);
  if (e != cudaSuccess) return fail(BCH_ECUDA, std::string("device set-up: ") + cudaGetErrorString(e));
  unsigned long long id = 0;
  if (!current_context_id(&id)) return fail(BCH_ECUDA, "cannot identify the current CUDA context");
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev] || g_ctx_id[dev] != id) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return fail(BCH_ECUDA, std::string("cudaGetSymbolAddress of the no-allocation scratch: ") +
                                 cudaGetErrorString(e));
    g_addr[dev] = p;
    g_ctx_id[dev] = id;
  }
  *out = g_addr[dev];
  return BCH_OK;
}

}  // namespace

extern "C" bch_status bch_hybrid_decode_noalloc(const bch_code *code, const bch_code *std_code,
                                                const bch_nms_params *p, const float *llr, int ld,
                                                int n_frames, const uint16_t *autos, uint64_t *hard,
                                                uint8_t *iters, uint8_t *flags, float *llr_out,
                                                void *stream) {
  // the same argument checks as bch_hybrid_decode, all before the first launch
  bch_status s = check_params(code, p);
  if (s == BCH_OK) s = check_osd(code, std_code, p->osd_order);
  if (s == BCH_OK) s = check_frames(code, llr, ld, n_frames);
  if (s != BCH_OK) return s;
  if (n_frames > kNoallocMaxFrames)
    return fail(BCH_EINVAL, "n_frames exceeds the 262144 frames the no-allocation scratch holds; "
                            "split the batch or use bch_hybrid_decode with a workspace");
  if (n_frames == 0) return BCH_OK;
  if (!hard || !flags) return fail(BCH_EINVAL, "hybrid decoding needs hard and flags");
  if (p->n_autos > 0 && !autos) return fail(BCH_EINVAL, "autos is null");
  if (p->osd_input == 1 && !llr_out)
    return fail(BCH_EINVAL, "osd_input = 1 needs llr_out (the NMS output the OSD reads)");
  void *base = nullptr;
  s = scratch_address(&base);
  if (s != BCH_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  unsigned char *ws = static_cast<unsigned char *>(base);
  unsigned *queue = reinterpret_cast<unsigned *>(ws + kQueueOff);
  // the array keeps the previous call's contents: the queue counters must start at 0
  cudaError_t e = cudaMemsetAsync(queue, 0, 16, st);
  if (e != cudaSuccess) return fail(BCH_ECUDA, std::string("clear scratch: ") + cudaGetErrorString(e));

  NmsArgs a;
  std::memset(&a, 0, sizeof(a));
  a.dc = code->dc;
  a.llr = llr;
  a.ld = ld;
  a.F = n_frames;
  a.autos = autos;
  a.P = p->n_autos;
  a.hard = hard;
  a.iters = iters;
  a.flags = flags;
  a.llr_out = llr_out;
  a.queue = queue;
  a.check = check_word();
  a.I = p->iters;
  a.early_stop = p->early_stop ? 1 : 0;
  a.msg = int(p->msg);
  a.rescale = p->rescale ? 1 : 0;
  a.qfrac = p->qfrac;
  for (int t = 0; t < 32; t++) a.alpha[t] = t < p->iters ? ldexpf(p->alpha[t], p->qfrac) : 0.0f;
  e = launch_nms(a, st);
  if (e != cudaSuccess) return fail(BCH_ECUDA, std::string("nms kernel: ") + cudaGetErrorString(e));

  uint32_t *counts = reinterpret_cast<uint32_t *>(ws + kCountsOff);
  uint32_t *list = reinterpret_cast<uint32_t *>(ws + kListOff);
  uint32_t *count = reinterpret_cast<uint32_t *>(ws + kCountOff);
  e = launch_compact(flags, n_frames, counts, list, count, st);
  if (e != cudaSuccess) return fail(BCH_ECUDA, std::string("compaction: ") + cudaGetErrorString(e));

  const int n = std_code->alg.n, M = n - std_code->alg.k;
  OsdArgs o;
  o.n = n;
  o.k = std_code->alg.k;
  o.M = M;
  o.rows = reinterpret_cast<const uint4 *>(std_code->dc.rowmask);
  o.cols = std_code->dc.colmask;
  o.llr = p->osd_input == 1 ? llr_out : llr;
  o.ld = ld;
  o.scale_input = p->osd_input == 1 ? 1 : 0;
  o.list = list;
  o.count = count;
  o.max_frames = n_frames;
  o.check = check_word();
  o.order = p->osd_order;
  o.hard = hard;
  o.flags = flags;
  o.queue = queue + 1;
  e = launch_osd(o, st);
  if (e != cudaSuccess) return fail(BCH_ECUDA, std::string("osd kernel: ") + cudaGetErrorString(e));
  return BCH_OK;
}
