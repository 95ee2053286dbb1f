// Host-memory decode pipeline (bch_decoder): chunked copy-in / hybrid decode /
// copy-out on two CUDA streams so transfers overlap the kernels of the other chunk.
// Chunks alternate between two device buffer sets; stream order makes a buffer's next
// copy-in wait for its previous copy-out.  With pinned host memory a GB300 moves
// about 210 GB/s each way; chunks of ~1M frames keep the copies hidden behind the
// decode while keeping few decode launches (each ends in a tail where the slowest
// frames of the last wave finish on a partly idle GPU).
#include <chrono>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "bch_kernels.cuh"

using namespace bchlib;

struct bch_decoder {
  const bch_code *code = nullptr;
  const bch_code *std_code = nullptr;
  bch_nms_params params{};
  std::vector<float> alpha;
  int ld = 0, chunk = 0, W64 = 1;
  cudaStream_t st[2] = {nullptr, nullptr};
  struct Slot {
    float *llr = nullptr;
    uint16_t *autos = nullptr;
    uint64_t *hard = nullptr;
    uint8_t *iters = nullptr;
    uint8_t *flags = nullptr;
    float *y = nullptr;  // final NMS output, when the OSD reads it (osd_input = 1)
    void *ws = nullptr;
  } slot[2];
  bool timing = false;
  bool in_place = true;  // decode device-accessible host buffers where they are
  bch_decoder_timing tm{};
};

namespace {
// Device address of [p, p + count) when the GPU can read and write that host memory in
// place -- page-locked memory mapped into the device's address space (under unified
// addressing at the same address) -- else nullptr.  Both ends are checked, so a range
// that leaves its mapped allocation is not taken.
template <class T>
T *device_view(T *p, size_t count) {
  if (!p || count == 0) return nullptr;
  cudaPointerAttributes a{}, b{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess || cudaPointerGetAttributes(&b, p + (count - 1)) != cudaSuccess) {
    cudaGetLastError();  // clear a non-sticky error of the query
    return nullptr;
  }
  if (a.type != cudaMemoryTypeHost || b.type != cudaMemoryTypeHost || !a.devicePointer || !b.devicePointer)
    return nullptr;
  T *da = static_cast<T *>(a.devicePointer), *db = static_cast<T *>(b.devicePointer);
  return db - da == std::ptrdiff_t(count - 1) ? da : nullptr;
}

void free_decoder(bch_decoder *d) {
  for (int b = 0; b < 2; b++) {
    cudaFree(d->slot[b].llr);
    cudaFree(d->slot[b].autos);
    cudaFree(d->slot[b].hard);
    cudaFree(d->slot[b].iters);
    cudaFree(d->slot[b].flags);
    cudaFree(d->slot[b].y);
    cudaFree(d->slot[b].ws);
    if (d->st[b]) cudaStreamDestroy(d->st[b]);
  }
  delete d;
}
}  // namespace

extern "C" {

bch_status bch_decoder_create(const bch_code *code, const bch_code *std_code,
                              const bch_nms_params *params, int ld, int chunk_frames,
                              bch_decoder **out) {
  if (!out || !code || !params || !params->alpha) return fail(BCH_EINVAL, "null argument");
  *out = nullptr;
  if (chunk_frames < 1 || ld < code->alg.n) return fail(BCH_EINVAL, "bad chunk or ld");
  if (params->iters < 1 || params->iters > 32) return fail(BCH_EINVAL, "iters must be in [1, 32]");
  bch_decoder *d = new (std::nothrow) bch_decoder();
  if (!d) return fail(BCH_ENOMEM, "host allocation");
  d->code = code;
  d->std_code = std_code;
  d->params = *params;
  d->alpha.assign(params->alpha, params->alpha + params->iters);
  d->params.alpha = d->alpha.data();
  d->ld = ld;
  d->chunk = chunk_frames;
  d->W64 = (code->alg.n + 63) / 64;
  size_t wsb = 0;
  bch_status s = bch_workspace_size(code, &d->params, chunk_frames, &wsb);
  if (s != BCH_OK) {
    delete d;
    return s;
  }
  const size_t F = size_t(chunk_frames);
  const int P = params->n_autos > 0 ? params->n_autos : 1;
  for (int b = 0; b < 2; b++) {
    auto &S = d->slot[b];
    bool ok = cudaStreamCreateWithFlags(&d->st[b], cudaStreamNonBlocking) == cudaSuccess &&
              cudaMalloc(&S.llr, F * ld * 4) == cudaSuccess &&
              cudaMalloc(&S.autos, F * P * 2) == cudaSuccess &&
              cudaMalloc(&S.hard, F * d->W64 * 8) == cudaSuccess &&
              cudaMalloc(&S.iters, F) == cudaSuccess && cudaMalloc(&S.flags, F) == cudaSuccess &&
              cudaMalloc(&S.ws, wsb) == cudaSuccess &&
              (params->osd_input != 1 || cudaMalloc(&S.y, F * ld * 4) == cudaSuccess);
    if (!ok) {
      free_decoder(d);
      return fail(BCH_ENOMEM, "decoder buffers");
    }
  }
  *out = d;
  return BCH_OK;
}

bch_status bch_decoder_run_host(bch_decoder *d, const float *llr, int n_frames, uint64_t autos_seed,
                                uint64_t frame0, uint64_t *hard, uint8_t *iters, uint8_t *flags) {
  if (!d) return fail(BCH_EINVAL, "null decoder");
  if (n_frames < 0 || (n_frames > 0 && (!llr || !hard))) return fail(BCH_EINVAL, "bad arguments");
  const int n = d->code->alg.n;
  const int nchunks = (n_frames + d->chunk - 1) / d->chunk;
  const auto t_wall = std::chrono::steady_clock::now();
  // per-phase timing: events before the copy-in, after it, after the decode and after
  // the copy-out of every chunk, read once the call's work has finished
  struct Events {  // destroyed on every return path
    std::vector<cudaEvent_t> v;
    ~Events() {
      for (cudaEvent_t e : v) cudaEventDestroy(e);
    }
  } evs;
  std::vector<cudaEvent_t> &ev = evs.v;
  auto mark = [&](cudaStream_t st) {
    if (!d->timing) return;
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) == cudaSuccess) {
      cudaEventRecord(e, st);
      ev.push_back(e);
    }
  };
  // In place: when the caller's buffers are page-locked host memory mapped into the
  // device's address space, the kernels read the LLRs and write the results there
  // directly (on a GB300 over the coherent CPU-GPU link), with no staging copies; the
  // chunks then only bound the automorphism and workspace buffers.  Otherwise each chunk
  // is copied in and its results copied out.
  const size_t Fz = size_t(n_frames);
  const float *llr_d = d->in_place ? device_view(llr, Fz * d->ld) : nullptr;
  uint64_t *hard_d = llr_d ? device_view(hard, Fz * d->W64) : nullptr;
  uint8_t *iters_d = hard_d && iters ? device_view(iters, Fz) : nullptr;
  uint8_t *flags_d = hard_d && flags ? device_view(flags, Fz) : nullptr;
  const bool zc = llr_d && hard_d && (!iters || iters_d) && (!flags || flags_d);
  for (int c = 0; c < nchunks; c++) {
    const int b = c & 1;
    auto &S = d->slot[b];
    cudaStream_t st = d->st[b];
    const int f0 = c * d->chunk;
    const int F = std::min(d->chunk, n_frames - f0);
    mark(st);
    cudaError_t e = cudaSuccess;
    if (!zc)
      e = cudaMemcpyAsync(S.llr, llr + size_t(f0) * d->ld, size_t(F) * d->ld * 4, cudaMemcpyHostToDevice, st);
    mark(st);
    if (e != cudaSuccess) return fail(BCH_ECUDA, std::string("copy in: ") + cudaGetErrorString(e));
    const float *cl = zc ? llr_d + size_t(f0) * d->ld : S.llr;
    uint64_t *ch = zc ? hard_d + size_t(f0) * d->W64 : S.hard;
    uint8_t *ci = zc && iters_d ? iters_d + f0 : S.iters;
    uint8_t *cf = zc && flags_d ? flags_d + f0 : S.flags;
    bch_status s = BCH_OK;
    if (d->params.n_autos > 0)
      s = bch_draw_automorphisms(n, d->params.n_autos, autos_seed, frame0 + uint64_t(f0), F, S.autos, st);
    if (s != BCH_OK) return s;
    if (d->std_code)
      s = bch_hybrid_decode(d->code, d->std_code, &d->params, cl, d->ld, F, S.autos, ch, ci, cf, S.y, nullptr,
                            nullptr, S.ws, st);
    else
      s = bch_nms_decode(d->code, &d->params, cl, d->ld, F, S.autos, ch, ci, cf, nullptr, S.ws, st);
    if (s != BCH_OK) return s;
    mark(st);
    if (!zc) {
      e = cudaMemcpyAsync(hard + size_t(f0) * d->W64, S.hard, size_t(F) * d->W64 * 8, cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess && iters) e = cudaMemcpyAsync(iters + f0, S.iters, F, cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess && flags) e = cudaMemcpyAsync(flags + f0, S.flags, F, cudaMemcpyDeviceToHost, st);
      if (e != cudaSuccess) return fail(BCH_ECUDA, std::string("copy out: ") + cudaGetErrorString(e));
    }
    mark(st);
  }
  for (int b = 0; b < 2; b++) {
    cudaError_t e = cudaStreamSynchronize(d->st[b]);
    if (e != cudaSuccess) return fail(BCH_ECUDA, std::string("decoder: ") + cudaGetErrorString(e));
  }
  if (d->timing) {
    d->tm.calls++;
    d->tm.chunks += nchunks;
    if (zc) d->tm.in_place_chunks += nchunks;
    d->tm.ms_wall +=
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_wall).count();
    double *acc[3] = {&d->tm.ms_h2d, &d->tm.ms_decode, &d->tm.ms_d2h};
    for (size_t c = 0; c + 4 <= ev.size(); c += 4)
      for (int q = 0; q < 3; q++) {
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, ev[c + q], ev[c + q + 1]) == cudaSuccess) *acc[q] += ms;
      }
  }
  return BCH_OK;
}

bch_status bch_decoder_set_timing(bch_decoder *d, int on) {
  if (!d) return fail(BCH_EINVAL, "null decoder");
  d->timing = on != 0;
  d->tm = bch_decoder_timing{};
  return BCH_OK;
}

bch_status bch_decoder_set_in_place(bch_decoder *d, int on) {
  if (!d) return fail(BCH_EINVAL, "null decoder");
  d->in_place = on != 0;
  return BCH_OK;
}

bch_status bch_decoder_get_timing(const bch_decoder *d, bch_decoder_timing *out) {
  if (!d || !out) return fail(BCH_EINVAL, "null argument");
  *out = d->tm;
  return BCH_OK;
}

void bch_decoder_destroy(bch_decoder *d) {
  if (!d) return;
  cudaStreamSynchronize(d->st[0]);
  cudaStreamSynchronize(d->st[1]);
  free_decoder(d);
}

}  // extern "C"
