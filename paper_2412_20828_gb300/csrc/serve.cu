// Continuous-batching server: requests of mixed codes and sizes are admitted into a
// persistent kernel as slots and HBM free up, and their frames are decoded by the
// hybrid decoder (enhanced NMS, OSD on the frames it fails) while other requests are
// already on the GPU.
//
// Device side: one warp per block; each lane decodes one frame at a time and, when
// its frame stops, takes the next unclaimed frame of the warp's code (requests of a
// code are published to that code's ring; claims are generation-checked CAS on a
// per-request counter and may span requests), so lanes never wait for a chunk's
// slowest frame.  A warp binds to one code while any lane has a frame and picks a
// code with published work when all its lanes are idle.  New frames are loaded by
// the whole warp with coalesced reads past L1.  Frames whose syndrome stays nonzero
// get OSD from the whole warp; after a warp barrier the finished frames are added to
// their requests' done counters (one atomic per request and warp), and the add that
// completes a request posts a completion record to a ring in host-mapped memory.
// Every wait is bounded: idle warps sleep and the kernel exits after `idle_exit_us`
// without work (the host relaunches it), and a stop flag ends it at the next
// iteration.  The loop itself is in serve_device.cuh; this file holds the host side
// and the precompiled kernel (the one specialised to a server's codes is generated
// at run time by jit.cpp).
//
// The automorphisms of a frame are drawn inside the kernel from (seed, frame index):
// admission launches no kernel, because the persistent kernel holds every SM's shared
// memory and a second kernel would not be scheduled until it exits.
//
// Host side: admission against the HBM budget (first-fit arena of 256-byte units),
// a FIFO of requests waiting for memory or a slot, submission through a host-mapped
// ring, completion polling, result fetch (which frees the request's memory).
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <random>
#include <string>
#include <thread>
#include <vector>

#include "bch_kernels.cuh"
#include "osd_device.cuh"
#include "serve_device.cuh"

using namespace bchlib;

namespace bchlib {

// P automorphism copies of one enhanced-NMS iteration for this lane's frame (rows of
// the warp's code read from global memory; columns of stride 32 in shared memory).
template <int WB>
__device__ __noinline__ void srv_copies(const SrvCode &cd, int P, float *y, float *acc, const uint32_t *ctx,
                                        float alpha) {
  SmemTables tb;
  tb.codes = const_cast<uint16_t *>(cd.dc.codes);
  tb.grp = const_cast<GroupDesc *>(cd.grp);
  tb.rowmask = reinterpret_cast<uint4 *>(const_cast<uint32_t *>(cd.dc.rowmask));
  tb.alpha = nullptr;
  tb.state = nullptr;
  const uint32_t n = uint32_t(cd.dc.n), m = uint32_t(cd.dc.m);
  for (int p = 0; p < P; p++) {
    const uint32_t cx = ctx[p * 32];
    enh_copy<kFP32, WB>(tb, cd.dc.n_groups, n, m, y, acc, cx & 0xffu, cx >> 8, 32u, alpha);
  }
}

// The precompiled copies: the code's rows read from its device tables.
struct SrvGenericCopies {
  __device__ __forceinline__ void operator()(int, const SrvCode &cd, int P, float *y, float *acc, float *,
                                             const uint32_t *ctx, float alpha) const {
    switch (cd.wb) {
      case 8: srv_copies<8>(cd, P, y, acc, ctx, alpha); break;
      case 16: srv_copies<16>(cd, P, y, acc, ctx, alpha); break;
      case 24: srv_copies<24>(cd, P, y, acc, ctx, alpha); break;
      case 32: srv_copies<32>(cd, P, y, acc, ctx, alpha); break;
      default: srv_copies<48>(cd, P, y, acc, ctx, alpha); break;
    }
  }
};

// The precompiled serving kernel (BCHDEC_NMS_KERNEL=generic, or when the specialised
// one cannot be compiled).
__global__ void __launch_bounds__(32) serve_kernel(const SrvArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  serve_loop(a, smem, SrvGenericCopies());
}

}  // namespace bchlib

// ------------------------------------------------------------------------- host side
namespace bchlib {
cudaKernel_t jit_serve_kernel(const bch_code *const *codes, int n_codes, std::string *err);
cudaKernel_t jit_serve_blocks_kernel(const bch_code *const *codes, int n_codes, std::string *err);
}  // namespace bchlib

struct bch_server {
  bch_server_config cfg{};
  std::vector<const bch_code *> codes, std_codes;
  std::vector<float> alpha;
  SrvArgs args{};
  cudaStream_t kst = nullptr, cst = nullptr;
  SrvShared *sh = nullptr;  // host pointer of the mapped block
  unsigned *sub_ring = nullptr;
  SrvComp *comp = nullptr;
  SrvSlot *slots_dev = nullptr;
  SrvDev *dv = nullptr;
  GroupDesc *grp_dev = nullptr;
  SrvCode *codes_dev = nullptr;
  float *alpha_dev = nullptr;
  SrvCode codes_host[kSrvMaxCodes];
  unsigned char *arena = nullptr;
  size_t arena_bytes = 0;
  std::map<size_t, size_t> free_list;  // offset -> bytes
  struct Req {
    unsigned long long id;
    int code, F, ld;
    const float *llr;
    uint64_t seed, frame0;
    size_t off = 0, bytes = 0;
    int slot = -1;
    bool done = false;
    bool cancelled = false;  // in flight when cancelled: released on completion, not reported
  };
  std::deque<Req> pending;
  std::map<unsigned long long, Req> active;
  std::vector<int> free_slots;
  std::vector<unsigned> slot_gen;
  SrvSlot *slot_mirror = nullptr;         // pinned host copies of the slot descriptors
  std::vector<cudaEvent_t> slot_ev;       // per slot: its admission copies are done
  std::deque<std::pair<unsigned, int>> staged;  // (ring entry, code) with copies in flight
  long long published_open = 0;           // published requests not yet completed
  unsigned sub_tail[kSrvMaxCodes] = {};
  unsigned comp_read = 0;
  unsigned long long next_id = 1;
  int blocks = 0, threads = 32;
  size_t smem = 0;
  const void *kfn = nullptr;  // the serving kernel: specialised to the codes, or precompiled
  std::string kinfo;
  std::mutex mu;
  bch_server_stats stats{};
};

namespace {

size_t align256s(size_t x) { return (x + 255) & ~size_t(255); }

struct Layout {
  size_t llr, hard, iters, flags, total;
};

Layout req_layout(const bch_server *s, int code, int F, int ld) {
  Layout L;
  const int W64 = (s->codes[code]->alg.n + 63) / 64;
  size_t off = 0;
  L.llr = off;
  off = align256s(off + size_t(F) * ld * 4);
  L.hard = off;
  off = align256s(off + size_t(F) * W64 * 8);
  L.iters = off;
  off = align256s(off + size_t(F));
  L.flags = off;
  off = align256s(off + size_t(F));
  L.total = off;
  return L;
}

bool arena_alloc(bch_server *s, size_t bytes, size_t *off) {
  for (auto it = s->free_list.begin(); it != s->free_list.end(); ++it) {
    if (it->second >= bytes) {
      *off = it->first;
      const size_t rest = it->second - bytes;
      const size_t noff = it->first + bytes;
      s->free_list.erase(it);
      if (rest) s->free_list[noff] = rest;
      return true;
    }
  }
  return false;
}

void arena_free(bch_server *s, size_t off, size_t bytes) {
  auto it = s->free_list.emplace(off, bytes).first;
  auto nx = std::next(it);
  if (nx != s->free_list.end() && it->first + it->second == nx->first) {
    it->second += nx->second;
    s->free_list.erase(nx);
  }
  if (it != s->free_list.begin()) {
    auto pv = std::prev(it);
    if (pv->first + pv->second == it->first) {
      pv->second += it->second;
      s->free_list.erase(it);
    }
  }
}

// Returns a finished request's arena memory and slot (the kernel no longer touches it).
void release_request(bch_server *s, std::map<unsigned long long, bch_server::Req>::iterator it) {
  arena_free(s, it->second.off, it->second.bytes);
  s->stats.bytes_in_use -= it->second.bytes;
  s->free_slots.push_back(it->second.slot);
  s->active.erase(it);
}

// Waits for stream `st` for at most `limit_s` seconds (no unbounded host wait on the
// persistent kernel or the copies): BCH_ETIMEOUT, with the server's state in the
// message, when it is still busy.
bch_status wait_stream(bch_server *s, cudaStream_t st, double limit_s, const char *what) {
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    const cudaError_t e = cudaStreamQuery(st);
    if (e == cudaSuccess) return BCH_OK;
    if (e != cudaErrorNotReady) return fail(BCH_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
    if (std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count() > limit_s) {
      // device counters, read on the legacy stream (the server's streams do not
      // block on it)
      SrvDev dv{};
      cudaMemcpy(&dv, s->dv, sizeof(dv), cudaMemcpyDeviceToHost);
      char msg[320];
      std::snprintf(msg, sizeof(msg),
                    "%s: still busy after %.0f s (running %u, live warps %u, completions %u, published open %lld, "
                    "pending %zu)",
                    what, limit_s, unsigned(s->sh->running), dv.live, dv.comp_tail, s->published_open,
                    s->pending.size());
      return fail(BCH_ETIMEOUT, msg);
    }
    // copies finish in microseconds: yield first, sleep only on long waits
    if (std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count() < 1e-3)
      std::this_thread::yield();
    else
      std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
}

bch_status launch_server_kernel(bch_server *s) {
  s->sh->running = 1;
  s->args.dv = s->dv;
  cudaError_t e = cudaMemsetAsync(&s->dv->live, 0, sizeof(unsigned), s->kst);
  if (e == cudaSuccess) {
    void *args[] = {&s->args};
    note_launch();
    e = cudaLaunchKernel(s->kfn, dim3(unsigned(s->blocks)), dim3(unsigned(s->threads)), args, s->smem, s->kst);
  }
  if (e != cudaSuccess) {
    s->sh->running = 0;
    return fail(BCH_ECUDA, std::string("serve kernel: ") + cudaGetErrorString(e));
  }
  return BCH_OK;
}

bch_status ensure_running(bch_server *s) {
  if (s->published_open > 0 && !s->sh->running) {
    // a previous instance that exited idle has finished (its last warp cleared the
    // flag on the way out)
    bch_status st = wait_stream(s, s->kst, 30.0, "serve kernel exit");
    if (st != BCH_OK) return st;
    st = launch_server_kernel(s);
    if (st != BCH_OK) return st;
    s->stats.kernel_launches++;
  }
  return BCH_OK;
}

// Publishes, in admission order, the staged requests whose copies have landed: their
// ring entries become visible to the kernel.  Caller holds the lock.
bch_status publish_staged(bch_server *s) {
  bool any = false;
  while (!s->staged.empty()) {
    const unsigned entry = s->staged.front().first;
    const int code = s->staged.front().second;
    const cudaError_t e = cudaEventQuery(s->slot_ev[entry & 0xffffu]);
    if (e == cudaErrorNotReady) break;
    if (e != cudaSuccess) return fail(BCH_ECUDA, std::string("admission copies: ") + cudaGetErrorString(e));
    const unsigned R = unsigned(s->cfg.max_requests);
    s->sub_ring[size_t(code) * R + s->sub_tail[code] % R] = entry;
    std::atomic_thread_fence(std::memory_order_release);
    s->sub_tail[code]++;
    s->sh->sub_tail[code] = s->sub_tail[code];
    s->staged.pop_front();
    s->published_open++;
    any = true;
  }
  std::atomic_thread_fence(std::memory_order_seq_cst);
  return any ? ensure_running(s) : BCH_OK;
}

// Admits a request: memory, slot, asynchronous copies of its LLRs and descriptor, then
// staging for publication once the copies are done (no host wait).  Caller holds the
// lock.
bch_status admit(bch_server *s, bch_server::Req &r, bool *admitted) {
  *admitted = false;
  if (s->free_slots.empty()) return BCH_OK;
  const Layout L = req_layout(s, r.code, r.F, r.ld);
  size_t off = 0;
  if (!arena_alloc(s, L.total, &off)) return BCH_OK;
  r.off = off;
  r.bytes = L.total;
  r.slot = s->free_slots.back();
  s->free_slots.pop_back();
  unsigned char *base = s->arena + off;
  SrvSlot &sl = s->slot_mirror[r.slot];  // no copy from this slot is in flight: it was free
  std::memset(&sl, 0, sizeof(sl));
  sl.llr = reinterpret_cast<const float *>(base + L.llr);
  sl.seed = r.seed;
  sl.frame0 = r.frame0;
  sl.hard = reinterpret_cast<uint64_t *>(base + L.hard);
  sl.iters = base + L.iters;
  sl.flags = base + L.flags;
  sl.id = r.id;
  sl.code = r.code;
  sl.F = r.F;
  sl.ld = r.ld;
  const unsigned gen = (s->slot_gen[r.slot] + 1) & 0xffffu;
  s->slot_gen[r.slot] = gen;
  sl.claim = (unsigned long long)gen << 32;
  sl.done = 0;
  cudaError_t e = cudaMemcpyAsync(const_cast<float *>(sl.llr), r.llr, size_t(r.F) * r.ld * 4, cudaMemcpyDefault,
                                  s->cst);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(s->slots_dev + r.slot, &sl, sizeof(sl), cudaMemcpyHostToDevice, s->cst);
  if (e == cudaSuccess) e = cudaEventRecord(s->slot_ev[r.slot], s->cst);
  if (e != cudaSuccess) return fail(BCH_ECUDA, std::string("admission copies: ") + cudaGetErrorString(e));
  s->staged.emplace_back(unsigned(r.slot) | (gen << 16), r.code);
  s->stats.admitted++;
  s->stats.bytes_in_use += L.total;
  *admitted = true;
  return publish_staged(s);
}

bch_status admit_pending(bch_server *s) {
  while (!s->pending.empty()) {
    bool ok = false;
    bch_server::Req r = s->pending.front();
    bch_status st = admit(s, r, &ok);
    if (st != BCH_OK) return st;
    if (!ok) break;
    s->pending.pop_front();
    s->active[r.id] = r;
  }
  return BCH_OK;
}

}  // namespace

extern "C" {

bch_status bch_server_create(const bch_server_config *cfg, bch_server **out) {
  if (!cfg || !out) return fail(BCH_EINVAL, "null argument");
  *out = nullptr;
  if (cfg->n_codes < 1 || cfg->n_codes > kSrvMaxCodes || !cfg->codes)
    return fail(BCH_EINVAL, "n_codes must be in [1, 8]");
  if (cfg->iters < 1 || cfg->iters > 32 || !cfg->alpha || cfg->n_autos < 1 || cfg->n_autos > 9 ||
      cfg->osd_order < 0 || cfg->osd_order > 2 || cfg->max_requests < 1 || cfg->budget_bytes < 4096)
    return fail(BCH_EINVAL, "bad server configuration");
  bch_server *s = new (std::nothrow) bch_server();
  if (!s) return fail(BCH_ENOMEM, "host allocation");
  s->cfg = *cfg;
  s->alpha.assign(cfg->alpha, cfg->alpha + cfg->iters);
  s->cfg.alpha = s->alpha.data();
  s->codes.assign(cfg->codes, cfg->codes + cfg->n_codes);
  s->std_codes.assign(cfg->n_codes, nullptr);
  if (cfg->std_codes) s->std_codes.assign(cfg->std_codes, cfg->std_codes + cfg->n_codes);
  s->cfg.codes = nullptr;
  s->cfg.std_codes = nullptr;
  auto cleanup = [s]() {
    if (s->kst) cudaStreamDestroy(s->kst);
    if (s->cst) cudaStreamDestroy(s->cst);
    if (s->sh) cudaFreeHost(s->sh);
    if (s->slot_mirror) cudaFreeHost(s->slot_mirror);
    for (cudaEvent_t ev : s->slot_ev) cudaEventDestroy(ev);
    cudaFree(s->slots_dev);
    cudaFree(s->dv);
    cudaFree(s->grp_dev);
    cudaFree(s->codes_dev);
    cudaFree(s->alpha_dev);
    cudaFree(s->arena);
    delete s;
  };
  SrvArgs &A = s->args;
  std::memset(&A, 0, sizeof(A));
  A.n_codes = cfg->n_codes;
  const int R = cfg->max_requests;
  // host-mapped control block, submission ring and completion ring in one allocation
  const size_t ring_off = 64;
  const size_t comp_off = (ring_off + size_t(kSrvMaxCodes) * R * 4 + 63) & ~size_t(63);
  const size_t shared_bytes = comp_off + size_t(R) * sizeof(SrvComp);
  void *hp = nullptr;
  if (cudaHostAlloc(&hp, shared_bytes, cudaHostAllocMapped) != cudaSuccess) {
    cleanup();
    return fail(BCH_ENOMEM, "mapped host memory");
  }
  std::memset(hp, 0, shared_bytes);
  s->sh = static_cast<SrvShared *>(hp);
  s->sub_ring = reinterpret_cast<unsigned *>(static_cast<unsigned char *>(hp) + ring_off);
  s->comp = reinterpret_cast<SrvComp *>(static_cast<unsigned char *>(hp) + comp_off);
  void *dsh = nullptr;
  if (cudaHostGetDevicePointer(&dsh, hp, 0) != cudaSuccess) {
    cleanup();
    return fail(BCH_ECUDA, "mapped device pointer");
  }
  A.sh = static_cast<SrvShared *>(dsh);
  A.sub_ring = reinterpret_cast<unsigned *>(static_cast<unsigned char *>(dsh) + ring_off);
  A.comp = reinterpret_cast<SrvComp *>(static_cast<unsigned char *>(dsh) + comp_off);
  A.ring = R;
  A.iters = cfg->iters;
  A.P = cfg->n_autos;
  A.order = cfg->osd_order;
  A.early_stop = 1;
  A.idle_ns = (unsigned long long)(cfg->idle_exit_us ? cfg->idle_exit_us : 200000) * 1000ull;
  if (cudaMalloc(&s->codes_dev, sizeof(SrvCode) * kSrvMaxCodes) != cudaSuccess ||
      cudaMalloc(&s->alpha_dev, sizeof(float) * 32) != cudaSuccess) {
    cleanup();
    return fail(BCH_ENOMEM, "server tables");
  }
  {
    float al[32];
    for (int t = 0; t < 32; t++) al[t] = t < cfg->iters ? cfg->alpha[t] : 0.0f;
    cudaMemcpy(s->alpha_dev, al, sizeof(al), cudaMemcpyHostToDevice);
  }
  std::memset(s->codes_host, 0, sizeof(s->codes_host));
  if (cudaMalloc(&s->slots_dev, sizeof(SrvSlot) * R) != cudaSuccess ||
      cudaMalloc(&s->dv, sizeof(SrvDev)) != cudaSuccess ||
      cudaMalloc(&s->grp_dev, sizeof(GroupDesc) * kMaxGroups * kSrvMaxCodes) != cudaSuccess) {
    cleanup();
    return fail(BCH_ENOMEM, "server tables");
  }
  cudaMemset(s->slots_dev, 0, sizeof(SrvSlot) * R);
  cudaMemset(s->dv, 0, sizeof(SrvDev));
  std::vector<GroupDesc> grp(size_t(kMaxGroups) * kSrvMaxCodes);
  for (int c = 0; c < cfg->n_codes; c++) {
    const bch_code *co = s->codes[c];
    const bch_code *sc = s->std_codes[c];
    if (!co || !co->dev_dc) {
      cleanup();
      return fail(BCH_EINVAL, "null code in the server configuration");
    }
    if (sc && (sc->kind != BCH_PCM_STANDARD || sc->alg.n != co->alg.n || sc->alg.k != co->alg.k ||
               sc->alg.n - sc->alg.k > 64)) {
      cleanup();
      return fail(BCH_EINVAL, "std_codes[i] must be the standard matrix of codes[i]");
    }
    SrvCode &sc_ = s->codes_host[c];
    sc_.dc = co->dc;
    for (int g = 0; g < kMaxGroups; g++) {
      GroupDesc d{};
      d.w = co->dc.group_w[g];
      d.rows = co->dc.group_rows[g];
      d.off = co->dc.group_off[g];
      grp[size_t(c) * kMaxGroups + g] = d;
    }
    sc_.grp = s->grp_dev + size_t(c) * kMaxGroups;
    sc_.std_cols = sc ? sc->dc.colmask : nullptr;
    sc_.M = sc ? sc->alg.n - sc->alg.k : 0;
    sc_.has_osd = sc ? 1 : 0;
    sc_.ord = 1;
    for (int x = 2 % co->alg.n; x != 1; x = (2 * x) % co->alg.n) sc_.ord++;
    const int mw = co->dc.max_w;
    sc_.wb = mw <= 8 ? 8 : mw <= 16 ? 16 : mw <= 24 ? 24 : mw <= 32 ? 32 : mw <= 48 ? 48 : 0;
    if (!sc_.wb) {
      cleanup();
      return fail(BCH_EINVAL, "row weight above 48");
    }
  }
  cudaMemcpy(s->grp_dev, grp.data(), sizeof(GroupDesc) * grp.size(), cudaMemcpyHostToDevice);
  cudaMemcpy(s->codes_dev, s->codes_host, sizeof(SrvCode) * kSrvMaxCodes, cudaMemcpyHostToDevice);
  A.codes = s->codes_dev;
  A.alpha = s->alpha_dev;
  s->arena_bytes = cfg->budget_bytes & ~size_t(255);
  if (cudaMalloc(&s->arena, s->arena_bytes) != cudaSuccess) {
    cleanup();
    return fail(BCH_ENOMEM, "HBM budget arena");
  }
  s->free_list[0] = s->arena_bytes;
  if (R > 65535) {
    cleanup();
    return fail(BCH_EINVAL, "max_requests above 65535");
  }
  for (int i = R - 1; i >= 0; i--) s->free_slots.push_back(i);
  s->slot_gen.assign(R, 0);
  if (cudaHostAlloc(reinterpret_cast<void **>(&s->slot_mirror), sizeof(SrvSlot) * R, cudaHostAllocDefault) !=
      cudaSuccess) {
    s->slot_mirror = nullptr;
    cleanup();
    return fail(BCH_ENOMEM, "pinned slot descriptors");
  }
  s->slot_ev.assign(R, nullptr);
  for (int i = 0; i < R; i++)
    if (cudaEventCreateWithFlags(&s->slot_ev[i], cudaEventDisableTiming) != cudaSuccess) {
      cleanup();
      return fail(BCH_ECUDA, "slot events");
    }
  A.slots = s->slots_dev;
  if (cudaStreamCreateWithFlags(&s->kst, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&s->cst, cudaStreamNonBlocking) != cudaSuccess) {
    cleanup();
    return fail(BCH_ECUDA, "streams");
  }
  // The serving kernel: by default the one compiled at run time with every code's rows
  // as straight-line code (cached in the process and on disk); the precompiled one
  // with BCHDEC_NMS_KERNEL=generic or when that compile fails (unless =jit).
  const char *mode = std::getenv("BCHDEC_NMS_KERNEL");
  A.scr_words = 0;
  s->kfn = reinterpret_cast<const void *>(serve_kernel);
  s->kinfo = "generic: selected by BCHDEC_NMS_KERNEL";
  if (!mode || std::strcmp(mode, "generic") != 0) {
    std::string err;
    cudaKernel_t k = jit_serve_kernel(s->codes.data(), cfg->n_codes, &err);
    if (k) {
      s->kfn = reinterpret_cast<const void *>(k);
      s->kinfo = "jit";
      for (const bch_code *co : s->codes)
        if (co->alg.n > 63) A.scr_words = std::max(A.scr_words, co->alg.n);
    } else if (mode && std::strcmp(mode, "jit") == 0) {
      cleanup();
      return fail(BCH_ECUDA, "serving kernel: " + err);
    } else {
      s->kinfo = "generic: " + err;
    }
  }
  // per warp: y and accumulator columns (128 x 32 FP32 each), scratch columns, OSD
  // scratch, automorphism parameters [9][32], claim segments [3][32]
  s->smem = sizeof(float) * 128 * 32 * 2 + sizeof(float) * size_t(A.scr_words) * 32 + sizeof(OsdSmem) +
            sizeof(uint32_t) * 9 * 32 + sizeof(int) * 3 * 32;
  s->threads = 32;
  // The block-bound serving kernel (default unless BCHDEC_SERVE_KERNEL=warps or the
  // precompiled kernel is selected): one 256-thread block per SM, bound to one code per
  // session, with the batch kernels' mappings.
  const char *sk = std::getenv("BCHDEC_SERVE_KERNEL");
  if (s->kinfo == "jit" && !(sk && std::strcmp(sk, "warps") == 0)) {
    A.blk_max_rows = 0;
    A.blk_flat_n = 0;
    A.blk_R = 16;
    for (const bch_code *co : s->codes) {
      A.blk_max_rows = std::max(A.blk_max_rows, int(co->rows.size()));
      if (co->alg.n <= 63) A.blk_flat_n = std::max(A.blk_flat_n, co->alg.n);
    }
    const SrvBlockLayout BL = srv_block_layout(A.blk_max_rows, A.blk_flat_n, A.P, A.blk_R, 127);
    std::string err;
    cudaKernel_t k = BL.total <= 227 * 1024 ? jit_serve_blocks_kernel(s->codes.data(), cfg->n_codes, &err) : nullptr;
    if (k) {
      s->kfn = reinterpret_cast<const void *>(k);
      s->kinfo = "jit-blocks";
      s->smem = BL.total;
      s->threads = kSrvBlockThreads;
    }
  }
  int sms = 0, per_sm = 0;
  if (launch_geometry(s->kfn, s->threads, s->smem, &sms, &per_sm) != cudaSuccess || per_sm < 1) {
    cleanup();
    return fail(BCH_ECUDA, "serve kernel attributes");
  }
  s->blocks = s->threads > 32 ? sms : (cfg->warps > 0 ? cfg->warps : sms * per_sm);
  // the set-up copies and clears above ran on the legacy stream: wait for those alone,
  // not for the device (another server's persistent kernel may be resident and busy)
  if (cudaStreamSynchronize(cudaStreamLegacy) != cudaSuccess) {
    cleanup();
    return fail(BCH_ECUDA, "server set-up copies");
  }
  *out = s;
  return BCH_OK;
}

bch_status bch_server_submit(bch_server *s, int code_id, const float *llr, int ld, int n_frames,
                             uint64_t autos_seed, uint64_t frame0, uint64_t *request_id) {
  if (!s || !llr || !request_id) return fail(BCH_EINVAL, "null argument");
  if (code_id < 0 || code_id >= int(s->codes.size())) return fail(BCH_EINVAL, "bad code id");
  if (n_frames < 1 || (s->cfg.max_frames_per_request > 0 && n_frames > s->cfg.max_frames_per_request) ||
      ld < s->codes[code_id]->alg.n)
    return fail(BCH_EINVAL, "bad request size");
  std::lock_guard<std::mutex> lk(s->mu);
  const Layout L = req_layout(s, code_id, n_frames, ld);
  if (L.total > s->arena_bytes) return fail(BCH_EBUDGET, "request larger than the HBM budget");
  bch_server::Req r;
  r.id = s->next_id++;
  r.code = code_id;
  r.F = n_frames;
  r.ld = ld;
  r.llr = llr;
  r.seed = autos_seed;
  r.frame0 = frame0;
  *request_id = r.id;
  s->stats.submitted++;
  if (s->pending.empty()) {
    bool ok = false;
    bch_status st = admit(s, r, &ok);
    if (st != BCH_OK) return st;
    if (ok) {
      s->active[r.id] = r;
      return BCH_OK;
    }
  }
  s->pending.push_back(r);
  s->stats.queued++;
  return BCH_OK;
}

bch_status bch_server_poll(bch_server *s, uint64_t *done_ids, int max_ids, int *n_done, int timeout_us) {
  if (!s || !done_ids || !n_done || max_ids < 1) return fail(BCH_EINVAL, "bad argument");
  *n_done = 0;
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    {
      std::lock_guard<std::mutex> lk(s->mu);
      while (*n_done < max_ids) {
        SrvComp *c = s->comp + (s->comp_read % unsigned(s->cfg.max_requests));
        if (*reinterpret_cast<volatile unsigned *>(&c->seq) != s->comp_read + 1) break;
        std::atomic_thread_fence(std::memory_order_acquire);
        const unsigned long long id = c->id;
        s->comp_read++;
        auto it = s->active.find(id);
        s->published_open--;
        s->stats.completed++;
        if (it != s->active.end() && it->second.cancelled) {
          // the kernel is done with a cancelled request: release it, report nothing
          release_request(s, it);
          continue;
        }
        if (it != s->active.end()) it->second.done = true;
        done_ids[(*n_done)++] = id;
      }
      bch_status st = admit_pending(s);
      if (st == BCH_OK) st = publish_staged(s);
      // a kernel instance that exited idle while published work is open: relaunch
      if (st == BCH_OK) st = ensure_running(s);
      if (st != BCH_OK) return st;
    }
    if (*n_done > 0 || timeout_us <= 0) break;
    const auto el = std::chrono::duration_cast<std::chrono::microseconds>(std::chrono::steady_clock::now() - t0);
    if (el.count() >= timeout_us) break;
    std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
  cudaError_t e = cudaStreamQuery(s->kst);
  if (e != cudaSuccess && e != cudaErrorNotReady)
    return fail(BCH_ECUDA, std::string("serve kernel: ") + cudaGetErrorString(e));
  return BCH_OK;
}

bch_status bch_server_fetch(bch_server *s, uint64_t id, uint64_t *hard, uint8_t *iters, uint8_t *flags) {
  if (!s || !hard) return fail(BCH_EINVAL, "null argument");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->active.find(id);
  if (it == s->active.end() || !it->second.done) return fail(BCH_EINVAL, "request not complete or unknown");
  bch_server::Req r = it->second;
  const Layout L = req_layout(s, r.code, r.F, r.ld);
  const int W64 = (s->codes[r.code]->alg.n + 63) / 64;
  unsigned char *base = s->arena + r.off;
  cudaError_t e = cudaMemcpyAsync(hard, base + L.hard, size_t(r.F) * W64 * 8, cudaMemcpyDefault, s->cst);
  if (e == cudaSuccess && iters) e = cudaMemcpyAsync(iters, base + L.iters, size_t(r.F), cudaMemcpyDefault, s->cst);
  if (e == cudaSuccess && flags) e = cudaMemcpyAsync(flags, base + L.flags, size_t(r.F), cudaMemcpyDefault, s->cst);
  if (e != cudaSuccess) return fail(BCH_ECUDA, std::string("fetch: ") + cudaGetErrorString(e));
  bch_status ws = wait_stream(s, s->cst, 30.0, "fetch copies");
  if (ws != BCH_OK) return ws;
  release_request(s, it);
  return admit_pending(s);
}

bch_status bch_server_cancel(bch_server *s, uint64_t id) {
  if (!s) return fail(BCH_EINVAL, "null server");
  std::lock_guard<std::mutex> lk(s->mu);
  for (auto it = s->pending.begin(); it != s->pending.end(); ++it)
    if (it->id == id) {  // never admitted: nothing on the device
      s->pending.erase(it);
      s->stats.cancelled++;
      return BCH_OK;
    }
  auto it = s->active.find(id);
  if (it == s->active.end() || it->second.cancelled) return fail(BCH_EINVAL, "unknown request");
  s->stats.cancelled++;
  if (it->second.done) {  // complete but not fetched
    release_request(s, it);
    return admit_pending(s);
  }
  it->second.cancelled = true;  // in flight: released when the kernel completes it
  return BCH_OK;
}

bch_status bch_server_kernel_info(bch_server *s, char *buf, size_t capacity) {
  if (!s || !buf || capacity == 0) return fail(BCH_EINVAL, "bad argument");
  std::snprintf(buf, capacity, "%s", s->kinfo.c_str());
  return BCH_OK;
}

bch_status bch_server_get_stats(bch_server *s, bch_server_stats *out) {
  if (!s || !out) return fail(BCH_EINVAL, "null argument");
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->stats;
  out->pending = (long long)s->pending.size();
  out->in_flight = (long long)s->active.size();
  return BCH_OK;
}

void bch_server_destroy(bch_server *s) {
  if (!s) return;
  s->sh->stop = 1;
  std::atomic_thread_fence(std::memory_order_seq_cst);
  // the kernel leaves at its next iteration; if it does not, its memory stays
  // allocated (freeing it under a running kernel would fault) and the error is kept
  if (wait_stream(s, s->kst, 30.0, "serve kernel stop") != BCH_OK ||
      wait_stream(s, s->cst, 30.0, "server copies") != BCH_OK)
    return;
  cudaStreamDestroy(s->kst);
  cudaStreamDestroy(s->cst);
  cudaFreeHost(s->sh);
  if (s->slot_mirror) cudaFreeHost(s->slot_mirror);
  for (cudaEvent_t ev : s->slot_ev) cudaEventDestroy(ev);
  cudaFree(s->slots_dev);
  cudaFree(s->dv);
  cudaFree(s->grp_dev);
  cudaFree(s->codes_dev);
  cudaFree(s->alpha_dev);
  cudaFree(s->arena);
  delete s;
}


// --------------------------------------------------------------------- benchmark
// Open-loop load generator: Poisson arrivals at rate_rps for duration_s; each request
// draws a code uniformly, a size F = floor(exp(u ln(max_frames + 1))) clipped to
// [1, max_frames] (log-uniform) and a contiguous range of that code's frame pool.
// Latency = scheduled arrival -> results in host memory.  static_batching = 1 runs the
// same arrival stream through plain batched launches instead of the server: requests
// are collected until batch_us after the first one or batch_frames frames, then every
// code's share is copied in, hybrid-decoded with one bch_hybrid_decode call and copied
// back before the batch's requests complete.  Without standard matrices or with
// osd_order = 0 the batches run the NMS decoder alone (n_autos = 0: the plain decoder).
bch_status bch_serve_bench(bch_server *srv, const bch_serve_bench_config *c, bch_serve_bench_result *res) {
  if (!c || !res || !c->pools || !c->pool_frames || !c->lds || !c->codes || c->n_codes < 1 ||
      c->n_codes > kSrvMaxCodes || c->rate_rps <= 0 || c->duration_s <= 0 || c->max_frames < 1)
    return fail(BCH_EINVAL, "bad benchmark configuration");
  if (!c->static_batching && !srv) return fail(BCH_EINVAL, "server required");
  std::memset(res, 0, sizeof(*res));
  using clk = std::chrono::steady_clock;
  std::mt19937_64 rng(c->seed);
  std::exponential_distribution<double> gap(c->rate_rps);
  std::uniform_real_distribution<double> uni(0.0, 1.0);
  struct Rq {
    int code, F, off;
    double t_arr;
    uint64_t id;
  };
  // pre-draw the arrival stream
  std::vector<Rq> reqs;
  double t = 0.0;
  long long offered_frames = 0;
  for (;;) {
    t += gap(rng);
    if (t > c->duration_s) break;
    Rq r;
    r.code = int(uni(rng) * c->n_codes) % c->n_codes;
    int F = int(std::floor(std::exp(uni(rng) * std::log(double(c->max_frames) + 1.0))));
    F = std::max(1, std::min(F, c->max_frames));
    F = std::min(F, c->pool_frames[r.code]);
    r.F = F;
    r.off = int(uni(rng) * double(c->pool_frames[r.code] - F + 1));
    r.t_arr = t;
    r.id = 0;
    reqs.push_back(r);
    offered_frames += F;
  }
  // results land in pinned host memory, as a latency-sensitive caller would have them
  struct Pinned {
    void *p = nullptr;
    explicit Pinned(size_t b) {
      if (cudaHostAlloc(&p, b, cudaHostAllocDefault) != cudaSuccess) p = nullptr;
    }
    ~Pinned() {
      if (p) cudaFreeHost(p);
    }
  };
  const size_t maxF = size_t(c->max_frames);
  const size_t capF = size_t(std::max(c->batch_frames, c->max_frames) + c->max_frames);
  Pinned hpin(capF * 16 * size_t(c->n_codes)), ipin(capF * size_t(c->n_codes)), fpin(capF * size_t(c->n_codes));
  if (!hpin.p || !ipin.p || !fpin.p) return fail(BCH_ENOMEM, "pinned result buffers");
  uint64_t *hbuf = static_cast<uint64_t *>(hpin.p);
  uint8_t *ibuf = static_cast<uint8_t *>(ipin.p), *fbuf = static_cast<uint8_t *>(fpin.p);
  (void)maxF;
  std::vector<double> lat;
  lat.reserve(reqs.size());
  long long frames_done = 0;
  const auto t0 = clk::now();
  auto now_s = [&]() { return std::chrono::duration<double>(clk::now() - t0).count(); };
  if (!c->static_batching) {
    std::map<uint64_t, size_t> by_id;
    size_t next = 0, done = 0;
    std::vector<uint64_t> ids(256);
    while (done < reqs.size()) {
      const double tn = now_s();
      while (next < reqs.size() && reqs[next].t_arr <= tn) {
        Rq &r = reqs[next];
        const float *src = c->pools[r.code] + size_t(r.off) * c->lds[r.code];
        bch_status st = bch_server_submit(srv, r.code, src, c->lds[r.code], r.F, c->seed ^ 0x5A5Aull,
                                          uint64_t(r.off), &r.id);
        if (st != BCH_OK) return st;
        by_id[r.id] = next;
        next++;
      }
      int nd = 0;
      bch_status st = bch_server_poll(srv, ids.data(), int(ids.size()), &nd, 0);
      if (st != BCH_OK) return st;
      for (int i = 0; i < nd; i++) {
        auto it = by_id.find(ids[i]);
        if (it == by_id.end()) continue;
        Rq &r = reqs[it->second];
        st = bch_server_fetch(srv, r.id, hbuf, ibuf, fbuf);
        if (st != BCH_OK) return st;
        lat.push_back(now_s() - r.t_arr);
        frames_done += r.F;
        done++;
        by_id.erase(it);
      }
      if (nd == 0 && next < reqs.size()) {
        const double wait = reqs[next].t_arr - now_s();
        if (wait > 20e-6) std::this_thread::sleep_for(std::chrono::microseconds(10));
      }
      if (now_s() > c->duration_s * 10 + 30) return fail(BCH_ETIMEOUT, "server benchmark did not drain");
    }
  } else {
    // static batching: per code, a device batch buffer and a hybrid decode per batch
    const int nc = c->n_codes;
    std::vector<float *> dllr(nc, nullptr);
    std::vector<uint16_t *> daut(nc, nullptr);
    std::vector<uint64_t *> dhard(nc, nullptr);
    std::vector<uint8_t *> dit(nc, nullptr), dfl(nc, nullptr);
    std::vector<void *> dws(nc, nullptr);
    const int cap = std::max(c->batch_frames, c->max_frames) + c->max_frames;
    bch_nms_params p{};
    p.iters = c->iters;
    p.alpha = c->alpha;
    p.n_autos = c->n_autos;
    p.early_stop = 1;
    p.msg = BCH_MSG_FP32;
    p.osd_order = c->osd_order;
    // stream-ordered allocations: unlike cudaFree, cudaFreeAsync does not wait for the
    // whole device, where a server's persistent kernel may still be resident
    cudaStream_t st;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    auto release = [&]() {
      auto drop = [&](void *q) {
        if (q) cudaFreeAsync(q, st);
      };
      for (int k = 0; k < nc; k++) {
        drop(dllr[k]);
        drop(daut[k]);
        drop(dhard[k]);
        drop(dit[k]);
        drop(dfl[k]);
        drop(dws[k]);
      }
      cudaStreamSynchronize(st);
      cudaStreamDestroy(st);
    };
    for (int k = 0; k < nc; k++) {
      size_t wsb = 0;
      bch_workspace_size(c->codes[k], &p, cap, &wsb);
      if (cudaMallocAsync(reinterpret_cast<void **>(&dllr[k]), size_t(cap) * c->lds[k] * 4, st) != cudaSuccess ||
          cudaMallocAsync(reinterpret_cast<void **>(&daut[k]), size_t(cap) * p.n_autos * 2, st) != cudaSuccess ||
          cudaMallocAsync(reinterpret_cast<void **>(&dhard[k]), size_t(cap) * 16, st) != cudaSuccess ||
          cudaMallocAsync(reinterpret_cast<void **>(&dit[k]), cap, st) != cudaSuccess ||
          cudaMallocAsync(reinterpret_cast<void **>(&dfl[k]), cap, st) != cudaSuccess ||
          cudaMallocAsync(&dws[k], wsb, st) != cudaSuccess) {
        release();
        return fail(BCH_ENOMEM, "static batching buffers");
      }
    }
    size_t next = 0;
    bch_status sfail = BCH_OK;
    while (next < reqs.size()) {
      if (now_s() > c->duration_s * 10 + 30) {
        sfail = fail(BCH_ETIMEOUT, "static batching benchmark did not drain");
        break;
      }
      // wait for the first request of the batch, then collect
      double tn = now_s();
      if (reqs[next].t_arr > tn) {
        std::this_thread::sleep_for(std::chrono::microseconds(10));
        continue;
      }
      const double t_first = reqs[next].t_arr;
      size_t end = next;
      long long frames = 0;
      for (;;) {
        tn = now_s();
        while (end < reqs.size() && reqs[end].t_arr <= tn && frames < c->batch_frames) {
          frames += reqs[end].F;
          end++;
        }
        if (frames >= c->batch_frames || tn - t_first >= c->batch_us * 1e-6 || end == reqs.size()) break;
        std::this_thread::sleep_for(std::chrono::microseconds(5));
      }
      for (int k = 0; k < nc; k++) {
        int tot = 0;
        for (size_t q = next; q < end; q++) {
          const Rq &r = reqs[q];
          if (r.code != k) continue;
          cudaMemcpyAsync(dllr[k] + size_t(tot) * c->lds[k], c->pools[k] + size_t(r.off) * c->lds[k],
                          size_t(r.F) * c->lds[k] * 4, cudaMemcpyDefault, st);
          if (p.n_autos > 0)
            bch_draw_automorphisms(c->codes[k]->alg.n, p.n_autos, c->seed ^ 0x5A5Aull, uint64_t(r.off), r.F,
                                   daut[k] + size_t(tot) * p.n_autos, st);
          tot += r.F;
        }
        if (!tot) continue;
        // the hybrid decoder, or (no OSD) the NMS decoder alone -- with n_autos = 0 the
        // single plain decoder on the given matrices
        bch_status s2 = (c->std_codes && p.osd_order > 0)
                            ? bch_hybrid_decode(c->codes[k], c->std_codes[k], &p, dllr[k], c->lds[k], tot,
                                                daut[k], dhard[k], dit[k], dfl[k], nullptr, nullptr, nullptr,
                                                dws[k], st)
                            : bch_nms_decode(c->codes[k], &p, dllr[k], c->lds[k], tot,
                                             p.n_autos > 0 ? daut[k] : nullptr, dhard[k], dit[k], dfl[k],
                                             nullptr, dws[k], st);
        if (s2 != BCH_OK) {
          sfail = s2;
          break;
        }
        const int W64 = (c->codes[k]->alg.n + 63) / 64;
        cudaMemcpyAsync(hbuf + size_t(k) * capF * 2, dhard[k], size_t(tot) * W64 * 8, cudaMemcpyDeviceToHost, st);
        cudaMemcpyAsync(ibuf + size_t(k) * capF, dit[k], tot, cudaMemcpyDeviceToHost, st);
        cudaMemcpyAsync(fbuf + size_t(k) * capF, dfl[k], tot, cudaMemcpyDeviceToHost, st);
      }
      if (sfail != BCH_OK) break;
      if (cudaStreamSynchronize(st) != cudaSuccess) {
        sfail = fail(BCH_ECUDA, "static batch");
        break;
      }
      tn = now_s();
      for (size_t q = next; q < end; q++) {
        lat.push_back(tn - reqs[q].t_arr);
        frames_done += reqs[q].F;
      }
      next = end;
    }
    cudaStreamSynchronize(st);
    release();
    if (sfail != BCH_OK) return sfail;
  }
  const double el = now_s();
  std::sort(lat.begin(), lat.end());
  auto pct = [&](double q) { return lat.empty() ? 0.0 : lat[std::min(lat.size() - 1, size_t(q * lat.size()))]; };
  double mean = 0;
  for (double v : lat) mean += v;
  res->requests = (long long)lat.size();
  res->frames = frames_done;
  res->p50_ms = pct(0.50) * 1e3;
  res->p99_ms = pct(0.99) * 1e3;
  res->mean_ms = lat.empty() ? 0 : mean / lat.size() * 1e3;
  res->max_ms = lat.empty() ? 0 : lat.back() * 1e3;
  res->elapsed_s = el;
  res->served_frames_per_s = frames_done / el;
  res->offered_frames_per_s = offered_frames / c->duration_s;
  res->offered_requests_per_s = reqs.size() / c->duration_s;
  return BCH_OK;
}

}  // extern "C"
