// Device side of the continuous-batching server, shared by the precompiled serving
// kernel (nvcc) and the serving kernel compiled at run time for a server's codes
// (NVRTC): the control structures the host and the kernel share, the claim of frames
// from the per-code submission rings, and the persistent loop.  The loop is a template
// on the step that runs one iteration's automorphism copies for a lane's frame: the
// precompiled kernel reads the rows from the code's tables, the specialised one has
// every code's rows as straight-line code.
#pragma once
#ifndef __CUDACC_RTC__
#include <stdint.h>

#include "autos_device.cuh"
#include "nms_device.cuh"
#include "osd_device.cuh"
#endif

namespace bchlib {

constexpr int kSrvMaxCodes = 8;

struct SrvCode {
  DevCode dc;
  const GroupDesc *grp;  // [kMaxGroups] in device memory
  const uint64_t *std_cols;  // standard H column masks (OSD)
  int M, has_osd, wb, ord;  // ord: order of 2 mod n (Frobenius exponents)
};

// claim = generation << 32 | next unclaimed frame: a claim is a CAS that only
// succeeds for the request currently in the slot.
struct SrvSlot {
  const float *llr;
  unsigned long long seed, frame0;  // automorphisms of frame f: draw (seed, frame0 + f)
  uint64_t *hard;
  uint8_t *iters;
  uint8_t *flags;
  unsigned long long id;
  unsigned long long claim;
  int code, F, ld;
  unsigned done;
};

struct SrvComp {
  unsigned long long id;
  unsigned long long t_ns;
  unsigned slot;
  unsigned seq;
};

// Host-mapped control block (written by the host: sub_ring / sub_tail / stop;
// written by the device: comp / running).
struct SrvShared {
  volatile unsigned sub_tail[kSrvMaxCodes];  // per code: requests published so far
  volatile unsigned stop;
  volatile unsigned running;
  unsigned pad[6];
};

static_assert(sizeof(SrvShared) <= 64, "the submission rings start at byte 64");

struct SrvDev {
  unsigned head[kSrvMaxCodes];  // per code: first ring entry not yet fully claimed
  unsigned comp_tail;
  unsigned live;
  unsigned pad[6];
};

struct SrvArgs {
  const SrvCode *codes;  // [kSrvMaxCodes] in device memory
  const float *alpha;    // [32] in device memory
  int n_codes;
  SrvSlot *slots;
  SrvShared *sh;
  unsigned *sub_ring;  // host-mapped [kSrvMaxCodes][ring]: slot | generation << 16
  SrvComp *comp;       // host-mapped [ring]
  SrvDev *dv;
  int ring;
  int iters, P, order, early_stop;
  int scr_words;  // per-lane scratch column (row sums of the specialised n = 127 copies)
  unsigned long long idle_ns;
  // block-bound serving kernel: largest row count, largest n <= 63 among the codes
  // (0: none), rows per partial exchange of the n = 127 sessions
  int blk_max_rows, blk_flat_n, blk_R;
};

__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ SrvSlot load_slot(const SrvSlot *p) {
  SrvSlot s;
  static_assert(sizeof(SrvSlot) % 8 == 0, "slot layout");
  const unsigned long long *src = reinterpret_cast<const unsigned long long *>(p);
  unsigned long long *dst = reinterpret_cast<unsigned long long *>(&s);
#pragma unroll
  for (int i = 0; i < int(sizeof(SrvSlot) / 8); i++) dst[i] = __ldcg(src + i);
  return s;
}

// Claims up to `want` frames of code c for a warp (lane 0 only): walks the code's
// submission ring from its head, taking frames from each request by a
// generation-checked CAS on the request's claim word and moving the head past
// requests that are fully claimed (or replaced).  Bounded attempts.  Writes the
// segments (slot, first frame, count) to seg[0..], seg[32..], seg[64..].
__device__ int srv_claim(const SrvArgs &a, int c, int want, int *seg) {
  int nseg = 0;
  unsigned *headp = a.dv->head + c;
  for (int tries = 0; tries < 8 && want > 0 && nseg < 32; tries++) {
    const unsigned h = *reinterpret_cast<volatile unsigned *>(headp);
    const unsigned tail = a.sh->sub_tail[c];
    if (h == tail) break;
    __threadfence_system();
    const unsigned e =
        *reinterpret_cast<volatile unsigned *>(&a.sub_ring[size_t(c) * a.ring + h % unsigned(a.ring)]);
    const int sidx = int(e & 0xffffu);
    const unsigned gen = e >> 16;
    SrvSlot *sp = a.slots + sidx;
    const unsigned long long cl = *reinterpret_cast<volatile unsigned long long *>(&sp->claim);
    const unsigned next = unsigned(cl);
    const int F = *reinterpret_cast<volatile int *>(&sp->F);
    if (((cl >> 32) & 0xffffu) != gen || int(next) >= F) {
      atomicCAS(headp, h, h + 1);  // fully claimed or replaced: move on
      continue;
    }
    const int take = min(want, F - int(next));
    if (atomicCAS(&sp->claim, cl, cl + (unsigned long long)take) == cl) {
      seg[nseg] = sidx;
      seg[32 + nseg] = int(next);
      seg[64 + nseg] = take;
      nseg++;
      want -= take;
      if (int(next) + take >= F) atomicCAS(headp, h, h + 1);
    }
  }
  return nseg;
}

// The persistent serving loop (the body of both serving kernels).  One warp per block; each lane decodes one frame at a
// time and, when its frame stops, takes the next frame of the same code (across
// request boundaries), so early stopping turns into throughput as in the batch
// kernels.  The warp binds to one code while any lane has a frame and picks a code
// with published work when all its lanes are idle.  Frames whose syndrome stays
// nonzero get order-p OSD from the whole warp before they are counted done.
// `copies(code, cd, P, y, acc, scr, ctx, alpha)` runs the P automorphism copies of
// one iteration for the calling lane's frame (columns of stride 32).
// Shared memory per warp: accumulator and y columns [128][32] FP32, the scratch
// columns [scr_words][32], OSD scratch, automorphism parameters [9][32], claim
// segments [3][32].
template <class Copies>
__device__ __forceinline__ void serve_loop(const SrvArgs &a, unsigned char *smem, const Copies &copies) {
  float *acc = reinterpret_cast<float *>(smem);
  float *y = acc + 128 * 32;
  float *scr = y + 128 * 32;
  OsdSmem &S = *reinterpret_cast<OsdSmem *>(scr + a.scr_words * 32);
  uint32_t *ctx = reinterpret_cast<uint32_t *>(reinterpret_cast<unsigned char *>(&S) + sizeof(OsdSmem));
  int *seg = reinterpret_cast<int *>(ctx + 9 * 32);
  const int lane = int(lane_id());
  if (lane == 0) atomicAdd(&a.dv->live, 1u);
  unsigned long long idle_since = globaltimer();
  unsigned sleep_ns = 64;
  int wc = -1;                    // the code this warp decodes (warp-uniform)
  int slot = -1, f = -1, t = 0;   // this lane's frame
  const float invP = 1.0f / float(a.P);
  for (;;) {
    if (a.sh->stop) break;
    // ---- an idle warp binds to a code with published work
    if (!__any_sync(kFull, f >= 0)) {
      int pick = -1;
      if (lane == 0) {
        for (int q = 0; q < a.n_codes; q++) {
          const int c = (wc + 1 + q + int(blockIdx.x)) % a.n_codes;
          if (*reinterpret_cast<volatile unsigned *>(&a.dv->head[c]) != a.sh->sub_tail[c]) {
            pick = c;
            break;
          }
        }
      }
      pick = __shfl_sync(kFull, pick, 0);
      if (pick < 0) {
        if (globaltimer() - idle_since > a.idle_ns) break;
        __nanosleep(sleep_ns);
        sleep_ns = sleep_ns < 20000 ? sleep_ns * 2 : sleep_ns;
        continue;
      }
      wc = pick;
    }
    const SrvCode &cd = a.codes[wc];  // device memory
    const int n = cd.dc.n;
    // ---- idle lanes take the next frames of the code
    const unsigned need = __ballot_sync(kFull, f < 0);
    if (need) {
      int nseg = 0;
      if (lane == 0) nseg = srv_claim(a, wc, __popc(need), seg);
      nseg = __shfl_sync(kFull, nseg, 0);
      __syncwarp();
      const float *src = nullptr;  // the LLR row of this lane's new frame
      if (f < 0 && nseg > 0) {
        int r = __popc(need & ((1u << lane) - 1u));
        for (int q = 0; q < nseg; q++) {
          const int cnt = seg[64 + q];
          if (r < cnt) {
            slot = seg[q];
            f = seg[32 + q] + r;
            break;
          }
          r -= cnt;
        }
        if (f >= 0) {
          // the host rewrites a slot between requests: read the descriptor past L1
          const SrvSlot sl = load_slot(a.slots + slot);
          src = sl.llr + size_t(f) * sl.ld;
          uint32_t va[9];
          draw_frame_autos(n, cd.ord, a.P, sl.seed, sl.frame0 + uint64_t(f), va);
          const uint32_t m = uint32_t(cd.dc.m);
          for (int p = 0; p < a.P; p++) {
            const uint32_t sh = va[p] & 0xffu, j = va[p] >> 8;
            // pi^-1(u) = rotr_m(u, j) + s' with s' = -rotr_m(s, j) mod n
            const uint32_t rs = j ? (((sh >> j) | (sh << (m - j))) & uint32_t(n)) : sh;
            ctx[p * 32 + lane] = j | ((rs ? uint32_t(n) - rs : 0u) << 8);
          }
          t = 0;
        }
      }
      __syncwarp();
      // the whole warp loads each new frame's row: coalesced reads (lane q takes
      // elements q, q + 32, ...) past L1, since copies rewrite the arena while the
      // kernel runs
      for (unsigned fm = __ballot_sync(kFull, src != nullptr); fm; fm &= fm - 1) {
        const int l = __ffs(fm) - 1;
        const float *row = reinterpret_cast<const float *>(
            __shfl_sync(kFull, reinterpret_cast<unsigned long long>(src), l));
        for (int i = lane; i < n; i += 32) {
          y[i * 32 + l] = __ldcg(row + i) + 0.0f;  // -0 -> +0
          acc[i * 32 + l] = 0.0f;
        }
      }
      __syncwarp();
    }
    const bool active = f >= 0;
    if (!__any_sync(kFull, active)) continue;
    sleep_ns = 64;
    idle_since = globaltimer();
    // ---- one iteration for the active lanes
    bool done = false;
    uint32_t nz = 0;
    uint32_t cb[4] = {0u, 0u, 0u, 0u};
    if (active) {
      const float alpha = __ldg(a.alpha + t);
      copies(wc, cd, a.P, y + lane, acc + lane, scr + lane, ctx + lane, alpha);
      float mx = 0.0f;
      for (int i = 0; i < n; i++) {
        const float yn = __fmaf_rn(acc[i * 32 + lane], invP, y[i * 32 + lane]);
        y[i * 32 + lane] = yn;
        acc[i * 32 + lane] = 0.0f;
        cb[i >> 5] |= (__float_as_uint(yn) >> 31) << (i & 31);
        mx = fmaxf(mx, fabsf(yn));
      }
      if (mx > 0x1p100f)  // exact renormalisation against FP32 overflow (see the batch kernels)
        for (int i = 0; i < n; i++) y[i * 32 + lane] *= 0x1p-64f;
      t++;
      nz = syndrome_nonzero<4>(reinterpret_cast<const uint4 *>(cd.dc.rowmask), cd.dc.rows, cb);
      done = t >= a.iters || (a.early_stop && nz == 0);
      if (done) {
        const SrvSlot sl = load_slot(a.slots + slot);
        const int W64 = (n + 63) / 64;
        sl.hard[size_t(f) * W64] = uint64_t(cb[0]) | (uint64_t(cb[1]) << 32);
        if (W64 > 1) sl.hard[size_t(f) * W64 + 1] = uint64_t(cb[2]) | (uint64_t(cb[3]) << 32);
        sl.iters[f] = uint8_t(t);
        sl.flags[f] = nz ? 0 : uint8_t(kFlagConverged);
      }
    }
    // ---- OSD of the frames that stopped with a nonzero syndrome (whole warp)
    const unsigned fail = __ballot_sync(kFull, done && nz != 0 && cd.has_osd);
    __syncwarp();
    for (unsigned fm = fail; fm; fm &= fm - 1) {
      const int l = __ffs(fm) - 1;
      const int sl_l = __shfl_sync(kFull, slot, l);
      const int f_l = __shfl_sync(kFull, f, l);
      const SrvSlot sl = load_slot(a.slots + sl_l);
      const int W64 = (n + 63) / 64;
      osd_one_frame(S, n, cd.dc.k, cd.M, cd.std_cols, sl.llr + size_t(f_l) * sl.ld, a.order,
                    sl.hard + size_t(f_l) * W64, sl.flags + f_l);
    }
    // ---- count finished frames: per request, one of the lanes that finished frames
    // of it adds them all to the request's done counter, and the add that completes
    // the request posts it.  The warp barrier orders every lane's result writes (the
    // OSD's, made by whichever lanes ran it, included) before the counting lane's
    // fence, and that fence is cumulative: it orders everything the counting lane has
    // observed before its add, so a warp that later completes the request (and fences
    // before posting it) publishes results that are all in memory.
    const unsigned dmask = __ballot_sync(kFull, done);
    if (dmask) {
      __syncwarp();
      if (done) {
        const unsigned peers = __match_any_sync(dmask, slot);
        if (lane == __ffs(peers) - 1) {
          const SrvSlot sl = load_slot(a.slots + slot);
          const unsigned cnt = unsigned(__popc(peers));
          __threadfence();
          const unsigned d = atomicAdd(&a.slots[slot].done, cnt) + cnt;
          if (int(d) == sl.F) {
            const unsigned ci = atomicAdd(&a.dv->comp_tail, 1u);
            SrvComp *c = a.comp + (ci % unsigned(a.ring));
            c->id = sl.id;
            c->t_ns = globaltimer();
            c->slot = unsigned(slot);
            __threadfence_system();
            *reinterpret_cast<volatile unsigned *>(&c->seq) = ci + 1;
          }
        }
        f = -1;
        slot = -1;
      }
    }
  }
  if (lane == 0) {
    if (atomicSub(&a.dv->live, 1u) == 1u) {
      __threadfence_system();
      a.sh->running = 0;
    }
  }
}


// ======================================================================================
// Block-bound serving kernel.  One 256-thread block per SM binds to one code for a
// session and decodes that code's frames with the batch kernels' own mapping -- one
// thread per frame in lockstep for n <= 63, the split mapping (two warps per 32 frames,
// half of the variables each) for n = 127 -- so an SM streams one code's straight-line
// rows at a time through its instruction cache.  Idle lanes claim frames of the bound
// code across request boundaries (srv_claim); a frame is loaded from its request's
// arena buffer, its automorphisms are drawn from (seed, frame0 + f), and when it stops
// its results go to the request's buffers, frames with a nonzero syndrome get OSD from
// their warp, and finished frames are counted per request (the add that completes a
// request posts it).  A session ends when the code has no claimable frame and every
// lane is idle, or, to rotate the SM across codes, once kSrvSessionIters iterations
// have run and the lanes in flight have finished.
constexpr int kSrvBlockThreads = 256;
constexpr int kSrvSessionIters = 48;

// Byte offsets of the block-bound kernel's shared memory: control words, alpha, the
// bound code's row masks, per-warp claim segments, then the session state (the
// largest of the one-thread-per-frame layout plus eight warps' OSD scratch and the
// split layout, whose partial buffers also hold the half-0 warps' OSD scratch).
struct SrvBlockLayout {
  size_t alpha, rowmask, seg, state, flat_osd, total;
};
__host__ __device__ inline SrvBlockLayout srv_block_layout(int max_rows, int flat_n, int P, int R, int n_split) {
  SrvBlockLayout L;
  L.alpha = 16;
  L.rowmask = 16 + 32 * 4;
  L.seg = L.rowmask + size_t(max_rows) * 16;
  L.state = (L.seg + size_t(kSrvBlockThreads / 32) * 96 * 4 + 15) & ~size_t(15);
  const size_t flat = flat_n > 0 ? size_t(kSrvBlockThreads) * (size_t(P) + 2 * size_t(flat_n)) * 4 : 0;
  L.flat_osd = L.state + flat;
  const size_t flat_total = flat_n > 0 ? flat + size_t(kSrvBlockThreads / 32) * sizeof(OsdSmem) : 0;
  const size_t Fs = 128;
  const size_t split = n_split > 0 ? Fs * 4 * 2 * size_t(P) + Fs * 4 * size_t(n_split) * 2 +
                                         Fs * 8 * 2 * 2 * size_t(R)
                                   : 0;
  L.total = L.state + (flat_total > split ? flat_total : split);
  return L;
}

// The lanes of a warp that need a frame claim frames of code c (lane 0 runs srv_claim;
// the segments go to the needing lanes in lane order).  A lane that gets a frame has
// slot and f set and returns true.
__device__ __forceinline__ bool warp_claim(const SrvArgs &a, int c, bool need, int *seg, int &slot, int &f) {
  const unsigned nm = __ballot_sync(kFull, need);
  if (!nm) return false;
  const int lane = int(lane_id());
  int nseg = 0;
  if (lane == 0) nseg = srv_claim(a, c, __popc(nm), seg);
  nseg = __shfl_sync(kFull, nseg, 0);
  __syncwarp();
  bool got = false;
  if (need && nseg > 0) {
    int r = __popc(nm & ((1u << lane) - 1u));
    for (int q = 0; q < nseg; q++) {
      const int cnt = seg[64 + q];
      if (r < cnt) {
        slot = seg[q];
        f = seg[32 + q] + r;
        got = true;
        break;
      }
      r -= cnt;
    }
  }
  __syncwarp();
  return got;
}

// The P automorphisms of frame f of a request, as the parameters (j | s' << 8) of
// pi^-1(u) = rotr_m(u, j) + s', written to ctx[p * stride].
__device__ __forceinline__ void srv_frame_ctx(const SrvCode &cd, int P, const SrvSlot &sl, int f,
                                              uint32_t *ctx, int stride) {
  uint32_t va[9];
  const int n = cd.dc.n;
  draw_frame_autos(n, cd.ord, P, sl.seed, sl.frame0 + uint64_t(f), va);
  const uint32_t m = uint32_t(cd.dc.m);
  for (int p = 0; p < P; p++) {
    const uint32_t sh = va[p] & 0xffu, j = va[p] >> 8;
    const uint32_t rs = j ? (((sh >> j) | (sh << (m - j))) & uint32_t(n)) : sh;
    ctx[p * stride] = j | ((rs ? uint32_t(n) - rs : 0u) << 8);
  }
}

// Warp-cooperative loads of new frames' LLR rows (positions [i0, i1)): for every lane
// whose src is set, the whole warp reads that row with coalesced reads past L1 (the
// host rewrites the arena between requests) into column col of y and clears acc.
__device__ __forceinline__ void warp_load_rows(const float *src, int col, int i0, int i1, float *y,
                                               float *acc, int stride) {
  const int lane = int(lane_id());
  for (unsigned fm = __ballot_sync(kFull, src != nullptr); fm; fm &= fm - 1) {
    const int l = __ffs(fm) - 1;
    const float *row = reinterpret_cast<const float *>(
        __shfl_sync(kFull, reinterpret_cast<unsigned long long>(src), l));
    const int cl = __shfl_sync(kFull, col, l);
    for (int i = i0 + lane; i < i1; i += 32) {
      y[i * stride + cl] = __ldcg(row + i) + 0.0f;  // -0 -> +0
      acc[i * stride + cl] = 0.0f;
    }
  }
  __syncwarp();
}

// A warp's frames that stopped this iteration (done): OSD of those with a nonzero
// syndrome (whole warp, in lane order), then the completion count of each request (as
// in serve_loop: a warp barrier orders every lane's result writes before the counting
// lane's cumulative fence and add).  Resets slot and f of the finished lanes.
__device__ __forceinline__ void warp_finish(const SrvArgs &a, const SrvCode &cd, bool done, uint32_t nz,
                                            int &slot, int &f, OsdSmem &S) {
  const int lane = int(lane_id());
  const int n = cd.dc.n;
  const unsigned fail = __ballot_sync(kFull, done && nz != 0 && cd.has_osd);
  __syncwarp();
  for (unsigned fm = fail; fm; fm &= fm - 1) {
    const int l = __ffs(fm) - 1;
    const int sl_l = __shfl_sync(kFull, slot, l);
    const int f_l = __shfl_sync(kFull, f, l);
    const SrvSlot sl = load_slot(a.slots + sl_l);
    const int W64 = (n + 63) / 64;
    osd_one_frame(S, n, cd.dc.k, cd.M, cd.std_cols, sl.llr + size_t(f_l) * sl.ld, a.order,
                  sl.hard + size_t(f_l) * W64, sl.flags + f_l);
  }
  const unsigned dmask = __ballot_sync(kFull, done);
  if (dmask) {
    __syncwarp();
    if (done) {
      const unsigned peers = __match_any_sync(dmask, slot);
      if (lane == __ffs(peers) - 1) {
        const SrvSlot sl = load_slot(a.slots + slot);
        const unsigned cnt = unsigned(__popc(peers));
        __threadfence();
        const unsigned d = atomicAdd(&a.slots[slot].done, cnt) + cnt;
        if (int(d) == sl.F) {
          const unsigned ci = atomicAdd(&a.dv->comp_tail, 1u);
          SrvComp *c = a.comp + (ci % unsigned(a.ring));
          c->id = sl.id;
          c->t_ns = globaltimer();
          c->slot = unsigned(slot);
          __threadfence_system();
          *reinterpret_cast<volatile unsigned *>(&c->seq) = ci + 1;
        }
      }
      f = -1;
      slot = -1;
    }
  }
}

__device__ __forceinline__ void srv_write_result(const SrvArgs &a, int slot, int f, int n, const uint32_t (&cb)[4],
                                                 int t, uint32_t nz) {
  const SrvSlot sl = load_slot(a.slots + slot);
  const int W64 = (n + 63) / 64;
  sl.hard[size_t(f) * W64] = uint64_t(cb[0]) | (uint64_t(cb[1]) << 32);
  if (W64 > 1) sl.hard[size_t(f) * W64 + 1] = uint64_t(cb[2]) | (uint64_t(cb[3]) << 32);
  sl.iters[f] = uint8_t(t);
  sl.flags[f] = nz ? 0 : uint8_t(kFlagConverged);
}

// Session of a code with n <= 63: one thread per frame, the block's warps in lockstep
// (the batch kernel's mapping; columns [x][thread] of stride 256).  Copy: the code's
// straight-line copy functor.
template <int NW, class Copy>
__device__ void serve_session_flat(const SrvArgs &a, int c, unsigned char *smem, const SrvBlockLayout &L,
                                   const Copy &copy) {
  constexpr int TPB = kSrvBlockThreads;
  const SrvCode &cd = a.codes[c];
  const int n = cd.dc.n, rows = cd.dc.rows;
  const uint32_t m = uint32_t(cd.dc.m);
  const int tid = int(threadIdx.x), warp = tid >> 5, lane = tid & 31;
  volatile int *claiming = reinterpret_cast<volatile int *>(smem);
  const float *alpha_s = reinterpret_cast<const float *>(smem + L.alpha);
  const uint4 *rowmask = reinterpret_cast<const uint4 *>(smem + L.rowmask);
  int *seg = reinterpret_cast<int *>(smem + L.seg) + warp * 96;
  uint32_t *ctx = reinterpret_cast<uint32_t *>(smem + L.state) + tid;
  float *acc_s = reinterpret_cast<float *>(smem + L.state) + size_t(a.P) * TPB;
  float *y_s = acc_s + size_t(n) * TPB;
  float *acc = acc_s + tid, *y = y_s + tid;
  OsdSmem &S = reinterpret_cast<OsdSmem *>(smem + L.flat_osd)[warp];
  SmemTables tb{};
  const float invP = 1.0f / float(a.P);
  for (int p = 0; p < a.P; p++) ctx[p * TPB] = 0u;
  int slot = -1, f = -1, t = 0, it = 0;
  for (;;) {
    if (*claiming) {
      const bool got = warp_claim(a, c, f < 0, seg, slot, f);
      const float *src = nullptr;
      if (got) {
        const SrvSlot sl = load_slot(a.slots + slot);
        src = sl.llr + size_t(f) * sl.ld;
        srv_frame_ctx(cd, a.P, sl, f, ctx, TPB);
        t = 0;
      }
      warp_load_rows(src, warp * 32 + lane, 0, n, y_s, acc_s, TPB);
    }
    if (!__syncthreads_or(f >= 0)) break;
    // after this iteration's first barrier every thread sees the decision
    if (tid == 0 && (++it >= kSrvSessionIters || a.sh->stop)) *claiming = 0;
    const float alpha = alpha_s[f >= 0 ? t : 0];
    for (int p = 0; p < a.P; p++) {
      __syncthreads();
      const uint32_t cx = f >= 0 ? ctx[p * TPB] : 0u;
      copy(tb, 0, uint32_t(n), m, y, acc, nullptr, cx & 0xffu, cx >> 8, uint32_t(TPB), alpha);
    }
    uint32_t cb[4] = {0u, 0u, 0u, 0u};
    float mx = 0.0f;
#pragma unroll
    for (int i = 0; i < NW * 32; i++) {
      if (i < n) {
        const float yn = __fmaf_rn(acc[i * TPB], invP, y[i * TPB]);
        y[i * TPB] = yn;
        acc[i * TPB] = 0.0f;
        cb[i >> 5] |= (__float_as_uint(yn) >> 31) << (i & 31);
        mx = fmaxf(mx, fabsf(yn));
      }
    }
    if (mx > 0x1p100f)  // exact renormalisation against FP32 overflow (as the batch kernels)
      for (int i = 0; i < n; i++) y[i * TPB] *= 0x1p-64f;
    bool done = false;
    uint32_t nz = 0;
    if (f >= 0) {
      t++;
      nz = syndrome_nonzero<4>(rowmask, rows, cb);
      done = t >= a.iters || (a.early_stop && nz == 0);
      if (done) srv_write_result(a, slot, f, n, cb, t, nz);
    }
    warp_finish(a, cd, done, nz, slot, f, S);
  }
}

// Session of a code with n = 127 in the split mapping of the batch kernel (two warps per
// 32 frames, warp half h owns the variables [64h, 64h + 64)): half 0 claims and hands
// the frames to half 1; each half loads its half of the LLRs and draws the
// automorphisms; after the merge the halves exchange hard-decision words and
// magnitudes; half 0 writes the results, runs the OSD (scratch in the partial buffers,
// unused between copies) and counts completions.
template <class Copy>
__device__ void serve_session_split(const SrvArgs &a, int c, unsigned char *smem, const SrvBlockLayout &L,
                                    const Copy &copy, int nchunk, int R) {
  constexpr int G = 4, Fs = 32 * G, TPB = 64 * G;
  const SrvCode &cd = a.codes[c];
  const int n = cd.dc.n, rows = cd.dc.rows;
  const int warp = int(threadIdx.x >> 5), lane = int(lane_id());
  const int h = (warp >> 1) & 1;
  const int s = ((warp & 1) + ((warp >> 2) << 1)) * 32 + lane;
  const int i0 = h * 64, i1 = h ? n : 64;
  volatile int *claiming = reinterpret_cast<volatile int *>(smem);
  const float *alpha_s = reinterpret_cast<const float *>(smem + L.alpha);
  const uint4 *rowmask = reinterpret_cast<const uint4 *>(smem + L.rowmask);
  int *seg = reinterpret_cast<int *>(smem + L.seg) + warp * 96;
  unsigned char *st = smem + L.state;
  uint32_t *ctx = reinterpret_cast<uint32_t *>(st) + size_t(h) * a.P * Fs + s;
  float *acc_s = reinterpret_cast<float *>(st + size_t(Fs) * 4 * 2 * a.P);
  float *y_s = acc_s + size_t(n) * Fs;
  unsigned char *pbase = reinterpret_cast<unsigned char *>(y_s + size_t(n) * Fs);
  float2 *part = reinterpret_cast<float2 *>(pbase);
  uint4 *xch = reinterpret_cast<uint4 *>(pbase);                           // [2][Fs]
  int2 *hand = reinterpret_cast<int2 *>(pbase + size_t(Fs) * 16 * 2);      // [Fs]
  OsdSmem &S = reinterpret_cast<OsdSmem *>(pbase + 8192)[warp >> 2 << 1 | (warp & 1)];
  float *acc = acc_s + s, *y = y_s + s;
  const float invP = 1.0f / float(a.P);
  for (int p = 0; p < a.P; p++) ctx[p * Fs] = 0u;
  int slot = -1, f = -1, t = 0, it = 0;
  for (;;) {
    const bool cl = *claiming != 0;
    const bool need = f < 0;
    if (h == 0) {
      if (cl) warp_claim(a, c, need, seg, slot, f);
      hand[s] = make_int2(slot, f);
    }
    bar_block(TPB);
    if (h == 1 && need) {
      const int2 hv = hand[s];
      slot = hv.x;
      f = hv.y;
    }
    const bool fresh = need && f >= 0;
    const float *src = nullptr;
    if (fresh) {
      const SrvSlot sl = load_slot(a.slots + slot);
      src = sl.llr + size_t(f) * sl.ld;
      srv_frame_ctx(cd, a.P, sl, f, ctx, Fs);
      t = 0;
    }
    warp_load_rows(src, s, i0, i1, y_s, acc_s, Fs);
    if (!__syncthreads_or(f >= 0)) break;
    if (threadIdx.x == 0 && (++it >= kSrvSessionIters || a.sh->stop)) *claiming = 0;
    const float alpha = alpha_s[f >= 0 ? t : 0];
    for (int p = 0; p < a.P; p++) {
      const uint32_t cx = f >= 0 ? ctx[p * Fs] : 0u;
      float2 *pa = part + (((p * nchunk) & 1) ? size_t(2) * R * Fs : 0) + s;
      float2 *pb = part + (((p * nchunk) & 1) ? 0 : size_t(2) * R * Fs) + s;
      copy(h, y, acc, pa, pb, cx & 0xffu, cx >> 8, alpha);
    }
    __syncthreads();
    uint32_t cw0 = 0, cw1 = 0;
    float mx = 0.0f;
    for (int i = i0; i < i1; i++) {
      const float yn = __fmaf_rn(acc[i * Fs], invP, y[i * Fs]);
      y[i * Fs] = yn;
      acc[i * Fs] = 0.0f;
      const uint32_t b = (__float_as_uint(yn) >> 31) << ((i - i0) & 31);
      if (i - i0 < 32) cw0 |= b; else cw1 |= b;
      mx = fmaxf(mx, fabsf(yn));
    }
    xch[h * Fs + s] = make_uint4(cw0, cw1, __float_as_uint(mx), 0u);
    __syncthreads();
    const uint4 o = xch[(1 - h) * Fs + s];
    uint32_t cb[4];
    cb[h * 2] = cw0;
    cb[h * 2 + 1] = cw1;
    cb[(1 - h) * 2] = o.x;
    cb[(1 - h) * 2 + 1] = o.y;
    mx = fmaxf(mx, __uint_as_float(o.z));
    if (mx > 0x1p100f && f >= 0)
      for (int i = i0; i < i1; i++) y[i * Fs] *= 0x1p-64f;
    bool done = false;
    uint32_t nz = 0;
    if (f >= 0) {
      t++;
      nz = syndrome_nonzero<4>(rowmask, rows, cb);
      done = t >= a.iters || (a.early_stop && nz == 0);
      if (done && h == 0) srv_write_result(a, slot, f, n, cb, t, nz);
    }
    // the OSD scratch lies in the partial buffers past the exchange and hand-off words;
    // the next copies start only after the loop-top barriers, once every OSD is done
    if (h == 0) {
      warp_finish(a, cd, done, nz, slot, f, S);
    } else if (done) {
      f = -1;
      slot = -1;
    }
  }
}

// The block-bound kernel's outer loop: thread 0 picks a code with published work
// (rotating its start per block and session) and the block runs a session of it;
// sessions(c, smem, L) dispatches to the code's session.  Idle blocks back off and exit
// after idle_ns without work; the stop flag ends the kernel between sessions and stops
// new claims inside one.
template <class Sessions>
__device__ __forceinline__ void serve_blocks(const SrvArgs &a, unsigned char *smem, const Sessions &sessions) {
  const int P = a.P;
  const SrvBlockLayout L = srv_block_layout(a.blk_max_rows, a.blk_flat_n, P, a.blk_R, 127);
  volatile int *ctl = reinterpret_cast<volatile int *>(smem);  // [0] claiming, [1] pick, [2] stop
  float *alpha_s = reinterpret_cast<float *>(smem + L.alpha);
  uint4 *rowmask = reinterpret_cast<uint4 *>(smem + L.rowmask);
  const int tid = int(threadIdx.x);
  if (tid < 32) alpha_s[tid] = __ldg(a.alpha + tid);
  if (tid == 0) atomicAdd(&a.dv->live, 1u);
  unsigned long long idle_since = globaltimer();
  unsigned sleep_ns = 64;
  int wc = int(blockIdx.x) % max(1, a.n_codes) - 1;
  for (;;) {
    if (tid == 0) {
      int pick = -1;
      const int stop = a.sh->stop ? 1 : 0;
      if (!stop) {
        for (int q = 0; q < a.n_codes; q++) {
          const int c = (wc + 1 + q) % a.n_codes;
          if (*reinterpret_cast<volatile unsigned *>(&a.dv->head[c]) != a.sh->sub_tail[c]) {
            pick = c;
            break;
          }
        }
      }
      ctl[1] = pick;
      ctl[2] = stop;
      ctl[0] = 1;
    }
    __syncthreads();
    const int pick = ctl[1], stop = ctl[2];
    if (stop) break;
    if (pick < 0) {
      if (globaltimer() - idle_since > a.idle_ns) break;
      __nanosleep(sleep_ns);
      sleep_ns = sleep_ns < 20000 ? sleep_ns * 2 : sleep_ns;
      __syncthreads();
      continue;
    }
    sleep_ns = 64;
    wc = pick;
    const SrvCode &cd = a.codes[pick];
    const uint4 *rm = reinterpret_cast<const uint4 *>(cd.dc.rowmask);
    for (int r = tid; r < cd.dc.rows; r += int(blockDim.x)) rowmask[r] = rm[r];
    __syncthreads();
    sessions(pick, smem, L);
    __syncthreads();
    idle_since = globaltimer();
  }
  if (tid == 0) {
    if (atomicSub(&a.dv->live, 1u) == 1u) {
      __threadfence_system();
      a.sh->running = 0;
    }
  }
}

}  // namespace bchlib
