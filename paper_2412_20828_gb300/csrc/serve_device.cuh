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

}  // namespace bchlib
