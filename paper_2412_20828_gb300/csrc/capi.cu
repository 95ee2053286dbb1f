// C ABI of the decoder library: argument checking, code objects, workspace layout and
// the launch sequences of the decode / training calls.  See include/bchdec.h.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <memory>
#include <string>
#include <vector>

#include "bch_kernels.cuh"

using namespace bchlib;

namespace bchlib {
cudaKernel_t jit_kernel(const bch_code *c, int msg, std::string *err, int qfrac = 0);
bool jit_compile_check(const bch_code *c, int msg, std::string *log);
bool jit_serve_compile_check(const bch_code *const *codes, int n_codes, std::string *log);
int jit_block_size(int n);
int jit_scratch_words(int n);
bool jit_split(int n);
int jit_split_groups();
int jit_split_chunk_rows();
size_t nms_table_bytes_host(const DevCode &dc);
}  // namespace bchlib

// Which enhanced-NMS kernel runs: the run-time specialised one ("jit") when it
// compiles, else the precompiled one.  BCHDEC_NMS_KERNEL=generic|jit|auto overrides.
static int kernel_mode() {
  const char *v = std::getenv("BCHDEC_NMS_KERNEL");
  if (!v) return 0;
  if (!std::strcmp(v, "generic")) return 1;
  if (!std::strcmp(v, "jit")) return 2;
  return 0;
}



namespace bchlib {

static thread_local std::string g_last_error;
static std::atomic<unsigned long long> g_launches{0};

void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

void set_error(const std::string &msg) { g_last_error = msg; }

bch_status fail(bch_status s, const std::string &msg) {
  set_error(msg);
  return s;
}

}  // namespace bchlib

namespace bchlib {
#ifdef BCH_CHECKED
// The checked build's check word: flags, count of invalid values, smallest frame with an
// invalid automorphism, smallest OSD list position with an invalid entry.
__device__ unsigned g_check_word[4] = {0u, 0u, 0xffffffffu, 0xffffffffu};
#endif

unsigned *check_word() {
#ifdef BCH_CHECKED
  void *p = nullptr;
  if (cudaGetSymbolAddress(&p, g_check_word) != cudaSuccess) {
    (void)cudaGetLastError();
    return nullptr;
  }
  return static_cast<unsigned *>(p);
#else
  return nullptr;
#endif
}

cudaError_t launch_geometry(const void *fn, int tpb, size_t smem, int *sms, int *per_sm) {
  // The shared-memory limit is one attribute per function (per device): it holds the
  // last value set, so it is raised to the largest size any launch has needed and never
  // lowered.  Occupancy depends on (block size, shared memory) and is remembered per
  // combination.
  struct Limit {
    int dev;
    const void *fn;
    size_t smem_max;
  };
  struct Geo {
    int dev;
    const void *fn;
    int tpb;
    size_t smem;
    int sms, per_sm;
  };
  static std::mutex mu;
  static std::vector<Limit> limits;
  static std::vector<Geo> known;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(mu);
  Limit *lim = nullptr;
  for (Limit &l : limits)
    if (l.dev == dev && l.fn == fn) lim = &l;
  if (!lim || lim->smem_max < smem) {
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    if (lim) {
      lim->smem_max = smem;
    } else {
      limits.push_back({dev, fn, smem});
    }
  }
  for (const Geo &g : known)
    if (g.dev == dev && g.fn == fn && g.tpb == tpb && g.smem == smem) {
      *sms = g.sms;
      *per_sm = g.per_sm;
      return cudaSuccess;
    }
  e = cudaDeviceGetAttribute(sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, fn, tpb, smem);
  if (e != cudaSuccess) return e;
  known.push_back({dev, fn, tpb, smem, *sms, *per_sm});
  return cudaSuccess;
}
}  // namespace bchlib

namespace {

bch_status cuda_fail(cudaError_t e, const char *what) {
  return fail(BCH_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define BCH_CUDA(call, what)                      \
  do {                                            \
    cudaError_t e_ = (call);                      \
    if (e_ != cudaSuccess) return cuda_fail(e_, what); \
  } while (0)

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Workspace layout (offsets in bytes from the 256-aligned base).
struct WsLayout {
  size_t queues = 0;  // u32 nms queue, u32 osd queue
  size_t counts = 0;  // u32 per 1024-frame block
  size_t list = 0;    // u32[F] failed frames
  size_t count = 0;   // u32 failed count
  size_t red = 0;     // float reductions (loss / backward partials)
  size_t total = 0;
};

WsLayout ws_layout(int F, int iters) {
  WsLayout L;
  size_t off = 0;
  L.queues = off;
  off = align256(off + 16);
  L.counts = off;
  off = align256(off + size_t((F + 1023) / 1024 + 1) * 4);
  L.list = off;
  off = align256(off + size_t(std::max(F, 1)) * 4);
  L.count = off;
  off = align256(off + 4);
  L.red = off;
  off = align256(off + std::max(bce_workspace(F), backward_workspace(F, std::max(iters, 1))));
  L.total = off;
  return L;
}

bool code_ok(const bch_code *c) { return c != nullptr && c->dev_dc != nullptr; }

}  // namespace

namespace bchlib {

bch_status check_params(const bch_code *code, const bch_nms_params *p) {
  if (!code_ok(code)) return fail(BCH_EINVAL, "null code");
  if (!p) return fail(BCH_EINVAL, "null params");
  if (p->iters < 1 || p->iters > 32) return fail(BCH_EINVAL, "iters must be in [1, 32]");
  if (!p->alpha) return fail(BCH_EINVAL, "alpha is null");
  if (p->n_autos < 0 || p->n_autos > 9) return fail(BCH_EINVAL, "n_autos must be in [0, 9]");
  if (p->msg < BCH_MSG_FP32 || p->msg > BCH_MSG_INT8) return fail(BCH_EINVAL, "bad msg type");
  if (p->n_autos == 0 && p->msg != BCH_MSG_FP32)
    return fail(BCH_EINVAL, "the plain decoder supports FP32 only");
  for (int t = 0; t < p->iters; t++)
    if (!std::isfinite(p->alpha[t])) return fail(BCH_EINVAL, "alpha must be finite");
  if (p->osd_input != 0 && p->osd_input != 1) return fail(BCH_EINVAL, "osd_input must be 0 or 1");
  if (p->qfrac < 0 || p->qfrac > 8) return fail(BCH_EINVAL, "qfrac must be in [0, 8]");
  if (p->qfrac > 0) {
    if (p->msg != BCH_MSG_INT8 || p->n_autos < 1)
      return fail(BCH_EINVAL, "qfrac applies to the enhanced decoder's 8-bit form only");
    for (int t = 0; t < p->iters; t++)
      if (!(p->alpha[t] >= 0.0f && p->alpha[t] <= 4.0f))
        return fail(BCH_EINVAL, "qfrac needs 0 <= alpha_t <= 4 (exact sums)");
  }
  return BCH_OK;
}

bch_status check_frames(const bch_code *code, const float *llr, int ld, int F) {
  if (F < 0) return fail(BCH_EINVAL, "n_frames < 0");
  if (ld < code->alg.n) return fail(BCH_EINVAL, "ld < n");
  if (F > 0 && !llr) return fail(BCH_EINVAL, "llr is null");
  return BCH_OK;
}

bch_status check_osd(const bch_code *code, const bch_code *std_code, int order) {
  if (!code_ok(std_code) || std_code->kind != BCH_PCM_STANDARD)
    return fail(BCH_EINVAL, "OSD needs the standard parity-check matrix");
  if (code && (!code_ok(code) || std_code->alg.n != code->alg.n || std_code->alg.k != code->alg.k))
    return fail(BCH_EINVAL, "std_code must be the standard matrix of the same code");
  if (order < 0 || order > 2) return fail(BCH_EINVAL, "OSD order must be 0, 1 or 2");
  if (std_code->alg.n - std_code->alg.k > 64) return fail(BCH_EINVAL, "OSD supports n-k <= 64");
  return BCH_OK;
}

}  // namespace bchlib

namespace {

// Builds the device image of a code: rows grouped by weight, column codes, row masks,
// parity words.
bch_status upload_code(bch_code *c) {
  const int n = c->alg.n, m = c->alg.m, k = c->alg.k;
  const int R = int(c->rows.size());
  std::vector<int> order(R);
  for (int i = 0; i < R; i++) order[i] = i;
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int b) { return c->rows[a].weight() < c->rows[b].weight(); });
  DevCode dc;
  std::memset(&dc, 0, sizeof(dc));
  dc.n = n;
  dc.k = k;
  dc.m = m;
  dc.rows = R;
  dc.nwords32 = (n + 31) / 32;
  std::vector<uint16_t> codes;
  int edges = 0, maxw = 0;
  for (int idx = 0; idx < R;) {
    const int w = c->rows[order[idx]].weight();
    if (w > 48) return fail(BCH_EINVAL, "row weight above 48 is not supported");
    if (w < 2) return fail(BCH_EINVAL, "row weight below 2");
    if (dc.n_groups >= kMaxGroups) return fail(BCH_EINVAL, "too many distinct row weights");
    const int g = dc.n_groups++;
    dc.group_w[g] = w;
    dc.group_off[g] = int(codes.size());
    int cnt = 0;
    while (idx < R && c->rows[order[idx]].weight() == w) {
      const Row &row = c->rows[order[idx]];
      int e = 0;
      for (int u = 0; u < n; u++)
        if (row.get(u)) {
          codes.push_back(uint16_t(u | (u << m)));
          e++;
        }
      while (e % 4) {
        codes.push_back(0);
        e++;
      }
      edges += w;
      maxw = std::max(maxw, w);
      cnt++;
      idx++;
    }
    dc.group_rows[g] = cnt;
  }
  dc.group_off[dc.n_groups] = int(codes.size());
  if (codes.size() % 2) codes.push_back(0);
  dc.edges = edges;
  dc.max_w = maxw;
  // device blob: codes | rowmask | par | colmask | descriptor
  const size_t off_codes = 0;
  const size_t off_mask = align256(off_codes + codes.size() * 2);
  const size_t off_par = align256(off_mask + size_t(R) * 16);
  const size_t off_cols = align256(off_par + size_t(k) * 8);
  const size_t off_desc = align256(off_cols + size_t(n) * 8);
  const size_t total = align256(off_desc + sizeof(DevCode));
  std::vector<unsigned char> host(total, 0);
  std::memcpy(host.data() + off_codes, codes.data(), codes.size() * 2);
  for (int r = 0; r < R; r++) {
    uint32_t w4[4];
    w4[0] = uint32_t(c->rows[r].w[0]);
    w4[1] = uint32_t(c->rows[r].w[0] >> 32);
    w4[2] = uint32_t(c->rows[r].w[1]);
    w4[3] = uint32_t(c->rows[r].w[1] >> 32);
    std::memcpy(host.data() + off_mask + size_t(r) * 16, w4, 16);
  }
  std::memcpy(host.data() + off_par, c->alg.par.data(), size_t(k) * 8);
  if (R <= 64) {  // column masks: bit r of column u = H[r][u] (the OSD elimination)
    for (int u = 0; u < n; u++) {
      uint64_t col = 0;
      for (int r = 0; r < R; r++)
        if (c->rows[r].get(u)) col |= 1ull << r;
      std::memcpy(host.data() + off_cols + size_t(u) * 8, &col, 8);
    }
  }
  void *blob = nullptr;
  if (cudaMalloc(&blob, total) != cudaSuccess) return fail(BCH_ENOMEM, "cudaMalloc for the code");
  unsigned char *b = static_cast<unsigned char *>(blob);
  dc.codes = reinterpret_cast<const uint16_t *>(b + off_codes);
  dc.rowmask = reinterpret_cast<const uint32_t *>(b + off_mask);
  dc.par = reinterpret_cast<const uint64_t *>(b + off_par);
  dc.colmask = reinterpret_cast<const uint64_t *>(b + off_cols);
  std::memcpy(host.data() + off_desc, &dc, sizeof(DevCode));
  cudaError_t e = cudaMemcpy(blob, host.data(), total, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(blob);
    return cuda_fail(e, "upload of the code");
  }
  c->dev_blob = blob;
  c->dc = dc;
  c->dev_dc = reinterpret_cast<DevCode *>(b + off_desc);
  return BCH_OK;
}

NmsArgs make_nms_args(const bch_code *code, const bch_nms_params *p, const float *llr, int ld, int F,
                      const uint16_t *autos, uint64_t *hard, uint8_t *iters, uint8_t *flags,
                      float *llr_out, unsigned *queue) {
  NmsArgs a;
  std::memset(&a, 0, sizeof(a));
  a.dc = code->dc;
  a.llr = llr;
  a.ld = ld;
  a.F = F;
  a.autos = autos;
  a.P = p->n_autos;
  a.hard = hard;
  a.iters = iters;
  a.flags = flags;
  a.llr_out = llr_out;
  a.ckpt = nullptr;
  a.queue = queue;
  a.check = check_word();
  a.I = p->iters;
  a.early_stop = p->early_stop ? 1 : 0;
  a.msg = int(p->msg);
  a.rescale = p->rescale ? 1 : 0;
  a.qfrac = p->qfrac;
  // with fractional bits the kernels round alpha 2^qfrac min (a power-of-two scale: exact)
  for (int t = 0; t < 32; t++) a.alpha[t] = t < p->iters ? ldexpf(p->alpha[t], p->qfrac) : 0.0f;
  return a;
}

}  // namespace

extern "C" {

const char *bch_status_str(bch_status s) {
  switch (s) {
    case BCH_OK: return "ok";
    case BCH_EINVAL: return "invalid argument";
    case BCH_ENOMEM: return "out of memory";
    case BCH_ECUDA: return "CUDA error";
    case BCH_ERANK: return "rank deficient parity-check matrix";
    case BCH_ETIMEOUT: return "timeout";
    case BCH_EBUDGET: return "over budget";
    case BCH_EBUSY: return "busy";
  }
  return "unknown status";
}

const char *bch_last_error(void) { return g_last_error.c_str(); }

const char *bch_version(void) { return "bchdec-gb300 1.0 (sm_103a)"; }

unsigned long long bch_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

int bch_is_checked(void) {
#ifdef BCH_CHECKED
  return 1;
#else
  return 0;
#endif
}

bch_status bch_check_read(uint32_t *word_out, int clear, void *stream) {
#ifdef BCH_CHECKED
  if (!word_out) return fail(BCH_EINVAL, "null word_out");
  unsigned *w = check_word();
  if (!w) return fail(BCH_ECUDA, "the check word's device address");
  BCH_CUDA(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)), "synchronise the stream");
  BCH_CUDA(cudaMemcpy(word_out, w, 4 * sizeof(unsigned), cudaMemcpyDeviceToHost), "read the check word");
  if (clear) {
    const unsigned init[4] = {0u, 0u, 0xffffffffu, 0xffffffffu};
    BCH_CUDA(cudaMemcpy(w, init, sizeof(init), cudaMemcpyHostToDevice), "clear the check word");
  }
  return BCH_OK;
#else
  (void)word_out;
  (void)clear;
  (void)stream;
  return fail(BCH_EINVAL, "this library was built without BCH_CHECKED");
#endif
}

static HoOptions ho_options(const bch_pcm_opts *opts) {
  HoOptions o;
  if (opts) {
    if (opts->q_rounds >= 0) o.q_rounds = opts->q_rounds;
    if (opts->sa_steps >= 0) o.sa_steps = opts->sa_steps;
    o.sa_lambda = opts->sa_lambda;
    if (opts->sa_t0_frac > 0) o.sa_t0_frac = opts->sa_t0_frac;
    if (opts->sa_cool > 0) o.sa_cool = opts->sa_cool;
  }
  return o;
}

static bch_status build_host(int n, int k, bch_pcm_kind kind, int m_rows, uint64_t seed,
                             const bch_pcm_opts *opts, bch_code *c) {
  std::string err;
  if (!make_algebra(n, k, &c->alg, &err)) return fail(BCH_EINVAL, err);
  c->kind = kind;
  if (kind == BCH_PCM_STANDARD) {
    c->rows = c->alg.std_h;
    return BCH_OK;
  }
  if (kind != BCH_PCM_OPTIMIZED) return fail(BCH_EINVAL, "unknown pcm kind");
  const HoOptions o = ho_options(opts);
  bch_status s = build_ho(c->alg, m_rows, seed, o, &c->rows, &c->r1_count, &err);
  if (s != BCH_OK) return fail(s, err);
  return BCH_OK;
}

bch_status bch_build_pcm_host(int n, int k, bch_pcm_kind kind, int m_rows, uint64_t seed,
                              const bch_pcm_opts *opts, uint8_t *dense, size_t capacity, int *rows) {
  if (!dense || !rows) return fail(BCH_EINVAL, "null output");
  bch_code c;
  bch_status s = build_host(n, k, kind, m_rows, seed, opts, &c);
  if (s != BCH_OK) return s;
  const size_t need = c.rows.size() * size_t(n);
  if (capacity < need) return fail(BCH_EINVAL, "capacity too small");
  for (size_t r = 0; r < c.rows.size(); r++)
    for (int i = 0; i < n; i++) dense[r * n + i] = c.rows[r].get(i) ? 1 : 0;
  *rows = int(c.rows.size());
  return BCH_OK;
}

bch_status bch_search_pcm(int n, int k, int m_rows, uint64_t seed, const bch_pcm_opts *opts,
                          int n_chains, long long *stats, uint8_t *dense_all, size_t capacity,
                          int *best, bch_code **out) {
  if (!out) return fail(BCH_EINVAL, "out is null");
  *out = nullptr;
  if (n_chains < 1 || n_chains > 4096) return fail(BCH_EINVAL, "n_chains must be in [1, 4096]");
  std::unique_ptr<bch_code> c(new (std::nothrow) bch_code());
  if (!c) return fail(BCH_ENOMEM, "host allocation");
  std::string err;
  if (!make_algebra(n, k, &c->alg, &err)) return fail(BCH_EINVAL, err);
  c->kind = BCH_PCM_OPTIMIZED;
  const HoOptions o = ho_options(opts);
  std::vector<Row> H0;
  uint64_t st0 = 0;
  bch_status s = prepare_ho(c->alg, m_rows, seed, o, &H0, &st0, &c->r1_count, &err);
  if (s != BCH_OK) return fail(s, err);
  const int Mo = int(H0.size()), M = n - k;
  if (Mo > 400) return fail(BCH_EINVAL, "the device search holds at most 400 rows");
  if (dense_all && capacity < size_t(n_chains) * Mo * n) return fail(BCH_EINVAL, "dense_all too small");
  // start temperature exactly as the host annealing computes it
  long long C4 = 0, SS = 0, E = 0;
  ho_loss_terms(n, H0, &C4, &SS, &E);
  const double lam = o.sa_lambda > 0.0 ? o.sa_lambda : double(n);
  const double loss0 = double(C4) + lam * (double(SS) - double(E) * double(E) / double(n)) / double(n);
  std::vector<ulonglong2> rows0(Mo);
  for (int r = 0; r < Mo; r++) rows0[r] = make_ulonglong2(H0[r].w[0], H0[r].w[1]);
  std::vector<uint64_t> states(n_chains);
  for (int ch = 0; ch < n_chains; ch++) states[ch] = st0 + uint64_t(ch) * 0xD1B54A32D192ED03ULL;
  ulonglong2 *d_rows0 = nullptr, *d_out = nullptr;
  uint64_t *d_st = nullptr;
  std::vector<ulonglong2> rows_out(size_t(n_chains) * Mo);
  cudaError_t e = cudaMalloc(&d_rows0, size_t(Mo) * sizeof(ulonglong2));
  if (e == cudaSuccess) e = cudaMalloc(&d_out, rows_out.size() * sizeof(ulonglong2));
  if (e == cudaSuccess) e = cudaMalloc(&d_st, size_t(n_chains) * 8);
  if (e == cudaSuccess) e = cudaMemcpy(d_rows0, rows0.data(), size_t(Mo) * sizeof(ulonglong2), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(d_st, states.data(), size_t(n_chains) * 8, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    AnnealArgs a;
    a.n = n;
    a.Mo = Mo;
    a.steps = o.sa_steps;
    a.chains = n_chains;
    a.lam = lam;
    a.T0 = o.sa_t0_frac * loss0;
    a.cool = o.sa_cool;
    a.rows0 = d_rows0;
    a.state0 = d_st;
    a.rows_out = d_out;
    e = launch_anneal(a, nullptr);
  }
  if (e == cudaSuccess) e = cudaMemcpy(rows_out.data(), d_out, rows_out.size() * sizeof(ulonglong2), cudaMemcpyDeviceToHost);
  cudaFree(d_rows0);
  cudaFree(d_out);
  cudaFree(d_st);
  if (e != cudaSuccess) return fail(BCH_ECUDA, std::string("annealing chains: ") + cudaGetErrorString(e));
  int kept = -1;
  double kept_loss = 0.0;
  std::vector<Row> best_rows;
  for (int ch = 0; ch < n_chains; ch++) {
    std::vector<Row> Hc(Mo);
    for (int r = 0; r < Mo; r++) {
      Hc[r].w[0] = rows_out[size_t(ch) * Mo + r].x;
      Hc[r].w[1] = rows_out[size_t(ch) * Mo + r].y;
    }
    const bool ok = repair_rank(n, M, Hc);
    long long c4 = 0, ss = 0, e2 = 0;
    ho_loss_terms(n, Hc, &c4, &ss, &e2);
    if (stats) {
      stats[size_t(ch) * 3] = c4;
      stats[size_t(ch) * 3 + 1] = ss;
      stats[size_t(ch) * 3 + 2] = ok ? 1 : 0;
    }
    if (dense_all)
      for (int r = 0; r < Mo; r++)
        for (int i = 0; i < n; i++) dense_all[(size_t(ch) * Mo + r) * n + i] = Hc[r].get(i) ? 1 : 0;
    const double loss = double(c4) + lam * (double(ss) - double(e2) * double(e2) / double(n)) / double(n);
    if (ok && (kept < 0 || loss < kept_loss)) {
      kept = ch;
      kept_loss = loss;
      best_rows = Hc;
    }
  }
  if (kept < 0) return fail(BCH_ERANK, "no annealing chain reached rank n-k");
  if (best) *best = kept;
  c->rows = std::move(best_rows);
  s = upload_code(c.get());
  if (s != BCH_OK) return s;
  *out = c.release();
  return BCH_OK;
}

bch_status bch_build_pcm(int n, int k, bch_pcm_kind kind, int m_rows, uint64_t seed,
                         const bch_pcm_opts *opts, bch_code **out) {
  if (!out) return fail(BCH_EINVAL, "out is null");
  *out = nullptr;
  bch_code *c = new (std::nothrow) bch_code();
  if (!c) return fail(BCH_ENOMEM, "host allocation");
  bch_status s0 = build_host(n, k, kind, m_rows, seed, opts, c);
  if (s0 != BCH_OK) {
    delete c;
    return s0;
  }
  bch_status s = upload_code(c);
  if (s != BCH_OK) {
    delete c;
    return s;
  }
  *out = c;
  return BCH_OK;
}

bch_status bch_nms_kernel_info(const bch_code *code, int msg, int n_autos, char *buf, size_t capacity) {
  if (!code_ok(code) || !buf || capacity == 0) return fail(BCH_EINVAL, "bad argument");
  std::string info;
  const int mode = kernel_mode();
  if (n_autos == 0) {
    info = "generic: plain decoder";
  } else if (mode == 1) {
    info = "generic: selected by BCHDEC_NMS_KERNEL";
  } else {
    std::string err;
    cudaKernel_t k = jit_kernel(code, msg, &err);
    info = k ? "jit" : "generic: " + err;
  }
  std::snprintf(buf, capacity, "%s", info.c_str());
  return BCH_OK;
}

bch_status bch_nms_jit_check(int n, int k, int m_rows, uint64_t seed, const bch_pcm_opts *opts, int msg,
                             char *log, size_t capacity) {
  if (!log || capacity == 0 || msg < BCH_MSG_FP32 || msg > BCH_MSG_INT8) return fail(BCH_EINVAL, "bad argument");
  log[0] = '\0';
  bch_code c;
  bch_status s = build_host(n, k, BCH_PCM_OPTIMIZED, m_rows, seed, opts, &c);
  if (s != BCH_OK) return s;
  std::string text;
  const bool ok = jit_compile_check(&c, msg, &text);
  std::snprintf(log, capacity, "%s", text.c_str());
  return ok ? BCH_OK : fail(BCH_ECUDA, "NVRTC compile failed");
}

bch_status bch_serve_jit_check(int n_codes, const int *n, const int *k, uint64_t seed, char *log,
                               size_t capacity) {
  if (!log || capacity == 0 || !n || !k || n_codes < 1 || n_codes > 8)
    return fail(BCH_EINVAL, "bad argument");
  log[0] = 0;
  std::unique_ptr<bch_code[]> cs(new bch_code[size_t(n_codes)]);
  std::vector<const bch_code *> ptrs;
  for (int i = 0; i < n_codes; i++) {
    bch_status st = build_host(n[i], k[i], BCH_PCM_OPTIMIZED, 0, seed, nullptr, &cs[size_t(i)]);
    if (st != BCH_OK) return st;
    ptrs.push_back(&cs[size_t(i)]);
  }
  std::string text;
  const bool ok = jit_serve_compile_check(ptrs.data(), n_codes, &text);
  std::snprintf(log, capacity, "%s", text.c_str());
  return ok ? BCH_OK : fail(BCH_ECUDA, "serving kernel compile failed");
}

bch_status bch_code_info(const bch_code *c, int *n, int *k, int *rows, int *edges, int *max_w) {
  if (!code_ok(c)) return fail(BCH_EINVAL, "null code");
  if (n) *n = c->alg.n;
  if (k) *k = c->alg.k;
  if (rows) *rows = int(c->rows.size());
  if (edges) *edges = c->dc.edges;
  if (max_w) *max_w = c->dc.max_w;
  return BCH_OK;
}

bch_status bch_pcm_export(const bch_code *c, uint8_t *dense, size_t capacity) {
  if (!code_ok(c) || !dense) return fail(BCH_EINVAL, "null argument");
  const size_t need = c->rows.size() * size_t(c->alg.n);
  if (capacity < need) return fail(BCH_EINVAL, "capacity too small");
  for (size_t r = 0; r < c->rows.size(); r++)
    for (int i = 0; i < c->alg.n; i++) dense[r * c->alg.n + i] = c->rows[r].get(i) ? 1 : 0;
  return BCH_OK;
}

void bch_code_free(bch_code *c) {
  if (!c) return;
  if (c->dev_blob) cudaFree(c->dev_blob);
  delete c;
}

bch_status bch_draw_automorphisms_host(int n, int n_autos, uint64_t seed, uint64_t frame0,
                                       int n_frames, uint16_t *out) {
  if (n != 15 && n != 63 && n != 127) return fail(BCH_EINVAL, "n must be 15, 63 or 127");
  if (n_autos < 1 || n_autos > 9) return fail(BCH_EINVAL, "n_autos must be in [1, 9]");
  if (n_frames < 0 || (n_frames > 0 && !out)) return fail(BCH_EINVAL, "bad output");
  draw_autos_host(n, n_autos, seed, frame0, n_frames, out);
  return BCH_OK;
}

bch_status bch_draw_automorphisms(int n, int n_autos, uint64_t seed, uint64_t frame0, int n_frames,
                                  uint16_t *out, void *stream) {
  if (n != 15 && n != 63 && n != 127) return fail(BCH_EINVAL, "n must be 15, 63 or 127");
  if (n_autos < 1 || n_autos > 9) return fail(BCH_EINVAL, "n_autos must be in [1, 9]");
  if (n_frames < 0 || (n_frames > 0 && !out)) return fail(BCH_EINVAL, "bad output");
  int ord = 1;
  for (int x = 2 % n; x != 1; x = (2 * x) % n) ord++;
  BCH_CUDA(launch_draw_autos(n, ord, n_autos, seed, frame0, n_frames, out,
                             static_cast<cudaStream_t>(stream)),
           "draw_autos");
  return BCH_OK;
}

bch_status bch_gen_frames(const bch_code *code, float ebn0_lo, float ebn0_hi, uint64_t seed,
                          uint64_t frame0, int n_frames, float *llr, int ld, uint64_t *codeword,
                          void *stream) {
  if (!code_ok(code)) return fail(BCH_EINVAL, "null code");
  if (n_frames < 0 || ld < code->alg.n || (n_frames > 0 && !llr)) return fail(BCH_EINVAL, "bad frames");
  if (code->alg.k > 128) return fail(BCH_EINVAL, "k > 128");
  GenArgs a;
  a.n = code->alg.n;
  a.k = code->alg.k;
  a.par = code->dc.par;
  a.ebn0_lo = ebn0_lo;
  a.ebn0_hi = ebn0_hi;
  a.seed = seed;
  a.frame0 = frame0;
  a.F = n_frames;
  a.ld = ld;
  a.llr = llr;
  a.codeword = codeword;
  BCH_CUDA(launch_gen_frames(a, static_cast<cudaStream_t>(stream)), "gen_frames");
  return BCH_OK;
}

bch_status bch_workspace_size(const bch_code *code, const bch_nms_params *params, int n_frames,
                              size_t *bytes) {
  if (!code_ok(code) || !bytes || n_frames < 0) return fail(BCH_EINVAL, "bad argument");
  const int it = params ? params->iters : 32;
  *bytes = ws_layout(n_frames, it).total;
  return BCH_OK;
}


static cudaError_t launch_jit(cudaKernel_t k, const bch_code *code, const NmsArgs &a, cudaStream_t st) {
  const int n = code->alg.n, tpb = jit_block_size(n), scr = jit_scratch_words(n);
  const size_t sa = a.msg == BCH_MSG_INT8 ? 4 : 4;
  const size_t sy = a.msg == BCH_MSG_FP32 ? 4 : (a.msg == BCH_MSG_FP16 ? 2 : 1);
  size_t smem = nms_table_bytes_host(code->dc) + 16 +
                size_t(tpb) * (size_t(a.P) * 4 + size_t(n) * (sa + sy) + size_t(scr) * sa);
  if (jit_split(n)) {  // two warps per 32 frames (see nms_split_persistent)
    const int G = jit_split_groups(), R = jit_split_chunk_rows();
    const size_t st = a.msg == BCH_MSG_FP32   ? SplitSmem<kFP32>::state_bytes(n, a.P, G, R)
                      : a.msg == BCH_MSG_FP16 ? SplitSmem<kFP16>::state_bytes(n, a.P, G, R)
                                              : SplitSmem<kINT8>::state_bytes(n, a.P, G, R);
    smem = nms_table_bytes_host(code->dc) + st;
  }
  if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
  const void *fn = reinterpret_cast<const void *>(k);
  int sms = 0, per_sm = 0;
  cudaError_t e = launch_geometry(fn, tpb, smem, &sms, &per_sm);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  long long blocks = (long long)sms * per_sm;
  const int fpb = jit_split(n) ? tpb / 2 : tpb;  // frames a block holds at a time
  const long long need = (a.F + fpb - 1) / fpb;
  if (blocks > need) blocks = need;
  if (blocks < 1) blocks = 1;
  void *args[] = {const_cast<NmsArgs *>(&a)};
  note_launch();
  return cudaLaunchKernel(fn, dim3(unsigned(blocks)), dim3(unsigned(tpb)), args, smem, st);
}

static cudaError_t launch_nms_code(const bch_code *code, const NmsArgs &a, cudaStream_t st,
                                   std::string *why) {
  const int mode = kernel_mode();
  // auto and jit: the specialised kernel (for n = 127 it spills but still runs 1.8x
  // faster than the precompiled one; its first compile takes tens of seconds and is
  // cached on disk); auto falls back to the precompiled kernel if it does not compile
  if (a.P > 0 && mode != 1) {
    std::string err;
    cudaKernel_t k = jit_kernel(code, a.msg, &err, a.qfrac);
    if (k) return launch_jit(k, code, a, st);
    if (why) *why = err;
    if (mode == 2) return cudaErrorNotSupported;
  }
  return launch_nms(a, st);
}

static bch_status run_nms(const bch_code *code, const bch_nms_params *params, const float *llr, int ld,
                          int n_frames, const uint16_t *autos, uint64_t *hard, uint8_t *iters,
                          uint8_t *flags, float *llr_out, float *ckpt, void *workspace,
                          cudaStream_t st) {
  bch_status s = check_params(code, params);
  if (s != BCH_OK) return s;
  s = check_frames(code, llr, ld, n_frames);
  if (s != BCH_OK) return s;
  if (n_frames == 0) return BCH_OK;
  if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255))
    return fail(BCH_EINVAL, "workspace must be non-null and 256-byte aligned");
  if (params->n_autos > 0 && !autos) return fail(BCH_EINVAL, "autos is null");
  const WsLayout L = ws_layout(n_frames, params->iters);
  unsigned char *ws = static_cast<unsigned char *>(workspace);
  unsigned *queue = reinterpret_cast<unsigned *>(ws + L.queues);
  BCH_CUDA(cudaMemsetAsync(queue, 0, 16, st), "clear queue");
  NmsArgs a = make_nms_args(code, params, llr, ld, n_frames, autos, hard, iters, flags, llr_out, queue);
  a.ckpt = ckpt;
  std::string why;
  cudaError_t e = launch_nms_code(code, a, st, &why);
  if (e != cudaSuccess) return fail(BCH_ECUDA, std::string("nms kernel: ") + cudaGetErrorString(e) + " " + why);
  return BCH_OK;
}

bch_status bch_nms_decode(const bch_code *code, const bch_nms_params *params, const float *llr, int ld,
                          int n_frames, const uint16_t *autos, uint64_t *hard, uint8_t *iters,
                          uint8_t *flags, float *llr_out, void *workspace, void *stream) {
  return run_nms(code, params, llr, ld, n_frames, autos, hard, iters, flags, llr_out, nullptr,
                 workspace, static_cast<cudaStream_t>(stream));
}

static bch_status run_osd(const bch_code *std_code, int order, const float *llr, int ld,
                          const uint32_t *list, const uint32_t *count, int max_frames, uint64_t *hard,
                          uint8_t *flags, unsigned *queue, cudaStream_t st, int scale_input = 0) {
  bch_status s = check_osd(nullptr, std_code, order);
  if (s != BCH_OK) return s;
  const int n = std_code->alg.n, M = n - std_code->alg.k;
  if (max_frames <= 0) return BCH_OK;
  OsdArgs a;
  a.n = n;
  a.k = std_code->alg.k;
  a.M = M;
  a.rows = reinterpret_cast<const uint4 *>(std_code->dc.rowmask);
  a.cols = std_code->dc.colmask;
  a.llr = llr;
  a.ld = ld;
  a.list = list;
  a.count = count;
  a.max_frames = max_frames;
  a.order = order;
  a.hard = hard;
  a.flags = flags;
  a.queue = queue;
  a.scale_input = scale_input;
  a.check = check_word();
  BCH_CUDA(launch_osd(a, st), "osd kernel");
  return BCH_OK;
}

bch_status bch_osd_decode(const bch_code *std_code, int order, const float *llr, int ld,
                          const uint32_t *frame_list, const uint32_t *count, int n_frames,
                          uint64_t *hard, uint8_t *flags, void *workspace, void *stream) {
  if (!frame_list || !count || !hard || !llr) return fail(BCH_EINVAL, "null argument");
  if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255))
    return fail(BCH_EINVAL, "workspace must be non-null and 256-byte aligned");
  if (code_ok(std_code) && ld < std_code->alg.n) return fail(BCH_EINVAL, "ld < n");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  unsigned *queue = reinterpret_cast<unsigned *>(workspace);
  BCH_CUDA(cudaMemsetAsync(queue, 0, 16, st), "clear queue");
  return run_osd(std_code, order, llr, ld, frame_list, count, n_frames, hard, flags, queue + 1, st);
}

bch_status bch_hybrid_decode(const bch_code *code, const bch_code *std_code, const bch_nms_params *params,
                             const float *llr, int ld, int n_frames, const uint16_t *autos, uint64_t *hard,
                             uint8_t *iters, uint8_t *flags, float *llr_out, uint32_t *failed_list,
                             uint32_t *failed_count, void *workspace, void *stream) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (!hard || !flags) return fail(BCH_EINVAL, "hybrid decoding needs hard and flags");
  // every argument is checked before the first launch, so a rejected call writes nothing
  bch_status s = check_params(code, params);
  if (s == BCH_OK) s = check_osd(code, std_code, params->osd_order);
  if (s != BCH_OK) return s;
  if (params->osd_input == 1 && !llr_out)
    return fail(BCH_EINVAL, "osd_input = 1 needs llr_out (the NMS output the OSD reads)");
  s = run_nms(code, params, llr, ld, n_frames, autos, hard, iters, flags, llr_out, nullptr,
                         workspace, st);
  if (s != BCH_OK || n_frames == 0) return s;
  const WsLayout L = ws_layout(n_frames, params->iters);
  unsigned char *ws = static_cast<unsigned char *>(workspace);
  uint32_t *list = failed_list ? failed_list : reinterpret_cast<uint32_t *>(ws + L.list);
  uint32_t *count = failed_count ? failed_count : reinterpret_cast<uint32_t *>(ws + L.count);
  BCH_CUDA(launch_compact(flags, n_frames, reinterpret_cast<uint32_t *>(ws + L.counts), list, count, st),
           "compaction");
  unsigned *queue = reinterpret_cast<unsigned *>(ws + L.queues);
  if (params->osd_input == 1)  // the failed frames' final y, scaled per frame in the OSD
    return run_osd(std_code, params->osd_order, llr_out, ld, list, count, n_frames, hard, flags, queue + 1,
                   st, 1);
  return run_osd(std_code, params->osd_order, llr, ld, list, count, n_frames, hard, flags, queue + 1, st);
}

bch_status bch_compact_failed(const uint8_t *flags, int n_frames, uint32_t *list, uint32_t *count,
                              void *workspace, void *stream) {
  if (n_frames < 0 || !count || (n_frames > 0 && (!flags || !list))) return fail(BCH_EINVAL, "bad argument");
  if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255))
    return fail(BCH_EINVAL, "workspace must be non-null and 256-byte aligned");
  const WsLayout L = ws_layout(n_frames, 1);
  BCH_CUDA(launch_compact(flags, n_frames,
                          reinterpret_cast<uint32_t *>(static_cast<unsigned char *>(workspace) + L.counts),
                          list, count, static_cast<cudaStream_t>(stream)),
           "compaction");
  return BCH_OK;
}

bch_status bch_count_errors(int n, const uint64_t *hard, const uint64_t *codeword, const uint8_t *iters,
                            const uint8_t *flags, int n_frames, long long *counters, void *stream) {
  if (n_frames < 0 || !counters || (n_frames > 0 && (!hard || !codeword)))
    return fail(BCH_EINVAL, "bad argument");
  BCH_CUDA(launch_count_errors(n, hard, codeword, iters, flags, n_frames, counters,
                               static_cast<cudaStream_t>(stream)),
           "count_errors");
  return BCH_OK;
}

bch_status bch_nms_forward_train(const bch_code *code, const bch_nms_params *params, const float *llr,
                                 int ld, int n_frames, const uint16_t *autos, float *ckpt, void *workspace,
                                 void *stream) {
  if (!ckpt) return fail(BCH_EINVAL, "ckpt is null");
  if (!params || params->msg != BCH_MSG_FP32 || params->n_autos < 1)
    return fail(BCH_EINVAL, "training runs the FP32 enhanced decoder");
  bch_nms_params p = *params;
  p.early_stop = 0;  // the training pass runs all iterations
  return run_nms(code, &p, llr, ld, n_frames, autos, nullptr, nullptr, nullptr, nullptr, ckpt, workspace,
                 static_cast<cudaStream_t>(stream));
}

bch_status bch_nms_backward(const bch_code *code, const bch_nms_params *params, const uint16_t *autos,
                            const float *ckpt, int ld, int n_frames, const float *grad_out, float *grad_llr,
                            float *grad_alpha, void *workspace, void *stream) {
  bch_status s = check_params(code, params);
  if (s != BCH_OK) return s;
  if (params->n_autos < 1) return fail(BCH_EINVAL, "backward needs n_autos >= 1");
  if (!ckpt || !grad_out || !grad_alpha || !autos) return fail(BCH_EINVAL, "null argument");
  if (ld < code->alg.n || n_frames < 0) return fail(BCH_EINVAL, "bad frames");
  if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255))
    return fail(BCH_EINVAL, "workspace must be non-null and 256-byte aligned");
  const WsLayout L = ws_layout(n_frames, params->iters);
  BwdArgs a;
  std::memset(&a, 0, sizeof(a));
  a.dc = code->dc;
  a.autos = autos;
  a.P = params->n_autos;
  a.ckpt = ckpt;
  a.ld = ld;
  a.F = n_frames;
  a.I = params->iters;
  a.grad_out = grad_out;
  a.grad_llr = grad_llr;
  a.partial = reinterpret_cast<float *>(static_cast<unsigned char *>(workspace) + L.red);
  a.check = check_word();
  for (int t = 0; t < 32; t++) a.alpha[t] = t < params->iters ? params->alpha[t] : 0.0f;
  BCH_CUDA(launch_backward(a, grad_alpha, static_cast<cudaStream_t>(stream)), "backward");
  return BCH_OK;
}

bch_status bch_bce_loss(int n, const float *y, int ld, const uint64_t *codeword, int n_frames, float *loss,
                        float *grad, void *workspace, void *stream) {
  if (!y || !codeword || !loss || n_frames < 0 || ld < n) return fail(BCH_EINVAL, "bad argument");
  if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255))
    return fail(BCH_EINVAL, "workspace must be non-null and 256-byte aligned");
  const WsLayout L = ws_layout(n_frames, 1);
  BCH_CUDA(launch_bce(n, y, ld, codeword, n_frames, loss, grad,
                      reinterpret_cast<float *>(static_cast<unsigned char *>(workspace) + L.red),
                      static_cast<cudaStream_t>(stream)),
           "bce");
  return BCH_OK;
}

bch_status bch_train_alpha(const bch_code *code, int n_autos, int iters, float *alpha_inout, int steps,
                           int batch, float ebn0_lo, float ebn0_hi, uint64_t seed, float lr,
                           float *loss_hist, void *stream) {
  return bch_train_alpha_resume(code, n_autos, iters, alpha_inout, nullptr, steps, batch, ebn0_lo, ebn0_hi,
                                seed, lr, loss_hist, stream);
}

bch_status bch_train_alpha_resume(const bch_code *code, int n_autos, int iters, float *alpha_inout,
                                  bch_adam_state *state, int steps, int batch, float ebn0_lo, float ebn0_hi,
                                  uint64_t seed, float lr, float *loss_hist, void *stream) {
  if (!code_ok(code) || !alpha_inout) return fail(BCH_EINVAL, "null argument");
  if (n_autos < 1 || n_autos > 9 || iters < 1 || iters > 32 || steps < 0 || batch < 1)
    return fail(BCH_EINVAL, "bad training shape");
  if (state && state->step != 0 && (state->iters != iters || state->step < 0 || state->batch != batch))
    return fail(BCH_EINVAL, "the saved training state belongs to another shape (iters or batch)");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int n = code->alg.n, ld = (n + 3) & ~3, W64 = (n + 63) / 64;
  const size_t fb = size_t(batch);
  float *llr = nullptr, *ckpt = nullptr, *gout = nullptr, *galpha = nullptr, *loss = nullptr;
  uint64_t *cw = nullptr;
  uint16_t *autos = nullptr;
  void *ws = nullptr;
  size_t wsb = ws_layout(batch, iters).total;
  bool ok = cudaMalloc(&llr, fb * ld * 4) == cudaSuccess &&
            cudaMalloc(&ckpt, size_t(iters + 1) * fb * ld * 4) == cudaSuccess &&
            cudaMalloc(&gout, fb * ld * 4) == cudaSuccess && cudaMalloc(&galpha, 32 * 4) == cudaSuccess &&
            cudaMalloc(&loss, 4) == cudaSuccess && cudaMalloc(&cw, fb * W64 * 8) == cudaSuccess &&
            cudaMalloc(&autos, fb * n_autos * 2) == cudaSuccess && cudaMalloc(&ws, wsb) == cudaSuccess;
  auto cleanup = [&]() {
    cudaFree(llr); cudaFree(ckpt); cudaFree(gout); cudaFree(galpha);
    cudaFree(loss); cudaFree(cw); cudaFree(autos); cudaFree(ws);
  };
  if (!ok) {
    cleanup();
    return fail(BCH_ENOMEM, "training buffers");
  }
  std::vector<double> m1(iters, 0.0), m2(iters, 0.0);
  long long step0 = 0;  // Adam steps (and frame batches) before this call
  if (state && state->step > 0) {
    step0 = state->step;
    for (int t = 0; t < iters; t++) {
      m1[t] = state->m[t];
      m2[t] = state->v[t];
    }
  }
  const double b1 = 0.9, b2 = 0.999, eps = 1e-8;
  bch_status s = BCH_OK;
  for (long long step = step0; step < step0 + steps && s == BCH_OK; step++) {
    bch_nms_params p;
    std::memset(&p, 0, sizeof(p));
    p.iters = iters;
    p.alpha = alpha_inout;
    p.n_autos = n_autos;
    p.early_stop = 0;
    p.msg = BCH_MSG_FP32;
    const uint64_t f0 = uint64_t(step) * uint64_t(batch);
    s = bch_gen_frames(code, ebn0_lo, ebn0_hi, seed, f0, batch, llr, ld, cw, st);
    if (s == BCH_OK) s = bch_draw_automorphisms(n, n_autos, seed ^ 0xA5A5A5A5ULL, f0, batch, autos, st);
    if (s == BCH_OK) s = bch_nms_forward_train(code, &p, llr, ld, batch, autos, ckpt, ws, st);
    if (s == BCH_OK)
      s = bch_bce_loss(n, ckpt + size_t(iters) * fb * ld, ld, cw, batch, loss, gout, ws, st);
    if (s == BCH_OK) s = bch_nms_backward(code, &p, autos, ckpt, ld, batch, gout, nullptr, galpha, ws, st);
    if (s != BCH_OK) break;
    float g[32], lv = 0;
    cudaError_t e = cudaMemcpyAsync(g, galpha, size_t(iters) * 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&lv, loss, 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
      s = cuda_fail(e, "training step");
      break;
    }
    if (loss_hist) loss_hist[step - step0] = lv;
    for (int t = 0; t < iters; t++) {
      m1[t] = b1 * m1[t] + (1 - b1) * g[t];
      m2[t] = b2 * m2[t] + (1 - b2) * double(g[t]) * g[t];
      const double mh = m1[t] / (1 - std::pow(b1, double(step + 1)));
      const double vh = m2[t] / (1 - std::pow(b2, double(step + 1)));
      alpha_inout[t] = float(alpha_inout[t] - lr * mh / (std::sqrt(vh) + eps));
    }
    if (state) {  // kept current after every completed step
      state->iters = iters;
      state->batch = batch;
      state->step = step + 1;
      for (int t = 0; t < iters; t++) {
        state->m[t] = m1[t];
        state->v[t] = m2[t];
      }
    }
  }
  cudaStreamSynchronize(st);
  cleanup();
  return s;
}

}  // extern "C"
