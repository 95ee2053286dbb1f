// Run-time specialisation of the enhanced min-sum kernel to one code's Tanner graph.
//
// The row loops of the precompiled kernel read column codes from shared memory and
// gather / scatter through per-frame permuted addresses for every edge.  Here the
// code's rows are emitted as straight-line CUDA source with the column indices as
// compile-time constants, so for one automorphism a thread first gathers the permuted
// word z_p[u] = y[pi_p^-1(u)] into registers (n loads), runs every check row on
// registers (min1 / min2 / sign product and the c2v sums S[u] for u in the row, 8
// lane-ops per edge) and finally scatters S into the frame's accumulator (n
// read-modify-writes).  For n <= 63 both z and S live in registers; for n = 127 z does
// and S lives in the thread's shared-memory column at compile-time offsets.
//
// Compiled with NVRTC (loaded with dlopen, so the library still loads on machines
// without it) for sm_103a and loaded with cudaLibraryLoadData; cached per source text.
#include <dlfcn.h>
#include <sys/stat.h>
#include <unistd.h>
#include <nvrtc.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "bch_internal.h"

namespace bchlib {

extern const char kDevTypesText[];
extern const char kNmsDeviceText[];
extern const char kAutosDeviceText[];
extern const char kOsdDeviceText[];
extern const char kServeDeviceText[];

namespace {

struct NvrtcApi {
  bool ok = false;
  std::string err;
  decltype(&nvrtcCreateProgram) create = nullptr;
  decltype(&nvrtcCompileProgram) compile = nullptr;
  decltype(&nvrtcGetProgramLogSize) log_size = nullptr;
  decltype(&nvrtcGetProgramLog) log = nullptr;
  decltype(&nvrtcGetCUBINSize) cubin_size = nullptr;
  decltype(&nvrtcGetCUBIN) cubin = nullptr;
  decltype(&nvrtcDestroyProgram) destroy = nullptr;
};

NvrtcApi &nvrtc() {
  static NvrtcApi api = [] {
    NvrtcApi a;
    void *h = dlopen("libnvrtc.so.13", RTLD_NOW | RTLD_LOCAL);
    if (!h) h = dlopen("/usr/local/cuda/lib64/libnvrtc.so.13", RTLD_NOW | RTLD_LOCAL);
    if (!h) {
      a.err = "libnvrtc.so.13 not found";
      return a;
    }
    a.create = reinterpret_cast<decltype(a.create)>(dlsym(h, "nvrtcCreateProgram"));
    a.compile = reinterpret_cast<decltype(a.compile)>(dlsym(h, "nvrtcCompileProgram"));
    a.log_size = reinterpret_cast<decltype(a.log_size)>(dlsym(h, "nvrtcGetProgramLogSize"));
    a.log = reinterpret_cast<decltype(a.log)>(dlsym(h, "nvrtcGetProgramLog"));
    a.cubin_size = reinterpret_cast<decltype(a.cubin_size)>(dlsym(h, "nvrtcGetCUBINSize"));
    a.cubin = reinterpret_cast<decltype(a.cubin)>(dlsym(h, "nvrtcGetCUBIN"));
    a.destroy = reinterpret_cast<decltype(a.destroy)>(dlsym(h, "nvrtcDestroyProgram"));
    a.ok = a.create && a.compile && a.log_size && a.log && a.cubin_size && a.cubin && a.destroy;
    if (!a.ok) a.err = "libnvrtc.so.13 lacks an entry point";
    return a;
  }();
  return api;
}

// Per-format definitions of the row macros used by the generated rows.  Within one
// automorphism z is fixed, so c2v(j,u) = sg_j sgn(z_u) alpha m_j(u) with sg_j the sign
// product of the whole row: the rows accumulate T[u] = sum_j sg_j alpha m_j(u) and the
// factor sgn(z_u) is applied once per variable at the end.  sg_j is the parity of the
// row's negative entries, taken from the copy's sign mask with the row mask as an
// immediate; BCH_RM receives it in bit 31 (popc << 31: one operation, no select) and
// applies it to alpha once (-alpha m rounds to exactly -(alpha m) in every format).  m_j(u) is min1 except at the row's minimum, handled by a predicated add
// of (v2 - v1) -- this keeps min/max/compare work on the ALU pipe down to ~4 operations
// per edge and moves the additions to the FMA pipe.  With the pair knob on, the two
// smallest magnitudes are tracked two edges at a time: with lo/hi the sorted pair,
// min1' = min(min1, lo) and min2' = min(max(min1, lo), min2, hi) (second smallest of
// four values with min1 <= min2), 5 operations per pair with a three-input minimum
// instead of 6.
const char *row_macros(int msg) {
  if (msg == 2)
    return R"(
#define BCH_VT int
#define BCH_R0 { int m1_ = 1 << 20, m2_ = 1 << 20;
#define BCH_R1(u) { const int a_ = abs(z[u]); m2_ = min(m2_, max(m1_, a_)); m1_ = min(m1_, a_); }
#define BCH_R1F(u, v) { const int p_ = abs(z[u]), q_ = abs(z[v]); m1_ = min(p_, q_); m2_ = max(p_, q_); }
#define BCH_R1P(u, v) { const int p_ = abs(z[u]), q_ = abs(z[v]); const int lo_ = min(p_, q_); \
  m2_ = __vimin3_s32(m2_, max(m1_, lo_), max(p_, q_)); m1_ = min(m1_, lo_); }
#define BCH_RM(SG) const float as_ = flip_sign(alpha, (SG)); \
  const int v1_ = rne_product(as_, m1_); const int dv_ = rne_product(as_, m2_) - v1_;
#define BCH_R2(u) BCH_SV(u) += v1_; if (abs(z[u]) == m1_) BCH_SV(u) += dv_;
#define BCH_R2I(u) BCH_SV(u) = v1_; if (abs(z[u]) == m1_) BCH_SV(u) += dv_;
#define BCH_R2F(u) BCH_R2(u)
#define BCH_RE }
#define BCH_FIN(u) ((z[u] < 0) ? -BCH_SV(u) : BCH_SV(u))
#define BCH_R0B int n1_ = 1 << 20, n2_ = 1 << 20;
#define BCH_R1B(u) { const int a_ = abs(z[u]); n2_ = min(n2_, max(n1_, a_)); n1_ = min(n1_, a_); }
#define BCH_RJ m2_ = __vimin3_s32(max(m1_, n1_), m2_, n2_); m1_ = min(m1_, n1_);
)";
  if (msg == 1)
    return R"(
#define BCH_VT float
#define BCH_R0 { float m1_ = FLT_MAX, m2_ = FLT_MAX;
#define BCH_R1(u) m2_ = fminf(m2_, fmaxf(m1_, fabsf(z[u]))); m1_ = fminf(m1_, fabsf(z[u]));
#define BCH_R1F(u, v) { const float a_ = fabsf(z[u]), b_ = fabsf(z[v]); \
  m1_ = fminf(a_, b_); m2_ = fmaxf(a_, b_); }
#define BCH_R1P(u, v) { const float a_ = fabsf(z[u]), b_ = fabsf(z[v]); const float lo_ = fminf(a_, b_); \
  m2_ = bch_min3f(m2_, fmaxf(m1_, lo_), fmaxf(a_, b_)); m1_ = fminf(m1_, lo_); }
#define BCH_RM(SG) const float as_ = flip_sign(alpha, (SG)); \
  const float v1_ = half_product(as_, m1_); const float dv_ = half_product(as_, m2_) - v1_;
#define BCH_R2(u) BCH_SV(u) += v1_; if (fabsf(z[u]) == m1_) BCH_SV(u) += dv_;
#define BCH_R2I(u) BCH_SV(u) = v1_; if (fabsf(z[u]) == m1_) BCH_SV(u) += dv_;
#define BCH_R2F(u) { const float p_ = (fabsf(z[u]) - m1_) * 0x1p100f; \
  BCH_SV(u) = __fmaf_rn(dv_, __saturatef(__fmaf_rn(-p_, 0x1p100f, 1.0f)), BCH_SV(u) + v1_); }
#define BCH_RE }
#define BCH_FIN(u) flip_sign(BCH_SV(u), __float_as_uint(z[u]))
#define BCH_R0B float n1_ = FLT_MAX, n2_ = FLT_MAX;
#define BCH_R1B(u) n2_ = fminf(n2_, fmaxf(n1_, fabsf(z[u]))); n1_ = fminf(n1_, fabsf(z[u]));
#define BCH_RJ m2_ = bch_min3f(fmaxf(m1_, n1_), m2_, n2_); m1_ = fminf(m1_, n1_);
)";
  return R"(
#define BCH_VT float
#define BCH_R0 { float m1_ = FLT_MAX, m2_ = FLT_MAX;
#define BCH_R1(u) m2_ = fminf(m2_, fmaxf(m1_, fabsf(z[u]))); m1_ = fminf(m1_, fabsf(z[u]));
#define BCH_R1F(u, v) { const float a_ = fabsf(z[u]), b_ = fabsf(z[v]); \
  m1_ = fminf(a_, b_); m2_ = fmaxf(a_, b_); }
#define BCH_R1P(u, v) { const float a_ = fabsf(z[u]), b_ = fabsf(z[v]); const float lo_ = fminf(a_, b_); \
  m2_ = bch_min3f(m2_, fmaxf(m1_, lo_), fmaxf(a_, b_)); m1_ = fminf(m1_, lo_); }
#define BCH_RM(SG) const float as_ = flip_sign(alpha, (SG)); \
  const float v1_ = as_ * m1_; const float dv_ = as_ * m2_ - v1_;
#define BCH_R2(u) BCH_SV(u) += v1_; if (fabsf(z[u]) == m1_) BCH_SV(u) += dv_;
#define BCH_R2I(u) BCH_SV(u) = v1_; if (fabsf(z[u]) == m1_) BCH_SV(u) += dv_;
#define BCH_R2F(u) { const float p_ = (fabsf(z[u]) - m1_) * 0x1p100f; \
  BCH_SV(u) = __fmaf_rn(dv_, __saturatef(__fmaf_rn(-p_, 0x1p100f, 1.0f)), BCH_SV(u) + v1_); }
#define BCH_RE }
#define BCH_FIN(u) flip_sign(BCH_SV(u), __float_as_uint(z[u]))
#define BCH_R0B float n1_ = FLT_MAX, n2_ = FLT_MAX;
#define BCH_R1B(u) n2_ = fminf(n2_, fmaxf(n1_, fabsf(z[u]))); n1_ = fminf(n1_, fabsf(z[u]));
#define BCH_RJ m2_ = bch_min3f(fmaxf(m1_, n1_), m2_, n2_); m1_ = fminf(m1_, n1_);
)";
}

// Macros of the split mapping (two warps per 32 frames, each owning half of the
// variables): BCH_PS stores the half's partial (min1 with the sign parity in its sign
// bit, min2) of row r into buffer B; BCH_Q combines both halves' partials of row r into
// m1_, m2_ and the row's sign parity sgp_ (bit 31; inside a BCH_R0 block).
const char *split_macros(int msg) {
  if (msg == 2)
    return R"(
#define BCH_PS(B, r, SG) B[((r) * 2 + BCH_H) * BCH_FS] = \
  make_float2(__int_as_float(m1_ | int(uint32_t(SG) & kSign)), __int_as_float(m2_));
#define BCH_Q(B, r) const float2 qa_ = B[((r) * 2) * BCH_FS], qb_ = B[((r) * 2 + 1) * BCH_FS]; \
  const int xa_ = __float_as_int(qa_.x), xb_ = __float_as_int(qb_.x); \
  const int a1_ = xa_ & 0x7fffffff, b1_ = xb_ & 0x7fffffff; \
  m1_ = min(a1_, b1_); m2_ = min(max(a1_, b1_), min(__float_as_int(qa_.y), __float_as_int(qb_.y))); \
  const uint32_t sgp_ = uint32_t(xa_ ^ xb_);
)";
  return R"(
#define BCH_PS(B, r, SG) B[((r) * 2 + BCH_H) * BCH_FS] = \
  make_float2(__uint_as_float(__float_as_uint(m1_) | (uint32_t(SG) & kSign)), m2_);
#define BCH_Q(B, r) const float2 qa_ = B[((r) * 2) * BCH_FS], qb_ = B[((r) * 2 + 1) * BCH_FS]; \
  const float a1_ = fabsf(qa_.x), b1_ = fabsf(qb_.x); \
  m1_ = fminf(a1_, b1_); m2_ = fminf(fmaxf(a1_, b1_), fminf(qa_.y, qb_.y)); \
  const uint32_t sgp_ = __float_as_uint(qa_.x) ^ __float_as_uint(qb_.x);
)";
}

struct Compiled {
  cudaLibrary_t lib = nullptr;
  cudaKernel_t kernel = nullptr;
  std::string err;
};

std::mutex g_mu;
std::map<std::string, std::shared_ptr<Compiled>> g_cache;

}  // namespace

namespace {
int env_int(const char *name, int lo, int hi, int dflt) {
  const char *v = std::getenv(name);
  if (!v) return dflt;
  const int x = std::atoi(v);
  return x >= lo && x <= hi ? x : dflt;
}
}  // namespace

// n = 127: the split mapping (two warps per 32 frames, half of the variables each, no
// spills) unless BCHDEC_JIT_SPLIT=0 selects the one-thread-per-frame kernel (a tuning
// and comparison knob; both compute identical results).
bool jit_split(int n) { return n > 63 && env_int("BCHDEC_JIT_SPLIT", 0, 1, 1) == 1; }
int jit_split_groups() { return 4; }      // 32-frame groups per block: 256 threads
int jit_split_chunk_rows() { return 16; } // rows per partial exchange

// Threads per block: 256 for n <= 63 (two warps per scheduler, all in lockstep so the
// straight-line body is fetched once per block; 255 registers hold the 2n
// register-resident values without spilling), 64 for n = 127.  BCHDEC_JIT_TPB (a
// multiple of 32, 64..512) overrides it for n <= 63 -- a tuning knob.  Measured on the
// (63,36) + (63,45) workload: 256 threads 187.1 M frames/s, 384 threads 186.0.
int jit_block_size(int n) {
  if (n > 63) return jit_split(n) ? 64 * jit_split_groups() : 64;
  const int t = env_int("BCHDEC_JIT_TPB", 64, 512, 256);
  return t % 32 == 0 ? t : 256;
}
// BCHDEC_JIT_PAIRS=1 tracks min1/min2 two edges at a time (tuning knob; off by default:
// it needs more registers and measured 1-2% slower).
bool jit_pairs() { return env_int("BCHDEC_JIT_PAIRS", 0, 1, 0) == 1; }
// BCHDEC_JIT_CHAINS=2 runs each row's first pass as two independent min1/min2 chains
// (even and odd edges) joined at the end -- min1 = min(a1, b1), min2 = min(max(a1, b1),
// a2, b2), the row's two smallest magnitudes whatever the order, so the results are
// bit-identical -- giving the scheduler two dependency chains per row (tuning knob).
int jit_chains() { return env_int("BCHDEC_JIT_CHAINS", 1, 2, 1); }
// Percentage of output-pass edges emitted in the compare-free form: with t = |z| - min1
// (>= 0), g = sat(1 - (t 2^100) 2^100) is exactly 1 when t = 0 and 0 otherwise
// (denormals included: t >= 2^-149), and fma(dv, g, S + v1) rounds like the
// predicated form (S + v1) + dv.  Five FMA-pipe operations replace one ALU compare and
// two additions.  BCHDEC_JIT_FMA_PCT (0..100) is a tuning knob.
int jit_fma_percent() { return env_int("BCHDEC_JIT_FMA_PCT", 0, 100, 0); }
bool jit_lockstep(int n) { return n <= 63; }
// Resident blocks per SM the register budget is sized for: 384 threads per SM for
// n <= 63 (at most 170 registers each, about the 2n register-resident values plus
// temporaries; a block of 256 gets 255).
int jit_min_blocks(int n) {
  const char *v = std::getenv("BCHDEC_JIT_MIN_BLOCKS");  // tuning knob (register budget)
  if (v && std::atoi(v) >= 1 && std::atoi(v) <= 8) return std::atoi(v);
  if (n <= 63) return std::max(1, 384 / jit_block_size(n));
  return jit_split(n) ? 1 : 2;
}
int jit_scratch_words(int n) { return n <= 63 || jit_split(n) ? 0 : n; }

// Common prologue of the generated sources: fixed-width types, the embedded device
// headers, the three-input minimum and the row macros of one storage format.
static void emit_prologue(std::ostringstream &o, int msg, bool serving) {
  o << "typedef unsigned int uint32_t;\ntypedef int int32_t;\ntypedef unsigned short uint16_t;\n"
       "typedef unsigned char uint8_t;\ntypedef signed char int8_t;\n"
       "typedef unsigned long long uint64_t;\ntypedef unsigned long long uintptr_t;\n"
       "#define FLT_MAX 3.402823466e+38f\n#include <cuda_fp16.h>\n";
  o << kDevTypesText << "\n" << kNmsDeviceText << "\n";
  if (serving) o << kAutosDeviceText << "\n" << kOsdDeviceText << "\n" << kServeDeviceText << "\n";
  o << "namespace bchlib {\n"
    << "__device__ __forceinline__ float bch_min3f(float a, float b, float c) {\n"
    << "  float d;\n  asm(\"min.f32 %0, %1, %2, %3;\" : \"=f\"(d) : \"f\"(a), \"f\"(b), \"f\"(c));\n"
    << "  return d;\n}\n"
    << row_macros(msg);
}

// The statements of one automorphism copy of code c: gather z_p from the frame's y
// column (element stride `stride`), the rows as straight-line code, scatter into the
// accumulator column.  They use y, acc, scr, jr, sp and alpha; with `scratch` the row
// sums live in the scratch column (same stride), else in registers.
// The gather and scatter positions of a copy as running offsets.  pi^-1(u) =
// rotr_m(u, j) + s' = u 2^-j + s' mod n (rotating right by j multiplies by 2^-j modulo
// 2^m - 1), so the element offset of variable u is sp stride + u (2^-j stride) mod
// n stride: four interleaved chains (u = k mod 4) step by 4 (2^-j stride) with one
// modular add per variable, instead of a bit-field extract, a modular add and a
// multiply -- the same positions.  Measured on the config-2 mix: FP32 0.540 of the
// peak against 0.515 (FP16 +5%, INT8 +1.5%); BCHDEC_JIT_INCR=0 restores the direct form.
bool jit_incr() { return env_int("BCHDEC_JIT_INCR", 0, 1, 1) == 1; }
// The first row of a column assigns its row sum instead of adding to zero (the same
// value but for the sign of a zero, which the accumulator, +0 at each iteration, cannot
// see); BCHDEC_JIT_FIRST_ASSIGN=0 adds as the rows after it do (a tuning knob).
bool jit_first_assign() { return env_int("BCHDEC_JIT_FIRST_ASSIGN", 0, 1, 1) == 1; }
// The lockstep kernel synchronises its block once per iteration; a block barrier before
// each automorphism copy as well (BCHDEC_JIT_COPY_BARRIER=1, a knob) measured 0.5%
// slower on the config-2 mix: a copy touches only its thread's columns.
bool jit_copy_barrier() { return env_int("BCHDEC_JIT_COPY_BARRIER", 0, 1, 0) == 1; }
// The statement that builds the sign words ng[] of count variables z[0..count): bit
// u & 31 of word u >> 5 is the sign of z_u.
static std::string sign_word_loop(int count, int msg, const char *indent) {
  const std::string bits = msg == 2 ? "uint32_t(z[u])" : "__float_as_uint(z[u])";
  std::ostringstream o;
  o << "#pragma unroll\n" << indent << "for (int u = 0; u < " << count << "; u++) ng[u >> 5] |= (" << bits
    << " >> 31) << (u & 31);\n";
  return o.str();
}

// The four running offsets o0_..o3_ of variables u0..u0 + 3 and their common step st4_
// (stride: a C expression; u0 u 2^-j is formed by doubling and adding at emission).
static void emit_offset_chains(std::ostringstream &o, int n, int m, const std::string &stride, int u0 = 0) {
  o << "      const uint32_t N_ = " << n << "u * (" << stride << ");\n"
    << "      const uint32_t st1_ = bfe32(1u | (1u << " << m << "), jr, " << m << ") * (" << stride << ");\n"
    << "      const uint32_t st2_ = addmod(st1_, st1_, N_), st3_ = addmod(st2_, st1_, N_);\n"
    << "      const uint32_t st4_ = addmod(st2_, st2_, N_);\n"
    << "      uint32_t o0_ = sp * (" << stride << ");\n";
  if (u0 > 0) {  // o0_ += u0 st1_ mod N_
    o << "      { uint32_t t_ = st1_;\n";
    for (int b = 0, v = u0; v; b++, v >>= 1) {
      if (v & 1) o << "        o0_ = addmod(o0_, t_, N_);\n";
      if (v >> 1) o << "        t_ = addmod(t_, t_, N_);\n";
    }
    o << "      }\n";
  }
  o << "      uint32_t o1_ = addmod(o0_, st1_, N_), o2_ = addmod(o0_, st2_, N_), o3_ = addmod(o0_, st3_, N_);\n";
}

// "STMT" with the variable index in U and its element offset in O, for every variable,
// through the offset chains.
static void emit_chain_loop(std::ostringstream &o, int n, const std::string &stmt_u_o) {
  for (int u = 0; u < n; u++) {
    const std::string ov = "o" + std::to_string(u & 3) + "_";
    std::string st = stmt_u_o;
    for (size_t q; (q = st.find("@U")) != std::string::npos;) st.replace(q, 2, std::to_string(u));
    for (size_t q; (q = st.find("@O")) != std::string::npos;) st.replace(q, 2, ov);
    o << "      " << st << "\n";
    if (u + 4 < n) o << "      " << ov << " = addmod(" << ov << ", st4_, N_);\n";
  }
}

static void emit_copy_body(std::ostringstream &o, const bch_code *c, int msg, int stride, bool scratch) {
  const int n = c->alg.n, m = c->alg.m;
  const int nw = (n + 31) / 32;
  o << "#undef BCH_SV\n";
  if (scratch)
    o << "#define BCH_SV(u) scr[(u) * " << stride << "]\n";
  else
    o << "#define BCH_SV(u) S[u]\n";
  o << "    BCH_VT z[" << n << "];\n";
  if (jit_incr()) {
    o << "    {\n";
    emit_offset_chains(o, n, m, std::to_string(stride) + "u");
    emit_chain_loop(o, n, "z[@U] = ld_y(y + @O);");
    o << "    }\n";
  } else {
    o << "#pragma unroll\n    for (int u = 0; u < " << n << "; u++) {\n"
      << "      const uint32_t i = addmod(bfe32(uint32_t(u) | (uint32_t(u) << " << m << "), jr, " << m
      << "), sp, " << n << ");\n      z[u] = ld_y(y + i * " << stride << ");\n    }\n";
  }
  if (scratch)
    o << "#pragma unroll\n    for (int u = 0; u < " << n << "; u++) BCH_SV(u) = 0;\n";
  else
    o << "    StoreT<" << msg << ">::A S[" << n << "];\n#pragma unroll\n    for (int u = 0; u < " << n
      << "; u++) S[u] = 0;\n";
  // sign mask of the permuted word: bit u = [z_u < 0]
  o << "    uint32_t ng[" << nw << "];\n#pragma unroll\n    for (int w = 0; w < " << nw << "; w++) ng[w] = 0u;\n"
    << sign_word_loop(n, msg, "    ");
  // rows, grouped by weight like the device image
  const int fma_pct = jit_fma_percent();
  int fma_acc = 0;
  // BCHDEC_JIT_ROW_FENCE=1: a compiler fence after each row keeps the scheduler from
  // overlapping the shared-memory row sums of many rows (n = 127: 0.55 KB of spills
  // instead of 2.5 KB, but measured 4% slower, so off by default)
  const bool fence = env_int("BCHDEC_JIT_ROW_FENCE", 0, 1, 0) == 1;
  std::vector<char> touched(n, 0);
  for (const Row &row : c->rows) {
    std::vector<int> cols;
    for (int u = 0; u < n; u++)
      if (row.get(u)) cols.push_back(u);
    uint32_t mw[4] = {0, 0, 0, 0};
    for (int u : cols) mw[u >> 5] |= 1u << (u & 31);
    std::ostringstream sg;
    sg << "(__popc(";
    bool first = true;
    for (int w = 0; w < nw; w++) {
      if (!mw[w]) continue;
      if (!first) sg << " ^ ";
      sg << "(ng[" << w << "] & 0x" << std::hex << mw[w] << std::dec << "u)";
      first = false;
    }
    sg << ") << 31)";
    o << "    BCH_R0";
    size_t e = 0;
    const bool pairs = jit_pairs();
    if (jit_chains() == 2 && cols.size() >= 4) {
      o << " BCH_R0B";
      for (size_t q = 0; q < cols.size(); q++) o << (q & 1 ? " BCH_R1B(" : " BCH_R1(") << cols[q] << ")";
      o << " BCH_RJ";
      e = cols.size();
    }
    if (pairs && e == 0 && cols.size() >= 2) {
      o << " BCH_R1F(" << cols[0] << ", " << cols[1] << ")";
      e = 2;
    }
    for (; pairs && e + 1 < cols.size(); e += 2) o << " BCH_R1P(" << cols[e] << ", " << cols[e + 1] << ")";
    for (; e < cols.size(); e++) o << " BCH_R1(" << cols[e] << ")";
    o << " BCH_RM(" << sg.str() << ")";
    // output pass: a share of the edges use the compare-free form (FMA pipe) so that
    // the ALU and FMA pipes carry similar loads; both forms round identically
    for (size_t q = 0; q < cols.size(); q++) {
      fma_acc += fma_pct;
      const bool f = fma_acc >= 100;
      if (f) fma_acc -= 100;
      // the first row of a column assigns its row sum: 0 + v1 = v1 but for the sign of a
      // zero, which no later addition to the accumulator (+0 at each iteration) can see
      if (!touched[cols[q]] && jit_first_assign()) {
        touched[cols[q]] = 1;
        o << " BCH_R2I(" << cols[q] << ")";
      } else {
        o << (f ? " BCH_R2F(" : " BCH_R2(") << cols[q] << ")";
      }
    }
    o << " BCH_RE" << (fence ? " asm volatile(\"\" ::: \"memory\");" : "") << "\n";
  }
  if (jit_incr()) {
    o << "    {\n";
    emit_offset_chains(o, n, m, std::to_string(stride) + "u");
    emit_chain_loop(o, n, "acc[@O] += BCH_FIN(@U);");
    o << "    }\n";
  } else {
    o << "#pragma unroll\n    for (int u = 0; u < " << n << "; u++) {\n"
      << "      const uint32_t i = addmod(bfe32(uint32_t(u) | (uint32_t(u) << " << m << "), jr, " << m
      << "), sp, " << n << ");\n      acc[i * " << stride << "] += BCH_FIN(u);\n    }\n";
  }
}

// The batch kernel's copy functor `name` (columns of stride `stride`).
static void emit_copy(std::ostringstream &o, const bch_code *c, int msg, const std::string &name, int stride,
                      bool scratch) {
  o << "struct " << name << " {\n  static constexpr int kScratch = " << (scratch ? c->alg.n : 0) << ";\n"
    << "  __device__ __forceinline__ void operator()(const SmemTables &, int, uint32_t, uint32_t,\n"
    << "      StoreT<" << msg << ">::Y *y, StoreT<" << msg << ">::A *acc, StoreT<" << msg
    << ">::A *scr, uint32_t jr, uint32_t sp, uint32_t, float alpha) const {\n";
  emit_copy_body(o, c, msg, stride, scratch);
  o << "  }\n};\n";
}

// The serving kernel's copy of code c (FP32) as a separate function, so that the
// compiler optimises each code's rows on their own: the lane's columns (stride 32)
// are found from the dynamic shared-memory base, in the serving layout (accumulator,
// y, scratch).
static void emit_serve_copy(std::ostringstream &o, const bch_code *c, const std::string &name, bool scratch) {
  o << "__device__ __noinline__ void " << name << "(uint32_t jr, uint32_t sp, float alpha) {\n"
    << "  extern __shared__ __align__(16) unsigned char smem[];\n"
    << "  float *acc = reinterpret_cast<float *>(smem) + lane_id();\n"
    << "  float *y = acc + 128 * 32;\n  float *scr = y + 128 * 32;\n  (void)scr;\n";
  emit_copy_body(o, c, 0, 32, scratch);
  o << "}\n";
}

// One half of the split mapping's automorphism copy: gather the half's 64 (or 63)
// values of z_p, for every chunk of R rows the first pass over the half's columns
// (partials to buffer A or B), a barrier, the second pass (combine, output pass), and
// finally scatter the half's row sums.  Both halves are emitted from the same chunk
// list, so they pass the same barriers.
static void emit_split_half(std::ostringstream &o, const bch_code *c, int msg, int h, int R,
                            const std::string &prefix = "split_half") {
  const int n = c->alg.n, m = c->alg.m;
  const int u0 = 64 * h, u1 = std::min(n, 64 * h + 64), nh = u1 - u0;
  const int nwh = (nh + 31) / 32;
  o << "__device__ " << (std::getenv("BCHDEC_JIT_SPLIT_NOINLINE") ? "__noinline__" : "__forceinline__") << " void "
    << prefix << h << "(StoreT<" << msg << ">::Y *y, StoreT<" << msg
    << ">::A *acc, float2 *pa, float2 *pb, uint32_t jr, uint32_t sp, float alpha) {\n"
    << "#undef BCH_SV\n#define BCH_SV(u) S[u]\n#undef BCH_H\n#define BCH_H " << h << "\n"
    << "  BCH_VT z[" << nh << "];\n";
  if (jit_incr()) {
    o << "  {\n";
    emit_offset_chains(o, n, m, "BCH_FS", u0);
    emit_chain_loop(o, nh, "z[@U] = ld_y(y + @O);");
    o << "  }\n";
  } else {
    o << "#pragma unroll\n  for (int u = 0; u < " << nh << "; u++) {\n"
      << "    const uint32_t uu = uint32_t(u + " << u0 << ");\n"
      << "    const uint32_t i = addmod(bfe32(uu | (uu << " << m << "), jr, " << m << "), sp, " << n << ");\n"
      << "    z[u] = ld_y(y + i * BCH_FS);\n  }\n";
  }
  o
    << "  StoreT<" << msg << ">::A S[" << nh << "];\n#pragma unroll\n  for (int u = 0; u < " << nh
    << "; u++) S[u] = 0;\n"
    << "  uint32_t ng[" << nwh << "];\n#pragma unroll\n  for (int w = 0; w < " << nwh << "; w++) ng[w] = 0u;\n"
    << sign_word_loop(nh, msg, "  ");
  // the half's columns (local indices) and its sign-parity expression, per row
  const int M = int(c->rows.size());
  std::vector<std::vector<int>> cols(M);
  std::vector<std::string> par(M);
  for (int r = 0; r < M; r++) {
    uint32_t mw[2] = {0, 0};
    for (int u = u0; u < u1; u++)
      if (c->rows[r].get(u)) {
        cols[r].push_back(u - u0);
        mw[(u - u0) >> 5] |= 1u << ((u - u0) & 31);
      }
    std::ostringstream sg;
    if (!mw[0] && !mw[1]) {
      sg << "0u";
    } else {
      sg << "(__popc(";
      bool first = true;
      for (int w = 0; w < 2; w++) {
        if (!mw[w]) continue;
        if (!first) sg << " ^ ";
        sg << "(ng[" << w << "] & 0x" << std::hex << mw[w] << std::dec << "u)";
        first = false;
      }
      sg << ") << 31)";
    }
    par[r] = sg.str();
  }
  const int nchunk = (M + R - 1) / R;
  auto pass1 = [&](int ch) {
    const char *buf = (ch & 1) ? "pb" : "pa";
    for (int r = ch * R; r < std::min(M, ch * R + R); r++) {
      o << "  BCH_R0";
      for (int u : cols[r]) o << " BCH_R1(" << u << ")";
      o << " BCH_PS(" << buf << ", " << (r - ch * R) << ", " << par[r] << ") BCH_RE\n";
    }
  };
  std::vector<char> touched(nh, 0);  // first row of a column assigns (see emit_copy_body)
  auto pass2 = [&](int ch) {
    const char *buf = (ch & 1) ? "pb" : "pa";
    for (int r = ch * R; r < std::min(M, ch * R + R); r++) {
      if (cols[r].empty()) continue;  // no edge of this half: nothing to add
      o << "  BCH_R0 BCH_Q(" << buf << ", " << (r - ch * R) << ") BCH_RM(sgp_)";
      for (int u : cols[r]) {
        o << (touched[u] || !jit_first_assign() ? " BCH_R2(" : " BCH_R2I(") << u << ")";
        touched[u] = 1;
      }
      o << " BCH_RE\n";
    }
  };
  pass1(0);
  for (int ch = 0; ch < nchunk; ch++) {
    o << "  bar_block(BCH_TPB);\n";
    pass2(ch);
    if (ch + 1 < nchunk) pass1(ch + 1);
  }
  if (jit_incr()) {
    o << "  {\n";
    emit_offset_chains(o, n, m, "BCH_FS", u0);
    emit_chain_loop(o, nh, "acc[@O] += BCH_FIN(@U);");
    o << "  }\n}\n";
  } else {
    o << "#pragma unroll\n  for (int u = 0; u < " << nh << "; u++) {\n"
      << "    const uint32_t uu = uint32_t(u + " << u0 << ");\n"
      << "    const uint32_t i = addmod(bfe32(uu | (uu << " << m << "), jr, " << m << "), sp, " << n << ");\n"
      << "    acc[i * BCH_FS] += BCH_FIN(u);\n  }\n}\n";
  }
}

static std::string jit_split_source(const bch_code *c, int msg) {
  const int G = jit_split_groups(), R = jit_split_chunk_rows();
  const int M = int(c->rows.size());
  std::ostringstream o;
  emit_prologue(o, msg, false);
  o << split_macros(msg) << "#define BCH_FS " << 32 * G << "\n#define BCH_TPB " << 64 * G << "\n";
  emit_split_half(o, c, msg, 0, R);
  emit_split_half(o, c, msg, 1, R);
  o << "struct SplitCopy {\n"
    << "  __device__ __forceinline__ void operator()(int h, StoreT<" << msg << ">::Y *y, StoreT<" << msg
    << ">::A *acc,\n      float2 *pa, float2 *pb, uint32_t jr, uint32_t sp, float alpha) const {\n"
    << "    if (h == 0) split_half0(y, acc, pa, pb, jr, sp, alpha);\n"
    << "    else split_half1(y, acc, pa, pb, jr, sp, alpha);\n  }\n};\n"
    << "}  // namespace bchlib\n"
    << "extern \"C\" __global__ void __launch_bounds__(" << 64 * G << ", 1) bch_nms_jit(const bchlib::NmsArgs a) {\n"
    << "  extern __shared__ __align__(16) unsigned char smem[];\n"
    << "  bchlib::nms_split_persistent<" << msg << ", " << G << ">(a, smem, bchlib::SplitCopy(), "
    << (M + R - 1) / R << ", " << R << ");\n}\n";
  return o.str();
}

// The block-bound serving kernel for a server's codes (FP32): per code a session with
// the batch kernels' mapping -- for n <= 63 the one-thread-per-frame copy functor on
// columns of stride 256, for n = 127 the two split halves -- and a dispatcher on the
// code a block is bound to.
std::string jit_serve_blocks_source(const bch_code *const *codes, int n_codes) {
  const int R = jit_split_chunk_rows();
  std::ostringstream o;
  emit_prologue(o, 0, true);
  o << split_macros(0) << "#define BCH_FS 128\n#define BCH_TPB 256\n";
  for (int i = 0; i < n_codes; i++) {
    const bch_code *c = codes[i];
    if (c->alg.n <= 63) {
      emit_copy(o, c, 0, "SrvFlat" + std::to_string(i), 256, false);
    } else {
      const std::string pre = "srv" + std::to_string(i) + "_half";
      emit_split_half(o, c, 0, 0, R, pre);
      emit_split_half(o, c, 0, 1, R, pre);
      o << "struct SrvSplit" << i << " {\n"
        << "  __device__ __forceinline__ void operator()(int h, float *y, float *acc, float2 *pa, float2 *pb,\n"
        << "      uint32_t jr, uint32_t sp, float alpha) const {\n"
        << "    if (h == 0) " << pre << "0(y, acc, pa, pb, jr, sp, alpha);\n"
        << "    else " << pre << "1(y, acc, pa, pb, jr, sp, alpha);\n  }\n};\n";
    }
  }
  o << "struct SrvBlockSessions {\n  const SrvArgs &a;\n"
    << "  __device__ __forceinline__ void operator()(int code, unsigned char *smem, const SrvBlockLayout &L) const {\n"
    << "    switch (code) {\n";
  for (int i = 0; i < n_codes; i++) {
    const bch_code *c = codes[i];
    o << "      case " << i << ": ";
    if (c->alg.n <= 63)
      o << "serve_session_flat<2>(a, " << i << ", smem, L, SrvFlat" << i << "()); break;\n";
    else
      o << "serve_session_split(a, " << i << ", smem, L, SrvSplit" << i << "(), "
        << (int(c->rows.size()) + R - 1) / R << ", " << R << "); break;\n";
  }
  o << "      default: break;\n    }\n  }\n};\n}  // namespace bchlib\n"
    << "extern \"C\" __global__ void __launch_bounds__(256, 1) bch_serve_blocks(const bchlib::SrvArgs a) {\n"
    << "  extern __shared__ __align__(16) unsigned char smem[];\n"
    << "  bchlib::serve_blocks(a, smem, bchlib::SrvBlockSessions{a});\n}\n";
  return o.str();
}

static std::string jit_body_source(const bch_code *c, int msg) {
  if (jit_split(c->alg.n)) return jit_split_source(c, msg);
  const int n = c->alg.n;
  const int tpb = jit_block_size(n);
  const int nw = (n + 31) / 32;
  std::ostringstream o;
  emit_prologue(o, msg, false);
  emit_copy(o, c, msg, "JitCopy", tpb, jit_scratch_words(n) > 0);
  o << "}  // namespace bchlib\n";
  o << "extern \"C\" __global__ void __launch_bounds__(" << tpb << ", " << jit_min_blocks(n)
    << ") bch_nms_jit(const bchlib::NmsArgs a) {\n"
    << "  extern __shared__ __align__(16) unsigned char smem[];\n"
    << "  bchlib::nms_persistent<" << msg << ", " << nw << ", " << (jit_lockstep(n) ? "true" : "false")
    << ", " << tpb << ">(a, smem, bchlib::JitCopy());\n}\n";
  return o.str();
}

// The serving kernel specialised to a server's codes (FP32 messages): one copy functor
// per code on columns of stride 32 (one warp per block), row sums in registers for
// n <= 63 and in the lane's scratch column for n = 127, dispatched on the warp's code.
std::string jit_serve_source(const bch_code *const *codes, int n_codes) {
  std::ostringstream o;
  emit_prologue(o, 0, true);
  for (int i = 0; i < n_codes; i++)
    emit_serve_copy(o, codes[i], "srv_copy_" + std::to_string(i), codes[i]->alg.n > 63);
  o << "struct SrvJitCopies {\n"
    << "  __device__ __forceinline__ void operator()(int code, const SrvCode &, int P, float *, float *,\n"
    << "      float *, const uint32_t *ctx, float alpha) const {\n"
    << "    switch (code) {\n";
  for (int i = 0; i < n_codes; i++)
    o << "      case " << i << ":\n        for (int p = 0; p < P; p++) {\n"
      << "          const uint32_t cx = ctx[p * 32];\n"
      << "          srv_copy_" << i << "(cx & 0xffu, cx >> 8, alpha);\n"
      << "        }\n        break;\n";
  o << "      default: break;\n    }\n  }\n};\n}  // namespace bchlib\n";
  o << "extern \"C\" __global__ void __launch_bounds__(32) bch_serve_jit(const bchlib::SrvArgs a) {\n"
    << "  extern __shared__ __align__(16) unsigned char smem[];\n"
    << "  bchlib::serve_loop(a, smem, bchlib::SrvJitCopies());\n}\n";
  return o.str();
}

// ---- on-disk cache of compiled kernels: <dir>/bchdec-jit-<hash>.cubin, keyed by the
// source text, the compile options and the NVRTC version.  Directory:
// BCHDEC_JIT_CACHE_DIR, else $XDG_CACHE_HOME/bchdec, else $HOME/.cache/bchdec;
// BCHDEC_JIT_CACHE_DIR=off disables the cache.
static uint64_t fnv1a(const void *p, size_t n, uint64_t h = 1469598103934665603ull) {
  const unsigned char *b = static_cast<const unsigned char *>(p);
  for (size_t i = 0; i < n; i++) h = (h ^ b[i]) * 1099511628211ull;
  return h;
}

static std::string cache_dir() {
  const char *d = std::getenv("BCHDEC_JIT_CACHE_DIR");
  if (d) return std::strcmp(d, "off") == 0 ? std::string() : std::string(d);
  if (const char *x = std::getenv("XDG_CACHE_HOME")) return std::string(x) + "/bchdec";
  if (const char *h = std::getenv("HOME")) return std::string(h) + "/.cache/bchdec";
  return std::string();
}

static std::string cache_path(const std::string &src, const char *const *opts, int nopt) {
  const std::string dir = cache_dir();
  if (dir.empty()) return dir;
  uint64_t h = fnv1a(src.data(), src.size());
  for (int i = 0; i < nopt; i++) h = fnv1a(opts[i], std::strlen(opts[i]), h);
  int major = 0, minor = 0;
  using VersionFn = nvrtcResult (*)(int *, int *);
  if (void *lib = dlopen("libnvrtc.so.13", RTLD_NOW | RTLD_LOCAL)) {
    if (auto fn = reinterpret_cast<VersionFn>(dlsym(lib, "nvrtcVersion"))) fn(&major, &minor);
  }
  const int ver[2] = {major, minor};
  h = fnv1a(ver, sizeof(ver), h);
  char name[64];
  std::snprintf(name, sizeof(name), "/bchdec-jit-%016llx.cubin", (unsigned long long)h);
  return dir + name;
}

static bool read_file(const std::string &path, std::vector<char> *out) {
  FILE *fp = std::fopen(path.c_str(), "rb");
  if (!fp) return false;
  std::fseek(fp, 0, SEEK_END);
  const long len = std::ftell(fp);
  std::fseek(fp, 0, SEEK_SET);
  bool ok = len > 0;
  if (ok) {
    out->resize(size_t(len));
    ok = std::fread(out->data(), 1, size_t(len), fp) == size_t(len);
  }
  std::fclose(fp);
  return ok;
}

static void write_file_atomic(const std::string &path, const std::vector<char> &data) {
  const std::string dir = path.substr(0, path.rfind('/'));
  // create the directory and its parents (best effort)
  for (size_t pos = 1; pos != std::string::npos;) {
    pos = dir.find('/', pos + 1);
    mkdir(dir.substr(0, pos).c_str(), 0755);
  }
  char tmp[64];
  std::snprintf(tmp, sizeof(tmp), ".tmp.%d", int(getpid()));
  const std::string tpath = path + tmp;
  FILE *fp = std::fopen(tpath.c_str(), "wb");
  if (!fp) return;
  const bool ok = std::fwrite(data.data(), 1, data.size(), fp) == data.size();
  std::fclose(fp);
  if (ok) std::rename(tpath.c_str(), path.c_str());
  else std::remove(tpath.c_str());
}

// Returns the specialised kernel for (code, msg), compiling it on first use (or
// loading it from the on-disk cache); on failure returns nullptr and sets *err.
cudaKernel_t jit_kernel_from_source(const bch_code *c, int msg, std::string *err, int qfrac);

// The tuning knobs that shape the generated source (read from the environment).
static std::string jit_knob_signature(int n) {
  char buf[96];
  std::snprintf(buf, sizeof(buf), "%d/%d/%d/%d/%d/%d/%d", jit_block_size(n), jit_min_blocks(n),
                int(jit_pairs()) + 2 * jit_chains(),
                jit_fma_percent(), env_int("BCHDEC_JIT_ROW_FENCE", 0, 1, 0), jit_scratch_words(n),
                int(jit_split(n)) + 2 * int(jit_incr()) + 4 * int(jit_first_assign()) +
                    8 * int(jit_copy_barrier()));
  return buf;
}

// The batch kernel's source for code c, format msg and qfrac fractional c2v bits (a
// compile-time constant, so the other forms carry none of its branches).
std::string jit_source(const bch_code *c, int msg, int qfrac) {
  return "#define BCH_JIT_QFRAC " + std::to_string(qfrac) + "\n" +
         (jit_copy_barrier() ? std::string() : std::string("#define BCH_JIT_NO_COPY_BARRIER 1\n")) +
         jit_body_source(c, msg);
}

cudaKernel_t jit_kernel(const bch_code *c, int msg, std::string *err, int qfrac) {
  const std::string key = std::to_string(msg) + "/" + std::to_string(qfrac) + ":" + jit_knob_signature(c->alg.n);
  {
    std::lock_guard<std::mutex> lk(c->jit_mu);
    for (const auto &m : c->jit_memo)
      if (m.key == key) {
        if (!m.kernel) *err = m.err;
        return static_cast<cudaKernel_t>(m.kernel);
      }
  }
  std::string why;
  cudaKernel_t k = jit_kernel_from_source(c, msg, &why, qfrac);
  {
    std::lock_guard<std::mutex> lk(c->jit_mu);
    c->jit_memo.push_back({key, static_cast<void *>(k), why});
  }
  if (!k) *err = why;
  return k;
}

// The library's own build defines, prepended to every run-time source: checked builds
// compile the specialised kernels with the same index checks as the precompiled ones
// (and, the define being part of the text, cache them apart).
static std::string with_build_defines(const std::string &src) {
#ifdef BCH_CHECKED
  return "#define BCH_CHECKED 1\n" + src;
#else
  return src;
#endif
}

// Compiles `src` (or loads it from the on-disk cache) and returns its kernel `entry`;
// cached in the process per source text.  On failure returns nullptr and sets *err.
static cudaKernel_t compile_source(const std::string &src_in, const char *entry, std::string *err) {
  const std::string src = with_build_defines(src_in);
  std::shared_ptr<Compiled> cp;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_cache.find(src);
    if (it != g_cache.end()) cp = it->second;
  }
  if (cp) {
    if (!cp->kernel) *err = cp->err;
    return cp->kernel;
  }
  cp = std::make_shared<Compiled>();
  NvrtcApi &api = nvrtc();
  const char *opts[] = {"--gpu-architecture=sm_103a", "-std=c++17", "-I/usr/local/cuda/include",
                        "-lineinfo"};
  const std::string cache_file = cache_path(src, opts, 4);
  std::vector<char> cached;
  if (!cache_file.empty() && read_file(cache_file, &cached) &&
      cudaLibraryLoadData(&cp->lib, cached.data(), nullptr, nullptr, 0, nullptr, nullptr, 0) == cudaSuccess &&
      cudaLibraryGetKernel(&cp->kernel, cp->lib, entry) == cudaSuccess) {
    // loaded a kernel compiled earlier from the same source
  } else if (!api.ok) {
    cp->kernel = nullptr;
    cp->err = api.err;
  } else {
    cp->kernel = nullptr;
    nvrtcProgram prog = nullptr;
    if (api.create(&prog, src.c_str(), (std::string(entry) + ".cu").c_str(), 0, nullptr, nullptr) !=
        NVRTC_SUCCESS) {
      cp->err = "nvrtcCreateProgram failed";
    } else {
      const nvrtcResult r = api.compile(prog, 4, opts);
      if (r != NVRTC_SUCCESS) {
        size_t ls = 0;
        api.log_size(prog, &ls);
        std::string log(ls, '\0');
        if (ls) api.log(prog, &log[0]);
        cp->err = "NVRTC compile failed: " + log.substr(0, 2000);
      } else {
        size_t cs = 0;
        api.cubin_size(prog, &cs);
        std::vector<char> cubin(cs);
        api.cubin(prog, cubin.data());
        cudaError_t e = cudaLibraryLoadData(&cp->lib, cubin.data(), nullptr, nullptr, 0, nullptr,
                                            nullptr, 0);
        if (e == cudaSuccess) e = cudaLibraryGetKernel(&cp->kernel, cp->lib, entry);
        if (e != cudaSuccess) {
          cp->kernel = nullptr;
          cp->err = std::string("loading the compiled kernel: ") + cudaGetErrorString(e);
        } else if (!cache_file.empty()) {
          write_file_atomic(cache_file, cubin);
        }
      }
      api.destroy(&prog);
    }
  }
  {
    std::lock_guard<std::mutex> lk(g_mu);
    g_cache[src] = cp;
  }
  if (!cp->kernel) *err = cp->err;
  return cp->kernel;
}

cudaKernel_t jit_kernel_from_source(const bch_code *c, int msg, std::string *err, int qfrac) {
  return compile_source(jit_source(c, msg, qfrac), "bch_nms_jit", err);
}

cudaKernel_t jit_serve_kernel(const bch_code *const *codes, int n_codes, std::string *err) {
  return compile_source(jit_serve_source(codes, n_codes), "bch_serve_jit", err);
}

cudaKernel_t jit_serve_blocks_kernel(const bch_code *const *codes, int n_codes, std::string *err) {
  return compile_source(jit_serve_blocks_source(codes, n_codes), "bch_serve_blocks", err);
}

// Compiles the specialised source with ptxas reporting on; no GPU is needed.  Returns
// false with *log holding the compiler output on failure.
static bool compile_check_source(const std::string &src, const char *entry, std::string *log);

bool jit_compile_check(const bch_code *c, int msg, std::string *log) {
  return compile_check_source(jit_source(c, msg, 0), "bch_nms_jit", log);
}

bool jit_serve_compile_check(const bch_code *const *codes, int n_codes, std::string *log) {
  if (!std::getenv("BCHDEC_SERVE_KERNEL") || std::strcmp(std::getenv("BCHDEC_SERVE_KERNEL"), "warps") != 0)
    return compile_check_source(jit_serve_blocks_source(codes, n_codes), "bch_serve_blocks", log);
  return compile_check_source(jit_serve_source(codes, n_codes), "bch_serve_jit", log);
}

static bool compile_check_source(const std::string &src_in, const char *entry, std::string *log) {
  const std::string src = with_build_defines(src_in);
  NvrtcApi &api = nvrtc();
  if (!api.ok) {
    *log = api.err;
    return false;
  }
  // BCHDEC_JIT_DUMP=<file>: also write the generated source there (a debugging aid)
  if (const char *dump = std::getenv("BCHDEC_JIT_DUMP")) {
    if (FILE *fp = std::fopen(dump, "w")) {
      std::fwrite(src.data(), 1, src.size(), fp);
      std::fclose(fp);
    }
  }
  nvrtcProgram prog = nullptr;
  if (api.create(&prog, src.c_str(), (std::string(entry) + ".cu").c_str(), 0, nullptr, nullptr) != NVRTC_SUCCESS) {
    *log = "nvrtcCreateProgram failed";
    return false;
  }
  const char *opts[] = {"--gpu-architecture=sm_103a", "-std=c++17", "-I/usr/local/cuda/include",
                        "-lineinfo", "--ptxas-options=-v"};
  const nvrtcResult r = api.compile(prog, 5, opts);
  size_t ls = 0;
  api.log_size(prog, &ls);
  std::string text(ls, '\0');
  if (ls) api.log(prog, &text[0]);
  while (!text.empty() && text.back() == '\0') text.pop_back();
  api.destroy(&prog);
  *log = text;
  return r == NVRTC_SUCCESS;
}

}  // namespace bchlib
