// Internal declarations shared by the library's translation units (host algebra,
// C-ABI layer and CUDA kernels).  Not installed; not part of the ABI.
#pragma once

#include <cstddef>
#include <cstdint>
#include <mutex>
#include <string>
#include <vector>

#include "bch_devtypes.h"
#include "bchdec.h"

namespace bchlib {

// A row of at most 128 bits: bit i = coefficient of x^i.
struct Row {
  uint64_t w[2] = {0, 0};
  bool get(int i) const { return (w[i >> 6] >> (i & 63)) & 1u; }
  void set(int i) { w[i >> 6] |= uint64_t(1) << (i & 63); }
  void flip(int i) { w[i >> 6] ^= uint64_t(1) << (i & 63); }
  int weight() const { return __builtin_popcountll(w[0]) + __builtin_popcountll(w[1]); }
  bool zero() const { return (w[0] | w[1]) == 0; }
  Row operator^(const Row &o) const {
    Row r;
    r.w[0] = w[0] ^ o.w[0];
    r.w[1] = w[1] ^ o.w[1];
    return r;
  }
  Row operator&(const Row &o) const {
    Row r;
    r.w[0] = w[0] & o.w[0];
    r.w[1] = w[1] & o.w[1];
    return r;
  }
  bool operator==(const Row &o) const { return w[0] == o.w[0] && w[1] == o.w[1]; }
  bool operator<(const Row &o) const { return w[1] != o.w[1] ? w[1] < o.w[1] : w[0] < o.w[0]; }
};

// Cyclic rotation by q (multiplication by x^q modulo x^n - 1).
Row rotate(const Row &r, int n, int q);

struct CodeAlgebra {
  int n = 0, k = 0, m = 0, ord = 0;
  std::vector<uint8_t> g;    // generator polynomial, n-k+1 coefficients
  std::vector<uint8_t> h;    // check polynomial, k+1 coefficients
  std::vector<Row> std_h;    // (n-k) standard rows
  std::vector<uint64_t> par; // parity word contributed by message bit i (n-k <= 64 bits)
};

// Returns false (with a message) for unsupported (n, k).
bool make_algebra(int n, int k, CodeAlgebra *out, std::string *err);

struct HoOptions {
  int q_rounds = 4;
  int sa_steps = 20000;
  double sa_lambda = 0.0;  // <= 0 -> n
  double sa_t0_frac = 0.05;
  double sa_cool = 0.9995;
};

// Builds H_o; returns BCH_OK, BCH_EINVAL or BCH_ERANK.
bch_status build_ho(const CodeAlgebra &alg, int m_rows, uint64_t seed, const HoOptions &opt,
                    std::vector<Row> *rows, int *r1_count, std::string *err);

// The construction split in its parts (build_ho = prepare, anneal, repair): steps 2-5
// (rows and the PRNG state after the padding), step 6 from a given state, rank repair.
bch_status prepare_ho(const CodeAlgebra &alg, int m_rows, uint64_t seed, const HoOptions &opt,
                      std::vector<Row> *rows, uint64_t *state, int *r1_count, std::string *err);
void anneal_ho(int n, std::vector<Row> &Ho, uint64_t state, const HoOptions &opt);
bool repair_rank(int n, int M, std::vector<Row> &Ho);
void ho_loss_terms(int n, const std::vector<Row> &Ho, long long *C4, long long *SS, long long *E);

int gf2_rank(std::vector<Row> rows, int n);

uint64_t splitmix64_next(uint64_t *state);
uint64_t splitmix64_mix(uint64_t z);
void draw_autos_host(int n, int P, uint64_t seed, uint64_t frame0, int F, uint16_t *out);

}  // namespace bchlib

struct bch_code {
  bchlib::CodeAlgebra alg;
  bch_pcm_kind kind;
  std::vector<bchlib::Row> rows;  // host copy, final row order
  int r1_count = 0;
  void *dev_blob = nullptr;  // device allocation holding the arrays below
  bchlib::DevCode dc;        // host-side descriptor with device pointers
  bchlib::DevCode *dev_dc = nullptr;  // descriptor copy in device memory
  // specialised kernels already looked up for this code, by (format, tuning knobs):
  // spares regenerating the kernel source on every decode call
  struct JitMemo {
    std::string key;
    void *kernel;
    std::string err;
  };
  mutable std::vector<JitMemo> jit_memo;
  mutable std::mutex jit_mu;
};

namespace bchlib {
void set_error(const std::string &msg);
bch_status fail(bch_status s, const std::string &msg);
// Counts one kernel launch of the library (bch_kernel_launches reports the total).
void note_launch();
// Argument checks shared by the decode entry points (BCH_EINVAL with a message).
bch_status check_params(const bch_code *code, const bch_nms_params *p);
bch_status check_frames(const bch_code *code, const float *llr, int ld, int F);
// The OSD stage's requirements: std_code is the standard matrix of the same code as
// `code` (when given), n - k <= 64, order in 0..2.
bch_status check_osd(const bch_code *code, const bch_code *std_code, int order);
}  // namespace bchlib
