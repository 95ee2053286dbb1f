// Host side of the decoder library: BCH code algebra, the standard parity-check
// matrix, the optimized matrix H_o (arXiv 2412.20828, Sec. III-A) and the host
// automorphism draw (Sec. III-B).  Rows are bit-packed into two 64-bit words.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <unordered_set>

#include "bch_internal.h"

namespace bchlib {

namespace {

using u128 = unsigned __int128;

u128 to128(const Row &r) { return (u128(r.w[1]) << 64) | u128(r.w[0]); }
Row from128(u128 x) {
  Row r;
  r.w[0] = uint64_t(x);
  r.w[1] = uint64_t(x >> 64);
  return r;
}
u128 mask_n(int n) { return n >= 128 ? ~u128(0) : ((u128(1) << n) - 1); }

// GF(2^m) element multiplication, primitive polynomial `prim` (with the x^m term).
int gf_mul(int a, int b, int m, int prim) {
  int r = 0;
  while (b) {
    if (b & 1) r ^= a;
    b >>= 1;
    a <<= 1;
    if (a & (1 << m)) a ^= prim;
  }
  return r;
}

int gf_pow(int a, int e, int m, int prim) {
  int r = 1;
  while (e > 0) {
    if (e & 1) r = gf_mul(r, a, m, prim);
    a = gf_mul(a, a, m, prim);
    e >>= 1;
  }
  return r;
}

// Evaluates the binary polynomial `poly` (bit i = coeff of x^i) at x in GF(2^m).
int eval_binary_poly(uint32_t poly, int deg, int x, int m, int prim) {
  int acc = 0;
  for (int i = deg; i >= 0; i--) acc = gf_mul(acc, x, m, prim) ^ int((poly >> i) & 1u);
  return acc;
}

// Product of binary polynomials held in 128-bit words.
u128 polymul2(u128 a, u128 b) {
  u128 r = 0;
  for (int i = 0; i < 128 && b; i++, b >>= 1)
    if (b & 1) r ^= a << i;
  return r;
}

int polydeg(u128 a) {
  int d = -1;
  for (int i = 0; i < 128; i++)
    if ((a >> i) & 1) d = i;
  return d;
}

}  // namespace

Row rotate(const Row &r, int n, int q) {
  q %= n;
  if (q < 0) q += n;
  if (q == 0) return r;
  u128 x = to128(r);
  u128 y = ((x << q) | (x >> (n - q))) & mask_n(n);
  return from128(y);
}

bool make_algebra(int n, int k, CodeAlgebra *out, std::string *err) {
  int m, prim;
  if (n == 15) {
    m = 4; prim = 0x13;
  } else if (n == 63) {
    m = 6; prim = 0x43;
  } else if (n == 127) {
    m = 7; prim = 0x89;
  } else {
    *err = "unsupported block length (n must be 15, 63 or 127)";
    return false;
  }
  if (k <= 0 || k >= n) {
    *err = "k out of range";
    return false;
  }
  CodeAlgebra A;
  A.n = n; A.k = k; A.m = m;
  A.ord = 1;
  for (int x = 2 % n; x != 1; x = (2 * x) % n) A.ord++;
  // Minimal polynomial of alpha^e: the binary polynomial of degree |coset(e)| with
  // alpha^e as a root, found by search over the 2^deg monic candidates.
  const int alpha = 2;
  std::vector<char> covered(n, 0);
  u128 g = 1;
  int deg = 0;
  for (int e = 1; deg < n - k; e += 2) {
    if (e >= n) {
      *err = "n-k is not a sum of cyclotomic coset sizes";
      return false;
    }
    if (covered[e]) continue;
    int csize = 0;
    int c = e;
    do {
      covered[c] = 1;
      csize++;
      c = (2 * c) % n;
    } while (c != e);
    int root = gf_pow(alpha, e, m, prim);
    uint32_t found = 0;
    for (uint32_t low = 0; low < (1u << csize); low++) {
      uint32_t cand = (1u << csize) | low;
      if (eval_binary_poly(cand, csize, root, m, prim) == 0) {
        found = cand;
        break;
      }
    }
    if (!found) {
      *err = "minimal polynomial search failed";
      return false;
    }
    g = polymul2(g, u128(found));
    deg += csize;
  }
  if (deg != n - k || polydeg(g) != n - k) {
    *err = "(n,k) is not a narrow-sense primitive BCH code";
    return false;
  }
  // h = (x^n + 1) / g by long division
  u128 num = (u128(1) << n) | 1;
  u128 q = 0;
  for (int i = n; i >= n - k; i--) {
    if ((num >> i) & 1) {
      int sh = i - (n - k);
      q |= u128(1) << sh;
      num ^= g << sh;
    }
  }
  if (num != 0) {
    *err = "g does not divide x^n + 1";
    return false;
  }
  A.g.resize(n - k + 1);
  for (int i = 0; i <= n - k; i++) A.g[i] = uint8_t((g >> i) & 1);
  A.h.resize(k + 1);
  for (int i = 0; i <= k; i++) A.h[i] = uint8_t((q >> i) & 1);
  // standard rows: x^r * reverse(h)
  u128 hrev = 0;
  for (int i = 0; i <= k; i++)
    if (A.h[k - i]) hrev |= u128(1) << i;
  A.std_h.resize(n - k);
  for (int r = 0; r < n - k; r++) A.std_h[r] = from128(hrev << r);
  // parity word of message bit i: x^(n-k+i) mod g
  A.par.resize(k);
  for (int i = 0; i < k; i++) {
    u128 rem = u128(1) << (n - k + i);
    for (int b = n - k + i; b >= n - k; b--)
      if ((rem >> b) & 1) rem ^= g << (b - (n - k));
    A.par[i] = uint64_t(rem);
  }
  *out = std::move(A);
  return true;
}

int gf2_rank(std::vector<Row> rows, int n) {
  int rank = 0;
  int M = int(rows.size());
  for (int c = 0; c < n && rank < M; c++) {
    int piv = -1;
    for (int r = rank; r < M; r++)
      if (rows[r].get(c)) {
        piv = r;
        break;
      }
    if (piv < 0) continue;
    std::swap(rows[piv], rows[rank]);
    for (int r = 0; r < M; r++)
      if (r != rank && rows[r].get(c)) rows[r] = rows[r] ^ rows[rank];
    rank++;
  }
  return rank;
}

uint64_t splitmix64_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

uint64_t splitmix64_next(uint64_t *state) {
  *state += 0x9E3779B97F4A7C15ULL;
  return splitmix64_mix(*state);
}

namespace {

uint64_t below(uint64_t x, uint64_t m) { return uint64_t((u128(x) * u128(m)) >> 64); }
double unit53(uint64_t x) { return double(x >> 11) * (1.0 / 9007199254740992.0); }

// Canonical member of a cyclic class: the numerically smallest rotation.
u128 canon(const Row &r, int n) {
  u128 best = to128(r);
  for (int q = 1; q < n; q++) {
    u128 v = to128(rotate(r, n, q));
    if (v < best) best = v;
  }
  return best;
}

struct U128Hash {
  size_t operator()(const u128 &x) const {
    return size_t(splitmix64_mix(uint64_t(x) ^ splitmix64_mix(uint64_t(x >> 64))));
  }
};

// Heuristic binary row summation (step 3; with shifts, one round of step 4).
std::vector<Row> row_sum_pass(const std::vector<Row> &in, int n, bool shifts) {
  std::vector<Row> out;
  std::unordered_set<u128, U128Hash> classes;
  std::vector<Row> sf;
  const int m = int(in.size());
  const int nq = shifts ? n : 1;
  for (int i = 0; i < m; i++) {
    const Row ri = in[i];
    int wg = ri.weight();
    sf.clear();
    sf.push_back(ri);
    for (int j = 0; j < m; j++) {
      if (j == i) continue;
      for (int qq = 1; qq <= nq; qq++) {
        int q = shifts ? qq % n : 0;
        Row t = ri ^ rotate(in[j], n, q);
        int w = t.weight();
        if (w == 0) continue;
        if (w == wg) {
          sf.push_back(t);
        } else if (w < wg) {
          wg = w;
          sf.clear();
          sf.push_back(t);
        }
      }
    }
    for (const Row &t : sf) {
      u128 c = canon(t, n);
      if (classes.insert(c).second) out.push_back(t);
    }
  }
  return out;
}

std::vector<Row> lightest(const std::vector<Row> &in, size_t cap) {
  std::vector<int> idx(in.size());
  for (size_t i = 0; i < in.size(); i++) idx[i] = int(i);
  std::stable_sort(idx.begin(), idx.end(),
                   [&](int a, int b) { return in[a].weight() < in[b].weight(); });
  std::vector<Row> out;
  for (size_t i = 0; i < idx.size() && out.size() < cap; i++) out.push_back(in[idx[i]]);
  return out;
}

int find_row(const std::vector<Row> &rows, const Row &r, int skip) {
  for (int i = 0; i < int(rows.size()); i++)
    if (i != skip && rows[i] == r) return i;
  return -1;
}

long long pairs(long long x) { return x * (x - 1) / 2; }

}  // namespace

// Steps 2-5 of the H_o construction: the padded row list and the PRNG state after the
// padding (the state the annealing of step 6 continues from).
bch_status prepare_ho(const CodeAlgebra &alg, int m_rows, uint64_t seed, const HoOptions &opt,
                      std::vector<Row> *rows_out, uint64_t *state_out, int *r1_count,
                      std::string *err) {
  const int n = alg.n, M = alg.n - alg.k;
  const bool want_default = m_rows <= 0;
  if (want_default) m_rows = 2 * M;
  if (m_rows < M) {
    *err = "m_rows below n-k";
    return BCH_EINVAL;
  }
  // step 2: reduced row echelon form of the standard matrix
  std::vector<Row> H = alg.std_h;
  {
    int rank = 0;
    for (int c = 0; c < n && rank < M; c++) {
      int piv = -1;
      for (int r = rank; r < M; r++)
        if (H[r].get(c)) {
          piv = r;
          break;
        }
      if (piv < 0) continue;
      std::swap(H[piv], H[rank]);
      for (int r = 0; r < M; r++)
        if (r != rank && H[r].get(c)) H[r] = H[r] ^ H[rank];
      rank++;
    }
  }
  // steps 3 and 4
  std::vector<Row> cur = row_sum_pass(H, n, false);
  for (int q = 0; q < opt.q_rounds; q++) {
    // a round works on the lightest 2 m_rows rows (stable) when there are more
    if (cur.size() > size_t(2 * m_rows)) cur = lightest(cur, size_t(2 * m_rows));
    cur = row_sum_pass(cur, n, true);
  }
  if (r1_count) *r1_count = int(cur.size());
  long long avail = 0;
  for (const Row &r : cur) {
    int per = n;
    for (int q = 1; q < n; q++)
      if (rotate(r, n, q) == r) {
        per = q;
        break;
      }
    avail += per;
  }
  if (want_default && m_rows > avail) m_rows = int(avail);
  if (m_rows > avail || m_rows < M) {
    *err = "m_rows exceeds the distinct rows reachable by the search";
    return BCH_EINVAL;
  }
  // step 5: lightest rows, then randomly shifted copies
  std::vector<Row> sorted = lightest(cur, cur.size());
  const int L = int(sorted.size());
  uint64_t st = seed;
  std::vector<Row> Ho;
  for (int i = 0; i < L && int(Ho.size()) < m_rows; i++) Ho.push_back(sorted[i]);
  int c = 0;
  while (int(Ho.size()) < m_rows) {
    if (L == 0 || c > 8 * m_rows + 8 * L) {
      *err = "padding did not find enough distinct shifted rows";
      return BCH_ERANK;
    }
    const Row src = sorted[c % L];
    c++;
    for (int a = 0; a < 4 * n; a++) {
      int q = int(below(splitmix64_next(&st), uint64_t(n)));
      Row cand = rotate(src, n, q);
      if (find_row(Ho, cand, -1) < 0) {
        Ho.push_back(cand);
        break;
      }
    }
  }
  *rows_out = std::move(Ho);
  *state_out = st;
  return BCH_OK;
}

// Loss terms of a row list: number of 4-cycles (row pairs' overlaps taken two at a
// time), sum of squared column weights, number of edges.
void ho_loss_terms(int n, const std::vector<Row> &Ho, long long *C4, long long *SS, long long *E) {
  const int Mo = int(Ho.size());
  long long c4 = 0, ss = 0, e = 0;
  for (int r = 0; r < Mo; r++)
    for (int r2 = r + 1; r2 < Mo; r2++) c4 += pairs((Ho[r] & Ho[r2]).weight());
  for (int i = 0; i < n; i++) {
    long long w = 0;
    for (int r = 0; r < Mo; r++) w += Ho[r].get(i) ? 1 : 0;
    ss += w * w;
    e += w;
  }
  *C4 = c4;
  *SS = ss;
  *E = e;
}

// Step 6: simulated annealing of the rows' cyclic shifts, PRNG state `st`.
void anneal_ho(int n, std::vector<Row> &Ho, uint64_t st, const HoOptions &opt) {
  const int Mo = int(Ho.size());
  const double lam = opt.sa_lambda > 0.0 ? opt.sa_lambda : double(n);
  std::vector<long long> ov(size_t(Mo) * Mo, 0), cyc(Mo, 0), nov(Mo, 0);
  std::vector<long long> colw(n, 0);
  long long E = 0;
  for (int r = 0; r < Mo; r++)
    for (int i = 0; i < n; i++)
      if (Ho[r].get(i)) {
        colw[i]++;
        E++;
      }
  long long C4 = 0;
  for (int r = 0; r < Mo; r++)
    for (int r2 = 0; r2 < Mo; r2++)
      if (r2 != r) ov[size_t(r) * Mo + r2] = (Ho[r] & Ho[r2]).weight();
  for (int r = 0; r < Mo; r++)
    for (int r2 = 0; r2 < Mo; r2++)
      if (r2 != r) cyc[r] += pairs(ov[size_t(r) * Mo + r2]);
  for (int r = 0; r < Mo; r++)
    for (int r2 = r + 1; r2 < Mo; r2++) C4 += pairs(ov[size_t(r) * Mo + r2]);
  long long SS = 0;
  for (int i = 0; i < n; i++) SS += colw[i] * colw[i];
  const double loss0 = double(C4) + lam * (double(SS) - double(E) * double(E) / double(n)) / double(n);
  double T = opt.sa_t0_frac * loss0;
  for (int s = 0; s < opt.sa_steps; s++) {
    const uint64_t x1 = splitmix64_next(&st);
    const uint64_t x2 = splitmix64_next(&st);
    const uint64_t x3 = splitmix64_next(&st);
    long long W = 0;
    for (int r = 0; r < Mo; r++) W += cyc[r] + 1;
    const long long tsel = (long long)below(x1, uint64_t(W));
    int r = 0;
    long long acc = 0;
    for (r = 0; r < Mo; r++) {
      acc += cyc[r] + 1;
      if (acc > tsel) break;
    }
    const int q = 1 + int(below(x2, uint64_t(n - 1)));
    const double u = unit53(x3);
    const Row old = Ho[r];
    const Row nr = rotate(old, n, q);
    if (find_row(Ho, nr, r) < 0) {
      long long dC4 = 0;
      for (int r2 = 0; r2 < Mo; r2++) {
        if (r2 == r) {
          nov[r2] = 0;
          continue;
        }
        nov[r2] = (nr & Ho[r2]).weight();
        dC4 += pairs(nov[r2]) - pairs(ov[size_t(r) * Mo + r2]);
      }
      long long dSS = 0;
      for (int i = 0; i < n; i++) {
        long long w1 = colw[i] - (old.get(i) ? 1 : 0) + (nr.get(i) ? 1 : 0);
        dSS += w1 * w1 - colw[i] * colw[i];
      }
      const double d = double(dC4) + lam * double(dSS) / double(n);
      bool accept = false;
      if (d <= 0.0)
        accept = true;
      else if (T > 0.0 && u < std::exp(-d / T))
        accept = true;
      if (accept) {
        for (int i = 0; i < n; i++) colw[i] += (nr.get(i) ? 1 : 0) - (old.get(i) ? 1 : 0);
        for (int r2 = 0; r2 < Mo; r2++) {
          if (r2 == r) continue;
          long long o = ov[size_t(r) * Mo + r2];
          cyc[r2] += pairs(nov[r2]) - pairs(o);
          ov[size_t(r) * Mo + r2] = nov[r2];
          ov[size_t(r2) * Mo + r] = nov[r2];
        }
        cyc[r] = 0;
        for (int r2 = 0; r2 < Mo; r2++)
          if (r2 != r) cyc[r] += pairs(ov[size_t(r) * Mo + r2]);
        C4 += dC4;
        Ho[r] = nr;
      }
    }
    T *= opt.sa_cool;
  }
}

// Rank repair: rows in order try the rotations q = 1 .. n-1 and keep the first that
// raises the rank, until the rank is n - k.  False if it stays below.
bool repair_rank(int n, int M, std::vector<Row> &Ho) {
  const int Mo = int(Ho.size());
  int rk = gf2_rank(Ho, n);
  for (int r = 0; r < Mo && rk < M; r++) {
    for (int q = 1; q < n; q++) {
      Row nr = rotate(Ho[r], n, q);
      if (find_row(Ho, nr, r) >= 0) continue;
      std::vector<Row> tmp = Ho;
      tmp[r] = nr;
      int r2 = gf2_rank(tmp, n);
      if (r2 > rk) {
        Ho[r] = nr;
        rk = r2;
        break;
      }
    }
  }
  return rk == M;
}

bch_status build_ho(const CodeAlgebra &alg, int m_rows, uint64_t seed, const HoOptions &opt,
                    std::vector<Row> *rows_out, int *r1_count, std::string *err) {
  std::vector<Row> Ho;
  uint64_t st = 0;
  bch_status s = prepare_ho(alg, m_rows, seed, opt, &Ho, &st, r1_count, err);
  if (s != BCH_OK) return s;
  anneal_ho(alg.n, Ho, st, opt);
  if (!repair_rank(alg.n, alg.n - alg.k, Ho)) {
    *err = "H_o did not reach rank n-k";
    return BCH_ERANK;
  }
  *rows_out = std::move(Ho);
  return BCH_OK;
}

void draw_autos_host(int n, int P, uint64_t seed, uint64_t frame0, int F, uint16_t *out) {
  int ord = 1;
  for (int x = 2 % n; x != 1; x = (2 * x) % n) ord++;
  for (int fi = 0; fi < F; fi++) {
    const uint64_t f = frame0 + uint64_t(fi);
    uint16_t *o = out + size_t(fi) * P;
    for (int p = 0; p < P; p++) {
      uint32_t s = 0, j = 0;
      for (int a = 0; a < 16; a++) {
        const uint64_t cnt = 1 + (f * uint64_t(P) + uint64_t(p)) * 16 + uint64_t(a);
        const uint64_t x = splitmix64_mix(seed + 0x9E3779B97F4A7C15ULL * cnt);
        s = uint32_t(((x & 0xffffffffULL) * uint64_t(n)) >> 32);
        j = uint32_t(((x >> 32) * uint64_t(ord)) >> 32);
        bool clash = false;
        for (int q = 0; q < p; q++)
          if ((o[q] & 0xffu) == s && (o[q] >> 8) == j) clash = true;
        if (!clash) break;
      }
      o[p] = uint16_t(s | (j << 8));
    }
  }
}

}  // namespace bchlib
