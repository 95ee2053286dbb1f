// Device-side search for the optimized parity-check matrix (arXiv 2412.20828, Sec. III-A,
// step 6): many simulated-annealing chains over the rows' cyclic shifts at once, one
// thread block per chain.  A chain is the host builder's annealing loop with its own
// PRNG stream; the sequential part of a proposal (three SplitMix64 draws, the row pick
// and the Metropolis test) runs on one thread and the parallel part on the block:
//  * the row pick: a warp-level prefix sum of the weights (4-cycles of the row + 1);
//  * the duplicate test of the shifted row against every other row;
//  * the change of the 4-cycle count: the new row's overlaps with all others as
//    popcounts of 128-bit ANDs, taken two at a time;
//  * the change of the squared column weights, one column per thread.
// The arithmetic, the order of the draws and the floating-point expressions are those
// of the host loop, so chain c reproduces the host annealing from the same state.
#include "bch_kernels.cuh"

namespace bchlib {

constexpr int kAnnealThreads = 256;

namespace {

__device__ __forceinline__ uint64_t sm64_next(uint64_t &st) {
  st += 0x9E3779B97F4A7C15ULL;
  return splitmix64_mix_d(st);
}
__device__ __forceinline__ uint64_t draw_below(uint64_t x, uint64_t m) { return __umul64hi(x, m); }
__device__ __forceinline__ long long pairs2(long long x) { return x * (x - 1) / 2; }
__device__ __forceinline__ int bit_at(const ulonglong2 &r, int i) {
  return int(((i < 64 ? r.x >> i : r.y >> (i - 64)) & 1ull));
}
__device__ __forceinline__ int popc128(const ulonglong2 &a, const ulonglong2 &b) {
  return __popcll(a.x & b.x) + __popcll(a.y & b.y);
}
// Cyclic rotation of the n-bit row r by q (0 < q < n): bit i moves to (i + q) mod n.
__device__ __forceinline__ ulonglong2 rot128(const ulonglong2 &r, int n, int q) {
  const unsigned __int128 x = (unsigned __int128)r.y << 64 | r.x;
  const unsigned __int128 mask = n >= 128 ? ~(unsigned __int128)0 : (((unsigned __int128)1 << n) - 1);
  const unsigned __int128 y = ((x << q) | (x >> (n - q))) & mask;
  return make_ulonglong2(uint64_t(y), uint64_t(y >> 64));
}

// Sum over the block (every thread calls it; two barriers).
__device__ long long block_sum(long long v, long long *red) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  const int w = int(threadIdx.x >> 5);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[w] = v;
  __syncthreads();
  long long s = 0;
  for (int i = 0; i < int(blockDim.x >> 5); i++) s += red[i];
  return s;
}

}  // namespace

__global__ void __launch_bounds__(kAnnealThreads) anneal_kernel(const AnnealArgs a) {
  extern __shared__ __align__(16) unsigned char sm[];
  const int Mo = a.Mo, n = a.n, tid = int(threadIdx.x), nt = int(blockDim.x);
  ulonglong2 *rows = reinterpret_cast<ulonglong2 *>(sm);                 // [Mo]
  int *cyc = reinterpret_cast<int *>(rows + Mo);                         // [Mo] 4-cycles of row r
  int *colw = cyc + Mo;                                                  // [128] column weights
  uint8_t *nov = reinterpret_cast<uint8_t *>(colw + 128);                // [Mo] new overlaps
  uint8_t *ov = nov + ((Mo + 15) & ~15);                                 // [Mo][Mo] overlaps
  __shared__ long long red[kAnnealThreads / 32];
  __shared__ uint64_t xs[3];
  __shared__ int sel_r, accept_f;
  const ulonglong2 *r0 = a.rows0;
  for (int r = tid; r < Mo; r += nt) rows[r] = r0[r];
  __syncthreads();
  for (int i = tid; i < 128; i += nt) {
    int w = 0;
    if (i < n)
      for (int r = 0; r < Mo; r++) w += bit_at(rows[r], i);
    colw[i] = w;
  }
  for (int e = tid; e < Mo * Mo; e += nt) {
    const int r = e / Mo, r2 = e - r * Mo;
    ov[e] = r == r2 ? 0 : uint8_t(popc128(rows[r], rows[r2]));
  }
  __syncthreads();
  for (int r = tid; r < Mo; r += nt) {
    long long c = 0;
    for (int r2 = 0; r2 < Mo; r2++)
      if (r2 != r) c += pairs2(ov[r * Mo + r2]);
    cyc[r] = int(c);
  }
  uint64_t st = a.state0[blockIdx.x];  // used by thread 0 only
  double T = a.T0;
  __syncthreads();
  const int seg = (Mo + 31) / 32;
  for (int s = 0; s < a.steps; s++) {
    if (tid == 0) {
      xs[0] = sm64_next(st);
      xs[1] = sm64_next(st);
      xs[2] = sm64_next(st);
    }
    __syncthreads();
    // row pick with probability proportional to (4-cycles + 1): warp 0 scans
    if (tid < 32) {
      const int lo = tid * seg, hi = min(Mo, lo + seg);
      long long part = 0;
      for (int r = lo; r < hi; r++) part += cyc[r] + 1;
      long long incl = part;
      for (int off = 1; off < 32; off <<= 1) {
        const long long o = __shfl_up_sync(0xffffffffu, incl, off);
        if (tid >= off) incl += o;
      }
      const long long W = __shfl_sync(0xffffffffu, incl, 31);
      const long long tsel = (long long)draw_below(xs[0], uint64_t(W));
      long long acc = incl - part;
      if (acc <= tsel && tsel < incl) {
        int r = lo;
        for (; r < hi; r++) {
          acc += cyc[r] + 1;
          if (acc > tsel) break;
        }
        sel_r = r;
      }
    }
    __syncthreads();
    const int r = sel_r;
    const int q = 1 + int(draw_below(xs[1], uint64_t(n - 1)));
    const double u = double(xs[2] >> 11) * (1.0 / 9007199254740992.0);
    const ulonglong2 old = rows[r];
    const ulonglong2 nr = rot128(old, n, q);
    bool dup = false;
    for (int r2 = tid; r2 < Mo; r2 += nt)
      if (r2 != r && rows[r2].x == nr.x && rows[r2].y == nr.y) dup = true;
    if (!__syncthreads_or(dup)) {
      long long pdc = 0, pds = 0;
      for (int r2 = tid; r2 < Mo; r2 += nt) {
        if (r2 == r) {
          nov[r2] = 0;
          continue;
        }
        const int nv = popc128(nr, rows[r2]);
        nov[r2] = uint8_t(nv);
        pdc += pairs2(nv) - pairs2(ov[r * Mo + r2]);
      }
      if (tid < n) {
        const long long c = colw[tid];
        const long long w1 = c - bit_at(old, tid) + bit_at(nr, tid);
        pds = w1 * w1 - c * c;
      }
      const long long dC4 = block_sum(pdc, red);
      const long long dSS = block_sum(pds, red);
      if (tid == 0) {
        const double d = double(dC4) + a.lam * double(dSS) / double(n);
        accept_f = (d <= 0.0) || (T > 0.0 && u < exp(-d / T));
      }
      __syncthreads();
      if (accept_f) {
        if (tid < n) colw[tid] += bit_at(nr, tid) - bit_at(old, tid);
        for (int r2 = tid; r2 < Mo; r2 += nt) {
          if (r2 == r) continue;
          const int o = ov[r * Mo + r2];
          cyc[r2] += int(pairs2(nov[r2]) - pairs2(o));
          ov[r * Mo + r2] = nov[r2];
          ov[r2 * Mo + r] = nov[r2];
        }
        __syncthreads();
        long long pc = 0;
        for (int r2 = tid; r2 < Mo; r2 += nt)
          if (r2 != r) pc += pairs2(ov[r * Mo + r2]);
        const long long c = block_sum(pc, red);
        if (tid == 0) {
          cyc[r] = int(c);
          rows[r] = nr;
        }
      }
    }
    if (tid == 0) T *= a.cool;
    __syncthreads();
  }
  ulonglong2 *out = a.rows_out + size_t(blockIdx.x) * Mo;
  for (int r = tid; r < Mo; r += nt) out[r] = rows[r];
}

size_t anneal_smem_bytes(int Mo) {
  return size_t(Mo) * 16 + size_t(Mo) * 4 + 128 * 4 + size_t((Mo + 15) & ~15) + size_t(Mo) * Mo;
}

cudaError_t launch_anneal(const AnnealArgs &a, cudaStream_t st) {
  const size_t smem = anneal_smem_bytes(a.Mo);
  if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
  cudaError_t e = cudaFuncSetAttribute(anneal_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  note_launch();
  anneal_kernel<<<unsigned(a.chains), kAnnealThreads, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace bchlib
