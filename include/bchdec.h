/*
 * bchdec.h -- C ABI of the GB300 (sm_103a) enhanced normalized min-sum decoder for
 * short BCH codes, after arXiv 2412.20828 (Li & Yu, "Effective Application of
 * Normalized Min-Sum Decoding for Short BCH Codes").
 *
 * Conventions shared by every entry point
 *  - Every function returns bch_status (BCH_OK = 0); no C++ exception crosses the ABI.
 *    bch_status_str() names a status; bch_last_error() returns the text of the most
 *    recent failure on the calling thread.
 *  - Codes: narrow-sense primitive BCH(n,k), n in {15, 63, 127}, GF(2^m) primitive
 *    polynomials x^4+x+1, x^6+x+1, x^7+x^3+1.
 *  - Bit order: bit i of a word is the coefficient of x^i; packed words hold bit i in
 *    64-bit word i/64, bit i%64.  Codeword layout is systematic: parity in positions
 *    0..n-k-1, message bit i at position n-k+i.
 *  - LLR sign (Eq. 1 of the paper): positive means bit 0; L = 2y/sigma^2.
 *  - Frame arrays are row-major [n_frames][ld] with ld >= n floats; ld a multiple of
 *    4 and 16-byte-aligned rows give 128-bit loads (ld = 64 for n = 63, 128 for 127).
 *  - Device-side calls are asynchronous on `stream` (a cudaStream_t; NULL = legacy
 *    default stream).  Pointers documented "device" must be device-accessible memory
 *    owned by the caller; the library owns only bch_code, bch_decoder and bch_server
 *    objects and what they allocate.  Decode calls allocate nothing: scratch comes
 *    from a caller-provided workspace sized by bch_workspace_size().
 *  - A CUDA error met during an asynchronous call surfaces as BCH_ECUDA from that
 *    call or a later one (errors are sticky, as in CUDA).
 */
#ifndef BCHDEC_H_
#define BCHDEC_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  BCH_OK = 0,
  BCH_EINVAL = 1,   /* bad argument (size, pointer, alignment, unsupported code)  */
  BCH_ENOMEM = 2,   /* host or device allocation failed (library-owned objects)   */
  BCH_ECUDA = 3,    /* a CUDA runtime call or kernel failed                        */
  BCH_ERANK = 4,    /* H_o could not reach rank n-k                                */
  BCH_ETIMEOUT = 5, /* a bounded device wait or host poll ran out                  */
  BCH_EBUDGET = 6,  /* request larger than the server's HBM budget                 */
  BCH_EBUSY = 7     /* server queue full / object in use                           */
} bch_status;

typedef enum { BCH_PCM_STANDARD = 0, BCH_PCM_OPTIMIZED = 1 } bch_pcm_kind;

/* Storage format of the per-frame LLR state y and of the row minima.
 *  FP32  float storage.
 *  FP16  binary16 storage, round-to-nearest-even, saturating at +-65504; the
 *        check-to-variable sums and the merge of Algorithm 1 stay FP32.
 *  INT8  8-bit saturating fixed point, LSB = 1/4 (q = clamp(rne(4x), -31, 31));
 *        minima, signs and check-to-variable values (rne(alpha q)) are integers,
 *        summed exactly in 16 bits, merged in FP32, re-quantised with saturation. */
typedef enum { BCH_MSG_FP32 = 0, BCH_MSG_FP16 = 1, BCH_MSG_INT8 = 2 } bch_msg_type;

/* Opaque code object: host and device copies of the standard H or H_o. */
typedef struct bch_code bch_code;

/* Options of the H_o construction (Sec. III-A, steps 3-6).  NULL = defaults. */
typedef struct {
  int q_rounds;      /* rounds of the shifted row-summation search (step 4); default 4   */
  int sa_steps;      /* simulated-annealing proposals (step 6); default 20000            */
  double sa_lambda;  /* weight of the column-weight variance in the loss; <= 0 means n  */
  double sa_t0_frac; /* initial temperature as a fraction of the initial loss; 0.05     */
  double sa_cool;    /* geometric cooling factor per proposal; default 0.9995           */
} bch_pcm_opts;

/* Decoder parameters. */
typedef struct {
  int iters;           /* maximum iterations I_m, 1..32                                 */
  const float *alpha;  /* host array of `iters` normalization factors alpha_1..alpha_t   */
  int n_autos;         /* P = automorphisms per frame, 1..9 (Algorithm 1); 0 selects the
                          plain flooding decoder of Eqs. (2)-(5) with per-edge messages */
  int early_stop;      /* 1: stop a frame at the first zero syndrome (Eq. 5)            */
  bch_msg_type msg;    /* storage format                                                 */
  int rescale;         /* 1 (FP16/INT8 only): renormalise each frame's y by a power of
                          two after every merge; min-sum is scale invariant, so only
                          quantisation changes.  0: plain saturation                     */
  int osd_order;       /* hybrid decoding only: OSD order 0..2                            */
  int osd_input;       /* hybrid decoding only: the reliabilities the OSD ranks and scores.
                          0: the channel LLR, the magnitude of Eq. (1) (Sec. II-B).
                          1: the frame's final NMS output y (the "improved" reliability
                          measure Sec. II-B allows), scaled by the power of two that puts
                          max_i |y_i| in [2^15, 2^16) -- exact, and the OSD's choice does
                          not depend on a common scale -- so that its integer weights
                          floor(|y| 2^24) resolve the values; needs llr_out, which
                          receives y and which the OSD reads                             */
  int qfrac;           /* 8-bit form only (msg = INT8, n_autos >= 1), 0..8: fractional
                          bits kept in the check-to-variable magnitudes.  0: c2v =
                          rne(alpha min_q) in units of the stored LSB (1/4).  f > 0: c2v =
                          rne(alpha min_q 2^f) in units of 2^-f LSB, summed exactly, and
                          the merge stores clamp(rne(N / D), +-31) of the exact quotient,
                          N = P 2^f q + sum, D = P 2^f (2^k more after k rescale
                          halvings); y keeps its 8-bit storage.  With rescale = 1 the
                          input is also quantised after the power of two 2^-k0 that keeps
                          max |4x| <= 31 (k0 starts the frame's exponent), so strong
                          inputs are not clipped.  Needs 0 <= alpha_t <= 4 (the sums stay
                          exact in FP32).  Zero-initialise the struct to leave it 0       */
} bch_nms_params;

/* Per-frame flag bits written by the decoders. */
#define BCH_FLAG_CONVERGED 1u /* the NMS hard decision has zero syndrome               */
#define BCH_FLAG_OSD 2u       /* the final word came from the OSD fallback             */

/* ---------------------------------------------------------------- codes (host) */

/* Build the parity-check matrix of BCH(n,k) on the host and upload it (Sec. III-A).
 * kind = STANDARD: the (n-k) x n cyclic matrix whose row r holds the reversed check
 *   polynomial from column r (attributes of Table I, "H" rows).
 * kind = OPTIMIZED: H_o by steps 1-6 of Sec. III-A: reduced row echelon form;
 *   heuristic binary row summation; q_rounds rounds with all cyclic shifts; selection
 *   of the m_rows lightest rows (or padding with randomly shifted copies); simulated
 *   annealing of cyclic row shifts against (#4-cycles + lambda var(column weights));
 *   rank repair.  m_rows = 0 selects 2(n-k), clamped to the number of distinct rows
 *   the search reached.  Deterministic in `seed` (SplitMix64).
 * Returns BCH_EINVAL for an unsupported (n,k), BCH_ERANK if rank n-k is unreachable.
 * *out is owned by the caller and released with bch_code_free(). */
bch_status bch_build_pcm(int n, int k, bch_pcm_kind kind, int m_rows, uint64_t seed,
                         const bch_pcm_opts *opts, bch_code **out);

/* Device-side search for H_o: step 6 of Sec. III-A (simulated annealing of the rows'
 * cyclic shifts) run as n_chains independent chains in parallel on the GPU, one thread
 * block per chain.  Steps 1-5 run on the host as in bch_build_pcm; chain c starts from
 * the builder's SplitMix64 state after step 5 advanced by c x 0xD1B54A32D192ED03, so
 * chain 0 is exactly the annealing bch_build_pcm(n, k, OPTIMIZED, m_rows, seed, opts)
 * runs.  Every chain's matrix gets the rank repair; the kept matrix is the one with the
 * lowest loss #4-cycles + lambda Var(column weights) among the chains that reach rank
 * n-k (ties: the lowest chain).  The paper anneals once; running many chains is this
 * library's use of the GPU for the step.  stats (nullable, host [n_chains][3]): each
 * chain's 4-cycles, sum of squared column weights, and 1 if it reached rank n-k, else 0.
 * dense_all (nullable, host, capacity bytes >= n_chains rows n): every chain's matrix,
 * [chain][row][column] bytes.  *best (nullable) receives the kept chain.  Synchronous;
 * allocates and frees its own device buffers.  BCH_EINVAL as bch_build_pcm, or for
 * n_chains outside 1..4096 or more than 400 rows; BCH_ERANK if no chain reaches rank
 * n-k.  *out is released with bch_code_free(). */
bch_status bch_search_pcm(int n, int k, int m_rows, uint64_t seed, const bch_pcm_opts *opts,
                          int n_chains, long long *stats, uint8_t *dense_all, size_t capacity,
                          int *best, bch_code **out);

/* Host-only variant of bch_build_pcm: runs the same construction and writes the matrix
 * as bytes (rows x n, row-major) into caller-owned host memory `dense` of `capacity`
 * bytes; *rows receives the row count.  Touches no GPU. */
bch_status bch_build_pcm_host(int n, int k, bch_pcm_kind kind, int m_rows, uint64_t seed,
                              const bch_pcm_opts *opts, uint8_t *dense, size_t capacity,
                              int *rows);

/* Names the enhanced-NMS kernel a decode of `code` with storage `msg` and n_autos
 * automorphisms runs: "jit" -- the kernel compiled at run time (NVRTC) for this code's
 * Tanner graph, rows as straight-line code on registers -- or "generic: <reason>" --
 * the precompiled kernel that reads the rows from shared memory.  The environment
 * variable BCHDEC_NMS_KERNEL=generic|jit|auto selects (default auto: jit when it
 * compiles, else generic; for n = 127 the specialised kernel is about 1.8x faster than
 * the precompiled one).  The first call for a code compiles (a few seconds for n <= 63,
 * 30-90 s for n = 127) and caches the kernel in the process and on disk
 * (BCHDEC_JIT_CACHE_DIR, default $XDG_CACHE_HOME/bchdec or $HOME/.cache/bchdec; "off"
 * disables it).  Tuning knobs of the specialised kernel, read when its source is
 * generated: BCHDEC_JIT_TPB (block size for n <= 63), BCHDEC_JIT_MIN_BLOCKS (register
 * budget), BCHDEC_JIT_PAIRS (min1/min2 two edges at a time), BCHDEC_JIT_FMA_PCT (share
 * of edges whose min2 correction runs on the FMA pipe), BCHDEC_JIT_ROW_FENCE (compiler
 * fence between rows), BCHDEC_JIT_DUMP (file receiving the source, with
 * bch_nms_jit_check).  Every setting computes the same results. */
bch_status bch_nms_kernel_info(const bch_code *code, int msg, int n_autos, char *buf,
                               size_t capacity);

/* Compiles the run-time specialised enhanced-NMS kernel for the optimized matrix that
 * bch_build_pcm(n, k, BCH_PCM_OPTIMIZED, m_rows, seed, opts) builds, for sm_103a with
 * NVRTC and ptxas reporting on, without loading it: no GPU is needed.  log
 * (caller-owned, capacity bytes, always NUL-terminated) receives the compiler output
 * -- registers, spills, shared memory -- or the errors.  BCH_ECUDA when the compile
 * fails or NVRTC is missing; the matrix builder's errors as bch_build_pcm.  No
 * counterpart in the paper: a build and tuning aid for the specialised kernel. */
bch_status bch_nms_jit_check(int n, int k, int m_rows, uint64_t seed, const bch_pcm_opts *opts,
                             int msg, char *log, size_t capacity);

/* Dimensions of a code object: n, k, rows, edges (ones in the matrix), max row weight. */
bch_status bch_code_info(const bch_code *code, int *n, int *k, int *rows, int *edges,
                         int *max_row_weight);

/* Copy the matrix out as bytes (rows x n, caller-owned host memory). */
bch_status bch_pcm_export(const bch_code *code, uint8_t *dense, size_t capacity);

void bch_code_free(bch_code *code);

/* ---------------------------------------------------------------- automorphisms */

/* Draw P automorphisms per frame (Sec. III-B): pairs (s, j) acting as
 * pi(i) = (2^j i + s) mod n, j a Frobenius power in [0, ord_n(2)), s a cyclic shift in
 * [0, n).  Stateless in (seed, frame index, slot): x = SplitMix64 output number
 * 1 + (f P + p) 16 + a from state `seed`; s = floor(lo32(x) n / 2^32),
 * j = floor(hi32(x) ord / 2^32); retried (a = 1..15) while the pair repeats an earlier
 * slot of the frame.  Output packed s | j << 8, layout [n_frames][n_autos].
 * bch_draw_automorphisms writes device memory on `stream`; the _host variant writes
 * host memory synchronously.  Both produce identical values. */
bch_status bch_draw_automorphisms(int n, int n_autos, uint64_t seed, uint64_t frame0,
                                  int n_frames, uint16_t *out, void *stream);
bch_status bch_draw_automorphisms_host(int n, int n_autos, uint64_t seed, uint64_t frame0,
                                       int n_frames, uint16_t *out);

/* ---------------------------------------------------------------- frames */

/* Synthetic BPSK/AWGN frames (Sec. II, Eq. 1) on the device, counter-based:
 * Philox4x32-10 keyed by seed, counter (frame, block, tag): tag 0 message bits,
 * tag 1 Box-Muller noise for positions 4b..4b+3, tag 2 a per-frame Eb/N0 uniform in
 * [ebn0_lo, ebn0_hi) when ebn0_hi > ebn0_lo.  Systematic encoding, s = 1 - 2c,
 * y = s + sigma n, L = 2y/sigma^2 with sigma^2 = 1/(2 (k/n) 10^(Eb/N0/10)).
 * llr: device [n_frames][ld] (padding columns written 0); codeword: device
 * [n_frames][ceil(n/64)] u64 or NULL. */
bch_status bch_gen_frames(const bch_code *code, float ebn0_lo, float ebn0_hi, uint64_t seed,
                          uint64_t frame0, int n_frames, float *llr, int ld, uint64_t *codeword,
                          void *stream);

/* ---------------------------------------------------------------- decoding */

/* Bytes of device scratch a decode call needs (frame queue counters, failed-frame
 * list of the hybrid decoder, training reductions).  Valid for any call with at most
 * n_frames frames and the same parameters. */
bch_status bch_workspace_size(const bch_code *code, const bch_nms_params *params, int n_frames,
                              size_t *bytes);

/* Enhanced NMS (Algorithm 1), or plain NMS (Eqs. 2-5) when params->n_autos == 0.
 * Algorithm 1 as implemented (reading A: the only state kept between iterations is y):
 *   for t = 1..I_m: for each automorphism p, z_p[pi_p(i)] = y[i]; on every edge (j,u)
 *   of H_o, c2v_p(j,u) = alpha_t prod_{u'!=u} sgn z_p[u'] min_{u'!=u} |z_p[u']|;
 *   y_t[i] = y[i] + (1/P) sum_p sum_{j: (j,pi_p(i)) edge} c2v_p(j, pi_p(i));
 *   c = [y_t < 0]; stop if H_o c^T = 0 (and early_stop), else y <- y_t.
 * llr: device [n_frames][ld] FP32 channel LLRs (read only).
 * autos: device [n_frames][n_autos] packed pairs (ignored when n_autos == 0).
 * hard: device [n_frames][ceil(n/64)] u64 final hard decision.
 * iters: device [n_frames] u8 iterations run.  flags: device [n_frames] u8
 * (BCH_FLAG_CONVERGED).  llr_out: device [n_frames][ld] final y (FP32) or NULL.
 * workspace: device, >= bch_workspace_size() bytes, 256-byte aligned.
 * n_frames = 0 is a no-op.  Frames are independent: the result of a frame does not
 * depend on the batch it is decoded in. */
bch_status bch_nms_decode(const bch_code *code, const bch_nms_params *params, const float *llr,
                          int ld, int n_frames, const uint16_t *autos, uint64_t *hard,
                          uint8_t *iters, uint8_t *flags, float *llr_out, void *workspace,
                          void *stream);

/* Hybrid decoder (Sec. IV, complexity discussion): enhanced NMS on `code`; frames
 * whose NMS hard decision has nonzero syndrome go to order-p OSD (Sec. II-B) on the
 * standard matrix `std_code`: positions sorted by FP32 |L| ascending (stable);
 * Gaussian elimination over GF(2) pivots on the least reliable independent columns;
 * the other k positions form the most reliable basis; every test pattern of weight
 * <= p on it is re-encoded and scored by sum over disagreeing positions of
 * floor(|L_i| 2^24) (exact integers); the first minimum wins.  OSD frames get
 * BCH_FLAG_OSD and their hard decision replaced.  failed_list (optional, device
 * [n_frames] u32) and failed_count (optional, device u32) receive the OSD frame
 * indices in ascending order and their count.  No host synchronisation. */
bch_status bch_hybrid_decode(const bch_code *code, const bch_code *std_code,
                             const bch_nms_params *params, const float *llr, int ld, int n_frames,
                             const uint16_t *autos, uint64_t *hard, uint8_t *iters, uint8_t *flags,
                             float *llr_out, uint32_t *failed_list, uint32_t *failed_count,
                             void *workspace, void *stream);

/* bch_hybrid_decode for callers that cannot allocate device memory when they decode
 * (real-time loops where cudaMalloc is forbidden or too slow after start-up, plug-ins
 * handed only pre-registered buffers): the same arguments minus the workspace, checked
 * by the same rules (n_autos = 0 selects the plain decoder) before anything is
 * launched, so a rejected call writes nothing.  The paper has no counterpart; this is
 * a deployment convenience.  Its scratch is one file-scope __device__ array of about
 * 1 MB that every GPU loading the library holds until exit, so n_frames is limited to
 * 262144 (larger batches return BCH_EINVAL).  The first call in a CUDA context looks
 * the array up (cudaGetSymbolAddress) with that context current -- again after the
 * context is re-created, e.g. by cudaDeviceReset; make that first call before any
 * stream capture.  Each device has its own array, shared by every call on that device:
 * calls that overlap on the same GPU (different streams at the same time) race and
 * must be serialised by the caller; each call clears what must start at zero.  No
 * cudaMalloc, cudaFree or allocating routine is called and only precompiled kernels
 * run; results equal bch_hybrid_decode's within the FP32 tolerance (bit-exact for
 * integer work). */
bch_status bch_hybrid_decode_noalloc(const bch_code *code, const bch_code *std_code,
                                     const bch_nms_params *params, const float *llr, int ld,
                                     int n_frames, const uint16_t *autos, uint64_t *hard,
                                     uint8_t *iters, uint8_t *flags, float *llr_out, void *stream);

/* Failed-frame compaction (the hybrid decoder's hand-off to OSD): writes to list
 * (device [n_frames] u32) the indices of the frames whose flags lack
 * BCH_FLAG_CONVERGED, in ascending order, and their number to *count (device u32).
 * Deterministic two-pass block scan; no host synchronisation. */
bch_status bch_compact_failed(const uint8_t *flags, int n_frames, uint32_t *list, uint32_t *count,
                              void *workspace, void *stream);

/* Order-p OSD alone on the listed frames (indices into llr), overwriting their hard
 * decision; used by the hybrid decoder and exposed for testing.  n_frames is the number
 * of frames in llr, hard and flags; the first min(*count, n_frames) entries of
 * frame_list (device u32) are read and each must be < n_frames (the checked build
 * skips and records any other). */
bch_status bch_osd_decode(const bch_code *std_code, int order, const float *llr, int ld,
                          const uint32_t *frame_list, const uint32_t *count, int n_frames,
                          uint64_t *hard, uint8_t *flags, void *workspace, void *stream);

/* Per-batch error counters (for FER/BER reporting) accumulated into
 * counters[8] (device int64): 0 frames, 1 frame errors, 2 bit errors, 3 undetected
 * errors (converged to a wrong codeword), 4 OSD frames, 5 total iterations,
 * 6 NMS-converged frames, 7 reserved.  codeword is the transmitted word. */
bch_status bch_count_errors(int n, const uint64_t *hard, const uint64_t *codeword,
                            const uint8_t *iters, const uint8_t *flags, int n_frames,
                            long long *counters, void *stream);

/* ---------------------------------------------------------------- host pipeline */

/* Decoder context for callers whose frames live in host memory.  It owns device
 * buffers for two chunks of `chunk_frames` frames and two CUDA streams, so the
 * host-to-device copy of one chunk, the hybrid decode of another and the copy-back
 * overlap.  params (alpha is copied) and ld are fixed at creation; std_code may be
 * NULL to run enhanced NMS only (no OSD). */
typedef struct bch_decoder bch_decoder;
bch_status bch_decoder_create(const bch_code *code, const bch_code *std_code,
                              const bch_nms_params *params, int ld, int chunk_frames,
                              bch_decoder **out);
/* Decodes n_frames frames from host memory: llr [n_frames][ld] FP32, automorphisms drawn
 * on the device from (autos_seed, frame0 + index), results to host arrays hard
 * [n_frames][ceil(n/64)], iters and flags [n_frames] (iters/flags nullable).  Returns
 * when all results are in host memory.  When every buffer is page-locked host memory
 * mapped into the device's address space (cudaHostAlloc, or torch's pin_memory, under
 * unified addressing) the kernels read the LLRs and write the results in place -- on a
 * GB300 over the coherent CPU-GPU link -- with no staging copies; otherwise (pageable
 * memory, or bch_decoder_set_in_place(dec, 0)) each chunk is copied in and its results
 * copied out on the two streams. */
bch_status bch_decoder_run_host(bch_decoder *dec, const float *llr, int n_frames,
                                uint64_t autos_seed, uint64_t frame0, uint64_t *hard,
                                uint8_t *iters, uint8_t *flags);
void bch_decoder_destroy(bch_decoder *dec);
/* Per-phase timing of bch_decoder_run_host, a measurement aid with no counterpart in
 * the paper.  bch_decoder_set_timing(dec, 1) clears the totals and makes every later
 * run_host call record four CUDA events per chunk on the chunk's stream (around the
 * copy-in, the decode and the copy-out) and its host wall time; set_timing(dec, 0)
 * stops.  bch_decoder_get_timing returns the totals since the last set_timing: calls,
 * chunks, ms_wall (host time inside run_host), and the device time of the copies in,
 * of the decode launches (automorphism draw, NMS, compaction, OSD) and of the copies
 * out.  The two streams overlap, so the three device sums can exceed ms_wall. */
typedef struct {
  long long calls, chunks, in_place_chunks; /* in_place_chunks: decoded without copies */
  double ms_wall, ms_h2d, ms_decode, ms_d2h;
} bch_decoder_timing;
bch_status bch_decoder_set_timing(bch_decoder *dec, int on);
/* 1 (default): decode mapped page-locked host buffers in place (see run_host); 0: always
 * stage the chunks through the decoder's device buffers with copies. */
bch_status bch_decoder_set_in_place(bch_decoder *dec, int on);
bch_status bch_decoder_get_timing(const bch_decoder *dec, bch_decoder_timing *out);

/* ---------------------------------------------------------------- serving */

/* Continuous-batching decode server.  Requests (one code, 1..max frames each) are
 * admitted as device slots as HBM (budget_bytes) and slots (max_requests) free up and
 * are decoded by the hybrid decoder (enhanced NMS, OSD on the frames it fails when
 * std_codes[i] is given) inside a persistent kernel, overlapping requests that are
 * already on the GPU.  Per-frame results do not depend on which other requests are
 * in flight.  All device waits are bounded: an idle kernel exits after idle_exit_us
 * (default 200 ms) and is relaunched on demand. */
typedef struct bch_server bch_server;
typedef struct {
  int n_codes;                           /* 1..8 code ids                              */
  const bch_code *const *codes;          /* [n_codes] matrices for NMS (H_o)           */
  const bch_code *const *std_codes;      /* [n_codes] standard H for OSD, or NULL      */
  int iters;                             /* I_m                                         */
  const float *alpha;                    /* [iters], copied                             */
  int n_autos;                           /* P                                           */
  int osd_order;                         /* 0..2                                        */
  size_t budget_bytes;                   /* HBM for request data (LLR, draws, results) */
  int max_requests;                      /* slots (requests in flight), <= 65535        */
  int max_frames_per_request;            /* 0: no limit beyond the budget               */
  int warps;                             /* persistent warps; 0: fill the GPU           */
  unsigned idle_exit_us;                 /* idle time before the kernel exits           */
} bch_server_config;

typedef struct {
  long long submitted, admitted, queued, completed, kernel_launches;
  long long bytes_in_use, pending, in_flight, cancelled;
} bch_server_stats;

bch_status bch_server_create(const bch_server_config *cfg, bch_server **out);
/* Submits a request: llr [n_frames][ld] FP32 (host or device memory; it must stay
 * valid until the request completes), automorphisms drawn from (autos_seed, frame0 +
 * index).  Admitted at once when memory and a slot are free, else queued in FIFO
 * order; BCH_EBUDGET if it can never fit the budget.  *request_id identifies it. */
bch_status bch_server_submit(bch_server *srv, int code_id, const float *llr, int ld,
                             int n_frames, uint64_t autos_seed, uint64_t frame0,
                             uint64_t *request_id);
/* Collects up to max_ids completed request ids (waiting up to timeout_us for at least
 * one) and admits queued requests that now fit.  Relaunching a kernel that exited
 * idle waits at most 30 s for the previous instance; past that BCH_ETIMEOUT, with
 * the kernel's live-warp and completion counters in bch_last_error(). */
bch_status bch_server_poll(bch_server *srv, uint64_t *done_ids, int max_ids, int *n_done,
                           int timeout_us);
/* Copies a completed request's results to caller memory (hard [n][ceil(n/64)], iters,
 * flags; host or device) and releases its memory and slot.  BCH_ETIMEOUT if the
 * copies have not finished within 30 s. */
bch_status bch_server_fetch(bch_server *srv, uint64_t request_id, uint64_t *hard,
                            uint8_t *iters, uint8_t *flags);
bch_status bch_server_get_stats(bch_server *srv, bch_server_stats *out);
/* Cancels a request: one still queued is dropped at once; one already on the GPU keeps
 * its frames in flight and is released (memory and slot) when the kernel completes it,
 * without being reported by bch_server_poll; a completed request not yet fetched is
 * released at once.  Either way bch_server_fetch of its id then returns BCH_EINVAL.
 * BCH_EINVAL for an unknown (or already cancelled) id.  No counterpart in the paper:
 * request management of the serving loop. */
bch_status bch_server_cancel(bch_server *srv, uint64_t request_id);
/* Names the serving kernel the server runs: "jit" -- compiled at server creation
 * (NVRTC) with every code's rows as straight-line code, one automorphism copy per code
 * as in the batch decoder's specialised kernel, cached in the process and on disk
 * like it -- or "generic: <reason>" -- the precompiled kernel reading the rows from the
 * codes' device tables.  BCHDEC_NMS_KERNEL (read at bch_server_create) selects as for
 * the batch decoders: generic, jit (creation fails if the compile fails) or auto
 * (default).  Both compute the same results, equal to the batch hybrid decoder's.
 * buf: caller-owned, capacity bytes, always NUL-terminated. */
bch_status bch_server_kernel_info(bch_server *srv, char *buf, size_t capacity);
/* Compiles, for sm_103a with ptxas reporting on, the serving kernel a server of the
 * optimized matrices of BCH(n[i], k[i]) (i < n_codes <= 8, default row counts, matrix
 * seed `seed`) would run, without loading it: no GPU is needed.  log as in
 * bch_nms_jit_check.  No counterpart in the paper: a build aid. */
bch_status bch_serve_jit_check(int n_codes, const int *n, const int *k, uint64_t seed, char *log,
                               size_t capacity);
/* Stops the kernel (at its next iteration) and frees everything.  If the kernel or
 * the server's copies are still running after 30 s, its memory is left allocated
 * (freeing it under a running kernel would fault) and the reason is kept for
 * bch_last_error(). */
void bch_server_destroy(bch_server *srv);

/* Serving benchmark (open loop).  Poisson arrivals at rate_rps for duration_s; each
 * request: code uniform over n_codes, size floor(exp(u ln(max_frames+1))) clipped to
 * [1, max_frames], frames = a contiguous range of that code's host frame pool.
 * Latency = scheduled arrival -> results in host memory.  static_batching = 1 sends the
 * same stream through plain batched launches (collect for batch_us after the first
 * request or batch_frames frames, one bch_hybrid_decode per code, copy back) instead of
 * the server (srv may then be NULL). */
typedef struct {
  double rate_rps, duration_s;
  int max_frames;
  uint64_t seed;
  int n_codes;
  const float *const *pools;  /* [n_codes] host frame pools [pool_frames][ld]            */
  const int *pool_frames;     /* [n_codes]                                               */
  const int *lds;             /* [n_codes]                                               */
  const bch_code *const *codes, *const *std_codes; /* used by static batching            */
  int iters; const float *alpha; int n_autos; int osd_order; /* static batching decoder */
  int static_batching, batch_us, batch_frames;
} bch_serve_bench_config;

typedef struct {
  long long requests, frames;
  double p50_ms, p99_ms, mean_ms, max_ms, elapsed_s;
  double served_frames_per_s, offered_frames_per_s, offered_requests_per_s;
} bch_serve_bench_result;

bch_status bch_serve_bench(bch_server *srv, const bch_serve_bench_config *cfg,
                           bch_serve_bench_result *res);

/* ---------------------------------------------------------------- training */

/* Training forward pass: all `iters` iterations without early stop (FP32 only),
 * checkpointing y^(0..I_m): ckpt device [iters+1][n_frames][ld] (y^(t) of frame f at
 * ckpt + (t n_frames + f) ld).  workspace as for bch_nms_decode. */
bch_status bch_nms_forward_train(const bch_code *code, const bch_nms_params *params,
                                 const float *llr, int ld, int n_frames, const uint16_t *autos,
                                 float *ckpt, void *workspace, void *stream);

/* Backward pass through the iterations (subgradient of min-sum): given
 * grad_out = dLoss/dy^(I_m) [n_frames][ld], writes grad_llr = dLoss/dy^(0)
 * [n_frames][ld] (nullable) and grad_alpha[iters] (device FP32, overwritten).
 * d c2v/d alpha_t = c2v/alpha_t; d c2v(j,u)/d z_a = alpha_t prod_{u'!=u} sgn z_u' sgn z_a
 * at a = argmin over the row without u (lowest column on ties); sign derivatives 0.
 * Recomputes each iteration from its checkpoint. */
bch_status bch_nms_backward(const bch_code *code, const bch_nms_params *params,
                            const uint16_t *autos, const float *ckpt, int ld, int n_frames,
                            const float *grad_out, float *grad_llr, float *grad_alpha,
                            void *workspace, void *stream);

/* Binary cross-entropy of the final LLRs against the transmitted word:
 * loss = mean_i softplus(-(1 - 2c_i) y_i) over frames and bits (device FP32 scalar,
 * overwritten) and grad = dloss/dy [n_frames][ld]. */
bch_status bch_bce_loss(int n, const float *y, int ld, const uint64_t *codeword, int n_frames,
                        float *loss, float *grad, void *workspace, void *stream);

/* Convenience loop: `steps` Adam steps (learning rate lr) on the per-iteration factors
 * alpha_inout[iters] (host, in/out) using `batch` frames per step generated on the
 * device at Eb/N0 uniform in [ebn0_lo, ebn0_hi).  loss_hist (host, nullable) gets the
 * loss of every step.  Allocates its own device buffers. */
bch_status bch_train_alpha(const bch_code *code, int n_autos, int iters, float *alpha_inout,
                           int steps, int batch, float ebn0_lo, float ebn0_hi, uint64_t seed,
                           float lr, float *loss_hist, void *stream);

/* Training state for resuming bch_train_alpha: the Adam moments of every factor and the
 * number of steps taken (which also fixes the frames of the next step: step s decodes
 * frames s batch ... (s + 1) batch - 1 of the simulated stream).  Plain data: a caller
 * saves it with alpha[] and restores both to continue where it stopped.  A zeroed state
 * (step = 0) starts fresh.  No counterpart in the paper: checkpointing of the training
 * loop. */
typedef struct {
  int iters, batch;  /* shape the state belongs to */
  long long step;    /* Adam steps taken */
  double m[32], v[32];
} bch_adam_state;

/* bch_train_alpha continued from (alpha_inout, *state): runs `steps` more Adam steps
 * and updates both after every step (so an interrupted run keeps a consistent pair).
 * state NULL behaves as bch_train_alpha.  N steps in one call and the same N split
 * over several calls that pass the state on give bit-identical alpha and losses.
 * BCH_EINVAL if a nonzero state belongs to another iters or batch. */
bch_status bch_train_alpha_resume(const bch_code *code, int n_autos, int iters, float *alpha_inout,
                                  bch_adam_state *state, int steps, int batch, float ebn0_lo,
                                  float ebn0_hi, uint64_t seed, float lr, float *loss_hist,
                                  void *stream);

/* ---------------------------------------------------------------- checked build */

/* The checked library is this library compiled with -DBCH_CHECKED
 * (paper_2412_20828_gb300/_build/checked/libbchdec.so; the Python binding loads it when
 * BCHDEC_CHECKED=1).  Its kernels validate every index they take from caller-supplied
 * device data before using it:
 *   - each packed automorphism s | j << 8 (Sec. III-B: pi(i) = 2^j i + s mod n) must
 *     have s < n and j < m, n = 2^m - 1 (enhanced NMS in every kernel variant, the
 *     hybrid, no-allocation and training entry points, the backward pass);
 *   - each OSD frame-list entry (bch_osd_decode) must be < n_frames.
 * An invalid value never traps: it is replaced by a harmless one (the identity
 * automorphism, so the frame is decoded as if that copy were unpermuted; a bad list
 * entry is skipped) and recorded in the current device's check word:
 *   word[0]  OR of BCH_CHECK_* bits,
 *   word[1]  number of invalid values met (a value read by several threads counts once
 *            per reader),
 *   word[2]  smallest frame index holding an invalid automorphism (0xffffffff: none),
 *   word[3]  smallest OSD list position holding an invalid entry (0xffffffff: none).
 * Automorphisms the library draws itself (host pipeline, server, simulation) are valid
 * by construction.  The ordinary build does the same work without the checks and
 * takes such values as given (results undefined for invalid ones).  No counterpart in
 * the paper: a debugging aid. */
#define BCH_CHECK_AUTOMORPHISM 1u
#define BCH_CHECK_OSD_FRAME 2u

/* 1 in the checked build, else 0. */
int bch_is_checked(void);

/* Synchronises `stream`, copies the current device's check word to word_out (host
 * u32 [4]) and, when clear != 0, resets it (0, 0, 0xffffffff, 0xffffffff).
 * BCH_EINVAL in the ordinary build or for a null word_out. */
bch_status bch_check_read(uint32_t *word_out, int clear, void *stream);

/* ---------------------------------------------------------------- misc */

const char *bch_status_str(bch_status s);
const char *bch_last_error(void);
/* Number of kernels this library has launched in the process so far (every device and
 * thread; incremented at each launch), e.g. to count the launches inside a timed
 * region.  No counterpart in the paper: a measurement aid. */
unsigned long long bch_kernel_launches(void);
/* Library version string. */
const char *bch_version(void);

#ifdef __cplusplus
}
#endif
#endif /* BCHDEC_H_ */
