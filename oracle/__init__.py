"""FP64 CPU oracle for the enhanced-NMS / OSD decoder of arXiv 2412.20828.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this package.
The decoder library never imports it and shares no code with it.

The arithmetic lives in ``bch_oracle.c`` (plain C, one byte per bit, double
precision); this module compiles it with gcc on first use and wraps it with numpy
arrays.  Functions whose parity against the paper is only partly pinned say so in
the C file's header: the H_o row set (``build_ho``) is "parity unpinned" against the
paper (pinned only by invariants), everything else is pinned by the tests listed
there.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bch_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, EARG, ECODE, ERANK, ENOMEM = 0, -1, -2, -3, -4


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (portable flags only: it builds on x86-64 and Arm)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = C.CDLL(build())
        P = C.c_void_p
        i, u64, d = C.c_int, C.c_uint64, C.c_double
        sig = {
            "or_ord2": (i, [i]),
            "or_gen_poly": (i, [i, i, P]),
            "or_std_h": (i, [i, i, P]),
            "or_encode": (i, [i, i, P, i, P]),
            "or_syndrome_weight": (i, [P, i, i, P]),
            "or_rank": (i, [P, i, i]),
            "or_sigma2": (d, [i, i, d]),
            "or_channel_llr": (None, [i, i, P, P, i, P, P, i]),
            "or_splitmix64": (u64, [P]),
            "or_philox4x32_10": (None, [P, P, P]),
            "or_framegen": (i, [i, i, u64, u64, i, d, d, P, i, P, P]),
            "or_draw_autos": (i, [i, i, u64, u64, i, P]),
            "or_build_ho": (i, [i, i, i, u64, i, i, d, d, d, P, P, P]),
            "or_build_ho_chain": (i, [i, i, i, u64, i, i, d, d, d, i, P, P, P, P]),
            "or_nms_plain": (i, [P, i, i, P, i, i, i, d, i, P, P, P, P, P, P]),
            "or_nms_enhanced": (i, [P, i, i, P, i, i, i, P, i, P, i, P, P, P, P, P, P, P]),
            "or_nms_plain_f32": (i, [P, i, i, P, i, i, i, C.c_float, i, P, P, P, P]),
            "or_nms_enhanced_f32": (i, [P, i, i, P, i, i, i, P, i, P, i, P, P, P, P]),
            "or_osd": (i, [P, i, i, P, i, i, i, P, P, P]),
            "or_q16": (d, [d]),
            "or_nms_enhanced_q": (i, [P, i, i, P, i, i, i, P, i, P, i, i, i, i, P, P, P, P, P]),
            "or_ml": (i, [i, i, P, i, i, P]),
            "or_nms_train_grad": (i, [P, i, i, P, i, i, i, P, i, P, P, P, P, P, P, P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _check(rc, what):
    if rc != OK:
        raise RuntimeError(f"oracle {what} failed with status {rc}")


# ----------------------------------------------------------------------------- algebra
def ord2(n: int) -> int:
    return _load().or_ord2(n)


def gen_poly(n: int, k: int) -> np.ndarray:
    g = np.zeros(n - k + 1, np.uint8)
    _check(_load().or_gen_poly(n, k, _p(g)), "gen_poly")
    return g


def std_h(n: int, k: int) -> np.ndarray:
    H = np.zeros((n - k, n), np.uint8)
    _check(_load().or_std_h(n, k, _p(H)), "std_h")
    return H


def encode(n: int, k: int, msg: np.ndarray) -> np.ndarray:
    msg = np.ascontiguousarray(msg, dtype=np.uint8).reshape(-1, k)
    cw = np.zeros((msg.shape[0], n), np.uint8)
    _check(_load().or_encode(n, k, _p(msg), msg.shape[0], _p(cw)), "encode")
    return cw


def syndrome_weight(H: np.ndarray, c: np.ndarray) -> int:
    H = np.ascontiguousarray(H, np.uint8)
    c = np.ascontiguousarray(c, np.uint8)
    return _load().or_syndrome_weight(_p(H), H.shape[0], H.shape[1], _p(c))


def rank(H: np.ndarray) -> int:
    H = np.ascontiguousarray(H, np.uint8)
    return _load().or_rank(_p(H), H.shape[0], H.shape[1])


def sigma2(n: int, k: int, ebn0_db: float) -> float:
    return _load().or_sigma2(n, k, float(ebn0_db))


def channel_llr(n: int, k: int, cw: np.ndarray, noise: np.ndarray, ebn0_db, ld: int | None = None):
    """FP32 LLRs of Eq. (1) for codewords ``cw`` [F, n] and standard normals ``noise``."""
    cw = np.ascontiguousarray(cw, np.uint8).reshape(-1, n)
    F = cw.shape[0]
    noise = np.ascontiguousarray(noise, np.float64).reshape(F, n)
    e = np.ascontiguousarray(np.broadcast_to(np.asarray(ebn0_db, np.float64), (F,)))
    ld = ld or n
    llr = np.zeros((F, ld), np.float32)
    _load().or_channel_llr(n, k, _p(cw), _p(noise), F, _p(e), _p(llr), ld)
    return llr


# ----------------------------------------------------------------------------- PRNGs
def splitmix64(state: int, count: int) -> list[int]:
    st = np.array([state], np.uint64)
    return [int(_load().or_splitmix64(_p(st))) for _ in range(count)]


def philox4x32_10(ctr, key) -> list[int]:
    c = np.array(ctr, np.uint32)
    kk = np.array(key, np.uint32)
    o = np.zeros(4, np.uint32)
    _load().or_philox4x32_10(_p(c), _p(kk), _p(o))
    return [int(x) for x in o]


def framegen(n, k, seed, frame0, F, ebn0_lo, ebn0_hi=None, ld=None):
    """Synthetic frames by the library's Philox/Box-Muller recipe, restated in FP64."""
    ld = ld or n
    ebn0_hi = ebn0_lo if ebn0_hi is None else ebn0_hi
    llr = np.zeros((F, ld), np.float32)
    cw = np.zeros((F, n), np.uint8)
    e = np.zeros(F, np.float64)
    _check(_load().or_framegen(n, k, seed, frame0, F, ebn0_lo, ebn0_hi, _p(llr), ld, _p(cw), _p(e)),
           "framegen")
    return llr, cw, e


# ----------------------------------------------------------------------------- graph
def draw_autos(n: int, P: int, seed: int, frame0: int, F: int) -> np.ndarray:
    out = np.zeros((F, P), np.uint16)
    _check(_load().or_draw_autos(n, P, seed, frame0, F, _p(out)), "draw_autos")
    return out


def auto_perm(v: int, n: int) -> np.ndarray:
    """pi as an index array: pi[i] = (2^j i + s) mod n."""
    s, j = v & 0xFF, v >> 8
    i = np.arange(n)
    return (pow(2, j, n) * i + s) % n


DEFAULT_Q_ROUNDS = 4
DEFAULT_SA_STEPS = 20000
DEFAULT_T0_FRAC = 0.05
DEFAULT_COOL = 0.9995


def build_ho(n, k, m_rows=0, seed=0x2412_20828, q_rounds=DEFAULT_Q_ROUNDS,
             sa_steps=DEFAULT_SA_STEPS, sa_lambda=None, t0_frac=DEFAULT_T0_FRAC,
             cool=DEFAULT_COOL, return_r1=False):
    lam = float(n) if sa_lambda is None else float(sa_lambda)
    H = np.zeros((max(m_rows, 2 * (n - k)), n), np.uint8)
    r1 = np.zeros(1, np.int32)
    mo = np.zeros(1, np.int32)
    _check(_load().or_build_ho(n, k, m_rows, seed, q_rounds, sa_steps, lam, t0_frac, cool,
                               _p(H), _p(r1), _p(mo)), "build_ho")
    H = np.ascontiguousarray(H[: int(mo[0])])
    return (H, int(r1[0])) if return_r1 else H


def build_ho_chain(n, k, chain, m_rows=0, seed=0x2412_20828, q_rounds=DEFAULT_Q_ROUNDS,
                   sa_steps=DEFAULT_SA_STEPS, sa_lambda=None, t0_frac=DEFAULT_T0_FRAC,
                   cool=DEFAULT_COOL):
    """H_o annealed by chain `chain` of a parallel annealing search (see the C file;
    chain 0 is build_ho).  Returns (H, number of 4-cycles, sum of squared column
    weights) of the final matrix."""
    lam = float(n) if sa_lambda is None else float(sa_lambda)
    H = np.zeros((max(m_rows, 2 * (n - k)), n), np.uint8)
    r1 = np.zeros(1, np.int32)
    mo = np.zeros(1, np.int32)
    st = np.zeros(2, np.int64)
    _check(_load().or_build_ho_chain(n, k, m_rows, seed, q_rounds, sa_steps, lam, t0_frac, cool,
                                     int(chain), _p(H), _p(r1), _p(mo), _p(st)), "build_ho_chain")
    return np.ascontiguousarray(H[: int(mo[0])]), int(st[0]), int(st[1])


# ----------------------------------------------------------------------------- decoders
def _pool_map(fn, F, chunk, threads):
    if threads is None:
        threads = os.cpu_count() or 1
    if threads <= 1 or F <= chunk:
        fn(0, F)
        return
    with ThreadPoolExecutor(threads) as ex:
        list(ex.map(lambda a: fn(a, min(F, a + chunk)), range(0, F, chunk)))


def nms_plain(H, llr, iters, alpha, early_stop=True, threads=1):
    H = np.ascontiguousarray(H, np.uint8)
    M, n = H.shape
    llr = np.ascontiguousarray(llr, np.float32)
    F, ld = llr.shape
    hard = np.zeros((F, n), np.uint8)
    it = np.zeros(F, np.int32)
    conv = np.zeros(F, np.uint8)
    y = np.zeros((F, n), np.float64)
    env = np.zeros(F, np.float64)
    mar = np.zeros(F, np.float64)
    lib = _load()

    def run(a, b):
        _check(lib.or_nms_plain(_p(H), M, n, _p(llr[a:]), ld, b - a, iters, float(alpha),
                                int(early_stop), _p(hard[a:]), _p(it[a:]), _p(conv[a:]),
                                _p(y[a:]), _p(env[a:]), _p(mar[a:])), "nms_plain")

    _pool_map(run, F, 256, threads)
    return dict(hard=hard, iters=it, converged=conv, y=y, env=env, margin_rel=mar)


def nms_enhanced(Ho, llr, autos, iters, alpha, early_stop=True, trace=False, threads=1):
    """Algorithm 1, reading A.  ``alpha`` is a scalar or one factor per iteration."""
    Ho = np.ascontiguousarray(Ho, np.uint8)
    M, n = Ho.shape
    llr = np.ascontiguousarray(llr, np.float32)
    F, ld = llr.shape
    autos = np.ascontiguousarray(autos, np.uint16).reshape(F, -1)
    P = autos.shape[1]
    al = np.ascontiguousarray(np.broadcast_to(np.asarray(alpha, np.float64), (iters,)))
    hard = np.zeros((F, n), np.uint8)
    it = np.zeros(F, np.int32)
    conv = np.zeros(F, np.uint8)
    y = np.zeros((F, n), np.float64)
    margin = np.zeros(F, np.float64)
    tr = np.zeros((F, iters + 1, n), np.float64) if trace else None
    mag = np.zeros((F, iters, n), np.float64) if trace else None
    lib = _load()

    def run(a, b):
        _check(lib.or_nms_enhanced(_p(Ho), M, n, _p(llr[a:]), ld, b - a, P, _p(autos[a:]), iters,
                                   _p(al), int(early_stop), _p(hard[a:]), _p(it[a:]),
                                   _p(conv[a:]), _p(y[a:]),
                                   _p(tr[a:]) if trace else None,
                                   _p(mag[a:]) if trace else None, _p(margin[a:])),
               "nms_enhanced")

    _pool_map(run, F, 256, threads)
    out = dict(hard=hard, iters=it, converged=conv, y=y, margin=margin)
    if trace:
        out["trace"] = tr
        out["mag"] = mag
    return out


def nms_plain_f32(H, llr, iters, alpha, early_stop=True, threads=1):
    """Eqs. (2)-(5) evaluated directly in FP32 (the loops of ``nms_plain``); see the C
    file: it measures how far a direct single-precision evaluation drifts from FP64."""
    H = np.ascontiguousarray(H, np.uint8)
    M, n = H.shape
    llr = np.ascontiguousarray(llr, np.float32)
    F, ld = llr.shape
    hard = np.zeros((F, n), np.uint8)
    it = np.zeros(F, np.int32)
    conv = np.zeros(F, np.uint8)
    y = np.zeros((F, n), np.float64)
    lib = _load()

    def run(a, b):
        _check(lib.or_nms_plain_f32(_p(H), M, n, _p(llr[a:]), ld, b - a, iters,
                                    float(np.float32(alpha)), int(early_stop), _p(hard[a:]),
                                    _p(it[a:]), _p(conv[a:]), _p(y[a:])), "nms_plain_f32")

    _pool_map(run, F, 256, threads)
    return dict(hard=hard, iters=it, converged=conv, y=y)


def nms_enhanced_f32(Ho, llr, autos, iters, alpha, early_stop=True, threads=1):
    """Algorithm 1 (reading A) evaluated directly in FP32 (the loops of
    ``nms_enhanced``); see the C file."""
    Ho = np.ascontiguousarray(Ho, np.uint8)
    M, n = Ho.shape
    llr = np.ascontiguousarray(llr, np.float32)
    F, ld = llr.shape
    autos = np.ascontiguousarray(autos, np.uint16).reshape(F, -1)
    P = autos.shape[1]
    al = np.ascontiguousarray(np.broadcast_to(np.asarray(alpha, np.float32), (iters,)))
    hard = np.zeros((F, n), np.uint8)
    it = np.zeros(F, np.int32)
    conv = np.zeros(F, np.uint8)
    y = np.zeros((F, n), np.float64)
    lib = _load()

    def run(a, b):
        _check(lib.or_nms_enhanced_f32(_p(Ho), M, n, _p(llr[a:]), ld, b - a, P, _p(autos[a:]),
                                       iters, _p(al), int(early_stop), _p(hard[a:]), _p(it[a:]),
                                       _p(conv[a:]), _p(y[a:])), "nms_enhanced_f32")

    _pool_map(run, F, 256, threads)
    return dict(hard=hard, iters=it, converged=conv, y=y)


def q16(x: float) -> float:
    return _load().or_q16(float(x))


def nms_enhanced_q(Ho, llr, autos, iters, alpha, fmt, rescale=False, early_stop=True, threads=1,
                   qfrac=0):
    """Algorithm 1 with FP16 (fmt=1) or 8-bit (fmt=2) storage; with qfrac > 0 (8-bit only)
    the check-to-variable magnitudes keep qfrac fractional bits and the merge rounds the
    exact quotient; see the C file."""
    Ho = np.ascontiguousarray(Ho, np.uint8)
    M, n = Ho.shape
    llr = np.ascontiguousarray(llr, np.float32)
    F, ld = llr.shape
    autos = np.ascontiguousarray(autos, np.uint16).reshape(F, -1)
    P = autos.shape[1]
    al = np.ascontiguousarray(np.broadcast_to(np.asarray(alpha, np.float64), (iters,)))
    hard = np.zeros((F, n), np.uint8)
    it = np.zeros(F, np.int32)
    conv = np.zeros(F, np.uint8)
    y = np.zeros((F, n), np.float64)
    margin = np.zeros(F, np.float64)
    lib = _load()

    def run(a, b):
        _check(lib.or_nms_enhanced_q(_p(Ho), M, n, _p(llr[a:]), ld, b - a, P, _p(autos[a:]), iters,
                                     _p(al), int(early_stop), fmt, int(rescale), int(qfrac), _p(hard[a:]),
                                     _p(it[a:]), _p(conv[a:]), _p(y[a:]), _p(margin[a:])),
               "nms_enhanced_q")

    _pool_map(run, F, 256, threads)
    # margin (FP16 only): smallest distance of a merged value, relative to its operand
    # magnitude, to zero or to a binary16 rounding boundary (see the C file)
    return dict(hard=hard, iters=it, converged=conv, y=y, margin=margin)


def osd(H, llr, order=2, threads=1, return_mrb=False):
    H = np.ascontiguousarray(H, np.uint8)
    M, n = H.shape
    llr = np.ascontiguousarray(llr, np.float32)
    F, ld = llr.shape
    cw = np.zeros((F, n), np.uint8)
    sc = np.zeros(F, np.uint64)
    mrb = np.zeros((F, n - M), np.int32)
    lib = _load()

    def run(a, b):
        _check(lib.or_osd(_p(H), M, n, _p(llr[a:]), ld, b - a, order, _p(cw[a:]), _p(sc[a:]),
                          _p(mrb[a:])), "osd")

    _pool_map(run, F, 16, threads)
    if return_mrb:
        return cw, sc, mrb
    return cw, sc


def ml(n, k, llr):
    llr = np.ascontiguousarray(llr, np.float32)
    F, ld = llr.shape
    cw = np.zeros((F, n), np.uint8)
    _check(_load().or_ml(n, k, _p(llr), ld, F, _p(cw)), "ml")
    return cw


def hybrid(Ho, Hstd, llr, autos, iters, alpha, order=2, threads=1):
    """Hybrid decoder (Sec. IV-B): the NMS word where its syndrome is zero, else OSD."""
    r = nms_enhanced(Ho, llr, autos, iters, alpha, early_stop=True, threads=threads)
    fail = np.nonzero(r["converged"] == 0)[0]
    final = r["hard"].copy()
    if fail.size:
        cw, _ = osd(Hstd, llr[fail], order, threads=threads)
        final[fail] = cw
    r["final"] = final
    r["osd_frames"] = fail
    return r


def hybrid_nms_reliability(Ho, Hstd, llr, autos, iters, alpha, order=2, threads=1):
    """Hybrid decoder with the OSD fallback ranking and scoring positions by the NMS
    output y of each failed frame instead of its channel LLR (the paper feeds OSD the
    channel LLR, Sec. II-B; this is the alternative input).  y grows by about an order
    of magnitude per iteration, past the OSD's integer weights floor(|L| 2^24) capped
    at 2^40, so each failed frame's y is first scaled by the power of two that puts
    max_i |y_i| in [2^15, 2^16) (exact) and rounded to FP32, the OSD's input format.
    Decisions do not depend on the scale: min-sum is homogeneous in its input and the
    scaling is per frame."""
    r = nms_enhanced(Ho, llr, autos, iters, alpha, early_stop=True, threads=threads)
    fail = np.nonzero(r["converged"] == 0)[0]
    final = r["hard"].copy()
    if fail.size:
        y = r["y"][fail]
        _, ex = np.frexp(np.max(np.abs(y), axis=1))  # max |y| = m 2^ex, m in [0.5, 1)
        ys = np.ldexp(y, (16 - ex)[:, None]).astype(np.float32)
        cw, _ = osd(Hstd, ys, order, threads=threads)
        final[fail] = cw
    r["final"] = final
    r["osd_frames"] = fail
    return r


def train_grad(Ho, llr, autos, iters, alpha, cw, return_margin=False):
    Ho = np.ascontiguousarray(Ho, np.uint8)
    M, n = Ho.shape
    llr = np.ascontiguousarray(llr, np.float32)
    F, ld = llr.shape
    autos = np.ascontiguousarray(autos, np.uint16).reshape(F, -1)
    P = autos.shape[1]
    al = np.ascontiguousarray(np.broadcast_to(np.asarray(alpha, np.float64), (iters,)))
    cw = np.ascontiguousarray(cw, np.uint8)
    loss = np.zeros(1, np.float64)
    da = np.zeros(iters, np.float64)
    dl = np.zeros((F, n), np.float64)
    y = np.zeros((F, n), np.float64)
    tm = np.zeros(F, np.float64)
    _check(_load().or_nms_train_grad(_p(Ho), M, n, _p(llr), ld, F, P, _p(autos), iters, _p(al),
                                     _p(cw), _p(loss), _p(da), _p(dl), _p(y), _p(tm)), "train_grad")
    if return_margin:
        return float(loss[0]), da, dl, y, tm
    return float(loss[0]), da, dl, y
