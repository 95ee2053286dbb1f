"""Thin Python binding of the C ABI in ``include/bchdec.h`` (ctypes).

Argument marshalling only: every step of decoding runs in the CUDA library.  Device
buffers are torch CUDA tensors (torch is used for memory and streams); the calls are
asynchronous on the current torch stream unless ``stream`` is given.  Loading fails
loudly when ``libbchdec.so`` has not been built -- there is no CPU fallback.  With
BCHDEC_CHECKED=1 in the environment the checked build (``_build/checked``, compiled
with -DBCH_CHECKED) is loaded instead.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libbchdec.so")
LIB_PATH_CHECKED = os.path.join(_HERE, "_build", "checked", "libbchdec.so")
CHECK_AUTOMORPHISM, CHECK_OSD_FRAME = 1, 2

OK, EINVAL, ENOMEM, ECUDA, ERANK, ETIMEOUT, EBUDGET, EBUSY = range(8)
PCM_STANDARD, PCM_OPTIMIZED = 0, 1
MSG_FP32, MSG_FP16, MSG_INT8 = 0, 1, 2
FLAG_CONVERGED, FLAG_OSD = 1, 2

# Every symbol the header declares (checked by the tests without a GPU).
EXPORTS = (
    "bch_build_pcm", "bch_build_pcm_host", "bch_search_pcm", "bch_nms_kernel_info", "bch_nms_jit_check", "bch_code_info", "bch_pcm_export", "bch_code_free",
    "bch_draw_automorphisms", "bch_draw_automorphisms_host", "bch_gen_frames",
    "bch_workspace_size", "bch_nms_decode", "bch_hybrid_decode", "bch_hybrid_decode_noalloc",
    "bch_osd_decode",
    "bch_compact_failed", "bch_count_errors", "bch_nms_forward_train", "bch_nms_backward", "bch_bce_loss",
    "bch_train_alpha", "bch_decoder_create", "bch_decoder_run_host", "bch_decoder_destroy",
    "bch_decoder_set_timing", "bch_decoder_get_timing", "bch_decoder_set_in_place", "bch_train_alpha_resume",
    "bch_kernel_launches",
    "bch_server_create", "bch_server_submit", "bch_server_poll", "bch_server_fetch",
    "bch_server_get_stats", "bch_server_cancel", "bch_server_kernel_info", "bch_serve_jit_check", "bch_server_destroy",
    "bch_serve_bench",
    "bch_is_checked", "bch_check_read",
    "bch_status_str", "bch_last_error", "bch_version",
)


class BchError(RuntimeError):
    def __init__(self, status, where, detail):
        super().__init__(f"{where}: status {status} ({detail})")
        self.status = status


class PcmOpts(C.Structure):
    _fields_ = [("q_rounds", C.c_int), ("sa_steps", C.c_int), ("sa_lambda", C.c_double),
                ("sa_t0_frac", C.c_double), ("sa_cool", C.c_double)]


class ServerConfig(C.Structure):
    _fields_ = [("n_codes", C.c_int), ("codes", C.POINTER(C.c_void_p)),
                ("std_codes", C.POINTER(C.c_void_p)), ("iters", C.c_int),
                ("alpha", C.POINTER(C.c_float)), ("n_autos", C.c_int), ("osd_order", C.c_int),
                ("budget_bytes", C.c_size_t), ("max_requests", C.c_int),
                ("max_frames_per_request", C.c_int), ("warps", C.c_int),
                ("idle_exit_us", C.c_uint)]


class ServerStats(C.Structure):
    _fields_ = [(nm, C.c_longlong) for nm in ("submitted", "admitted", "queued", "completed",
                                               "kernel_launches", "bytes_in_use", "pending",
                                               "in_flight", "cancelled")]


class ServeBenchConfig(C.Structure):
    _fields_ = [("rate_rps", C.c_double), ("duration_s", C.c_double), ("max_frames", C.c_int),
                ("seed", C.c_uint64), ("n_codes", C.c_int), ("pools", C.POINTER(C.c_void_p)),
                ("pool_frames", C.POINTER(C.c_int)), ("lds", C.POINTER(C.c_int)),
                ("codes", C.POINTER(C.c_void_p)), ("std_codes", C.POINTER(C.c_void_p)),
                ("iters", C.c_int), ("alpha", C.POINTER(C.c_float)), ("n_autos", C.c_int),
                ("osd_order", C.c_int), ("static_batching", C.c_int), ("batch_us", C.c_int),
                ("batch_frames", C.c_int)]


class ServeBenchResult(C.Structure):
    _fields_ = [("requests", C.c_longlong), ("frames", C.c_longlong), ("p50_ms", C.c_double),
                ("p99_ms", C.c_double), ("mean_ms", C.c_double), ("max_ms", C.c_double),
                ("elapsed_s", C.c_double), ("served_frames_per_s", C.c_double),
                ("offered_frames_per_s", C.c_double), ("offered_requests_per_s", C.c_double)]


class NmsParams(C.Structure):
    _fields_ = [("iters", C.c_int), ("alpha", C.POINTER(C.c_float)), ("n_autos", C.c_int),
                ("early_stop", C.c_int), ("msg", C.c_int), ("rescale", C.c_int),
                ("osd_order", C.c_int), ("osd_input", C.c_int), ("qfrac", C.c_int)]


_lock = threading.Lock()
_lib = None


def load():
    """Loads libbchdec.so (built by ``paper_2412_20828_gb300.build.build()``)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = LIB_PATH_CHECKED if os.environ.get("BCHDEC_CHECKED") == "1" else LIB_PATH
        if not os.path.exists(path):
            raise RuntimeError(
                f"{path} is missing: build it with "
                "`python -c 'import __graft_entry__ as g; g.build()'` (no CPU fallback exists)")
        lib = C.CDLL(path)
        P, i, u64, f, sz = C.c_void_p, C.c_int, C.c_uint64, C.c_float, C.c_size_t
        st = C.c_int
        sig = {
            "bch_build_pcm": (st, [i, i, i, i, u64, C.POINTER(PcmOpts), C.POINTER(P)]),
            "bch_build_pcm_host": (st, [i, i, i, i, u64, C.POINTER(PcmOpts), P, sz, C.POINTER(i)]),
            "bch_search_pcm": (st, [i, i, i, u64, C.POINTER(PcmOpts), i, P, P, sz, C.POINTER(i),
                                    C.POINTER(P)]),
            "bch_nms_kernel_info": (st, [P, i, i, C.c_char_p, sz]),
            "bch_nms_jit_check": (st, [i, i, i, u64, P, i, C.c_char_p, sz]),
            "bch_code_info": (st, [P, C.POINTER(i), C.POINTER(i), C.POINTER(i), C.POINTER(i),
                                   C.POINTER(i)]),
            "bch_pcm_export": (st, [P, P, sz]),
            "bch_code_free": (None, [P]),
            "bch_draw_automorphisms": (st, [i, i, u64, u64, i, P, P]),
            "bch_draw_automorphisms_host": (st, [i, i, u64, u64, i, P]),
            "bch_gen_frames": (st, [P, f, f, u64, u64, i, P, i, P, P]),
            "bch_workspace_size": (st, [P, C.POINTER(NmsParams), i, C.POINTER(sz)]),
            "bch_nms_decode": (st, [P, C.POINTER(NmsParams), P, i, i, P, P, P, P, P, P, P]),
            "bch_hybrid_decode": (st, [P, P, C.POINTER(NmsParams), P, i, i, P, P, P, P, P, P, P,
                                       P, P]),
            "bch_hybrid_decode_noalloc": (st, [P, P, C.POINTER(NmsParams), P, i, i, P, P, P, P, P,
                                               P]),
            "bch_osd_decode": (st, [P, i, P, i, P, P, i, P, P, P, P]),
            "bch_compact_failed": (st, [P, i, P, P, P, P]),
            "bch_count_errors": (st, [i, P, P, P, P, i, P, P]),
            "bch_nms_forward_train": (st, [P, C.POINTER(NmsParams), P, i, i, P, P, P, P]),
            "bch_nms_backward": (st, [P, C.POINTER(NmsParams), P, P, i, i, P, P, P, P, P]),
            "bch_bce_loss": (st, [i, P, i, P, i, P, P, P, P]),
            "bch_train_alpha": (st, [P, i, i, P, i, i, f, f, u64, f, P, P]),
            "bch_train_alpha_resume": (st, [P, i, i, P, C.POINTER(AdamState), i, i, f, f, u64, f, P, P]),
            "bch_decoder_create": (st, [P, P, C.POINTER(NmsParams), i, i, C.POINTER(P)]),
            "bch_decoder_run_host": (st, [P, P, i, u64, u64, P, P, P]),
            "bch_decoder_destroy": (None, [P]),
            "bch_decoder_set_timing": (st, [P, i]),
            "bch_decoder_get_timing": (st, [P, C.POINTER(DecoderTiming)]),
            "bch_decoder_set_in_place": (st, [P, i]),
            "bch_kernel_launches": (C.c_ulonglong, []),
            "bch_server_create": (st, [C.POINTER(ServerConfig), C.POINTER(P)]),
            "bch_server_submit": (st, [P, i, P, i, i, u64, u64, C.POINTER(u64)]),
            "bch_server_poll": (st, [P, P, i, C.POINTER(i), i]),
            "bch_server_fetch": (st, [P, u64, P, P, P]),
            "bch_server_get_stats": (st, [P, C.POINTER(ServerStats)]),
            "bch_server_cancel": (st, [P, u64]),
            "bch_server_kernel_info": (st, [P, C.c_char_p, sz]),
            "bch_serve_jit_check": (st, [i, C.POINTER(C.c_int), C.POINTER(C.c_int), u64, C.c_char_p, sz]),
            "bch_server_destroy": (None, [P]),
            "bch_serve_bench": (st, [P, C.POINTER(ServeBenchConfig), C.POINTER(ServeBenchResult)]),
            "bch_is_checked": (i, []),
            "bch_check_read": (st, [P, i, P]),
            "bch_status_str": (C.c_char_p, [i]),
            "bch_last_error": (C.c_char_p, []),
            "bch_version": (C.c_char_p, []),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _check(rc, where):
    if rc != OK:
        lib = load()
        raise BchError(rc, where, lib.bch_last_error().decode(errors="replace"))


def _ptr(t):
    """Raw pointer of a torch tensor / numpy array (None stays NULL)."""
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data_as(C.c_void_p)
    if not t.is_contiguous():
        raise ValueError("tensors passed to the library must be contiguous")
    return C.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is not None:
        return C.c_void_p(stream)
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dev(t, dtype, name):
    import torch
    if t is None:
        return None
    if not (isinstance(t, torch.Tensor) and t.is_cuda):
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    return t


class Code:
    """A BCH code object (standard H or optimized H_o) owned by the library."""

    def __init__(self, n, k, kind=PCM_OPTIMIZED, m_rows=0, seed=0x2412_20828, q_rounds=4,
                 sa_steps=20000, sa_lambda=0.0, sa_t0_frac=0.05, sa_cool=0.9995):
        lib = load()
        self._h = C.c_void_p()
        opts = PcmOpts(q_rounds, sa_steps, sa_lambda, sa_t0_frac, sa_cool)
        _check(lib.bch_build_pcm(n, k, kind, m_rows, seed, C.byref(opts), C.byref(self._h)),
               "bch_build_pcm")
        a = [C.c_int() for _ in range(5)]
        _check(lib.bch_code_info(self._h, *[C.byref(x) for x in a]), "bch_code_info")
        self.n, self.k, self.rows, self.edges, self.max_row_weight = (x.value for x in a)
        self.kind = kind

    @classmethod
    def _adopt(cls, handle, kind):
        """Wraps a code object the library created (ownership passes to the wrapper)."""
        self = cls.__new__(cls)
        self._h = handle
        a = [C.c_int() for _ in range(5)]
        _check(load().bch_code_info(self._h, *[C.byref(x) for x in a]), "bch_code_info")
        self.n, self.k, self.rows, self.edges, self.max_row_weight = (x.value for x in a)
        self.kind = kind
        return self

    @property
    def handle(self):
        return self._h

    def kernel_info(self, msg=MSG_FP32, n_autos=3) -> str:
        buf = C.create_string_buffer(4096)
        _check(load().bch_nms_kernel_info(self._h, msg, n_autos, buf, 4096), "bch_nms_kernel_info")
        return buf.value.decode()

    def dense(self) -> np.ndarray:
        out = np.zeros((self.rows, self.n), np.uint8)
        _check(load().bch_pcm_export(self._h, _ptr(out), out.nbytes), "bch_pcm_export")
        return out

    def close(self):
        if self._h:
            load().bch_code_free(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def search_pcm(n, k, n_chains, m_rows=0, seed=0x2412_20828, q_rounds=4, sa_steps=20000,
               sa_lambda=0.0, sa_t0_frac=0.05, sa_cool=0.9995, return_all=False):
    """bch_search_pcm: the annealing step of H_o as n_chains parallel chains on the GPU;
    returns (Code of the kept chain, kept chain, stats [n_chains][3]) and, with
    return_all, every chain's matrix [n_chains][rows][n]."""
    rows = max(m_rows, 2 * (n - k))  # capacity; the matrices are [n_chains][rows of H_o][n]
    stats = np.zeros((n_chains, 3), np.int64)
    dense = np.zeros(n_chains * rows * n, np.uint8) if return_all else None
    best = C.c_int(-1)
    h = C.c_void_p()
    opts = PcmOpts(q_rounds, sa_steps, sa_lambda, sa_t0_frac, sa_cool)
    _check(load().bch_search_pcm(n, k, m_rows, seed, C.byref(opts), n_chains, _ptr(stats),
                                 _ptr(dense), dense.nbytes if dense is not None else 0,
                                 C.byref(best), C.byref(h)), "bch_search_pcm")
    code = Code._adopt(h, PCM_OPTIMIZED)
    if return_all:
        return code, best.value, stats, dense[: n_chains * code.rows * n].reshape(n_chains, code.rows, n)
    return code, best.value, stats


def build_pcm(n, k, kind=PCM_OPTIMIZED, m_rows=0, seed=0x2412_20828, **opts) -> Code:
    return Code(n, k, kind, m_rows, seed, **opts)


def build_pcm_host(n, k, kind=PCM_OPTIMIZED, m_rows=0, seed=0x2412_20828, q_rounds=4,
                   sa_steps=20000, sa_lambda=0.0, sa_t0_frac=0.05, sa_cool=0.9995) -> np.ndarray:
    """The matrix of bch_build_pcm computed on the host only (no GPU), as bytes."""
    rows_cap = max(m_rows, 2 * (n - k))
    out = np.zeros((rows_cap, n), np.uint8)
    rows = C.c_int()
    opts = PcmOpts(q_rounds, sa_steps, sa_lambda, sa_t0_frac, sa_cool)
    _check(load().bch_build_pcm_host(n, k, kind, m_rows, seed, C.byref(opts), _ptr(out), out.nbytes,
                                     C.byref(rows)), "bch_build_pcm_host")
    return np.ascontiguousarray(out[: rows.value])


def nms_jit_check(n, k, msg=MSG_FP32, m_rows=0, seed=0x2412_20828) -> str:
    """Compiles the specialised kernel of the optimized matrix of BCH(n, k) (no GPU
    needed); returns the compiler report (registers, spills) or raises BchError with
    the compile errors."""
    buf = C.create_string_buffer(1 << 16)
    rc = load().bch_nms_jit_check(n, k, m_rows, seed, None, msg, buf, 1 << 16)
    if rc != OK:
        raise BchError(rc, "bch_nms_jit_check",
                       buf.value.decode(errors="replace") or load().bch_last_error().decode())
    return buf.value.decode(errors="replace")


def serve_jit_check(codes, seed=0x2412_20828) -> str:
    """Compiles the serving kernel specialised to the optimized matrices of the codes
    [(n, k), ...] (no GPU needed); returns the compiler report or raises BchError."""
    nn = (C.c_int * len(codes))(*[n for n, _ in codes])
    kk = (C.c_int * len(codes))(*[k for _, k in codes])
    buf = C.create_string_buffer(1 << 16)
    rc = load().bch_serve_jit_check(len(codes), nn, kk, seed, buf, 1 << 16)
    if rc != OK:
        raise BchError(rc, "bch_serve_jit_check",
                       buf.value.decode(errors="replace") or load().bch_last_error().decode())
    return buf.value.decode(errors="replace")


OSD_CHANNEL, OSD_NMS_OUTPUT = 0, 1


def params(iters, alpha, n_autos=3, early_stop=True, msg=MSG_FP32, rescale=False, osd_order=2,
           osd_input=OSD_CHANNEL, qfrac=0):
    """Builds a bch_nms_params; ``alpha`` is a scalar or one factor per iteration; ``qfrac``
    fractional bits of the 8-bit form's check-to-variable magnitudes (see the header)."""
    al = np.ascontiguousarray(np.broadcast_to(np.asarray(alpha, np.float32), (iters,)))
    p = NmsParams(iters, al.ctypes.data_as(C.POINTER(C.c_float)), n_autos, int(early_stop), msg,
                  int(rescale), osd_order, int(osd_input), int(qfrac))
    p._alpha_keepalive = al  # the C struct points into this array
    return p


def workspace_size(code: Code, p: NmsParams, n_frames: int) -> int:
    b = C.c_size_t()
    _check(load().bch_workspace_size(code.handle, C.byref(p), n_frames, C.byref(b)),
           "bch_workspace_size")
    return b.value


def workspace(code: Code, p: NmsParams, n_frames: int, device="cuda"):
    import torch
    nb = workspace_size(code, p, n_frames)
    return torch.empty(max(nb, 256), dtype=torch.uint8, device=device)


def draw_automorphisms(n, n_autos, seed, frame0, out, stream=None):
    import torch
    _dev(out, torch.int16, "out")
    F = out.shape[0]
    _check(load().bch_draw_automorphisms(n, n_autos, seed, frame0, F, _ptr(out), _stream(stream)),
           "bch_draw_automorphisms")
    return out


def draw_automorphisms_host(n, n_autos, seed, frame0, n_frames) -> np.ndarray:
    out = np.zeros((n_frames, n_autos), np.uint16)
    _check(load().bch_draw_automorphisms_host(n, n_autos, seed, frame0, n_frames, _ptr(out)),
           "bch_draw_automorphisms_host")
    return out


def gen_frames(code: Code, ebn0_lo, ebn0_hi, seed, frame0, llr, codeword=None, stream=None):
    import torch
    _dev(llr, torch.float32, "llr")
    _dev(codeword, torch.int64, "codeword")
    F, ld = llr.shape
    _check(load().bch_gen_frames(code.handle, float(ebn0_lo), float(ebn0_hi), seed, frame0, F,
                                 _ptr(llr), ld, _ptr(codeword), _stream(stream)), "bch_gen_frames")


def nms_decode(code: Code, p: NmsParams, llr, autos, hard, iters=None, flags=None, llr_out=None,
               ws=None, stream=None):
    import torch
    _dev(llr, torch.float32, "llr")
    _dev(hard, torch.int64, "hard")
    F, ld = llr.shape
    ws = ws if ws is not None else workspace(code, p, F)
    _check(load().bch_nms_decode(code.handle, C.byref(p), _ptr(llr), ld, F, _ptr(autos), _ptr(hard),
                                 _ptr(iters), _ptr(flags), _ptr(llr_out), _ptr(ws), _stream(stream)),
           "bch_nms_decode")


def hybrid_decode(code: Code, std_code: Code, p: NmsParams, llr, autos, hard, iters, flags,
                  llr_out=None, failed_list=None, failed_count=None, ws=None, stream=None):
    import torch
    _dev(llr, torch.float32, "llr")
    F, ld = llr.shape
    ws = ws if ws is not None else workspace(code, p, F)
    _check(load().bch_hybrid_decode(code.handle, std_code.handle, C.byref(p), _ptr(llr), ld, F,
                                    _ptr(autos), _ptr(hard), _ptr(iters), _ptr(flags),
                                    _ptr(llr_out), _ptr(failed_list), _ptr(failed_count), _ptr(ws),
                                    _stream(stream)), "bch_hybrid_decode")


def hybrid_decode_noalloc(code: Code, std_code: Code, p: NmsParams, llr, autos, hard, iters, flags,
                          llr_out=None, stream=None):
    """bch_hybrid_decode without a workspace: for callers that cannot allocate device
    memory while decoding (scratch is a fixed ~1 MB device array; n_frames <= 262144)."""
    import torch
    _dev(llr, torch.float32, "llr")
    F, ld = llr.shape
    _check(load().bch_hybrid_decode_noalloc(code.handle, std_code.handle, C.byref(p), _ptr(llr), ld,
                                            F, _ptr(autos), _ptr(hard), _ptr(iters), _ptr(flags),
                                            _ptr(llr_out), _stream(stream)),
           "bch_hybrid_decode_noalloc")


def osd_decode(std_code: Code, order, llr, frame_list, count, hard, flags=None, ws=None,
               stream=None):
    """Order-p OSD on the first min(count, len(llr)) frames listed in frame_list (device
    u32 indices into llr, each < len(llr))."""
    import torch
    F, ld = llr.shape
    ws = ws if ws is not None else torch.zeros(256, dtype=torch.uint8, device=llr.device)
    _check(load().bch_osd_decode(std_code.handle, order, _ptr(llr), ld, _ptr(frame_list),
                                 _ptr(count), F, _ptr(hard), _ptr(flags),
                                 _ptr(ws), _stream(stream)), "bch_osd_decode")


def compact_failed(flags, lst, count, ws, n_frames=None, stream=None):
    F = flags.shape[0] if n_frames is None else n_frames
    _check(load().bch_compact_failed(_ptr(flags), F, _ptr(lst), _ptr(count), _ptr(ws),
                                     _stream(stream)), "bch_compact_failed")


def count_errors(n, hard, codeword, iters, flags, counters, stream=None):
    F = hard.shape[0]
    _check(load().bch_count_errors(n, _ptr(hard), _ptr(codeword), _ptr(iters), _ptr(flags), F,
                                   _ptr(counters), _stream(stream)), "bch_count_errors")


def nms_forward_train(code: Code, p: NmsParams, llr, autos, ckpt, ws=None, stream=None):
    F, ld = llr.shape
    ws = ws if ws is not None else workspace(code, p, F)
    _check(load().bch_nms_forward_train(code.handle, C.byref(p), _ptr(llr), ld, F, _ptr(autos),
                                        _ptr(ckpt), _ptr(ws), _stream(stream)),
           "bch_nms_forward_train")


def nms_backward(code: Code, p: NmsParams, autos, ckpt, grad_out, grad_llr, grad_alpha, ws=None,
                 stream=None):
    F, ld = grad_out.shape
    ws = ws if ws is not None else workspace(code, p, F)
    _check(load().bch_nms_backward(code.handle, C.byref(p), _ptr(autos), _ptr(ckpt), ld, F,
                                   _ptr(grad_out), _ptr(grad_llr), _ptr(grad_alpha), _ptr(ws),
                                   _stream(stream)), "bch_nms_backward")


def bce_loss(n, y, codeword, loss, grad, ws, stream=None):
    F, ld = y.shape
    _check(load().bch_bce_loss(n, _ptr(y), ld, _ptr(codeword), F, _ptr(loss), _ptr(grad), _ptr(ws),
                               _stream(stream)), "bch_bce_loss")


def train_alpha(code: Code, n_autos, iters, alpha, steps, batch, ebn0_lo, ebn0_hi, seed, lr,
                stream=None):
    al = np.ascontiguousarray(np.broadcast_to(np.asarray(alpha, np.float32), (iters,))).copy()
    hist = np.zeros(max(steps, 1), np.float32)
    _check(load().bch_train_alpha(code.handle, n_autos, iters, _ptr(al), steps, batch,
                                  float(ebn0_lo), float(ebn0_hi), seed, float(lr), _ptr(hist),
                                  _stream(stream)), "bch_train_alpha")
    return al, hist[:steps]


class AdamState(C.Structure):
    """bch_adam_state: the training loop's resumable state."""
    _fields_ = [("iters", C.c_int), ("batch", C.c_int), ("step", C.c_longlong),
                ("m", C.c_double * 32), ("v", C.c_double * 32)]

    def to_arrays(self) -> dict:
        return {"iters": self.iters, "batch": self.batch, "step": self.step,
                "m": np.array(self.m[:]), "v": np.array(self.v[:])}

    @classmethod
    def from_arrays(cls, d) -> "AdamState":
        s = cls()
        s.iters, s.batch, s.step = int(d["iters"]), int(d["batch"]), int(d["step"])
        for t in range(32):
            s.m[t] = float(d["m"][t])
            s.v[t] = float(d["v"][t])
        return s


def save_training(path, alpha, state: AdamState):
    """Writes alpha and the Adam state to an .npz file (exact doubles and floats)."""
    d = state.to_arrays()
    np.savez(path, alpha=np.asarray(alpha, np.float32), **d)


def load_training(path):
    """(alpha, AdamState) from a file written by save_training."""
    with np.load(path) as z:
        return z["alpha"].copy(), AdamState.from_arrays(z)


def train_alpha_resume(code, n_autos, iters, alpha, state, steps, batch, ebn0_lo, ebn0_hi, seed, lr,
                       stream=None):
    """bch_train_alpha_resume: continues from (alpha, state); returns (alpha, losses) and
    updates state in place."""
    al = np.ascontiguousarray(np.broadcast_to(np.asarray(alpha, np.float32), (iters,))).copy()
    hist = np.zeros(max(steps, 1), np.float32)
    _check(load().bch_train_alpha_resume(code.handle, n_autos, iters, _ptr(al), C.byref(state), steps,
                                         batch, float(ebn0_lo), float(ebn0_hi), seed, float(lr),
                                         _ptr(hist), _stream(stream)), "bch_train_alpha_resume")
    return al, hist[:steps]


class DecoderTiming(C.Structure):
    _fields_ = [("calls", C.c_longlong), ("chunks", C.c_longlong), ("in_place_chunks", C.c_longlong),
                ("ms_wall", C.c_double),
                ("ms_h2d", C.c_double), ("ms_decode", C.c_double), ("ms_d2h", C.c_double)]


def is_checked() -> bool:
    """True when the loaded library is the checked build (-DBCH_CHECKED)."""
    return bool(load().bch_is_checked())


def check_read(clear=True, stream=None) -> np.ndarray:
    """The checked build's device check word (u32 [4]: CHECK_* bits, number of invalid
    values, smallest frame with an invalid automorphism, smallest OSD list position with
    an invalid entry; 0xffffffff where none); synchronises the stream."""
    w = np.zeros(4, np.uint32)
    _check(load().bch_check_read(w.ctypes.data, 1 if clear else 0, _stream(stream)), "bch_check_read")
    return w


def kernel_launches() -> int:
    """Kernels the library has launched in this process (bch_kernel_launches)."""
    return int(load().bch_kernel_launches())


class HostDecoder:
    """bch_decoder: decodes frames held in host memory with overlapped transfers."""

    def __init__(self, code: Code, std_code, p: NmsParams, ld: int, chunk_frames: int = 1 << 20):
        self._h = C.c_void_p()
        self._p = p
        self.code, self.std = code, std_code
        _check(load().bch_decoder_create(code.handle, std_code.handle if std_code else None,
                                         C.byref(p), ld, chunk_frames, C.byref(self._h)),
               "bch_decoder_create")
        self.ld = ld

    def run(self, llr, autos_seed, frame0, hard, iters=None, flags=None):
        """llr / hard / iters / flags: host numpy arrays or pinned CPU torch tensors."""
        F = llr.shape[0]
        _check(load().bch_decoder_run_host(self._h, _ptr(llr), F, autos_seed, frame0, _ptr(hard),
                                           _ptr(iters), _ptr(flags)), "bch_decoder_run_host")

    def set_in_place(self, on=True):
        """Decode mapped page-locked host buffers in place (default) or stage copies."""
        _check(load().bch_decoder_set_in_place(self._h, int(on)), "bch_decoder_set_in_place")

    def set_timing(self, on=True):
        """Per-phase timing of the later run() calls (bch_decoder_set_timing)."""
        _check(load().bch_decoder_set_timing(self._h, int(on)), "bch_decoder_set_timing")

    def timing(self) -> dict:
        t = DecoderTiming()
        _check(load().bch_decoder_get_timing(self._h, C.byref(t)), "bch_decoder_get_timing")
        return {f: getattr(t, f) for f, _ in DecoderTiming._fields_}

    def close(self):
        if self._h:
            load().bch_decoder_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """bch_server: continuous-batching hybrid decoding of requests of mixed codes."""

    def __init__(self, codes, std_codes, iters, alpha, n_autos=3, osd_order=2,
                 budget_bytes=16 << 30, max_requests=1024, max_frames_per_request=4096, warps=0,
                 idle_exit_us=200000):
        self.codes, self.std_codes = list(codes), list(std_codes) if std_codes else None
        self._al = np.ascontiguousarray(np.broadcast_to(np.asarray(alpha, np.float32), (iters,)))
        n = len(self.codes)
        self._ch = (C.c_void_p * n)(*[c.handle.value for c in self.codes])
        self._sh = (C.c_void_p * n)(*[c.handle.value if c else None for c in self.std_codes]) \
            if self.std_codes else None
        cfg = ServerConfig(n, C.cast(self._ch, C.POINTER(C.c_void_p)),
                           C.cast(self._sh, C.POINTER(C.c_void_p)) if self._sh else None,
                           iters, self._al.ctypes.data_as(C.POINTER(C.c_float)), n_autos, osd_order,
                           budget_bytes, max_requests, max_frames_per_request, warps, idle_exit_us)
        self._h = C.c_void_p()
        _check(load().bch_server_create(C.byref(cfg), C.byref(self._h)), "bch_server_create")
        self._keep = {}

    def submit(self, code_id, llr, autos_seed, frame0):
        """llr: [F, ld] FP32 numpy array (host) or CUDA tensor; kept alive until fetched."""
        F, ld = llr.shape
        rid = C.c_uint64()
        _check(load().bch_server_submit(self._h, code_id, _ptr(llr), ld, F, autos_seed, frame0,
                                        C.byref(rid)), "bch_server_submit")
        self._keep[rid.value] = (llr, code_id, F)
        return rid.value

    def poll(self, max_ids=256, timeout_us=0):
        ids = np.zeros(max_ids, np.uint64)
        nd = C.c_int()
        _check(load().bch_server_poll(self._h, _ptr(ids), max_ids, C.byref(nd), timeout_us),
               "bch_server_poll")
        return [int(x) for x in ids[: nd.value]]

    def fetch(self, rid):
        if rid not in self._keep:  # unknown, cancelled or already fetched
            raise BchError(EINVAL, "bch_server_fetch", "request not complete or unknown")
        llr, code_id, F = self._keep[rid]
        n = self.codes[code_id].n
        hard = np.zeros((F, (n + 63) // 64), np.uint64)
        it = np.zeros(F, np.uint8)
        fl = np.zeros(F, np.uint8)
        _check(load().bch_server_fetch(self._h, rid, _ptr(hard), _ptr(it), _ptr(fl)),
               "bch_server_fetch")
        del self._keep[rid]
        return hard.view(np.int64), it, fl

    def kernel_info(self) -> str:
        """"jit" (serving kernel specialised to the codes) or "generic: <reason>"."""
        buf = C.create_string_buffer(4096)
        _check(load().bch_server_kernel_info(self._h, buf, 4096), "bch_server_kernel_info")
        return buf.value.decode()

    def cancel(self, rid):
        """bch_server_cancel: drops a queued request, or releases one on the GPU when the
        kernel completes it (it is then never reported by poll)."""
        _check(load().bch_server_cancel(self._h, C.c_uint64(rid)), "bch_server_cancel")
        self._keep.pop(rid, None)

    def stats(self):
        st = ServerStats()
        _check(load().bch_server_get_stats(self._h, C.byref(st)), "bch_server_get_stats")
        return {k: getattr(st, k) for k, _ in ServerStats._fields_}

    def close(self):
        if self._h:
            load().bch_server_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def serve_bench(server, codes, std_codes, pools, rate_rps, duration_s, max_frames=4096, seed=1,
                iters=12, alpha=0.78, n_autos=3, osd_order=2, static_batching=False,
                batch_us=1000, batch_frames=65536):
    """bch_serve_bench: pools are pinned host tensors / numpy arrays [pool_frames, ld]."""
    n = len(pools)
    al = np.ascontiguousarray(np.broadcast_to(np.asarray(alpha, np.float32), (iters,)))
    pp = (C.c_void_p * n)(*[_ptr(p).value for p in pools])
    pf = (C.c_int * n)(*[int(p.shape[0]) for p in pools])
    ld = (C.c_int * n)(*[int(p.shape[1]) for p in pools])
    ch = (C.c_void_p * n)(*[c.handle.value for c in codes])
    sh = (C.c_void_p * n)(*[c.handle.value for c in std_codes]) if std_codes else None
    cfg = ServeBenchConfig(rate_rps, duration_s, max_frames, seed, n,
                           C.cast(pp, C.POINTER(C.c_void_p)), pf, ld,
                           C.cast(ch, C.POINTER(C.c_void_p)),
                           C.cast(sh, C.POINTER(C.c_void_p)) if sh else None, iters,
                           al.ctypes.data_as(C.POINTER(C.c_float)), n_autos, osd_order,
                           int(static_batching), batch_us, batch_frames)
    res = ServeBenchResult()
    _check(load().bch_serve_bench(server._h if server else None, C.byref(cfg), C.byref(res)),
           "bch_serve_bench")
    return {k: getattr(res, k) for k, _ in ServeBenchResult._fields_}


def unpack_bits(words: np.ndarray, n: int) -> np.ndarray:
    """[F, ceil(n/64)] packed words (int64/uint64) -> [F, n] uint8 bits."""
    w = np.ascontiguousarray(words).view(np.uint64).reshape(words.shape[0], -1)
    bits = np.zeros((w.shape[0], n), np.uint8)
    for i in range(n):
        bits[:, i] = (w[:, i >> 6] >> np.uint64(i & 63)) & np.uint64(1)
    return bits


def pack_bits(bits: np.ndarray) -> np.ndarray:
    """[F, n] bits -> [F, ceil(n/64)] int64 words (bit i of word i//64)."""
    F, n = bits.shape
    W = (n + 63) // 64
    out = np.zeros((F, W), np.uint64)
    for i in range(n):
        out[:, i >> 6] |= bits[:, i].astype(np.uint64) << np.uint64(i & 63)
    return out.view(np.int64)
