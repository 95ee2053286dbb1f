"""GPU parity of the decoding path (called through the C ABI) against the FP64 oracle:
automorphism draws, frame generation, enhanced NMS (Algorithm 1), plain NMS
(Eqs. 2-5), OSD and the hybrid decoder, plus edge cases."""
import numpy as np
import pytest

import oracle as O
from helpers import (ambiguous_frames, autos_dev, check_trajectory, frame_envelope, frames, rel_close,
                     to_dev)
from paper_2412_20828_gb300 import bchdec as B

pytestmark = pytest.mark.gpu

CODES = [(15, 7), (63, 36), (63, 45), (127, 64), (127, 78), (127, 99)]


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    from paper_2412_20828_gb300 import build
    build.build()
    B.load()
    return torch


_codes = {}


def code(n, k, kind=B.PCM_OPTIMIZED):
    key = (n, k, kind)
    if key not in _codes:
        _codes[key] = B.Code(n, k, kind=kind)
    return _codes[key]


def W64(n):
    return (n + 63) // 64


def run_nms(torch, c, llr, autos, iters, alpha, early_stop=True, msg=B.MSG_FP32, rescale=False,
            n_autos=3):
    F, ld = llr.shape
    p = B.params(iters, alpha, n_autos=n_autos, early_stop=early_stop, msg=msg, rescale=rescale)
    d_llr = to_dev(llr)
    d_aut = autos_dev(autos) if autos is not None else None
    hard = torch.zeros((F, W64(c.n)), dtype=torch.int64, device="cuda")
    it = torch.zeros(F, dtype=torch.uint8, device="cuda")
    fl = torch.zeros(F, dtype=torch.uint8, device="cuda")
    yo = torch.full((F, ld), 7.0, dtype=torch.float32, device="cuda")
    B.nms_decode(c, p, d_llr, d_aut, hard, it, fl, yo)
    torch.cuda.synchronize()
    return dict(hard=B.unpack_bits(hard.cpu().numpy(), c.n), iters=it.cpu().numpy(),
                flags=fl.cpu().numpy(), y=yo.cpu().numpy())


# ------------------------------------------------------------------ draws and frames
@pytest.mark.parametrize("n,P", [(63, 3), (127, 3), (127, 9), (15, 3)])
def test_autos_device_bit_exact(torch_cuda, n, P):
    torch = torch_cuda
    F = 10007
    out = torch.zeros((F, P), dtype=torch.int16, device="cuda")
    B.draw_automorphisms(n, P, 99, 123, out)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy().view(np.uint16), O.draw_autos(n, P, 99, 123, F))


@pytest.mark.parametrize("nk,ld,lo,hi", [((63, 36), 64, 3.0, 3.0), ((127, 64), 128, 2.0, 5.0),
                                         ((63, 45), 63, 1.0, 6.0), ((15, 7), 16, 4.0, 4.0)])
def test_framegen_matches_oracle(torch_cuda, nk, ld, lo, hi):
    torch = torch_cuda
    n, k = nk
    F = 3001
    c = code(n, k)
    llr = torch.full((F, ld), 5.0, dtype=torch.float32, device="cuda")
    cw = torch.zeros((F, W64(n)), dtype=torch.int64, device="cuda")
    B.gen_frames(c, lo, hi, 77, 1000, llr, cw)
    torch.cuda.synchronize()
    ref_llr, ref_cw, ref_e = O.framegen(n, k, 77, 1000, F, lo, hi, ld=ld)
    assert np.array_equal(B.unpack_bits(cw.cpu().numpy(), n), ref_cw)
    got = llr.cpu().numpy()
    scale = np.array([2.0 / O.sigma2(n, k, e) for e in ref_e])[:, None]
    tol = 1e-5 * np.maximum(np.abs(ref_llr), scale)
    assert np.all(np.abs(got - ref_llr) <= tol)
    assert np.all(got[:, n:] == 0)


# ------------------------------------------------------------------ enhanced NMS
@pytest.mark.parametrize("nk", CODES)
def test_enhanced_one_iteration(torch_cuda, nk):
    n, k = nk
    c = code(n, k)
    F = 1000  # not a multiple of the warp or block size
    cw, llr = frames(n, k, F, 2.0, 100 + n + k, ld=(n + 3) & ~3)
    autos = O.draw_autos(n, 3, 5, 0, F)
    g = run_nms(torch_cuda, c, llr, autos, 1, 0.78, early_stop=False)
    ref = O.nms_enhanced(c.dense(), llr, autos, 1, 0.78, early_stop=False, trace=True)
    ok = rel_close(g["y"][:, :n], ref["y"], ref["mag"][:, 0, :])
    assert ok.all(), f"{(~ok).sum()} entries out of tolerance"
    assert np.all(g["y"][:, n:] == 7.0)  # padding columns untouched
    assert np.all(g["iters"] == 1)


@pytest.mark.parametrize("nk", CODES)
@pytest.mark.parametrize("ebn0", [1.5, 3.5])
def test_enhanced_full_decode(torch_cuda, nk, ebn0):
    n, k = nk
    c = code(n, k)
    F = 1500
    cw, llr = frames(n, k, F, ebn0, 200 + n + k, ld=(n + 3) & ~3)
    autos = O.draw_autos(n, 3, 11, 0, F)
    alpha = np.linspace(0.7, 0.9, 12)
    g = run_nms(torch_cuda, c, llr, autos, 12, alpha)
    ref = O.nms_enhanced(c.dense(), llr, autos, 12, alpha, trace=True, threads=None)
    amb = ambiguous_frames(llr, ref, n)
    assert amb.mean() < 0.1
    ok = ~amb
    assert np.array_equal(g["iters"][ok], ref["iters"][ok])
    assert np.array_equal(g["hard"][ok], ref["hard"][ok])
    assert np.array_equal(g["flags"][ok] & 1, ref["converged"][ok])
    # trajectory: against the drift of the direct FP32 evaluation of the same frames
    env = frame_envelope(ref)[:, None]
    f32 = O.nms_enhanced_f32(c.dense(), llr, autos, 12, alpha, threads=None)
    check_trajectory(g["y"][:, :n], ref["y"], f32["y"], env, ok, "enhanced", 12)


def test_enhanced_nine_automorphisms_and_unaligned_ld(torch_cuda):
    n, k = 63, 45
    c = code(n, k)
    F = 333
    cw, llr = frames(n, k, F, 2.5, 300, ld=n)  # ld = 63: scalar load path
    autos = O.draw_autos(n, 9, 3, 0, F)
    g = run_nms(torch_cuda, c, llr, autos, 6, 0.8, n_autos=9)
    ref = O.nms_enhanced(c.dense(), llr, autos, 6, 0.8, trace=True)
    ok = ~ambiguous_frames(llr, ref, n)
    assert np.array_equal(g["hard"][ok], ref["hard"][ok])
    assert np.array_equal(g["iters"][ok], ref["iters"][ok])


def test_enhanced_noiseless_one_iteration(torch_cuda):
    for n, k in CODES:
        c = code(n, k)
        cw = O.encode(n, k, np.random.default_rng(n).integers(0, 2, (77, k), dtype=np.uint8))
        llr = (3.0 * (1 - 2.0 * cw)).astype(np.float32)
        g = run_nms(torch_cuda, c, llr, O.draw_autos(n, 3, 1, 0, 77), 12, 0.78)
        assert np.all(g["iters"] == 1) and np.all(g["flags"] & 1)
        assert np.array_equal(g["hard"], cw)


def test_zero_frames_is_noop(torch_cuda):
    torch = torch_cuda
    c = code(63, 45)
    p = B.params(12, 0.78)
    empty = torch.zeros((0, 64), dtype=torch.float32, device="cuda")
    hard = torch.zeros((0, 1), dtype=torch.int64, device="cuda")
    B.nms_decode(c, p, empty, torch.zeros((0, 3), dtype=torch.int16, device="cuda"), hard)
    torch.cuda.synchronize()


def test_invalid_arguments_rejected(torch_cuda):
    torch = torch_cuda
    c = code(63, 45)
    llr = torch.zeros((4, 64), dtype=torch.float32, device="cuda")
    hard = torch.zeros((4, 1), dtype=torch.int64, device="cuda")
    with pytest.raises(B.BchError) as e:
        B.nms_decode(c, B.params(33, 0.78), llr, None, hard)
    assert e.value.status == B.EINVAL
    with pytest.raises(B.BchError):
        B.nms_decode(c, B.params(12, 0.78, n_autos=3), llr, None, hard)  # autos missing
    with pytest.raises(B.BchError):
        B.nms_decode(c, B.params(12, 0.78), llr[:, :32].contiguous(), None, hard)  # ld < n


def test_batch_independence(torch_cuda):
    # a frame decodes to the same bits whatever batch it is in (persistent scheduling)
    n, k = 127, 64
    c = code(n, k)
    F = 700
    _, llr = frames(n, k, F, 2.0, 400, ld=128)
    autos = O.draw_autos(n, 3, 2, 0, F)
    full = run_nms(torch_cuda, c, llr, autos, 12, 0.78)
    part = run_nms(torch_cuda, c, llr[350:400], autos[350:400], 12, 0.78)
    assert np.array_equal(full["hard"][350:400], part["hard"])
    assert np.array_equal(full["y"][350:400], part["y"])


# ------------------------------------------------------------------ plain NMS
@pytest.mark.parametrize("ebn0", [2.0, 3.0])
def test_plain_nms_standard_h(torch_cuda, ebn0):
    n, k = 63, 36
    c = code(n, k, B.PCM_STANDARD)
    F = 1200
    cw, llr = frames(n, k, F, ebn0, 500, ld=64)
    g = run_nms(torch_cuda, c, llr, None, 8, 0.78, n_autos=0)
    ref = O.nms_plain(c.dense(), llr, 8, 0.78, threads=None)
    # a sign is decided by rounding when a value is within a few FP32 ulps (times the
    # iterations) of zero relative to its own operands: 2e-5 leaves a 4x margin
    amb = np.any(np.abs(llr[:, :n]) < 1e-3, axis=1) | (ref["margin_rel"] < 2e-5)
    assert amb.mean() < 0.1
    ok = ~amb
    assert np.array_equal(g["iters"][ok], ref["iters"][ok])
    assert np.array_equal(g["hard"][ok], ref["hard"][ok])
    env = ref["env"][:, None]
    f32 = O.nms_plain_f32(c.dense(), llr, 8, 0.78, threads=None)
    check_trajectory(g["y"][:, :n], ref["y"], f32["y"], env, ok, "plain", 8)
    # one iteration from the same input: element-wise against the operand magnitude
    g1 = run_nms(torch_cuda, c, llr, None, 1, 0.78, n_autos=0, early_stop=False)
    r1 = O.nms_plain(c.dense(), llr, 1, 0.78, early_stop=False)
    assert rel_close(g1["y"][:, :n], r1["y"], r1["env"][:, None]).all()


# ------------------------------------------------------------------ OSD and hybrid
@pytest.mark.parametrize("nk", CODES)
def test_osd_order2_bit_exact(torch_cuda, nk):
    torch = torch_cuda
    n, k = nk
    std = code(n, k, B.PCM_STANDARD)
    F = 150 if n == 127 else 400
    cw, llr = frames(n, k, F, 1.5, 600 + n + k, ld=(n + 3) & ~3)
    d_llr = to_dev(llr)
    lst = torch.arange(F, dtype=torch.int32, device="cuda")
    cnt = torch.tensor([F], dtype=torch.int32, device="cuda")
    hard = torch.zeros((F, W64(n)), dtype=torch.int64, device="cuda")
    fl = torch.zeros(F, dtype=torch.uint8, device="cuda")
    B.osd_decode(std, 2, d_llr, lst, cnt, hard, fl)
    torch.cuda.synchronize()
    ref, _ = O.osd(std.dense(), llr, order=2, threads=None)
    assert np.array_equal(B.unpack_bits(hard.cpu().numpy(), n), ref)
    assert np.all(fl.cpu().numpy() == B.FLAG_OSD)


def test_osd_partial_list(torch_cuda):
    torch = torch_cuda
    n, k = 63, 45
    std = code(n, k, B.PCM_STANDARD)
    F = 100
    cw, llr = frames(n, k, F, 2.0, 650, ld=64)
    sel = np.array([3, 17, 50, 99], np.int32)
    hard = torch.full((F, 1), -1, dtype=torch.int64, device="cuda")
    B.osd_decode(std, 1, to_dev(llr), to_dev(sel), to_dev(np.array([4], np.int32)), hard)
    torch.cuda.synchronize()
    h = hard.cpu().numpy()
    ref, _ = O.osd(std.dense(), llr[sel], order=1)
    assert np.array_equal(B.unpack_bits(h[sel], n), ref)
    others = np.setdiff1d(np.arange(F), sel)
    assert np.all(h[others] == -1)


@pytest.mark.parametrize("nk,ebn0", [((127, 99), 3.0), ((127, 78), 3.0), ((127, 64), 2.5),
                                     ((63, 36), 2.0), ((15, 7), 2.0)])
def test_hybrid_matches_oracle(torch_cuda, nk, ebn0):
    torch = torch_cuda
    n, k = nk
    c, std = code(n, k), code(n, k, B.PCM_STANDARD)
    F = 600
    cw, llr = frames(n, k, F, ebn0, 700 + n + k, ld=(n + 3) & ~3)
    autos = O.draw_autos(n, 3, 13, 0, F)
    p = B.params(12, 0.78, osd_order=2)
    hard = torch.zeros((F, W64(n)), dtype=torch.int64, device="cuda")
    it = torch.zeros(F, dtype=torch.uint8, device="cuda")
    fl = torch.zeros(F, dtype=torch.uint8, device="cuda")
    lst = torch.zeros(F, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    B.hybrid_decode(c, std, p, to_dev(llr), autos_dev(autos), hard, it, fl, failed_list=lst,
                    failed_count=cnt)
    torch.cuda.synchronize()
    ref = O.hybrid(c.dense(), std.dense(), llr, autos, 12, 0.78, threads=None)
    refe = O.nms_enhanced(c.dense(), llr, autos, 12, 0.78, trace=True, threads=None)
    ok = ~ambiguous_frames(llr, refe, n)
    got = B.unpack_bits(hard.cpu().numpy(), n)
    assert np.array_equal(got[ok], ref["final"][ok])
    flags = fl.cpu().numpy()
    osd_frames = np.nonzero(flags & B.FLAG_OSD)[0]
    fails = np.nonzero((flags & B.FLAG_CONVERGED) == 0)[0]
    assert np.array_equal(osd_frames, fails)
    nf = int(cnt.cpu().numpy()[0])
    assert nf == fails.size
    assert np.array_equal(lst.cpu().numpy()[:nf], fails)  # ascending frame order
    # OSD output is a codeword
    H = std.dense()
    assert np.all((got[osd_frames].astype(np.int64) @ H.T) % 2 == 0)


def test_rejected_hybrid_call_writes_nothing(torch_cuda):
    # every argument check of the hybrid decoder (the OSD stage's included) precedes the
    # first launch: a call with OSD order 3 or an optimized matrix as std_code fails
    # with BCH_EINVAL and leaves the outputs as they were
    torch = torch_cuda
    n, k = 63, 45
    c, std = code(n, k), code(n, k, B.PCM_STANDARD)
    F = 100
    _, llr = frames(n, k, F, 3.0, 660, ld=64)
    autos = autos_dev(O.draw_autos(n, 3, 1, 0, F))
    hard = torch.full((F, 1), 7, dtype=torch.int64, device="cuda")
    fl = torch.full((F,), 9, dtype=torch.uint8, device="cuda")
    for other, order in ((std, 3), (c, 2)):
        with pytest.raises(B.BchError) as e:
            B.hybrid_decode(c, other, B.params(12, 0.78, osd_order=order), to_dev(llr), autos,
                            hard, None, fl)
        assert e.value.status == B.EINVAL
    torch.cuda.synchronize()
    assert bool((hard == 7).all()) and bool((fl == 9).all())


def test_count_errors(torch_cuda):
    torch = torch_cuda
    n = 127
    rng = np.random.default_rng(5)
    F = 5000
    a = rng.integers(0, 2, (F, n), dtype=np.uint8)
    b = a.copy()
    flip = rng.random((F, n)) < 0.002
    b[flip] ^= 1
    it = rng.integers(1, 13, F).astype(np.uint8)
    fl = rng.integers(0, 4, F).astype(np.uint8)
    ctr = torch.zeros(8, dtype=torch.int64, device="cuda")
    B.count_errors(n, to_dev(B.pack_bits(b)), to_dev(B.pack_bits(a)), to_dev(it), to_dev(fl), ctr)
    torch.cuda.synchronize()
    got = ctr.cpu().numpy()
    fe = flip.any(1)
    assert got[0] == F and got[1] == fe.sum() and got[2] == flip.sum()
    assert got[3] == (fe & ((fl & 1) == 1) & ((fl & 2) == 0)).sum()
    assert got[4] == ((fl & 2) > 0).sum() and got[5] == it.sum() and got[6] == (fl & 1).sum()


# ------------------------------------------------------------------ kernel variants
@pytest.mark.parametrize("nk", [(63, 36), (127, 64)])
@pytest.mark.parametrize("msg", [B.MSG_FP32, B.MSG_INT8])
def test_jit_and_generic_kernels_agree(torch_cuda, msg, nk, monkeypatch):
    # the run-time specialised kernel and the precompiled kernel compute the same
    # decoder: INT8 sums are exact integers (bit-exact), FP32 differs only in the
    # association of the c2v sums
    n, k = nk
    c = code(n, k)
    assert c.kernel_info(msg) == "jit"
    F = 2000
    cw, llr = frames(n, k, F, 2.0 if n == 63 else 3.0, 1234, ld=64 if n == 63 else 128)
    autos = O.draw_autos(n, 3, 77, 0, F)
    a = run_nms(torch_cuda, c, llr, autos, 12, 0.78, msg=msg)
    monkeypatch.setenv("BCHDEC_NMS_KERNEL", "generic")
    assert c.kernel_info(msg).startswith("generic")
    b = run_nms(torch_cuda, c, llr, autos, 12, 0.78, msg=msg)
    if msg == B.MSG_INT8:
        for key in ("hard", "iters", "flags", "y"):
            assert np.array_equal(a[key], b[key]), key
    else:
        ref = O.nms_enhanced(c.dense(), llr, autos, 12, 0.78, trace=True, threads=None)
        ok = ~ambiguous_frames(llr, ref, n)
        assert np.array_equal(a["hard"][ok], b["hard"][ok])
        assert np.array_equal(a["iters"][ok], b["iters"][ok])


@pytest.mark.parametrize("msg", [B.MSG_FP32, B.MSG_FP16])
def test_compare_free_edge_form_is_bit_identical(torch_cuda, msg, monkeypatch):
    """The specialised kernel's two forms of the min2 correction -- predicated add after
    a compare, and fma(dv, sat(1 - (t 2^100) 2^100), S + v1) -- round identically, so
    kernels built with either form give the same bits (hard, iterations, final y)."""
    n, k = 63, 45
    c = code(n, k)
    F = 3000
    cw, llr = frames(n, k, F, 2.5, 4321, ld=64)
    # include exact ties and tiny magnitudes (denormal differences t)
    llr[:50, :8] = np.float32(1.5)
    llr[50:100, :8] = np.float32(1e-40)
    autos = O.draw_autos(n, 3, 88, 0, F)
    monkeypatch.setenv("BCHDEC_JIT_FMA_PCT", "0")
    a = run_nms(torch_cuda, c, llr, autos, 12, 0.78, msg=msg)
    monkeypatch.setenv("BCHDEC_JIT_FMA_PCT", "100")
    b = run_nms(torch_cuda, c, llr, autos, 12, 0.78, msg=msg)
    monkeypatch.setenv("BCHDEC_JIT_FMA_PCT", "50")
    d = run_nms(torch_cuda, c, llr, autos, 12, 0.78, msg=msg)
    for key in ("hard", "iters", "flags", "y"):
        assert np.array_equal(a[key], b[key]), key
        assert np.array_equal(a[key], d[key]), key


@pytest.mark.parametrize("ebn0", [2.0, 4.0])
def test_bch15_hybrid_and_osd_vs_exhaustive_ml(torch_cuda, ebn0):
    """BCH(15,7) at 10^5 frames against exhaustive maximum-likelihood decoding over all
    128 codewords (oracle): the GPU hybrid equals the oracle hybrid frame by frame
    (unambiguous frames), ML is a lower bound on its errors and every excess error is
    an NMS frame that converged to a wrong codeword (undetected, so never sent to OSD);
    OSD(2) alone on every frame reaches the ML frame error rate."""
    torch = torch_cuda
    n, k, F = 15, 7, 100_000
    c, std = code(n, k), code(n, k, B.PCM_STANDARD)
    cw, llr = frames(n, k, F, ebn0, 1507 + int(ebn0), ld=16)
    autos = O.draw_autos(n, 3, 29, 0, F)
    p = B.params(12, 0.78, osd_order=2)
    hard = torch.zeros((F, 1), dtype=torch.int64, device="cuda")
    it = torch.zeros(F, dtype=torch.uint8, device="cuda")
    fl = torch.zeros(F, dtype=torch.uint8, device="cuda")
    d_llr = to_dev(llr)
    B.hybrid_decode(c, std, p, d_llr, autos_dev(autos), hard, it, fl)
    # OSD(2) alone on every frame
    hard_o = torch.zeros((F, 1), dtype=torch.int64, device="cuda")
    lst = torch.arange(F, dtype=torch.int32, device="cuda")
    cnt = torch.tensor([F], dtype=torch.int32, device="cuda")
    B.osd_decode(std, 2, d_llr, lst, cnt, hard_o)
    torch.cuda.synchronize()
    got = B.unpack_bits(hard.cpu().numpy(), n)
    got_o = B.unpack_bits(hard_o.cpu().numpy(), n)
    flags = fl.cpu().numpy()
    ml = O.ml(n, k, llr)
    ref = O.hybrid(c.dense(), std.dense(), llr, autos, 12, 0.78, threads=None)
    refe = O.nms_enhanced(c.dense(), llr, autos, 12, 0.78, trace=True, threads=None)
    ok = ~ambiguous_frames(llr, refe, n)
    assert np.array_equal(got[ok], ref["final"][ok])
    err_h = np.any(got != cw, axis=1)
    err_ml = np.any(ml != cw, axis=1)
    err_o = np.any(got_o != cw, axis=1)
    e_h, e_ml, e_o = int(err_h.sum()), int(err_ml.sum()), int(err_o.sum())
    assert e_ml > 30
    sd = np.sqrt(e_h + e_ml)
    assert e_h >= e_ml - 3 * sd
    undetected = err_h & ((flags & B.FLAG_OSD) == 0)
    excess = err_h & ~err_ml  # the hybrid errs where ML does not
    assert int((excess & ~undetected).sum()) <= 0.01 * e_ml + 3, (e_h, e_ml)
    assert abs(e_o - e_ml) <= 0.01 * e_ml + 3 * np.sqrt(e_o + e_ml), (e_o, e_ml)


@pytest.mark.parametrize("nk", [(63, 36), (127, 64)])
def test_maximum_iterations_no_overflow(torch_cuda, nk):
    """The API's largest iteration count without early stop: y grows about tenfold per
    iteration (past the FP32 range for BCH(127,64) after 32 iterations), and the decoder
    renormalises exactly by powers of two, so decisions and final LLRs still follow the
    FP64 oracle."""
    n, k = nk
    c = code(n, k)
    F = 200
    cw, llr = frames(n, k, F, 2.0, 5, ld=(n + 3) & ~3)
    autos = O.draw_autos(n, 3, 1, 0, F)
    g = run_nms(torch_cuda, c, llr, autos, 32, 0.78, early_stop=False)
    ref = O.nms_enhanced(c.dense(), llr, autos, 32, 0.78, early_stop=False, trace=True, threads=None)
    ok = ~ambiguous_frames(llr, ref, n)
    assert ok.mean() > 0.8
    y = g["y"][:, :n].astype(np.float64)
    assert not np.any(np.isnan(y))
    assert np.array_equal(g["hard"][ok], ref["hard"][ok])
    assert np.all(g["iters"] == 32)
    # the FP32 output holds +-inf only where the final LLR is at the FP32 range's edge
    inf = np.isinf(y)
    assert np.all(np.abs(ref["y"][inf]) > 1e38)
    assert np.all(np.sign(y[inf]) == np.sign(ref["y"][inf]))
    # trajectory: against the drift of the direct FP32 evaluation (which keeps y in
    # range the same way) of the same frames over the same 32 iterations
    env = frame_envelope(ref)[:, None]
    f32 = O.nms_enhanced_f32(c.dense(), llr, autos, 32, 0.78, early_stop=False, threads=None)
    check_trajectory(y, ref["y"], f32["y"], env, ok, "enhanced", 32)
