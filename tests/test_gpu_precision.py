"""GPU parity of the reduced-precision message formats against the quantised oracle.

INT8 (with and without power-of-two renormalisation): every quantiser input is an
exact integer combination or a correctly-rounded division whose .5 ties are exact, so
hard decisions, iteration counts and final values are bit-exact on every frame.
FP16: the binary16 check-to-variable values are formed exactly and rounded once on
both sides, so the only difference is that the kernel accumulates them in FP32 where
the oracle's sums are exact.  Its FP32 sum of K terms errs by at most (K + 2) 2^-24
of the operand magnitude (K <= 3 x column weight + 4, below 5e-6 for every code here),
so a stored binary16 value can differ only where the exact merged value lies within
that distance of a binary16 rounding boundary or of zero.  The oracle reports, per
frame, the smallest such distance over the whole decode (``margin``); frames whose
margin is below FP16_AMBIG = 2e-5 (4x the error bound) or whose channel LLR has some
|L| < 1e-3 are ambiguous, and every other frame must be bit-exact: hard decisions,
iteration counts, flags and final values.
"""
import numpy as np
import pytest

import oracle as O
from helpers import autos_dev, frames, to_dev
from paper_2412_20828_gb300 import bchdec as B

pytestmark = pytest.mark.gpu

ALPHA = float(np.float32(0.78))
FP16_AMBIG = 2e-5


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    from paper_2412_20828_gb300 import build
    build.build()
    B.load()
    return torch


def decode(torch, c, llr, autos, iters, msg, rescale, early_stop=True, qfrac=0):
    F, ld = llr.shape
    p = B.params(iters, ALPHA, n_autos=autos.shape[1], early_stop=early_stop, msg=msg,
                 rescale=rescale, qfrac=qfrac)
    hard = torch.zeros((F, (c.n + 63) // 64), dtype=torch.int64, device="cuda")
    it = torch.zeros(F, dtype=torch.uint8, device="cuda")
    fl = torch.zeros(F, dtype=torch.uint8, device="cuda")
    yo = torch.zeros((F, ld), dtype=torch.float32, device="cuda")
    B.nms_decode(c, p, to_dev(llr), autos_dev(autos), hard, it, fl, yo)
    torch.cuda.synchronize()
    return dict(hard=B.unpack_bits(hard.cpu().numpy(), c.n), iters=it.cpu().numpy(),
                flags=fl.cpu().numpy(), y=yo.cpu().numpy()[:, :c.n])


@pytest.mark.parametrize("nk", [(63, 36), (63, 45), (127, 64), (127, 99)])
@pytest.mark.parametrize("rescale", [False, True])
def test_int8_bit_exact(torch_cuda, nk, rescale):
    n, k = nk
    c = B.Code(n, k)
    F = 800
    cw, llr = frames(n, k, F, 2.5, 900 + n + k, ld=(n + 3) & ~3)
    autos = O.draw_autos(n, 3, 31, 0, F)
    g = decode(torch_cuda, c, llr, autos, 12, B.MSG_INT8, rescale)
    ref = O.nms_enhanced_q(c.dense(), llr, autos, 12, ALPHA, 2, rescale=rescale, threads=None)
    assert np.array_equal(g["iters"], ref["iters"])
    assert np.array_equal(g["hard"], ref["hard"])
    assert np.array_equal(g["flags"] & 1, ref["converged"])
    assert np.array_equal(g["y"].astype(np.float64), ref["y"])


@pytest.mark.parametrize("nk", [(63, 36), (63, 45), (127, 64), (127, 99)])
@pytest.mark.parametrize("rescale", [False, True])
@pytest.mark.parametrize("kernel", ["jit", "generic"])
def test_int8_fractional_bit_exact(torch_cuda, nk, rescale, kernel, monkeypatch):
    """The 8-bit form with 8 fractional c2v bits: integer sums and a merge that rounds
    the exact quotient, so every output is bit-exact with the oracle's qfrac branch
    (pinned by hand examples), on the specialised kernels (n = 127: split mapping) and
    the precompiled one."""
    if kernel == "generic":
        monkeypatch.setenv("BCHDEC_NMS_KERNEL", "generic")
    n, k = nk
    c = B.Code(n, k)
    F = 800
    cw, llr = frames(n, k, F, 3.0, 1900 + n + k, ld=(n + 3) & ~3)
    autos = O.draw_autos(n, 3, 41, 0, F)
    g = decode(torch_cuda, c, llr, autos, 12, B.MSG_INT8, rescale, qfrac=8)
    ref = O.nms_enhanced_q(c.dense(), llr, autos, 12, ALPHA, 2, rescale=rescale, threads=None,
                           qfrac=8)
    assert np.array_equal(g["iters"], ref["iters"])
    assert np.array_equal(g["hard"], ref["hard"])
    assert np.array_equal(g["flags"] & 1, ref["converged"])
    assert np.array_equal(g["y"].astype(np.float64), ref["y"])


def test_fractional_bits_rejected_outside_the_8_bit_form(torch_cuda):
    c = B.Code(63, 45)
    for kw in (dict(msg=B.MSG_FP32, qfrac=8), dict(msg=B.MSG_INT8, qfrac=9),
               dict(msg=B.MSG_INT8, qfrac=8, n_autos=0)):
        p = B.params(4, ALPHA, **{"n_autos": 3, **kw})
        with pytest.raises(B.BchError) as e:
            B.nms_decode(
                c, p, to_dev(np.zeros((4, 64), np.float32)), autos_dev(np.zeros((4, 3), np.uint16)),
                torch_cuda.zeros((4, 1), dtype=torch_cuda.int64, device="cuda"))
        assert e.value.status == B.EINVAL


@pytest.mark.parametrize("nk,ebn0", [((63, 45), 2.5), ((127, 64), 3.5), ((127, 99), 3.5)])
@pytest.mark.parametrize("rescale", [False, True])
def test_fp16_close_to_oracle(torch_cuda, nk, ebn0, rescale):
    n, k = nk
    c = B.Code(n, k)
    F = 800
    cw, llr = frames(n, k, F, ebn0, 950 + n + k, ld=(n + 3) & ~3)
    autos = O.draw_autos(n, 3, 37, 0, F)
    # first iteration: within one binary16 ulp of the oracle
    g1 = decode(torch_cuda, c, llr, autos, 1, B.MSG_FP16, rescale, early_stop=False)
    r1 = O.nms_enhanced_q(c.dense(), llr, autos, 1, ALPHA, 1, rescale=rescale, early_stop=False)
    ulp = np.array([O.q16(abs(v) * (1 + 2 ** -10)) - O.q16(abs(v)) if v != 0 else 2 ** -24
                    for v in r1["y"].ravel()]).reshape(r1["y"].shape)
    assert np.all(np.abs(g1["y"] - r1["y"]) <= np.maximum(ulp, 2 ** -24) * 1.0001)
    g = decode(torch_cuda, c, llr, autos, 12, B.MSG_FP16, rescale)
    ref = O.nms_enhanced_q(c.dense(), llr, autos, 12, ALPHA, 1, rescale=rescale, threads=None)
    amb = (ref["margin"] < FP16_AMBIG) | np.any(np.abs(llr[:, :n]) < 1e-3, axis=1)
    # long decodes of BCH(127,64) meet many non-exact merges (saturated or renormalised
    # frames next to tiny values), about a quarter of its frames
    assert amb.mean() < 0.3
    # over all frames (the ambiguous ones included) the frame error counts agree
    e_g = int(np.any(g["hard"] != cw, axis=1).sum())
    e_r = int(np.any(ref["hard"] != cw, axis=1).sum())
    assert abs(e_g - e_r) <= 3 * np.sqrt(e_g + e_r + 1)
    ok = ~amb
    assert np.array_equal(g["hard"][ok], ref["hard"][ok])
    assert np.array_equal(g["iters"][ok], ref["iters"][ok])
    assert np.array_equal(g["flags"][ok] & 1, ref["converged"][ok])
    assert np.array_equal(g["y"][ok].astype(np.float64), ref["y"][ok])


def test_fer_sweep_small(torch_cuda):
    """The precision sweep: FP32 NMS FER equals a direct decode of the same frames, and
    the FP16 / INT8 forms stay close to FP32 at 2 x 20 000 frames."""
    torch = torch_cuda
    from paper_2412_20828_gb300 import fer_sweep as FS
    res = FS.run(codes=[(63, 45)], points=[3.0, 4.0], frames=20000, chunk=8192, hybrid=True)
    e = res["codes"]["(63,45)"]["variants"]
    # direct FP32 decode of point 0 (frame indices 0.., seed as the sweep draws them)
    c = B.Code(63, 45)
    llr = torch.empty((20000, 64), dtype=torch.float32, device="cuda")
    cw = torch.empty((20000, 1), dtype=torch.int64, device="cuda")
    aut = torch.empty((20000, 3), dtype=torch.int16, device="cuda")
    B.gen_frames(c, 3.0, 3.0, 0x5EED, 0, llr, cw)
    B.draw_automorphisms(63, 3, 0x5EED + 1, 0, aut)
    hard = torch.empty((20000, 1), dtype=torch.int64, device="cuda")
    B.nms_decode(c, B.params(12, 0.78), llr, aut, hard)
    torch.cuda.synchronize()
    fe = int((hard != cw).any(dim=1).sum())
    assert e["fp32"]["nms"]["frame_errors"][0] == fe
    for name in ("fp16", "int8", "int8_rescale"):
        for stage in ("nms", "hybrid"):
            a = np.array(e[name][stage]["frame_errors"], float)
            b = np.array(e["fp32"][stage]["frame_errors"], float)
            assert np.all(np.abs(a - b) <= 0.25 * b + 4 * np.sqrt(b + 1)), (name, stage, a, b)
    assert "loss_db_vs_fp32" in e["int8"]["nms"]
