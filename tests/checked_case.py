"""The checked library's index checks on the GPU (run by test_gpu_checked.py in a process
of its own with BCHDEC_CHECKED=1, so that the checked build is the one loaded).

Every invalid value below reaches only the checked build's kernels, which test it before
any use: an automorphism with s >= n or j >= m is replaced by the identity, an OSD list
entry >= n_frames is skipped; each is recorded in the device's check word.  Checks:
  * valid inputs leave the word clear and decode as the oracle does (Algorithm 1);
  * invalid automorphisms (generic and specialised kernels, n = 63 and the n = 127 split
    mapping; the no-allocation entry point; the backward pass) set the flag, the count
    and the smallest bad frame, and the decode equals the decode with those pairs set to
    the identity, bit for bit;
  * invalid OSD list entries set their flag and smallest list position, and the valid
    entries' frames are decoded as the oracle's OSD decodes them.
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
sys.path.insert(0, HERE)

import numpy as np  # noqa: E402
import torch  # noqa: E402

import oracle as O  # noqa: E402
from helpers import ambiguous_frames, autos_dev, frames, to_dev  # noqa: E402
from paper_2412_20828_gb300 import bchdec as B  # noqa: E402
from paper_2412_20828_gb300 import build  # noqa: E402

NONE = 0xFFFFFFFF
CLEAR = [0, 0, NONE, NONE]


def corrupt(autos, n):
    """Invalid pairs at four frames (s = n; j = m; s = 255; 0xffff) and the same array with
    those pairs replaced by the identity (0)."""
    m = int(np.log2(n + 1))
    F = autos.shape[0]
    bad = autos.copy()
    where = [(5, 0, n), (17, 2, (m << 8) | 1), (F // 2, 1, 0x00FF), (F - 1, 1, 0xFFFF)]
    for f, p, v in where:
        bad[f, p] = v
    fixed = bad.copy()
    for f, p, _ in where:
        fixed[f, p] = 0
    return bad, fixed, len(where), min(f for f, _, _ in where)


def nms(code, llr, autos, F, n):
    hard = torch.zeros((F, (n + 63) // 64), dtype=torch.int64, device="cuda")
    it = torch.zeros(F, dtype=torch.uint8, device="cuda")
    fl = torch.zeros(F, dtype=torch.uint8, device="cuda")
    B.nms_decode(code, B.params(12, 0.78), to_dev(llr), autos_dev(autos), hard, it, fl)
    torch.cuda.synchronize()
    return hard.cpu().numpy(), it.cpu().numpy(), fl.cpu().numpy()


def check_nms(kernel, n, k, F, ebn0):
    if kernel == "generic":
        os.environ["BCHDEC_NMS_KERNEL"] = "generic"
    else:
        os.environ.pop("BCHDEC_NMS_KERNEL", None)
    code = B.Code(n, k)
    info = code.kernel_info()
    assert info.startswith("generic") == (kernel == "generic"), info
    cw, llr = frames(n, k, F, ebn0, 9100 + n + k, ld=(n + 3) & ~3)
    autos = O.draw_autos(n, 3, 11, 0, F)
    # valid automorphisms: the word stays clear; words and iterations equal the oracle's
    h0, i0, f0 = nms(code, llr, autos, F, n)
    assert list(B.check_read()) == CLEAR
    ref = O.nms_enhanced(code.dense(), llr, autos, 12, 0.78, trace=True, threads=None)
    ok = ~ambiguous_frames(llr, ref, n)
    assert ok.mean() > 0.9
    assert np.array_equal(B.unpack_bits(h0, n)[ok], ref["hard"][ok])
    assert np.array_equal(i0[ok], ref["iters"][ok])
    # invalid ones: recorded, and decoded as the identity
    bad, fixed, nbad, first = corrupt(autos, n)
    h1, i1, f1 = nms(code, llr, bad, F, n)
    w = B.check_read()
    assert w[0] == B.CHECK_AUTOMORPHISM and w[1] >= nbad and w[2] == first and w[3] == NONE, (kernel, n, w)
    h2, i2, f2 = nms(code, llr, fixed, F, n)
    assert list(B.check_read()) == CLEAR
    assert np.array_equal(h1, h2) and np.array_equal(i1, i2) and np.array_equal(f1, f2)
    # frames with no bad pair are unchanged
    same = np.ones(F, bool)
    same[np.any(bad != autos, axis=1)] = False
    assert np.array_equal(h1[same], h0[same]) and np.array_equal(i1[same], i0[same])
    print(f"  nms {kernel} ({n},{k}) [{info}]: word {list(w)}")
    os.environ.pop("BCHDEC_NMS_KERNEL", None)


def check_noalloc():
    n, k, F = 63, 36, 1500
    code, std = B.Code(n, k), B.Code(n, k, kind=B.PCM_STANDARD)
    cw, llr = frames(n, k, F, 2.0, 9200, ld=64)
    bad, fixed, nbad, first = corrupt(O.draw_autos(n, 3, 12, 0, F), n)
    p = B.params(12, 0.78, osd_order=2)
    outs = []
    for a in (bad, fixed):
        h = torch.zeros((F, 1), dtype=torch.int64, device="cuda")
        it = torch.zeros(F, dtype=torch.uint8, device="cuda")
        fl = torch.zeros(F, dtype=torch.uint8, device="cuda")
        B.hybrid_decode_noalloc(code, std, p, to_dev(llr), autos_dev(a), h, it, fl)
        torch.cuda.synchronize()
        outs.append((h.cpu().numpy(), it.cpu().numpy(), fl.cpu().numpy(), B.check_read()))
    w = outs[0][3]
    assert w[0] == B.CHECK_AUTOMORPHISM and w[1] >= nbad and w[2] == first, w
    assert list(outs[1][3]) == CLEAR
    for x, y in zip(outs[0][:3], outs[1][:3]):
        assert np.array_equal(x, y)
    print(f"  noalloc hybrid (63,36): word {list(w)}")


def check_backward():
    n, k, F, I = 63, 45, 800, 6
    code = B.Code(n, k)
    cw, llr = frames(n, k, F, 2.5, 9300, ld=64)
    bad, fixed, nbad, first = corrupt(O.draw_autos(n, 3, 13, 0, F), n)
    p = B.params(I, 0.78, early_stop=False)
    res = []
    for a in (bad, fixed):
        ckpt = torch.zeros((I + 1, F, 64), dtype=torch.float32, device="cuda")
        B.nms_forward_train(code, p, to_dev(llr), autos_dev(a), ckpt)
        g_out = torch.ones((F, 64), dtype=torch.float32, device="cuda")
        g_llr = torch.zeros((F, 64), dtype=torch.float32, device="cuda")
        g_al = torch.zeros(I, dtype=torch.float32, device="cuda")
        B.nms_backward(code, p, autos_dev(a), ckpt, g_out, g_llr, g_al)
        torch.cuda.synchronize()
        res.append((ckpt.cpu().numpy(), g_llr.cpu().numpy(), g_al.cpu().numpy(), B.check_read()))
    w = res[0][3]
    assert w[0] == B.CHECK_AUTOMORPHISM and w[1] >= 2 * nbad and w[2] == first, w  # forward + backward
    assert list(res[1][3]) == CLEAR
    for x, y in zip(res[0][:3], res[1][:3]):
        assert np.array_equal(x, y)
    print(f"  forward + backward (63,45): word {list(w)}")


def check_osd():
    n, k, F = 63, 45, 300
    std = B.Code(n, k, kind=B.PCM_STANDARD)
    cw, llr = frames(n, k, F, 2.0, 9400, ld=64)
    lst = np.array([0, 5, F, 7, 0x7FFFFFFF, 299], np.uint32)
    valid = lst[lst < F]
    hard = torch.full((F, 1), -1, dtype=torch.int64, device="cuda")
    B.osd_decode(std, 2, to_dev(llr), to_dev(lst.view(np.int32)), to_dev(np.array([len(lst)], np.int32)), hard)
    w = B.check_read()
    assert w[0] == B.CHECK_OSD_FRAME and w[1] == 2 and w[2] == NONE and w[3] == 2, w
    h = hard.cpu().numpy()
    ref, _ = O.osd(std.dense(), llr[valid], order=2)
    assert np.array_equal(B.unpack_bits(h[valid], n), ref)
    others = np.setdiff1d(np.arange(F), valid)
    assert np.all(h[others] == -1)
    print(f"  osd list: word {list(w)}")


def main():
    build.build(checked=True)
    assert B.is_checked()
    torch.cuda.set_device(0)
    B.check_read()  # start from a clear word
    for kernel in ("jit", "generic"):
        check_nms(kernel, 63, 45, 2000, 3.0)
        check_nms(kernel, 127, 64, 1000, 3.0)
    check_noalloc()
    check_backward()
    check_osd()
    print("checked build ok")


if __name__ == "__main__":
    main()
