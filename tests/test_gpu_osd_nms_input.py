"""The hybrid decoder with the OSD reading the NMS output (bch_nms_params.osd_input = 1):
Sec. II-B allows an improved reliability measure for the OSD; this one ranks and
scores positions by the failed frame's final y, scaled per frame by the power of two
that puts max |y| in [2^15, 2^16).

Each stage is checked against the oracle:
 * the NMS output y follows the FP64 oracle within the trajectory tolerance, with
   identical decisions on unambiguous frames (as for the plain hybrid decoder);
 * the OSD stage is integer work on its input, so on every frame it decodes its word
   equals the oracle's OSD of that frame's own y (the GPU's FP32 values), scaled as
   stated: bit-exact;
 * end to end, the frame errors agree with the oracle's hybrid_nms_reliability (FP64
   y) within three standard deviations (frame by frame the two can differ: the FP32
   and FP64 y differ by the trajectory drift, which can reorder near-equal
   reliabilities)."""
import numpy as np
import pytest

import oracle as O
from helpers import (ambiguous_frames, autos_dev, check_trajectory, frame_envelope, frames,
                     to_dev)
from paper_2412_20828_gb300 import bchdec as B

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("nk,ebn0", [((63, 36), 2.0), ((127, 99), 3.0), ((127, 64), 2.5)])
def test_hybrid_with_osd_on_nms_output(nk, ebn0):
    import torch
    from paper_2412_20828_gb300 import build
    build.build()
    n, k = nk
    c, std = B.Code(n, k), B.Code(n, k, kind=B.PCM_STANDARD)
    F = 800
    ld = (n + 3) & ~3
    cw, llr = frames(n, k, F, ebn0, 7300 + n + k, ld=ld)
    autos = O.draw_autos(n, 3, 17, 0, F)
    p = B.params(12, 0.78, osd_order=2, osd_input=B.OSD_NMS_OUTPUT)
    W64 = (n + 63) // 64
    hard = torch.zeros((F, W64), dtype=torch.int64, device="cuda")
    it = torch.zeros(F, dtype=torch.uint8, device="cuda")
    fl = torch.zeros(F, dtype=torch.uint8, device="cuda")
    yo = torch.zeros((F, ld), dtype=torch.float32, device="cuda")
    B.hybrid_decode(c, std, p, to_dev(llr), autos_dev(autos), hard, it, fl, llr_out=yo)
    torch.cuda.synchronize()
    got = B.unpack_bits(hard.cpu().numpy(), n)
    flags = fl.cpu().numpy()
    y = yo.cpu().numpy()[:, :n]
    # NMS stage
    ref = O.nms_enhanced(c.dense(), llr, autos, 12, 0.78, trace=True, threads=None)
    ok = ~ambiguous_frames(llr, ref, n)
    assert np.array_equal(it.cpu().numpy()[ok], ref["iters"][ok])
    assert np.array_equal((flags & B.FLAG_CONVERGED)[ok], ref["converged"][ok])
    f32 = O.nms_enhanced_f32(c.dense(), llr, autos, 12, 0.78, threads=None)
    check_trajectory(y, ref["y"], f32["y"], frame_envelope(ref)[:, None], ok, "enhanced", 12)
    # OSD stage on the GPU's own y: bit-exact
    osd = np.nonzero(flags & B.FLAG_OSD)[0]
    assert np.array_equal(osd, np.nonzero((flags & B.FLAG_CONVERGED) == 0)[0])
    assert osd.size > 20
    _, ex = np.frexp(np.max(np.abs(y[osd].astype(np.float64)), axis=1))
    ys = np.ldexp(y[osd].astype(np.float64), (16 - ex)[:, None]).astype(np.float32)
    assert np.array_equal(ys.astype(np.float64), np.ldexp(y[osd].astype(np.float64), (16 - ex)[:, None]))
    words, _ = O.osd(std.dense(), ys, 2, threads=None)
    assert np.array_equal(got[osd], words)
    # the NMS frames keep their NMS word
    nms_frames = np.setdiff1d(np.arange(F), osd)
    assert np.array_equal(got[nms_frames][ok[nms_frames]], ref["hard"][nms_frames][ok[nms_frames]])
    # end to end against the oracle's FP64 variant
    hyb = O.hybrid_nms_reliability(c.dense(), std.dense(), llr, autos, 12, 0.78, threads=None)
    e_g = int(np.any(got != cw, axis=1).sum())
    e_r = int(np.any(hyb["final"] != cw, axis=1).sum())
    assert abs(e_g - e_r) <= 3 * np.sqrt(e_g + e_r + 1), (e_g, e_r)
    print(f"OSD frames {osd.size}, identical to the FP64 variant: "
          f"{np.all(got[osd] == hyb['final'][osd], axis=1).mean():.3f}")


def test_osd_on_nms_output_needs_the_output_buffer():
    import torch
    n, k = 63, 45
    c, std = B.Code(n, k), B.Code(n, k, kind=B.PCM_STANDARD)
    llr = torch.zeros((8, 64), dtype=torch.float32, device="cuda")
    hard = torch.full((8, 1), 5, dtype=torch.int64, device="cuda")
    fl = torch.zeros(8, dtype=torch.uint8, device="cuda")
    aut = torch.zeros((8, 3), dtype=torch.int16, device="cuda")
    with pytest.raises(B.BchError) as e:
        B.hybrid_decode(c, std, B.params(12, 0.78, osd_input=B.OSD_NMS_OUTPUT), llr, aut, hard, None, fl)
    assert e.value.status == B.EINVAL
    torch.cuda.synchronize()
    assert bool((hard == 5).all())
