"""The no-allocation entry point (collected last on purpose).

bch_hybrid_decode_noalloc serves callers that cannot allocate device memory while they
decode: its scratch is a fixed device array owned by the library.  Two calls in a row
must each reproduce bch_hybrid_decode's result (the array keeps the previous call's
contents, so a missing clear would show on the second call), within the tolerance the
other parity tests use: identical words, flags and iteration counts on every frame whose
decoding meets no sign-ambiguous value.
"""
import numpy as np
import pytest

import oracle as O
from helpers import ambiguous_frames, autos_dev, frames, to_dev
from paper_2412_20828_gb300 import bchdec as B

pytestmark = pytest.mark.gpu


def test_noalloc_matches_workspace_entry_point():
    import torch
    from paper_2412_20828_gb300 import build
    build.build()
    n, k = 63, 36
    code = B.Code(n, k)
    std = B.Code(n, k, kind=B.PCM_STANDARD)
    F = 3000
    cw, llr = frames(n, k, F, 2.0, 4242, ld=64)
    autos = O.draw_autos(n, 3, 5, 0, F)
    p = B.params(12, 0.78, osd_order=2)
    d_llr, d_aut = to_dev(llr), autos_dev(autos)

    def outputs():
        return (torch.zeros((F, 1), dtype=torch.int64, device="cuda"),
                torch.zeros(F, dtype=torch.uint8, device="cuda"),
                torch.zeros(F, dtype=torch.uint8, device="cuda"))

    h0, i0, f0 = outputs()
    B.hybrid_decode(code, std, p, d_llr, d_aut, h0, i0, f0)
    torch.cuda.synchronize()
    ref = O.nms_enhanced(code.dense(), llr, autos, 12, 0.78, trace=True, threads=None)
    ok = ~ambiguous_frames(llr, ref, n)
    assert ok.mean() > 0.9
    # the hybrid decoder of the oracle (Sec. IV): NMS word where its syndrome is zero,
    # else the order-2 OSD word
    hyb = O.hybrid(code.dense(), std.dense(), llr, autos, 12, 0.78, threads=None)
    for _ in range(2):  # two calls in a row on the shared scratch
        h1, i1, f1 = outputs()
        B.hybrid_decode_noalloc(code, std, p, d_llr, d_aut, h1, i1, f1)
        torch.cuda.synchronize()
        assert np.array_equal(h1.cpu().numpy()[ok], h0.cpu().numpy()[ok])
        assert np.array_equal(i1.cpu().numpy()[ok], i0.cpu().numpy()[ok])
        assert np.array_equal(f1.cpu().numpy()[ok], f0.cpu().numpy()[ok])
        words = B.unpack_bits(h1.cpu().numpy(), n)
        assert np.array_equal(words[ok], hyb["final"][ok])
        assert np.array_equal(i1.cpu().numpy()[ok], hyb["iters"][ok])
    # a rejected call (OSD order 3) writes nothing: every check precedes the first launch
    h2 = torch.full((F, 1), 7, dtype=torch.int64, device="cuda")
    with pytest.raises(B.BchError) as e:
        B.hybrid_decode_noalloc(code, std, B.params(12, 0.78, osd_order=3), d_llr, d_aut, h2,
                                None, torch.zeros(F, dtype=torch.uint8, device="cuda"))
    assert e.value.status == B.EINVAL
    torch.cuda.synchronize()
    assert bool((h2 == 7).all())
    # beyond the scratch limit: a clear error, nothing launched
    big = torch.zeros((262145, 64), dtype=torch.float32, device="cuda")
    with pytest.raises(B.BchError) as e:
        B.hybrid_decode_noalloc(code, std, p, big, torch.zeros((262145, 3), dtype=torch.int16,
                                                                device="cuda"),
                                torch.zeros((262145, 1), dtype=torch.int64, device="cuda"),
                                None, torch.zeros(262145, dtype=torch.uint8, device="cuda"))
    assert e.value.status == B.EINVAL and "262144" in str(e.value)
