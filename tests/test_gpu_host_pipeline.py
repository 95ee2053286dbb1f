"""The host pipeline (bch_decoder_run_host: frames in host memory, chunked copies on two
streams, automorphisms drawn on the device from frame0 + index) against the oracle's
hybrid decoder (Sec. IV) and against the device entry point on the same frames.

The run spans several chunks and ends on a partial one, with a nonzero frame0, so the
per-chunk frame offsets of the automorphism draw, the reuse of the two chunk buffers and
the short last chunk are all exercised, in both modes: page-locked host buffers decoded
in place and pageable ones staged through copies."""
import numpy as np
import pytest

import oracle as O
from helpers import ambiguous_frames, autos_dev, frames, to_dev
from paper_2412_20828_gb300 import bchdec as B

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("nk,ebn0,with_osd,memory", [((63, 36), 2.5, True, "pinned"),
                                                      ((63, 36), 2.5, True, "pageable"),
                                                      ((127, 99), 3.5, True, "pinned"),
                                                      ((63, 45), 3.0, False, "pageable")])
def test_host_pipeline_matches_oracle_and_device_call(nk, ebn0, with_osd, memory):
    """Page-locked buffers are decoded in place (the kernels read and write host memory),
    pageable ones through staged copies; both give the oracle's and the device call's
    results."""
    import torch
    from paper_2412_20828_gb300 import build
    build.build()
    n, k = nk
    code = B.Code(n, k)
    std = B.Code(n, k, kind=B.PCM_STANDARD) if with_osd else None
    ld = (n + 3) & ~3
    F, chunk, frame0, seed = 3500, 1000, 123457, 99  # chunks 1000, 1000, 1000, 500
    cw, llr = frames(n, k, F, ebn0, 8100 + n + k, ld=ld)
    p = B.params(12, 0.78, osd_order=2)
    dec = B.HostDecoder(code, std, p, ld, chunk_frames=chunk)
    W64 = (n + 63) // 64
    if memory == "pinned":
        t_llr = torch.from_numpy(llr).pin_memory()
        t_h = torch.zeros((F, W64), dtype=torch.int64).pin_memory()
        t_i = torch.zeros(F, dtype=torch.uint8).pin_memory()
        t_f = torch.zeros(F, dtype=torch.uint8).pin_memory()
        args = (t_llr, seed, frame0, t_h, t_i, t_f)
    else:
        hard = np.zeros((F, W64), np.uint64)
        it = np.zeros(F, np.uint8)
        fl = np.zeros(F, np.uint8)
        args = (llr, seed, frame0, hard, it, fl)
    try:
        dec.set_timing(True)
        dec.run(*args)
        tm = dec.timing()
    finally:
        dec.close()
    assert tm["calls"] == 1 and tm["chunks"] == 4
    assert tm["in_place_chunks"] == (4 if memory == "pinned" else 0)
    if memory == "pinned":
        hard, it, fl = t_h.numpy().view(np.uint64), t_i.numpy(), t_f.numpy()
    got = B.unpack_bits(hard.view(np.int64), n)
    # the oracle on the automorphisms of frames frame0 .. frame0 + F - 1
    autos = O.draw_autos(n, 3, seed, frame0, F)
    trace = O.nms_enhanced(code.dense(), llr, autos, 12, 0.78, trace=True, threads=None)
    ok = ~ambiguous_frames(llr, trace, n)
    assert ok.mean() > 0.9
    if with_osd:
        ref = O.hybrid(code.dense(), std.dense(), llr, autos, 12, 0.78, threads=None)["final"]
    else:
        ref = trace["hard"]
    assert np.array_equal(got[ok], ref[ok])
    assert np.array_equal(it[ok], trace["iters"][ok])
    assert np.array_equal((fl & B.FLAG_CONVERGED)[ok], trace["converged"][ok])
    # the device entry point on the same frames and draws gives the same bits everywhere
    d_h = torch.zeros((F, W64), dtype=torch.int64, device="cuda")
    d_i = torch.zeros(F, dtype=torch.uint8, device="cuda")
    d_f = torch.zeros(F, dtype=torch.uint8, device="cuda")
    if with_osd:
        B.hybrid_decode(code, std, p, to_dev(llr), autos_dev(autos), d_h, d_i, d_f)
    else:
        B.nms_decode(code, p, to_dev(llr), autos_dev(autos), d_h, d_i, d_f)
    torch.cuda.synchronize()
    assert np.array_equal(d_h.cpu().numpy(), hard.view(np.int64))
    assert np.array_equal(d_i.cpu().numpy(), it)
    assert np.array_equal(d_f.cpu().numpy(), fl)
