"""Parity at the full benchmark size, in the benchmark's launch configuration: one
hybrid decode (specialised NMS kernel, P = 3, 12 iterations, OSD(2)) over 11 Eb/N0
points x 10^6 frames of BCH(63,36), automorphisms drawn on the device as the benchmark
does, then frames sampled across the whole batch -- the first and last two of every
point and seeded random ones -- against the oracle, frame by frame.  The frames come
from the seeded host draws and the oracle's encoder and channel."""
import numpy as np
import pytest

import oracle as O
from helpers import ambiguous_frames, frames
from paper_2412_20828_gb300 import bchdec as B

pytestmark = pytest.mark.gpu

POINTS = [1.0 + 0.5 * i for i in range(11)]


def test_full_size_hybrid_sampled_against_oracle():
    import torch
    from paper_2412_20828_gb300 import build
    build.build()
    n, k = 63, 36
    c, std = B.Code(n, k), B.Code(n, k, kind=B.PCM_STANDARD)
    assert c.kernel_info(B.MSG_FP32) == "jit"
    Bp = 1_000_000
    F = Bp * len(POINTS)
    llr = torch.empty((F, 64), dtype=torch.float32, device="cuda")
    aut = torch.empty((F, 3), dtype=torch.int16, device="cuda")
    rng = np.random.default_rng(77)
    picks, host_llr = [], []
    for pi, e in enumerate(POINTS):
        _, llr_p = frames(n, k, Bp, e, 9100 + pi, ld=64)
        llr[pi * Bp:(pi + 1) * Bp].copy_(torch.from_numpy(llr_p))
        B.draw_automorphisms(n, 3, 0x5EED, pi * 10_000_000, aut[pi * Bp:(pi + 1) * Bp])
        loc = np.unique(np.concatenate([[0, 1, Bp - 2, Bp - 1], rng.integers(0, Bp, 136)]))
        picks.append(pi * Bp + loc)
        host_llr.append(llr_p[loc])
        del llr_p
    idx = np.concatenate(picks)
    llr_o = np.ascontiguousarray(np.concatenate(host_llr))
    hard = torch.empty((F, 1), dtype=torch.int64, device="cuda")
    it = torch.empty(F, dtype=torch.uint8, device="cuda")
    fl = torch.empty(F, dtype=torch.uint8, device="cuda")
    B.hybrid_decode(c, std, B.params(12, 0.78, osd_order=2), llr, aut, hard, it, fl)
    torch.cuda.synchronize()
    aut_o = np.concatenate([O.draw_autos(n, 3, 0x5EED, (i // Bp) * 10_000_000 + i % Bp, 1) for i in idx])
    ref = O.hybrid(c.dense(), std.dense(), llr_o, aut_o, 12, 0.78, threads=None)
    refe = O.nms_enhanced(c.dense(), llr_o, aut_o, 12, 0.78, trace=True, threads=None)
    ok = ~ambiguous_frames(llr_o, refe, n)
    assert ok.mean() > 0.95 and idx.size > 1000
    sel = torch.from_numpy(idx).cuda()
    got = B.unpack_bits(hard[sel].cpu().numpy(), n)
    assert np.array_equal(got[ok], ref["final"][ok])
    assert np.array_equal(it[sel].cpu().numpy()[ok], ref["iters"][ok])
    osd = (fl[sel].cpu().numpy() & B.FLAG_OSD) != 0
    assert np.array_equal(osd[ok], ref["converged"][ok] == 0)
