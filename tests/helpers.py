"""Shared helpers of the GPU parity tests: seeded inputs (oracle encoder + channel on
draws from ``synth``), device marshalling and the tolerance rules.

Tolerance rules (FP32 kernel vs FP64 oracle, same FP32 input bytes):
 * one iteration from the same input: a sum of terms is compared relative to the sum
   of the terms' magnitudes (the "operand magnitude" returned by the oracle):
   |gpu - ref| <= 1e-5 max(|ref|, mag, 1);
 * after several iterations no FP32 evaluation of the decoder stays within 1e-5 of the
   FP64 result: each iteration's rounding is carried into the next, and the min-sum
   update can amplify a small value's error by up to about 1 + alpha x (column weight)
   while the frame grows by about tenfold.  The oracle's direct FP32 restatement of the
   same loops (``nms_enhanced_f32``, ``nms_plain_f32``) measures that drift,
   drift(f) = max_i |y32 - y64| / max(|y64|, env(f)) with env(f) the largest operand
   magnitude met while decoding frame f.  Its largest value over the parity workloads
   is recorded per decoder and iteration count in tests/golden/fp32_drift.txt (written
   by tests/golden/make_fp32_drift.py from the oracle alone; a CPU test re-measures
   it).  A kernel's drift over the unambiguous frames must stay within DRIFT_FACTOR
   times that value, and its median drift within DRIFT_FACTOR times the restatement's
   median on the same frames (the median is a stable statistic of a few hundred frames;
   the largest drift of one frame is not: it depends on how that frame's roundings
   happen to line up).  DRIFT_FACTOR = 4: per edge the kernel rounds up to three times
   where the direct evaluation rounds once (the row sum S + alpha m1, the difference
   alpha m2 - alpha m1 and the corrected sum at the row's minimum; the c2v product
   itself is rounded identically), and it merges the P copies with one fused
   multiply-add by fl(1/P) instead of a division, so its per-iteration rounding error
   is at most about three times the direct one plus 2^-24 of the merged sum, and both
   errors go through the same iterated map;
 * hard decisions and iteration counts must be identical on every frame whose
   decoding never met a sign-ambiguous value: |y| < 1e-3 on the channel LLR, or any
   |y^(t)| below 1e-4 of its operand magnitude in a later iteration (there the sign is
   decided by rounding order, and a flipped sign legitimately changes the rest).  The
   direct FP32 restatement meets this rule on every workload of the tests (a CPU test
   checks it), which is the evidence that 1e-4 covers FP32 rounding;
 * integer work (matrices, permutations, syndromes, OSD) is bit-exact.
"""
import numpy as np

import oracle as O
from paper_2412_20828_gb300 import synth

REL_TOL = 1e-5
DRIFT_FACTOR = 4.0
AMBIG_LLR = 1e-3
AMBIG_REL = 1e-4


def frames(n, k, F, ebn0, seed, ld=None):
    msg = synth.messages(F, k, seed)
    cw = O.encode(n, k, msg)
    llr = O.channel_llr(n, k, cw, synth.normals(F, n, seed), ebn0, ld=ld or n)
    return cw, llr


def to_dev(x, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(x))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def autos_dev(autos):
    return to_dev(autos.view(np.int16))


def ambiguous_frames(llr, ref, n):
    """Frames whose oracle trace meets a sign-ambiguous value (see module doc)."""
    amb = np.any(np.abs(llr[:, :n]) < AMBIG_LLR, axis=1)
    if "trace" in ref:
        tr = ref["trace"][:, 1:, :]
        mg = np.maximum(ref["mag"], 1.0)
        amb |= np.any(np.abs(tr) < AMBIG_REL * mg, axis=(1, 2))
    return amb


def frame_envelope(ref):
    """Largest operand magnitude met while decoding each frame (from the trace)."""
    return np.max(ref["mag"], axis=(1, 2))


def rel_close(gpu, ref, mag=None):
    scale = np.abs(ref)
    if mag is not None:
        scale = np.maximum(scale, mag)
    scale = np.maximum(scale, 1.0)
    return np.abs(gpu - ref) <= REL_TOL * scale


def drift(y, ref_y, env):
    """Per-frame largest deviation of y from the FP64 result, relative to
    max(|ref|, the frame's envelope).  Entries where both are infinite (an FP32 output
    at the edge of the range) count as equal."""
    y = np.asarray(y, np.float64)
    d = np.abs(y - ref_y)
    d[np.isinf(y) & (np.sign(y) == np.sign(ref_y))] = 0.0
    return np.max(d / np.maximum(np.abs(ref_y), env), axis=1)


def drift_table():
    """{(decoder, iterations): largest drift of the direct FP32 restatement}."""
    import os
    out = {}
    with open(os.path.join(os.path.dirname(__file__), "golden", "fp32_drift.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                dec, it, d = line.split()[:3]
                out[(dec, int(it))] = float(d)
    return out


def check_trajectory(y, ref_y, f32_y, env, ok, decoder, iters):
    """Asserts the multi-iteration tolerance of the module doc on the frames `ok` and
    returns (kernel max, bound, kernel median, median bound) for reporting."""
    d = drift(y, ref_y, env)[ok]
    d32 = drift(f32_y, ref_y, env)[ok]
    bound = max(REL_TOL, DRIFT_FACTOR * drift_table()[(decoder, iters)])
    med_bound = max(REL_TOL, DRIFT_FACTOR * float(np.median(d32)))
    print(f"drift kernel max {d.max():.3g} (bound {bound:.3g}), median {np.median(d):.3g} "
          f"(bound {med_bound:.3g}); FP32 restatement max {d32.max():.3g}")
    assert d.max() <= bound, f"worst drift {d.max():.3g} > {bound:.3g}"
    assert np.median(d) <= med_bound, f"median drift {np.median(d):.3g} > {med_bound:.3g}"
    return d.max(), bound, float(np.median(d)), med_bound
