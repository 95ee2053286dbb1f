"""Pins for the oracle's direct FP32 restatements of the decoders (``nms_plain_f32``,
``nms_enhanced_f32``), the evidence behind the trajectory tolerance of the GPU parity
tests.

* the hand-derived examples (tests/golden/nms_hand_examples.txt, exact binary
  fractions) come out exactly;
* one iteration from the same FP32 input stays within the textbook bound of a
  floating-point sum: each c2v product is rounded once (relative error <= u = 2^-24)
  and a sum of K terms accumulated left to right errs by at most (K - 1) u times the
  sum of the terms' magnitudes (Higham, Accuracy and Stability of Numerical
  Algorithms, 2nd ed., Sec. 4.2), so |y32 - y64| <= (K + 2) u mag with K the number of
  terms and mag the oracle's operand magnitude.  A dropped or doubled term, a wrong
  sign or a wrong permutation breaks this bound by orders of magnitude;
* over full decodes the restatement takes the FP64 decoder's decisions and iteration
  counts on every frame the ambiguity rule keeps, on every code and SNR of the GPU
  parity tests, and its drift grows with the iterations run.
"""
import numpy as np
import pytest

import oracle as O
from helpers import ambiguous_frames, drift, frame_envelope, frames

H4 = np.array([[1, 1, 1, 0], [0, 1, 1, 1]], np.uint8)
U = 2.0 ** -24


def _gold(key):
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "nms_hand_examples.txt")) as f:
        for line in f:
            if line.startswith(key + " "):
                return np.array([float(x) for x in line.split()[1:]])
    raise KeyError(key)


def test_fp32_restatements_reproduce_hand_examples():
    L = _gold("plain_L").astype(np.float32)[None, :]
    r1 = O.nms_plain_f32(H4, L, iters=5, alpha=0.5)
    assert r1["iters"][0] == 1 and r1["converged"][0] == 1
    assert np.array_equal(r1["y"][0], _gold("plain_x1"))
    r2 = O.nms_plain_f32(H4, L, iters=2, alpha=0.5, early_stop=False)
    assert np.array_equal(r2["y"][0], _gold("plain_x2"))
    assert r2["hard"][0].tolist() == [0, 1, 0, 0]
    y0 = _gold("enh_y0").astype(np.float32)[None, :]
    r = O.nms_enhanced_f32(H4, y0, np.array([[0, 1]], np.uint16), iters=1, alpha=0.5)
    assert np.array_equal(r["y"][0], _gold("enh_y1"))


@pytest.mark.parametrize("nk", [(15, 7), (63, 36), (127, 99)])
def test_enhanced_fp32_one_iteration_within_sum_error_bound(nk):
    n, k = nk
    Ho = O.build_ho(n, k)
    F, P = 300, 3
    _, llr = frames(n, k, F, 2.0, 40 + n, ld=n)
    autos = O.draw_autos(n, P, 3, 0, F)
    ref = O.nms_enhanced(Ho, llr, autos, 1, 0.78, early_stop=False, trace=True)
    r32 = O.nms_enhanced_f32(Ho, llr, autos, 1, 0.78, early_stop=False)
    K = int(Ho.sum(axis=0).max()) * P + P + 1  # column sums, copy sums, the merge
    err = np.abs(r32["y"] - ref["y"])
    # alpha itself is rounded to FP32 on the restatement's side: |0.78 - fl(0.78)| < u
    assert np.all(err <= (K + 3) * U * ref["mag"][:, 0, :])
    # the bound is not vacuous: the restatement does differ from FP64, by far less
    assert err.max() > 0 and (err / ref["mag"][:, 0, :]).max() < 1e-6


def test_plain_fp32_one_iteration_within_sum_error_bound():
    n, k = 63, 36
    H = O.std_h(n, k)
    _, llr = frames(n, k, 300, 2.0, 41, ld=64)
    ref = O.nms_plain(H, llr, 1, 0.78, early_stop=False)
    r32 = O.nms_plain_f32(H, llr, 1, 0.78, early_stop=False)
    K = int(H.sum(axis=0).max()) + 1
    err = np.abs(r32["y"] - ref["y"])
    assert np.all(err <= (K + 3) * U * ref["env"][:, None])
    assert err.max() > 0


@pytest.mark.parametrize("nk", [(63, 36), (63, 45), (127, 64), (127, 99)])
def test_enhanced_fp32_decisions_follow_fp64_on_unambiguous_frames(nk):
    n, k = nk
    Ho = O.build_ho(n, k)
    F = 300
    alpha = np.linspace(0.7, 0.9, 12)
    worst = []
    for ebn0 in (1.5, 3.5):
        _, llr = frames(n, k, F, ebn0, 200 + n + k, ld=(n + 3) & ~3)
        autos = O.draw_autos(n, 3, 11, 0, F)
        ref = O.nms_enhanced(Ho, llr, autos, 12, alpha, trace=True, threads=None)
        r32 = O.nms_enhanced_f32(Ho, llr, autos, 12, alpha, threads=None)
        ok = ~ambiguous_frames(llr, ref, n)
        assert ok.mean() > 0.85
        assert np.array_equal(r32["hard"][ok], ref["hard"][ok])
        assert np.array_equal(r32["iters"][ok], ref["iters"][ok])
        assert np.array_equal(r32["converged"][ok], ref["converged"][ok])
        worst.append(drift(r32["y"], ref["y"], frame_envelope(ref)[:, None])[ok].max())
    # a direct FP32 evaluation drifts well past 1e-5 over 12 iterations on these codes,
    # and stays far below a sign change
    assert max(worst) > 1e-6 and max(worst) < 1e-2


def test_plain_fp32_decisions_follow_fp64_on_unambiguous_frames():
    n, k = 63, 36
    H = O.std_h(n, k)
    _, llr = frames(n, k, 600, 2.0, 500, ld=64)
    ref = O.nms_plain(H, llr, 8, 0.78, threads=None)
    r32 = O.nms_plain_f32(H, llr, 8, 0.78, threads=None)
    ok = ~(np.any(np.abs(llr[:, :n]) < 1e-3, axis=1) | (ref["margin_rel"] < 2e-5))
    assert np.array_equal(r32["hard"][ok], ref["hard"][ok])
    assert np.array_equal(r32["iters"][ok], ref["iters"][ok])


def test_fp32_range_renormalisation_is_exact():
    # 32 iterations of BCH(127,64) without early stop take y past the FP32 range; the
    # restatement's power-of-two renormalisation keeps it finite and close to FP64
    n, k = 127, 64
    Ho = O.build_ho(n, k)
    _, llr = frames(n, k, 200, 2.0, 5, ld=128)
    autos = O.draw_autos(n, 3, 1, 0, 200)
    ref = O.nms_enhanced(Ho, llr, autos, 32, 0.78, early_stop=False, trace=True, threads=None)
    r32 = O.nms_enhanced_f32(Ho, llr, autos, 32, 0.78, early_stop=False, threads=None)
    assert np.abs(ref["y"]).max() > 3.4e38  # past FLT_MAX in FP64
    assert np.all(np.isfinite(r32["y"]))
    ok = ~ambiguous_frames(llr, ref, n)
    assert np.array_equal(r32["hard"][ok], ref["hard"][ok])
    assert drift(r32["y"], ref["y"], frame_envelope(ref)[:, None])[ok].max() < 1e-2


def test_drift_table_matches_a_fresh_measurement():
    # tests/golden/fp32_drift.txt (written by make_fp32_drift.py from the oracle) bounds
    # the restatement's drift on a fresh, smaller sample of the same workloads, and the
    # 12-iteration entry is reached within a factor 100 (the table is not vacuous; a
    # sample's largest drift sits in a heavy tail, so smaller samples reach less of it)
    from helpers import drift_table
    tab = drift_table()
    alpha = np.linspace(0.7, 0.9, 12)
    worst = 0.0
    for n, k in [(63, 36), (127, 99)]:
        Ho = O.build_ho(n, k)
        _, llr = frames(n, k, 300, 3.5, 200 + n + k, ld=(n + 3) & ~3)
        autos = O.draw_autos(n, 3, 11, 0, 300)
        ref = O.nms_enhanced(Ho, llr, autos, 12, alpha, trace=True, threads=None)
        r32 = O.nms_enhanced_f32(Ho, llr, autos, 12, alpha, threads=None)
        ok = ~ambiguous_frames(llr, ref, n)
        worst = max(worst, drift(r32["y"], ref["y"], frame_envelope(ref)[:, None])[ok].max())
    assert tab[("enhanced", 12)] / 100 <= worst <= tab[("enhanced", 12)]
    assert tab[("enhanced", 12)] < tab[("enhanced", 32)]
