"""Pins for the oracle's reduced-precision decoder (``nms_enhanced_q``) against
hand-derived examples (tests/golden/quantised_hand_examples.txt): ties to even in the
8-bit check-to-variable rounding rne(alpha min_q) on odd minima, saturation at +-31 of
the input and of the merged values, binary16 saturation at 65504 and ties to even of
the binary16 store, and two iterations of the power-of-two renormalisation (8-bit) and
one of the binary16 one.  Each example states the value a plausible mistake (ties away
from zero, a missing clamp, a wrong exponent count) would give instead."""
import os

import numpy as np

import oracle as O

H4 = np.array([[1, 1, 1, 0], [0, 1, 1, 1]], np.uint8)
IDENT = np.zeros((1, 1), np.uint16)


def _gold(key):
    with open(os.path.join(os.path.dirname(__file__), "golden", "quantised_hand_examples.txt")) as f:
        for line in f:
            if line.startswith(key + " "):
                return np.array([float(x) for x in line.split()[1:]])
    raise KeyError(key)


def _run(key, iters, alpha, fmt, rescale=False):
    L = _gold(key).astype(np.float32)[None, :]
    return O.nms_enhanced_q(H4, L, IDENT, iters, alpha, fmt, rescale=rescale, early_stop=False)


def test_int8_c2v_rounds_ties_to_even():
    r = _run("q1_L", 1, 0.5, 2)
    assert np.array_equal(r["y"][0], _gold("q1_y1"))
    assert r["hard"][0].tolist() == [0, 0, 0, 0]


def test_int8_saturates_input_and_merge_at_31():
    r = _run("q2_L", 1, 1.0, 2)
    assert np.array_equal(r["y"][0], _gold("q2_y1"))
    assert r["hard"][0].tolist() == [1, 1, 0, 1] and r["converged"][0] == 1


def test_fp16_saturates_at_65504_and_rounds_ties_to_even():
    r = _run("q3_L", 1, 1.0, 1)
    assert np.array_equal(r["y"][0], _gold("q3_y1"))
    r = _run("q3_L", 1, 1.0, 1, rescale=True)
    assert np.array_equal(r["y"][0], _gold("q3r_y1"))


def test_int8_rescale_two_iterations():
    r = _run("q4_L", 2, 1.0, 2)
    assert np.array_equal(r["y"][0], _gold("q4_y2")) and r["iters"][0] == 2
    r = _run("q4_L", 2, 1.0, 2, rescale=True)
    assert np.array_equal(r["y"][0], _gold("q4r_y2")) and r["iters"][0] == 2
    assert r["hard"][0].tolist() == [0, 0, 0, 0]
