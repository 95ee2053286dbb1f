"""Pins for the oracle's reduced-precision decoder (``nms_enhanced_q``) against
hand-derived examples (tests/golden/quantised_hand_examples.txt): ties to even in the
8-bit check-to-variable rounding rne(alpha min_q) on odd minima, saturation at +-31 of
the input and of the merged values, binary16 saturation at 65504 and ties to even of
the binary16 store, two iterations of the power-of-two renormalisation (8-bit) and
one of the binary16 one, and the 8-bit form with fractional check-to-variable bits
(qfrac = 8: exact fractional c2v, ties to even in the merge of the exact quotient,
the renormalisation on the exact numerators, and with it the power-of-two scaling of
the input that avoids clipping strong inputs).  Each example states the value a plausible mistake (ties away
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


def _run(key, iters, alpha, fmt, rescale=False, qfrac=0):
    L = _gold(key).astype(np.float32)[None, :]
    return O.nms_enhanced_q(H4, L, IDENT, iters, alpha, fmt, rescale=rescale, early_stop=False,
                            qfrac=qfrac)


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


def test_int8_fractional_c2v_merge_rounds_exact_quotient_ties_to_even():
    r = _run("q1_L", 1, 0.5, 2, qfrac=8)
    assert np.array_equal(r["y"][0], _gold("q5_y1"))
    assert r["hard"][0].tolist() == [0, 0, 0, 0]


def test_int8_fractional_c2v_keeps_fraction_of_alpha_min():
    r = _run("q1_L", 1, float(np.float32(0.78)), 2, qfrac=8)
    assert np.array_equal(r["y"][0], _gold("q6_y1"))
    assert r["hard"][0].tolist() == [1, 0, 0, 0]
    # the same input without fractional bits rounds each c2v first: v1 merges to 2
    r0 = _run("q1_L", 1, float(np.float32(0.78)), 2)
    assert np.array_equal(r0["y"][0], [-0.25, 0.5, 0.5, 0.75])


def test_int8_fractional_c2v_rescale_on_exact_numerators():
    r = _run("q4_L", 1, 0.75, 2, rescale=True, qfrac=8)
    assert np.array_equal(r["y"][0], _gold("q7_y1"))
    r = _run("q4_L", 1, 0.75, 2, qfrac=8)
    assert np.array_equal(r["y"][0], _gold("q7n_y1"))


def test_fractional_bits_rejected_outside_the_8_bit_form():
    import pytest
    L = _gold("q1_L").astype(np.float32)[None, :]
    with pytest.raises(Exception):
        O.nms_enhanced_q(H4, L, IDENT, 1, 0.5, 1, qfrac=8)
    with pytest.raises(Exception):
        O.nms_enhanced_q(H4, L, IDENT, 1, 0.5, 2, qfrac=9)


def test_int8_fractional_rescale_scales_the_input_instead_of_clipping():
    r = _run("q2_L", 1, 1.0, 2, rescale=True, qfrac=8)
    assert np.array_equal(r["y"][0], _gold("q8_y1"))
    assert r["hard"][0].tolist() == [1, 1, 0, 1]
