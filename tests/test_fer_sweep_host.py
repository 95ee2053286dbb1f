"""Host logic of the precision sweep: the SNR-loss interpolation on FER curves."""
import math

import pytest

from paper_2412_20828_gb300.fer_sweep import fer_loss_db, interp_ebn0_at_fer


def test_interp_on_exact_exponential_curve():
    # FER = 10^(-e): log10 FER is linear in dB, so interpolation is exact
    pts = [1.0, 2.0, 3.0, 4.0]
    fer = [10 ** -e for e in pts]
    assert interp_ebn0_at_fer(pts, fer, 10 ** -2.5) == pytest.approx(2.5)
    assert interp_ebn0_at_fer(pts, fer, 10 ** -1) == pytest.approx(1.0)
    assert interp_ebn0_at_fer(pts, fer, 10 ** -4) == pytest.approx(4.0)
    assert interp_ebn0_at_fer(pts, fer, 1.0) is None  # above the curve
    assert interp_ebn0_at_fer(pts, fer, 1e-6) is None  # below the curve


def test_loss_of_shifted_curve():
    # a curve shifted right by 0.2 dB loses 0.2 dB wherever it lies inside the reference
    pts = [1.0, 1.5, 2.0, 2.5, 3.0]
    ref = [10 ** -e for e in pts]
    var = [10 ** -(e - 0.2) for e in pts]
    loss = fer_loss_db(pts, ref, var, [1000] * 5)
    assert loss[0] is None  # FER above the reference's range
    for x in loss[1:]:
        assert x == pytest.approx(0.2)
    # too few errors: no claim
    assert fer_loss_db(pts, ref, var, [10] * 5) == [None] * 5


def test_zero_error_points_are_skipped():
    pts = [1.0, 2.0, 3.0]
    ref = [0.1, 0.01, 0.0]
    assert interp_ebn0_at_fer(pts, ref, 0.0316227766) == pytest.approx(1.5)
    assert interp_ebn0_at_fer(pts, ref, 0.001) is None
    assert math.isclose(fer_loss_db(pts, ref, ref, [100, 100, 0])[1], 0.0, abs_tol=1e-12)
