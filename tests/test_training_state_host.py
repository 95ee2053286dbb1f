"""The training loop's resumable state (bch_adam_state) round-trips through a file
exactly: alpha as FP32, the Adam moments as doubles, the step count (host only)."""
import ctypes as C

import numpy as np

from paper_2412_20828_gb300 import bchdec as B


def test_adam_state_layout_matches_the_c_struct():
    # int iters, int batch, long long step, double m[32], double v[32]
    assert C.sizeof(B.AdamState) == 4 + 4 + 8 + 32 * 8 * 2
    assert B.AdamState.step.offset == 8 and B.AdamState.m.offset == 16


def test_training_state_round_trips_through_a_file(tmp_path):
    rng = np.random.default_rng(7)
    s = B.AdamState()
    s.iters, s.batch, s.step = 12, 65536, 137
    for t in range(32):
        s.m[t] = float(rng.standard_normal() * 1e-3)
        s.v[t] = float(rng.random() * 1e-6)
    alpha = rng.random(12).astype(np.float32)
    path = tmp_path / "train_state.npz"
    B.save_training(path, alpha, s)
    a2, s2 = B.load_training(path)
    assert np.array_equal(a2, alpha) and a2.dtype == np.float32
    assert (s2.iters, s2.batch, s2.step) == (12, 65536, 137)
    assert bytes(s2) == bytes(s)  # every double bit for bit
