"""Writes tests/golden/fp32_drift.txt: the largest drift of the oracle's direct FP32
restatement of the decoders from the FP64 oracle, over the parity tests' workloads.

drift(f) = max_i |y32_i - y64_i| / max(|y64_i|, env(f)), env(f) the largest operand
magnitude met while decoding frame f, over the frames the ambiguity rule keeps.  The
GPU parity tests hold the kernels to DRIFT_FACTOR times these values (tests/helpers.py).
Calls only the oracle.  Run from the repository root:
    python tests/golden/make_fp32_drift.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))
sys.path.insert(0, os.path.dirname(HERE))

import oracle as O  # noqa: E402
from helpers import ambiguous_frames, drift, frame_envelope, frames  # noqa: E402

CODES = [(15, 7), (63, 36), (63, 45), (127, 64), (127, 78), (127, 99)]


def enhanced(n, k, F, ebn0, seed, iters, alpha, early_stop):
    Ho = O.build_ho(n, k)
    _, llr = frames(n, k, F, ebn0, seed, ld=(n + 3) & ~3)
    autos = O.draw_autos(n, 3, 11, 0, F)
    ref = O.nms_enhanced(Ho, llr, autos, iters, alpha, early_stop=early_stop, trace=True,
                         threads=None)
    r32 = O.nms_enhanced_f32(Ho, llr, autos, iters, alpha, early_stop=early_stop, threads=None)
    ok = ~ambiguous_frames(llr, ref, n)
    return float(drift(r32["y"], ref["y"], frame_envelope(ref)[:, None])[ok].max())


def plain(ebn0, F=1200):
    n, k = 63, 36
    H = O.std_h(n, k)
    _, llr = frames(n, k, F, ebn0, 500, ld=64)
    ref = O.nms_plain(H, llr, 8, 0.78, threads=None)
    r32 = O.nms_plain_f32(H, llr, 8, 0.78, threads=None)
    ok = ~(np.any(np.abs(llr[:, :n]) < 1e-3, axis=1) | (ref["margin_rel"] < 2e-5))
    return float(drift(r32["y"], ref["y"], ref["env"][:, None])[ok].max())


def main():
    rows = []
    # enhanced NMS, 12 iterations with early stop, alpha ramp 0.7 .. 0.9: every code at
    # 1.5 and 3.5 dB, 1500 frames each
    d12 = max(enhanced(n, k, 1500, e, 200 + n + k, 12, np.linspace(0.7, 0.9, 12), True)
              for n, k in CODES for e in (1.5, 3.5))
    rows.append(("enhanced", 12, d12, "6 codes x {1.5, 3.5} dB x 1500 frames, alpha 0.7..0.9"))
    # enhanced NMS, 32 iterations without early stop (the API's maximum), alpha 0.78
    d32 = max(enhanced(n, k, 1000, e, 900 + n + k, 32, 0.78, False)
              for n, k in [(63, 36), (127, 64)] for e in (1.5, 2.0, 3.5))
    rows.append(("enhanced", 32, d32, "(63,36), (127,64) x {1.5, 2, 3.5} dB x 1000 frames, "
                                      "alpha 0.78, no early stop"))
    # plain NMS on the standard H of BCH(63,36), 8 iterations, alpha 0.78
    d8 = max(plain(e) for e in (2.0, 3.0))
    rows.append(("plain", 8, d8, "(63,36) standard H x {2, 3} dB x 1200 frames, alpha 0.78"))
    with open(os.path.join(HERE, "fp32_drift.txt"), "w") as f:
        f.write("# Largest drift of a direct FP32 evaluation from the FP64 oracle (see\n"
                "# make_fp32_drift.py, which wrote this file): decoder iterations drift workload\n")
        for dec, it, d, what in rows:
            f.write(f"{dec} {it} {d:.4e} {what}\n")


if __name__ == "__main__":
    main()
