"""Seeded synthetic inputs shared by the decoder's tests, smoke check and benchmark.

This module draws random numbers only: message bits and standard-normal noise from
numpy's PCG64 generator.  It holds none of the decoder's arithmetic (no encoding, no
channel model, no decoding); the tests pass its draws to the CPU oracle's encoder and
channel, and the resulting FP32 LLR bytes go unchanged to both the oracle and the
CUDA library.  The workload recipe (codes, Eb/N0 grid, frame counts) follows the
BPSK/AWGN setting of Sec. II and the simulation section of arXiv 2412.20828.
"""
from __future__ import annotations

import numpy as np

# Codes evaluated in the paper (Sec. IV) plus the tiny code checked against
# exhaustive maximum likelihood.
CODES = {
    (15, 7): "BCH(15,7) t=2",
    (63, 36): "BCH(63,36) t=5",
    (63, 45): "BCH(63,45) t=3",
    (127, 64): "BCH(127,64) t=10",
    (127, 78): "BCH(127,78) t=7",
    (127, 99): "BCH(127,99) t=4",
}

# Eb/N0 grid of the enhanced-NMS sweep: 1.0 .. 6.0 dB in 0.5 dB steps.
EBN0_GRID_DB = tuple(1.0 + 0.5 * i for i in range(11))


def rng(seed: int, stream: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64([int(seed) & (2**63 - 1), int(stream)]))


def messages(F: int, k: int, seed: int, stream: int = 0) -> np.ndarray:
    """Uniform i.i.d. message bits, shape [F, k], uint8."""
    return rng(seed, 2 * stream).integers(0, 2, size=(F, k), dtype=np.uint8)


def normals(F: int, n: int, seed: int, stream: int = 0) -> np.ndarray:
    """Standard normal draws, shape [F, n], float64."""
    return rng(seed, 2 * stream + 1).standard_normal((F, n))


def uniform(F: int, lo: float, hi: float, seed: int, stream: int = 0) -> np.ndarray:
    """Per-frame uniform draws in [lo, hi), e.g. a per-frame Eb/N0."""
    return rng(seed, 1000 + stream).uniform(lo, hi, size=F)
