"""The FP16 form's check-to-variable rounding (half_product in the decoder's device
header: the FP32 product rounded to odd, then once to binary16) equals the binary16
value nearest to the exact product alpha * m, ties to even, saturating at 65504.  The
reference is numpy's float16 conversion of the exact FP64 product (24 + 11 significant
bits), the same reference that pins the oracle's binary16 rounding.  Cases: every
finite positive binary16 m with several alphas (0.78 among them), and alphas placing
the product exactly on, one FP32 ulp below and one above a binary16 midpoint."""
import os
import shutil
import subprocess

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _cases():
    rng = np.random.default_rng(5)
    hv = np.arange(1, 0x7C00, dtype=np.uint16).view(np.float16).astype(np.float32)
    A, M = [], []
    for al in [0.78, 0.75, 0.5, 1.0, 0.6049, 1.3, 3.9] + list(rng.uniform(0.1, 2.0, 8)):
        A.append(np.full(hv.size, al, np.float32))
        M.append(hv)
    k = rng.integers(0, hv.size - 1, 100_000)
    m = hv[rng.integers(0, hv.size, 100_000)]
    mid = (hv[k].astype(np.float64) + hv[k + 1].astype(np.float64)) / 2
    a0 = (mid / m.astype(np.float64)).astype(np.float32)
    for d in (-1, 0, 1):
        A.append((a0.view(np.int32) + d).view(np.float32))
        M.append(m)
    # products that are exactly a binary16 midpoint (the ties-to-even cases); with m a
    # power of two, alpha = midpoint / m is exact
    ties = int(np.sum(a0.astype(np.float64) * m.astype(np.float64) == mid))
    k2 = rng.integers(0, hv.size - 1, 50_000)
    m2 = (2.0 ** rng.integers(-14, 15, 50_000)).astype(np.float32)
    mid2 = (hv[k2].astype(np.float64) + hv[k2 + 1].astype(np.float64)) / 2
    a2 = (mid2 / m2.astype(np.float64)).astype(np.float32)
    ties += int(np.sum(a2.astype(np.float64) * m2.astype(np.float64) == mid2))
    A.append(a2)
    M.append(m2)
    A = np.concatenate(A).astype(np.float32)
    M = np.concatenate(M).astype(np.float32)
    ok = np.isfinite(A) & (A > 0)
    return A[ok], M[ok], ties


def test_half_product_is_the_correctly_rounded_binary16_product(tmp_path):
    nvcc = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
    if not os.path.exists(nvcc) and not shutil.which("nvcc"):
        pytest.fail("nvcc is needed to build the test driver")
    exe = str(tmp_path / "half_product_case")
    subprocess.run([nvcc if os.path.exists(nvcc) else "nvcc", "-gencode", "arch=compute_103a,code=sm_103a",
                    "-O2", "-I", os.path.join(ROOT, "paper_2412_20828_gb300", "csrc"),
                    "-I", os.path.join(ROOT, "include"), "-o", exe,
                    os.path.join(HERE, "half_product_case.cu")], check=True)
    A, M, ties = _cases()
    fin, fout = tmp_path / "in.bin", tmp_path / "out.bin"
    with open(fin, "wb") as f:
        np.array([A.size], np.int32).tofile(f)
        A.tofile(f)
        M.tofile(f)
    subprocess.run([exe, str(fin), str(fout)], check=True, timeout=300)
    out = np.fromfile(fout, np.float32)
    exact = A.astype(np.float64) * M.astype(np.float64)
    ref = np.minimum(exact, 65504.0).astype(np.float16).astype(np.float32)
    bad = np.flatnonzero(out != ref)
    assert bad.size == 0, np.stack([A[bad[:5]], M[bad[:5]], out[bad[:5]], ref[bad[:5]]], 1)
    assert ties > 40_000 and out.size > 500_000
