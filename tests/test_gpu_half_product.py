"""The FP16 form's roundings in the decoder's device header, against numpy's float16
conversion of exact FP64 values (the reference that pins the oracle's binary16
rounding):
  * half_product(alpha, m) -- the check-to-variable magnitude: the FP32 product rounded
    to odd, then once to binary16 -- must be the binary16 value nearest to the exact
    product alpha m (24 + 11 significant bits: exact in FP64), ties to even, saturating
    at 65504.  Cases: every finite positive binary16 m with several alphas (0.78 among
    them), alphas putting the product on, one FP32 ulp below and one above a binary16
    midpoint, and 50 000 exact midpoints (m a power of two);
  * half_of_quotient(num, P) -- the merge: the correctly rounded FP32 quotient rounded to
    odd with its exact remainder, then once to binary16 -- must be the binary16 value
    nearest to num / P (ties to even, saturating, zero stored as +0).  The FP64 quotient
    of an FP32 num by P <= 9 is a binary16 midpoint only if the exact quotient is (the
    two differ by less than half an FP64 ulp, while num - mid P is a nonzero multiple of
    num's FP32 ulp otherwise), so its float16 conversion is exact.  Cases: log-uniform
    magnitudes of both signs, exact midpoints num = mid P and their FP32 neighbours,
    saturation, zeros."""
import os
import shutil
import subprocess

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    nvcc = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
    if not os.path.exists(nvcc):
        nvcc = shutil.which("nvcc")
    assert nvcc, "nvcc is needed to build the test driver"
    d = tmp_path_factory.mktemp("half")
    exe = str(d / "half_product_case")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O2",
                    "-I", os.path.join(ROOT, "paper_2412_20828_gb300", "csrc"),
                    "-I", os.path.join(ROOT, "include"), "-o", exe,
                    os.path.join(HERE, "half_product_case.cu")], check=True)

    def run(a, b, mode):
        fin, fout = d / f"{mode}_in.bin", d / f"{mode}_out.bin"
        with open(fin, "wb") as f:
            np.array([a.size], np.int32).tofile(f)
            a.astype(np.float32).tofile(f)
            b.astype(np.float32).tofile(f)
        subprocess.run([exe, str(fin), str(fout), mode], check=True, timeout=300)
        return np.fromfile(fout, np.float32)
    return run


def _binary16_positive():
    return np.arange(1, 0x7C00, dtype=np.uint16).view(np.float16).astype(np.float32)


def _product_cases():
    rng = np.random.default_rng(5)
    hv = _binary16_positive()
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


def test_half_product_is_the_correctly_rounded_binary16_product(driver):
    A, M, ties = _product_cases()
    out = driver(A, M, "product")
    exact = A.astype(np.float64) * M.astype(np.float64)
    ref = np.minimum(exact, 65504.0).astype(np.float16).astype(np.float32)
    bad = np.flatnonzero(out != ref)
    assert bad.size == 0, np.stack([A[bad[:5]], M[bad[:5]], out[bad[:5]], ref[bad[:5]]], 1)
    assert ties > 40_000 and out.size > 500_000


def test_half_of_quotient_is_the_correctly_rounded_binary16_quotient(driver):
    rng = np.random.default_rng(6)
    hv = _binary16_positive()
    N = 400_000
    num = (rng.choice([-1.0, 1.0], N) * 2.0 ** rng.uniform(-20, 19, N)).astype(np.float32)
    P = rng.integers(1, 10, N).astype(np.float32)
    # exact midpoints: num = mid P (mid has 12 significant bits, P at most 4: exact)
    k = rng.integers(0, hv.size - 1, 100_000)
    Pm = rng.integers(1, 10, 100_000).astype(np.float64)
    mid = (hv[k].astype(np.float64) + hv[k + 1].astype(np.float64)) / 2
    nm = (mid * Pm * rng.choice([-1.0, 1.0], 100_000)).astype(np.float32)
    nums = [num, nm, (nm.view(np.int32) - 1).view(np.float32), (nm.view(np.int32) + 1).view(np.float32),
            np.array([0.0, -0.0, 65504.0 * 9, -70000.0, 65519.0 * 3, 65521.0 * 3], np.float32)]
    Ps = [P, Pm.astype(np.float32), Pm.astype(np.float32), Pm.astype(np.float32),
          np.array([1, 3, 9, 1, 3, 3], np.float32)]
    A = np.concatenate(nums)
    B = np.concatenate(Ps)
    out = driver(A, B, "quotient")
    q = A.astype(np.float64) / B.astype(np.float64)
    ref = np.clip(q, -65504.0, 65504.0).astype(np.float16).astype(np.float32)
    bad = np.flatnonzero(out != ref)
    assert bad.size == 0, np.stack([A[bad[:5]], B[bad[:5]], out[bad[:5]], ref[bad[:5]]], 1)
    assert not np.any(np.signbit(out[out == 0.0]))  # zero is stored as +0
    assert int(np.sum(A[N:N + 100_000].astype(np.float64) / B[N:N + 100_000].astype(np.float64)
                      == np.abs(mid) * np.sign(A[N:N + 100_000]))) > 90_000  # exact ties
