"""C-ABI checks that need no GPU: the library builds, loads and exports every symbol
declared in include/bchdec.h, and its host-side logic (code algebra, H_o
construction, automorphism draws) is bit-exact against the independent oracle."""
import os
import re

import numpy as np
import pytest

import oracle as O
from paper_2412_20828_gb300 import bchdec as B
from paper_2412_20828_gb300 import build as libbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def lib():
    libbuild.build()
    return B.load()


def test_exports_every_declared_symbol(lib):
    hdr = open(os.path.join(ROOT, "include", "bchdec.h")).read()
    declared = set(re.findall(r"\b(bch_[a-z0-9_]+)\(", hdr))
    assert declared == set(B.EXPORTS)
    for name in declared:
        assert getattr(lib, name) is not None


def test_checked_build_is_separate_and_exports_every_symbol(lib):
    """The ordinary library reports no checks and refuses to read a check word (before
    any CUDA call); the checked one (-DBCH_CHECKED, loaded in a child process) exports
    the same symbols and reports its checks."""
    import ctypes as C
    import subprocess
    import sys
    import numpy as np
    assert lib.bch_is_checked() == 0
    w = np.zeros(4, np.uint32)
    assert lib.bch_check_read(w.ctypes.data, 1, None) == B.EINVAL
    assert b"BCH_CHECKED" in lib.bch_last_error()
    from paper_2412_20828_gb300 import build
    path = build.build(checked=True)
    assert path == B.LIB_PATH_CHECKED
    code = ("import ctypes, sys\n"
            f"lib = ctypes.CDLL({path!r})\n"
            f"names = {list(B.EXPORTS)!r}\n"
            "assert all(getattr(lib, n) is not None for n in names)\n"
            "print(lib.bch_is_checked())\n")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == "1"


def test_status_strings(lib):
    assert lib.bch_status_str(0) == b"ok"
    assert lib.bch_status_str(4).startswith(b"rank")
    assert b"sm_103a" in lib.bch_version()


@pytest.mark.parametrize("nk", [(15, 7), (63, 36), (63, 45), (127, 64), (127, 78), (127, 99)])
def test_pcm_bit_exact_with_oracle(nk):
    n, k = nk
    assert np.array_equal(B.build_pcm_host(n, k, kind=B.PCM_STANDARD), O.std_h(n, k))
    assert np.array_equal(B.build_pcm_host(n, k), O.build_ho(n, k))


@pytest.mark.parametrize("n,k,m_rows", [(63, 36, 27), (63, 36, 47), (63, 36, 122), (63, 36, 269), (63, 36, 316),
                                         (63, 45, 33), (63, 45, 78), (127, 64, 72), (127, 78, 57), (127, 99, 33)])
def test_pcm_paper_sizes_bit_exact(n, k, m_rows):
    # the row counts of Table I and of the redundancy ladder of Sec. III-A, including
    # the padded matrices (more rows than the search's distinct classes)
    a = B.build_pcm_host(n, k, m_rows=m_rows)
    assert a.shape == (m_rows, n)
    assert np.array_equal(a, O.build_ho(n, k, m_rows=m_rows))


@pytest.mark.parametrize("seed,m_rows,q,sa", [(1, 0, 4, 20000), (99, 40, 2, 5000), (7, 60, 1, 300)])
def test_pcm_options_bit_exact(seed, m_rows, q, sa):
    a = B.build_pcm_host(63, 45, m_rows=m_rows, seed=seed, q_rounds=q, sa_steps=sa)
    b = O.build_ho(63, 45, m_rows=m_rows, seed=seed, q_rounds=q, sa_steps=sa)
    assert np.array_equal(a, b)


def test_pcm_rejects_bad_arguments():
    with pytest.raises(B.BchError) as e:
        B.build_pcm_host(64, 45)
    assert e.value.status == B.EINVAL
    with pytest.raises(B.BchError):
        B.build_pcm_host(63, 44)  # not a BCH dimension
    with pytest.raises(B.BchError):
        B.build_pcm_host(63, 45, m_rows=10)


@pytest.mark.parametrize("n,P", [(15, 3), (63, 3), (127, 3), (127, 9), (63, 1)])
def test_automorphism_draw_bit_exact(n, P):
    a = B.draw_automorphisms_host(n, P, 1234, 5000, 3000)
    b = O.draw_autos(n, P, 1234, 5000, 3000)
    assert np.array_equal(a, b)


def test_bit_packing_roundtrip():
    rng = np.random.default_rng(0)
    bits = rng.integers(0, 2, (50, 127), dtype=np.uint8)
    assert np.array_equal(B.unpack_bits(B.pack_bits(bits), 127), bits)


@pytest.mark.parametrize("msg", [0, 1, 2])
def test_specialised_kernel_compiles_without_gpu(msg):
    """The run-time specialised enhanced-NMS kernel of BCH(63,45) compiles for sm_103a
    (NVRTC, no GPU) in every message format."""
    report = B.nms_jit_check(63, 45, msg)
    assert "registers" in report


def test_serving_kernel_compiles_without_gpu(monkeypatch):
    """The serving kernels specialised to a server's codes compile for sm_103a (NVRTC,
    no GPU) without spilling: the block-bound kernel (the default) and the per-warp one
    with one separate copy function per code."""
    report = B.serve_jit_check([(63, 45), (63, 36)])
    assert "bch_serve_blocks" in report
    lines = report.splitlines()
    props = lines[lines.index(next(l for l in lines if "Function properties for bch_serve_blocks" in l)) + 1]
    assert "0 bytes spill stores" in props
    monkeypatch.setenv("BCHDEC_SERVE_KERNEL", "warps")
    report = B.serve_jit_check([(63, 45), (63, 36)])
    assert "bch_serve_jit" in report
    assert "srv_copy_0" in report and "srv_copy_1" in report
    for line in report.splitlines():
        if "srv_copy" in line:
            props = report.splitlines()[report.splitlines().index(line) + 1]
            assert "0 bytes spill stores" in props
    with pytest.raises(B.BchError):
        B.serve_jit_check([(63, 45)] * 9)  # at most 8 codes
