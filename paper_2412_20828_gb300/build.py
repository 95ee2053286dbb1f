"""Builds the decoder library in-tree: libbchdec.so for sm_103a.

CUDA sources are compiled by nvcc with ``-gencode arch=compute_103a,code=sm_103a``
and the host algebra by g++ (portable flags only: the same sources build on x86-64
and on Arm), in parallel, then linked by nvcc into
``paper_2412_20828_gb300/_build/libbchdec.so``.  ``build(checked=True)`` compiles the
same sources with ``-DBCH_CHECKED`` into ``_build/checked/libbchdec.so``: kernels that
validate every index taken from caller-supplied device data (bch_check_read).
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libbchdec.so")
OUT_CHECKED = os.path.join(OUT, "checked")
LIB_CHECKED = os.path.join(OUT_CHECKED, "libbchdec.so")
INCLUDE = os.path.join(ROOT, "include")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

CU_SOURCES = ["k_nms.cu", "k_nms_fp32.cu", "k_nms_fp16.cu", "k_nms_int8.cu", "k_osd.cu", "k_misc.cu",
              "k_train.cu", "k_search.cu", "capi.cu", "runtime.cu", "noalloc.cu", "serve.cu"]
CPP_SOURCES = ["bch_host.cpp", "jit.cpp"]


def _deps_mtime() -> float:
    paths = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    paths.append(os.path.join(INCLUDE, "bchdec.h"))
    paths.append(os.path.abspath(__file__))
    return max(os.path.getmtime(p) for p in paths)


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    out_dir, lib = (OUT_CHECKED, LIB_CHECKED) if checked else (OUT, LIB)
    defs = ["-DBCH_CHECKED"] if checked else []
    os.makedirs(out_dir, exist_ok=True)
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= _deps_mtime():
        return lib
    inc = ["-I", CSRC, "-I", INCLUDE, *defs]
    procs = []
    objs = []
    # the device headers the run-time compiler needs, embedded as text
    gen = os.path.join(out_dir, "gen_device_text.cpp")
    with open(gen, "w") as f:
        f.write("namespace bchlib {\n")
        for sym, name in (("kDevTypesText", "bch_devtypes.h"), ("kNmsDeviceText", "nms_device.cuh"),
                          ("kAutosDeviceText", "autos_device.cuh"), ("kOsdDeviceText", "osd_device.cuh"),
                          ("kServeDeviceText", "serve_device.cuh")):
            with open(os.path.join(CSRC, name)) as g:
                text = g.read()
            assert ")__BCHTEXT__" not in text
            f.write(f'extern const char {sym}[] = R"__BCHTEXT__({text})__BCHTEXT__";\n')
        f.write("}  // namespace bchlib\n")
    gobj = gen + ".o"
    procs.append(("gen_device_text.cpp", subprocess.Popen(
        ["g++", "-O1", "-std=c++17", "-fPIC", "-c", gen, "-o", gobj],
        stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    objs.append(gobj)
    for src in CU_SOURCES:
        obj = os.path.join(out_dir, src + ".o")
        cmd = [NVCC, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
               "-Xcompiler", "-ffp-contract=off", "--expt-relaxed-constexpr", *inc,
               "-c", os.path.join(CSRC, src), "-o", obj]
        procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
        objs.append(obj)
    for src in CPP_SOURCES:
        obj = os.path.join(out_dir, src + ".o")
        cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-ffp-contract=off",
               "-I", "/usr/local/cuda/include", *inc, "-c", os.path.join(CSRC, src), "-o", obj]
        procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
        objs.append(obj)
    failed = []
    for src, p in procs:
        out, _ = p.communicate()
        text = out.decode(errors="replace")
        if p.returncode != 0:
            failed.append((src, text))
        elif verbose and text.strip():
            print(f"[{src}]\n{text}", file=sys.stderr)
    if failed:
        msg = "\n".join(f"--- {s}\n{t}" for s, t in failed)
        raise RuntimeError(f"building libbchdec failed:\n{msg}")
    tmp = lib + f".{os.getpid()}.tmp"
    cmd = [NVCC, *ARCH, "-shared", "-cudart", "shared", "-Xlinker", "-rpath,/usr/local/cuda/lib64",
           "-o", tmp, *objs]
    subprocess.run(cmd, check=True)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, checked="--checked" in sys.argv))
