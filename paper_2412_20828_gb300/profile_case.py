"""One small decode case for profiling a kernel with ncu: frames generated on the device,
then a warm-up decode and a second decode of the same frames (skip the first launch of
the kernel of interest with ncu's -s to capture the second).

    python -m paper_2412_20828_gb300.profile_case --code 127,64 --frames 400000
    ncu --set full --clock-control none -k regex:bch_nms_jit -s 1 -c 1 -o prof \\
        python -m paper_2412_20828_gb300.profile_case --code 127,64 --frames 400000
"""
from __future__ import annotations

import argparse


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--code", default="127,64", help="n,k")
    ap.add_argument("--frames", type=int, default=400_000)
    ap.add_argument("--ebn0", type=float, default=3.0)
    ap.add_argument("--msg", default="fp32", choices=["fp32", "fp16", "int8"])
    ap.add_argument("--hybrid", action="store_true", help="also run compaction and OSD")
    ap.add_argument("--m-rows", type=int, default=0, help="rows of H_o (0: 2(n-k))")
    a = ap.parse_args(argv)
    import torch
    from . import bchdec as B
    B.load()
    n, k = (int(x) for x in a.code.split(","))
    msg = {"fp32": B.MSG_FP32, "fp16": B.MSG_FP16, "int8": B.MSG_INT8}[a.msg]
    code = B.Code(n, k, m_rows=a.m_rows)
    std = B.Code(n, k, kind=B.PCM_STANDARD) if a.hybrid else None
    F, ld, W64 = a.frames, (n + 3) & ~3, (n + 63) // 64
    llr = torch.empty((F, ld), dtype=torch.float32, device="cuda")
    B.gen_frames(code, a.ebn0, a.ebn0, 7, 0, llr)
    aut = torch.empty((F, 3), dtype=torch.int16, device="cuda")
    B.draw_automorphisms(n, 3, 8, 0, aut)
    p = B.params(12, 0.78, msg=msg, osd_order=2)
    hard = torch.zeros((F, W64), dtype=torch.int64, device="cuda")
    it = torch.zeros(F, dtype=torch.uint8, device="cuda")
    fl = torch.zeros(F, dtype=torch.uint8, device="cuda")
    ws = B.workspace(code, p, F)
    for _ in range(2):
        if std is not None:
            B.hybrid_decode(code, std, p, llr, aut, hard, it, fl, ws=ws)
        else:
            B.nms_decode(code, p, llr, aut, hard, it, fl, ws=ws)
    torch.cuda.synchronize()
    print(f"BCH({n},{k}) {F} frames at {a.ebn0} dB, {a.msg}: kernel {code.kernel_info(msg)}, "
          f"mean iterations {float(it.float().mean()):.3f}, edges {code.edges}")


if __name__ == "__main__":
    main()
