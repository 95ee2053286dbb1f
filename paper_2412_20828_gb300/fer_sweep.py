"""FER / BER curves of the enhanced NMS decoder per message precision, and the SNR loss
of each reduced-precision form against FP32.

For every code and Eb/N0 point the same frames (device Philox draw) and automorphisms
are decoded with FP32, FP16 and 8-bit saturating messages (optionally with the
per-frame power-of-two rescale), NMS alone and as the hybrid NMS + OSD-2 decoder
(Sec. II-B, Sec. IV).  The loss in dB of a variant at a point is how much higher the
variant's Eb/N0 is than the Eb/N0 at which the FP32 curve (log10 FER linear in dB
between points) reaches the same FER.

    python -m paper_2412_20828_gb300.fer_sweep --frames 1000000 --json out.json
"""
from __future__ import annotations

import argparse
import json
import math
import sys
import time

import numpy as np

# (name, message format, power-of-two rescale, fractional c2v bits of the 8-bit form)
VARIANTS = (("fp32", 0, False, 0), ("fp16", 1, False, 0), ("int8", 2, False, 0), ("int8_rescale", 2, True, 0),
            ("int8f", 2, False, 8), ("int8f_rescale", 2, True, 8))
DEFAULT_CODES = ((63, 45), (63, 36))
DEFAULT_POINTS = tuple(1.0 + 0.5 * i for i in range(11))


def interp_ebn0_at_fer(points, fer, target):
    """Eb/N0 at which a FER curve reaches ``target`` (log10 FER linear in dB between
    points; None outside the curve's range or where the curve has no errors)."""
    pts = [(e, f) for e, f in zip(points, fer) if f > 0]
    if not pts or target <= 0:
        return None
    lt = math.log10(target)
    for (e0, f0), (e1, f1) in zip(pts, pts[1:]):
        l0, l1 = math.log10(f0), math.log10(f1)
        if (l0 - lt) * (l1 - lt) <= 0 and l0 != l1:
            return e0 + (lt - l0) * (e1 - e0) / (l1 - l0)
        if l0 == lt:
            return e0
    if math.log10(pts[-1][1]) == lt:
        return pts[-1][0]
    return None


def fer_loss_db(points, fer_ref, fer_var, errors_var, min_errors=50):
    """Per point: the variant's SNR loss against the reference curve (None where the
    variant saw fewer than ``min_errors`` frame errors or the FER lies outside the
    reference curve)."""
    out = []
    for e, f, ne in zip(points, fer_var, errors_var):
        if ne < min_errors:
            out.append(None)
            continue
        e_ref = interp_ebn0_at_fer(points, fer_ref, f)
        out.append(None if e_ref is None else e - e_ref)
    return out


def run(codes=DEFAULT_CODES, points=DEFAULT_POINTS, frames=1_000_000, iters=12, alpha=0.78,
        n_autos=3, chunk=1 << 20, seed=0x5EED, hybrid=True, variants=None, log=sys.stderr):
    import torch
    from . import bchdec as B
    B.load()
    vlist = [v for v in VARIANTS if variants is None or v[0] in variants]
    if not vlist or vlist[0][0] != "fp32":
        raise ValueError("the variants must include fp32 (the reference curve)")
    res = {"points": list(points), "frames_per_point": frames, "iters": iters, "alpha": alpha,
           "n_autos": n_autos, "codes": {}}
    for n, k in codes:
        code = B.Code(n, k)
        std = B.Code(n, k, kind=B.PCM_STANDARD)
        ld = 64 if n <= 64 else 128
        W = (n + 63) // 64
        Fc = min(chunk, frames)
        llr = torch.empty((Fc, ld), dtype=torch.float32, device="cuda")
        cw = torch.empty((Fc, W), dtype=torch.int64, device="cuda")
        aut = torch.empty((Fc, n_autos), dtype=torch.int16, device="cuda")
        hard = torch.empty((Fc, W), dtype=torch.int64, device="cuda")
        its = torch.empty(Fc, dtype=torch.uint8, device="cuda")
        flg = torch.empty(Fc, dtype=torch.uint8, device="cuda")
        ctr = torch.zeros((len(vlist), 2, len(points), 8), dtype=torch.int64, device="cuda")
        ps = {name: B.params(iters, alpha, n_autos=n_autos, msg=msg, rescale=rs, qfrac=qf)
              for name, msg, rs, qf in vlist}
        ws = B.workspace(code, ps["fp32"], Fc)
        ev = []  # (variant, stage, point, start, end): device time of each decode call
        stream = torch.cuda.current_stream()

        def timed(vi, si, pi, fn):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            ev.append((vi, si, pi, a, b))
        t0 = time.time()
        for pi, e in enumerate(points):
            for f0 in range(0, frames, Fc):
                F = min(Fc, frames - f0)
                base = pi * 10**9 + f0
                B.gen_frames(code, e, e, seed, base, llr[:F], cw[:F])
                B.draw_automorphisms(n, n_autos, seed + 1, base, aut[:F])
                for vi, (name, *_) in enumerate(vlist):
                    timed(vi, 0, pi, lambda: B.nms_decode(code, ps[name], llr[:F], aut[:F], hard[:F],
                                                          its[:F], flg[:F], ws=ws))
                    B.count_errors(n, hard[:F], cw[:F], its[:F], flg[:F], ctr[vi, 0, pi])
                    if hybrid:
                        timed(vi, 1, pi, lambda: B.hybrid_decode(code, std, ps[name], llr[:F], aut[:F],
                                                                 hard[:F], its[:F], flg[:F], ws=ws))
                        B.count_errors(n, hard[:F], cw[:F], its[:F], flg[:F], ctr[vi, 1, pi])
        torch.cuda.synchronize()
        c = ctr.cpu().numpy()
        dev_s = np.zeros((len(vlist), 2, len(points)))
        for vi, si, pi, a, b in ev:
            dev_s[vi, si, pi] += a.elapsed_time(b) / 1e3
        entry = {"seconds": time.time() - t0, "variants": {}}
        for vi, (name, *_) in enumerate(vlist):
            v = {}
            for si, stage in enumerate(("nms", "hybrid")):
                if stage == "hybrid" and not hybrid:
                    continue
                fr = c[vi, si, :, 0]
                v[stage] = {"frame_errors": c[vi, si, :, 1].tolist(),
                            "fer": (c[vi, si, :, 1] / fr).tolist(),
                            "ber": (c[vi, si, :, 2] / (fr * n)).tolist(),
                            "avg_iters": (c[vi, si, :, 5] / fr).tolist(),
                            "frames_per_s": (fr / np.maximum(dev_s[vi, si], 1e-12)).tolist(),
                            # edge-updates per second: NMS iterations run x P x edges over
                            # the stage's device time (OSD time included for the hybrid)
                            "edge_updates_per_s": (c[vi, si, :, 5] * n_autos * code.edges /
                                                   np.maximum(dev_s[vi, si], 1e-12)).tolist()}
            entry["variants"][name] = v
        for stage in ("nms", "hybrid") if hybrid else ("nms",):
            ref = entry["variants"]["fp32"][stage]["fer"]
            for name, *_ in vlist[1:]:
                v = entry["variants"][name][stage]
                v["loss_db_vs_fp32"] = fer_loss_db(points, ref, v["fer"], v["frame_errors"])
        res["codes"][f"({n},{k})"] = entry
        print(f"({n},{k}) done in {entry['seconds']:.1f} s", file=log)
        code.close()
        std.close()
    return res


def format_table(res):
    lines = []
    pts = res["points"]
    for cname, entry in res["codes"].items():
        for stage in ("nms", "hybrid"):
            if stage not in entry["variants"]["fp32"]:
                continue
            lines.append(f"BCH{cname} {stage}: FER per Eb/N0 (dB) and loss vs FP32 (dB)")
            lines.append("| variant | " + " | ".join(f"{e:g}" for e in pts) + " |")
            lines.append("|---|" + "---|" * len(pts))
            for name, v in entry["variants"].items():
                s = v[stage]
                cells = []
                for i in range(len(pts)):
                    f = s["fer"][i]
                    cell = f"{f:.2e}" if f > 0 else "0"
                    loss = s.get("loss_db_vs_fp32")
                    if loss is not None and loss[i] is not None:
                        cell += f" ({loss[i]:+.3f})"
                    cells.append(cell)
                lines.append(f"| {name} | " + " | ".join(cells) + " |")
            lines.append("")
    return "\n".join(lines)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--codes", default="63,45;63,36")
    ap.add_argument("--frames", type=int, default=1_000_000)
    ap.add_argument("--iters", type=int, default=12)
    ap.add_argument("--alpha", type=float, default=0.78)
    ap.add_argument("--points", default=",".join(f"{e:g}" for e in DEFAULT_POINTS))
    ap.add_argument("--no-hybrid", action="store_true")
    ap.add_argument("--variants", default=",".join(v[0] for v in VARIANTS))
    ap.add_argument("--json", default=None)
    a = ap.parse_args(argv)
    codes = [tuple(int(x) for x in c.split(",")) for c in a.codes.split(";")]
    points = [float(x) for x in a.points.split(",")]
    res = run(codes, points, a.frames, a.iters, a.alpha, hybrid=not a.no_hybrid,
              variants=a.variants.split(","))
    print(format_table(res))
    if a.json:
        with open(a.json, "w") as f:
            json.dump(res, f, indent=1)


if __name__ == "__main__":
    main()
