"""Shared helpers of the GPU parity tests: seeded inputs (oracle encoder + channel on
draws from ``synth``), device marshalling and the tolerance rules.

Tolerance rules (FP32 kernel vs FP64 oracle, same FP32 input bytes):
 * one iteration from the same input: a sum of terms is compared relative to the sum
   of the terms' magnitudes (the "operand magnitude" returned by the oracle):
   |gpu - ref| <= 1e-5 max(|ref|, mag, 1);
 * after several iterations the FP32 and FP64 trajectories drift apart in magnitude
   (rounding of a frame's largest values reaches its small ones through the
   cancellations of the updates, and each iteration can amplify it), so the final
   state of a multi-iteration decode is compared against the frame's largest operand
   magnitude env with the trajectory tolerance TRAJ_TOL:
   |gpu - ref| <= 1e-3 max(|ref|, env) -- while decisions stay exact (next rule);
 * hard decisions and iteration counts must be identical on every frame whose
   decoding never met a sign-ambiguous value: |y| < 1e-3 on the channel LLR, or any
   |y^(t)| below 1e-4 of its operand magnitude in a later iteration (there the sign is
   decided by rounding order, and a flipped sign legitimately changes the rest);
 * integer work (matrices, permutations, syndromes, OSD) is bit-exact.
"""
import numpy as np

import oracle as O
from paper_2412_20828_gb300 import synth

REL_TOL = 1e-5
TRAJ_TOL = 1e-3
AMBIG_LLR = 1e-3
AMBIG_REL = 1e-4


def frames(n, k, F, ebn0, seed, ld=None):
    msg = synth.messages(F, k, seed)
    cw = O.encode(n, k, msg)
    llr = O.channel_llr(n, k, cw, synth.normals(F, n, seed), ebn0, ld=ld or n)
    return cw, llr


def to_dev(x, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(x))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def autos_dev(autos):
    return to_dev(autos.view(np.int16))


def ambiguous_frames(llr, ref, n):
    """Frames whose oracle trace meets a sign-ambiguous value (see module doc)."""
    amb = np.any(np.abs(llr[:, :n]) < AMBIG_LLR, axis=1)
    if "trace" in ref:
        tr = ref["trace"][:, 1:, :]
        mg = np.maximum(ref["mag"], 1.0)
        amb |= np.any(np.abs(tr) < AMBIG_REL * mg, axis=(1, 2))
    return amb


def frame_envelope(ref):
    """Largest operand magnitude met while decoding each frame (from the trace)."""
    return np.max(ref["mag"], axis=(1, 2))


def rel_close(gpu, ref, mag=None):
    scale = np.abs(ref)
    if mag is not None:
        scale = np.maximum(scale, mag)
    scale = np.maximum(scale, 1.0)
    return np.abs(gpu - ref) <= REL_TOL * scale
