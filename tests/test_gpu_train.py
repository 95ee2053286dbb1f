"""GPU parity of the training path: checkpointed forward pass, the hand-written
backward kernel (subgradient through min1/min2) and the BCE loss, against the FP64
oracle gradient (itself pinned by central finite differences)."""
import numpy as np
import pytest

import oracle as O
from helpers import ambiguous_frames, autos_dev, frame_envelope, frames, rel_close, to_dev
from paper_2412_20828_gb300 import bchdec as B

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    from paper_2412_20828_gb300 import build
    build.build()
    B.load()
    return torch


@pytest.mark.parametrize("nk", [(63, 45), (127, 64)])
def test_forward_checkpoints_and_backward(torch_cuda, nk):
    torch = torch_cuda
    n, k = nk
    c = B.Code(n, k)
    Ho = c.dense()
    I = 4
    alpha = np.array([0.7, 0.75, 0.8, 0.85])
    F0 = 256
    cw, llr = frames(n, k, F0, 3.0, 800 + n, ld=(n + 3) & ~3)
    autos = O.draw_autos(n, 3, 21, 0, F0)
    # keep frames whose subgradient is unique (no near-tie of the two smallest |z|)
    _, _, _, _, tm = O.train_grad(Ho, llr, autos, I, alpha, cw, return_margin=True)
    tr0 = O.nms_enhanced(Ho, llr, autos, I, alpha, early_stop=False, trace=True)
    sel = np.nonzero((tm > 1e-4) & ~ambiguous_frames(llr, tr0, n))[0][:96]
    assert sel.size >= 48
    cw, llr, autos = cw[sel], np.ascontiguousarray(llr[sel]), np.ascontiguousarray(autos[sel])
    F, ld = llr.shape
    loss_ref, da_ref, dl_ref, y_ref = O.train_grad(Ho, llr, autos, I, alpha, cw)
    p = B.params(I, alpha, n_autos=3, early_stop=False)
    d_llr, d_aut = to_dev(llr), autos_dev(autos)
    ckpt = torch.zeros((I + 1, F, ld), dtype=torch.float32, device="cuda")
    ws = B.workspace(c, p, F)
    B.nms_forward_train(c, p, d_llr, d_aut, ckpt, ws)
    # checkpoints against the oracle trace
    tr = O.nms_enhanced(Ho, llr, autos, I, alpha, early_stop=False, trace=True)
    ck = ckpt.cpu().numpy()
    env = frame_envelope(tr)[:, None]
    for t in range(I + 1):
        mag = tr["mag"][:, t - 1, :] if t == 1 else (env if t > 1 else None)
        assert rel_close(ck[t, :, :n], tr["trace"][:, t, :], mag).all(), t
    # loss and its gradient
    d_cw = to_dev(B.pack_bits(cw))
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    gout = torch.zeros((F, ld), dtype=torch.float32, device="cuda")
    B.bce_loss(n, ckpt[I], d_cw, loss, gout, ws)
    torch.cuda.synchronize()
    assert float(loss.cpu()[0]) == pytest.approx(loss_ref, rel=1e-4)
    # backward
    gl = torch.zeros((F, ld), dtype=torch.float32, device="cuda")
    ga = torch.zeros(I, dtype=torch.float32, device="cuda")
    B.nms_backward(c, p, d_aut, ckpt, gout, gl, ga, ws)
    torch.cuda.synchronize()
    assert np.allclose(ga.cpu().numpy(), da_ref, rtol=2e-3, atol=1e-6 * np.abs(da_ref).max())
    g = gl.cpu().numpy()[:, :n]
    scale = np.abs(dl_ref).max(axis=1, keepdims=True)
    assert np.all(np.abs(g - dl_ref) <= 1e-3 * scale + 1e-12)


def test_train_alpha_reduces_loss(torch_cuda):
    c = B.Code(63, 45)
    alpha, hist = B.train_alpha(c, 3, 6, np.full(6, 0.5), steps=30, batch=4096, ebn0_lo=2.0,
                                ebn0_hi=5.0, seed=3, lr=0.02)
    assert np.all(np.isfinite(alpha)) and np.all(np.isfinite(hist))
    assert hist[-5:].mean() < hist[:5].mean()


def test_autograd_function_matches_oracle_gradient(torch_cuda):
    """The torch.autograd front end gives the oracle's dLoss/dalpha and dLoss/dllr."""
    torch = torch_cuda
    from paper_2412_20828_gb300 import autograd as AG
    n, k = 63, 45
    c = B.Code(n, k)
    Ho = c.dense()
    I = 5
    alpha0 = np.array([0.6, 0.7, 0.75, 0.8, 0.85])
    cw, llr = frames(n, k, 256, 2.5, 913, ld=64)
    autos = O.draw_autos(n, 3, 17, 0, 256)
    _, _, _, _, tm = O.train_grad(Ho, llr, autos, I, alpha0, cw, return_margin=True)
    tr0 = O.nms_enhanced(Ho, llr, autos, I, alpha0, early_stop=False, trace=True)
    sel = np.nonzero((tm > 1e-4) & ~ambiguous_frames(llr, tr0, n))[0][:96]
    assert sel.size >= 48
    cw, llr, autos = cw[sel], np.ascontiguousarray(llr[sel]), np.ascontiguousarray(autos[sel])
    loss_ref, da_ref, dl_ref, _ = O.train_grad(Ho, llr, autos, I, alpha0, cw)
    x = to_dev(llr).requires_grad_(True)
    alpha = torch.tensor(alpha0, dtype=torch.float32, device="cuda", requires_grad=True)
    y = AG.enhanced_nms(x, alpha, c, autos_dev(autos))
    loss = AG.bce(y, to_dev(B.pack_bits(cw)), c)
    loss.backward()
    assert float(loss) == pytest.approx(loss_ref, rel=1e-4)
    assert np.allclose(alpha.grad.cpu().numpy(), da_ref, rtol=2e-3,
                       atol=1e-6 * np.abs(da_ref).max())
    g = x.grad.cpu().numpy()[:, :n]
    scale = np.abs(dl_ref).max(axis=1, keepdims=True)
    assert np.all(np.abs(g - dl_ref) <= 1e-3 * scale + 1e-12)


def test_autograd_training_loop_on_simulated_frames(torch_cuda):
    """alpha_t trained by torch.optim through the backward kernel on frames the decoder
    simulates itself (Eb/N0 uniform in [2, 5] dB): the loss falls."""
    torch = torch_cuda
    from paper_2412_20828_gb300 import autograd as AG
    c = B.Code(63, 36)
    I, F = 6, 8192
    alpha = AG.alpha_init(I, 0.5)
    opt = torch.optim.Adam([alpha], lr=0.02)
    llr = torch.empty((F, 64), dtype=torch.float32, device="cuda")
    cw = torch.empty((F, 1), dtype=torch.int64, device="cuda")
    aut = torch.empty((F, 3), dtype=torch.int16, device="cuda")
    hist = []
    for step in range(25):
        B.gen_frames(c, 2.0, 5.0, 77, step * F, llr, cw)
        B.draw_automorphisms(63, 3, 78, step * F, aut)
        opt.zero_grad()
        loss = AG.bce(AG.enhanced_nms(llr, alpha, c, aut), cw, c)
        loss.backward()
        opt.step()
        hist.append(float(loss))
    assert np.all(np.isfinite(hist)) and torch.isfinite(alpha).all()
    assert np.mean(hist[-5:]) < np.mean(hist[:5])


def test_training_resumes_bit_exactly(tmp_path):
    """Six Adam steps in one call equal three steps, a save to disk and a load, and three
    more steps that continue from the saved state: identical alpha and losses (the frames
    of step s are frames s x batch ... of the simulated stream in both runs)."""
    from paper_2412_20828_gb300 import build
    build.build()
    code = B.Code(63, 45)
    kw = dict(n_autos=3, iters=8, steps=6, batch=4096, ebn0_lo=2.0, ebn0_hi=4.0, seed=31, lr=0.01)
    a_full, h_full = B.train_alpha(code, kw["n_autos"], kw["iters"], 0.78, kw["steps"], kw["batch"],
                                   kw["ebn0_lo"], kw["ebn0_hi"], kw["seed"], kw["lr"])
    st = B.AdamState()
    a1, h1 = B.train_alpha_resume(code, 3, 8, 0.78, st, 3, 4096, 2.0, 4.0, 31, 0.01)
    assert st.step == 3
    B.save_training(tmp_path / "s.npz", a1, st)
    a1b, st2 = B.load_training(tmp_path / "s.npz")
    a2, h2 = B.train_alpha_resume(code, 3, 8, a1b, st2, 3, 4096, 2.0, 4.0, 31, 0.01)
    assert st2.step == 6
    assert np.array_equal(np.concatenate([h1, h2]), h_full)
    assert np.array_equal(a2, a_full)
    with pytest.raises(B.BchError):  # a state of another shape is refused
        B.train_alpha_resume(code, 3, 8, a2, st2, 1, 2048, 2.0, 4.0, 31, 0.01)
