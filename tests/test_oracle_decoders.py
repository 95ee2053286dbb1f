"""Pins for the oracle's channel, generators, automorphisms and decoders.

Expectations come from hand-derived examples (tests/golden/nms_hand_examples.txt),
published known-answer vectors, closed forms of the channel, group properties of the
automorphisms, coding-theory facts (d_min of BCH(15,7)) and brute force.
"""
import os

import numpy as np
import pytest

import oracle as O
from paper_2412_20828_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")
H4 = np.array([[1, 1, 1, 0], [0, 1, 1, 1]], np.uint8)


def _gold(key):
    with open(os.path.join(GOLD, "nms_hand_examples.txt")) as f:
        for line in f:
            if line.startswith(key + " "):
                return np.array([float(x) for x in line.split()[1:]])
    raise KeyError(key)


def _frames(n, k, F, ebn0, seed):
    msg = synth.messages(F, k, seed)
    cw = O.encode(n, k, msg)
    llr = O.channel_llr(n, k, cw, synth.normals(F, n, seed), ebn0)
    return cw, llr


# ------------------------------------------------------------------ generators
def test_philox_known_answers():
    # Known-answer vectors published with Philox4x32-10 (Salmon et al., SC'11, Random123)
    assert O.philox4x32_10([0, 0, 0, 0], [0, 0]) == [0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8]
    assert O.philox4x32_10([0xFFFFFFFF] * 4, [0xFFFFFFFF] * 2) == [
        0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD]
    assert O.philox4x32_10([0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344],
                           [0xA4093822, 0x299F31D0]) == [0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1]


def test_splitmix64_first_output():
    # SplitMix64 from state 0 (Steele et al., OOPSLA 2014; reference implementation)
    assert O.splitmix64(0, 1)[0] == 0xE220A8397B1DCDAF


def test_sigma2_closed_form():
    # sigma^2 = 1 / (2 R Eb/N0): values at 3 dB
    assert O.sigma2(63, 36, 3.0) == pytest.approx(0.43857, abs=1e-4)
    assert O.sigma2(127, 99, 3.0) == pytest.approx(0.32146, abs=1e-4)


def test_channel_llr_statistics():
    # Gaussian LLR consistency (Eq. 1): for c = 0, L ~ N(2/s2, 4/s2)
    n, k, F = 63, 36, 4000
    cw = np.zeros((F, n), np.uint8)
    llr = O.channel_llr(n, k, cw, synth.normals(F, n, 3), 2.0).astype(np.float64)
    s2 = O.sigma2(n, k, 2.0)
    assert llr.mean() == pytest.approx(2 / s2, rel=0.01)
    assert llr.var() == pytest.approx(4 / s2, rel=0.02)
    # antipodal symmetry: L(c = 1, noise) = -L(c = 0, -noise)
    cw1 = np.ones((F, n), np.uint8)
    llr1 = O.channel_llr(n, k, cw1, -synth.normals(F, n, 3), 2.0)
    assert np.allclose(llr1, -llr, rtol=0, atol=1e-4 * np.abs(llr).max())


def test_framegen_recipe_properties():
    n, k = 127, 64
    llr, cw, e = O.framegen(n, k, seed=99, frame0=1000, F=3000, ebn0_lo=2.0, ebn0_hi=5.0, ld=128)
    H = O.std_h(n, k)
    assert np.all((cw.astype(np.int64) @ H.T.astype(np.int64)) % 2 == 0)
    assert abs(cw[:, n - k:].mean() - 0.5) < 0.02  # message bits uniform
    assert e.min() >= 2.0 and e.max() < 5.0 and abs(e.mean() - 3.5) < 0.05
    # recover the unit normals from the LLRs and check N(0,1)
    s2 = np.array([O.sigma2(n, k, x) for x in e])
    y = llr[:, :n].astype(np.float64) * s2[:, None] / 2
    z = (y - (1 - 2.0 * cw)) / np.sqrt(s2)[:, None]
    assert abs(z.mean()) < 0.01 and abs(z.var() - 1) < 0.01
    assert np.all(llr[:, n:] == 0)
    # frame index addressing: frames 1000.. regenerate identically from frame0 = 1500
    llr2, cw2, _ = O.framegen(n, k, seed=99, frame0=1500, F=10, ebn0_lo=2.0, ebn0_hi=5.0, ld=128)
    assert np.array_equal(llr2, llr[500:510]) and np.array_equal(cw2, cw[500:510])


# ------------------------------------------------------------------ automorphisms
@pytest.mark.parametrize("nk", [(15, 7), (63, 36), (63, 45), (127, 64), (127, 99)])
def test_automorphisms_map_codewords_to_codewords(nk):
    n, k = nk
    H = O.std_h(n, k)
    aut = O.draw_autos(n, 3, seed=7, frame0=0, F=200)
    ordn = O.ord2(n)
    assert ordn == {15: 4, 63: 6, 127: 7}[n]
    s, j = aut & 0xFF, aut >> 8
    assert s.max() < n and j.max() < ordn
    # pairs are distinct within a frame
    assert all(len(set(r.tolist())) == 3 for r in aut)
    cw = O.encode(n, k, synth.messages(200, k, 5))
    for f in range(200):
        for p in range(3):
            pi = O.auto_perm(int(aut[f, p]), n)
            assert len(set(pi.tolist())) == n
            z = np.zeros(n, np.uint8)
            z[pi] = cw[f]
            assert O.syndrome_weight(H, z) == 0


def test_automorphism_draw_is_counter_based():
    a = O.draw_autos(127, 3, seed=3, frame0=0, F=100)
    b = O.draw_autos(127, 3, seed=3, frame0=40, F=10)
    assert np.array_equal(a[40:50], b)
    assert not np.array_equal(a, O.draw_autos(127, 3, seed=4, frame0=0, F=100))


# ------------------------------------------------------------------ plain NMS
def test_plain_nms_hand_example():
    L = _gold("plain_L").astype(np.float32)[None, :]
    r1 = O.nms_plain(H4, L, iters=5, alpha=0.5, early_stop=True)
    assert r1["iters"][0] == 1 and r1["converged"][0] == 1
    assert np.array_equal(r1["y"][0], _gold("plain_x1"))
    r2 = O.nms_plain(H4, L, iters=2, alpha=0.5, early_stop=False)
    assert r2["iters"][0] == 2 and r2["converged"][0] == 0
    assert np.array_equal(r2["y"][0], _gold("plain_x2"))
    assert r2["hard"][0].tolist() == [0, 1, 0, 0]


@pytest.mark.parametrize("nk", [(63, 36), (127, 64)])
def test_plain_nms_noiseless_one_iteration(nk):
    n, k = nk
    cw = O.encode(n, k, synth.messages(20, k, 1))
    llr = (4.0 * (1 - 2.0 * cw)).astype(np.float32)
    r = O.nms_plain(O.std_h(n, k), llr, iters=8, alpha=0.78)
    assert np.all(r["iters"] == 1) and np.all(r["converged"] == 1)
    assert np.array_equal(r["hard"], cw)


# ------------------------------------------------------------------ enhanced NMS
def test_enhanced_hand_example():
    y0 = _gold("enh_y0").astype(np.float32)[None, :]
    aut = np.array([[0, 1]], np.uint16)
    r = O.nms_enhanced(H4, y0, aut, iters=1, alpha=0.5, trace=True)
    assert np.array_equal(r["y"][0], _gold("enh_y1"))
    assert r["iters"][0] == 1


def test_enhanced_first_iteration_equals_plain_with_identity():
    # With P copies all equal to the identity, iteration 1 of Algorithm 1 is iteration 1
    # of Eqs. (2)-(4) (both start from c2v^(0) = 0).
    n, k = 63, 45
    Ho = O.build_ho(n, k)
    _, llr = _frames(n, k, 30, 2.0, 21)
    aut = np.zeros((30, 3), np.uint16)
    e = O.nms_enhanced(Ho, llr, aut, iters=1, alpha=0.7, early_stop=False)
    p = O.nms_plain(Ho, llr, iters=1, alpha=0.7, early_stop=False)
    assert np.allclose(e["y"], p["y"], rtol=1e-12, atol=1e-12)


def _compose(v, a_s, a_j, n):
    # pi_p o sigma^{-1} for pi_p = (s, j) and sigma(i) = 2^a_j i + a_s
    s, j = v & 0xFF, v >> 8
    ordn = O.ord2(n)
    jj = (j - a_j) % ordn
    ss = (s - pow(2, jj, n) * a_s) % n
    return ss | (jj << 8)


@pytest.mark.parametrize("nk", [(63, 36), (127, 99)])
def test_enhanced_permutation_equivariance(nk):
    # D(sigma(y); {pi_p sigma^-1}) = sigma(D(y; {pi_p})): fails if any permutation is
    # applied in the wrong direction in the dilation or the un-permutation step.
    n, k = nk
    Ho = O.build_ho(n, k)
    F = 12
    _, llr = _frames(n, k, F, 2.5, 31)
    aut = O.draw_autos(n, 3, 9, 0, F)
    base = O.nms_enhanced(Ho, llr, aut, iters=3, alpha=0.8, early_stop=False)
    a_s, a_j = 17 % n, 2
    sig = O.auto_perm(a_s | (a_j << 8), n)
    llr2 = np.zeros_like(llr)
    llr2[:, sig] = llr
    aut2 = np.vectorize(lambda v: _compose(int(v), a_s, a_j, n))(aut).astype(np.uint16)
    r2 = O.nms_enhanced(Ho, llr2, aut2, iters=3, alpha=0.8, early_stop=False)
    exp = np.zeros_like(base["y"])
    exp[:, sig] = base["y"]
    assert np.allclose(r2["y"], exp, rtol=1e-12, atol=1e-9)


@pytest.mark.parametrize("nk", [(63, 36), (63, 45), (127, 64), (127, 99)])
def test_enhanced_noiseless_one_iteration(nk):
    n, k = nk
    Ho = O.build_ho(n, k)
    cw = O.encode(n, k, synth.messages(10, k, 2))
    llr = (3.0 * (1 - 2.0 * cw)).astype(np.float32)
    r = O.nms_enhanced(Ho, llr, O.draw_autos(n, 3, 1, 0, 10), iters=12, alpha=0.78)
    assert np.all(r["iters"] == 1) and np.all(r["converged"] == 1)
    assert np.array_equal(r["hard"], cw)


def test_enhanced_stop_rule_from_trace():
    # Algorithm 1 stops at the first iteration whose hard decision has zero H_o syndrome
    n, k = 63, 36
    Ho = O.build_ho(n, k)
    _, llr = _frames(n, k, 60, 2.0, 41)
    aut = O.draw_autos(n, 3, 2, 0, 60)
    r = O.nms_enhanced(Ho, llr, aut, iters=12, alpha=0.78, trace=True)
    for f in range(60):
        t_run = r["iters"][f]
        for t in range(1, t_run + 1):
            c = (r["trace"][f, t] < 0).astype(np.uint8)
            zero = O.syndrome_weight(Ho, c) == 0
            assert zero == (t == t_run and r["converged"][f] == 1)


def test_syndrome_ho_equals_standard_h():
    # H_o and the standard H have the same row space, so their zero-syndrome tests agree
    n, k = 127, 64
    Ho = O.build_ho(n, k)
    H = O.std_h(n, k)
    rng = np.random.default_rng(0)
    words = rng.integers(0, 2, (300, n), dtype=np.uint8)
    words[:100] = O.encode(n, k, synth.messages(100, k, 3))
    for w in words:
        assert (O.syndrome_weight(Ho, w) == 0) == (O.syndrome_weight(H, w) == 0)


# ------------------------------------------------------------------ OSD and ML
def test_ml_corrects_up_to_two_errors():
    # BCH(15,7) has d_min = 5: with hard +-1 inputs ML is minimum-distance decoding and
    # corrects every pattern of at most 2 errors.
    n, k = 15, 7
    cw = O.encode(n, k, synth.messages(8, k, 4))
    rows = []
    truth = []
    for c in cw:
        s = 1.0 - 2.0 * c
        rows.append(s.copy())
        truth.append(c)
        for a in range(n):
            x = s.copy(); x[a] = -x[a]
            rows.append(x); truth.append(c)
            for b in range(a + 1, n):
                y = x.copy(); y[b] = -y[b]
                rows.append(y); truth.append(c)
    llr = np.array(rows, np.float32)
    out = O.ml(n, k, llr)
    assert np.array_equal(out, np.array(truth))


def test_osd_order_k_equals_ml_on_bch15_7():
    n, k = 15, 7
    _, llr = _frames(n, k, 400, 1.0, 51)
    ml = O.ml(n, k, llr)
    cw, _ = O.osd(O.std_h(n, k), llr, order=k)
    assert np.array_equal(cw, ml)


def _gf2_rank(A):
    A = A.copy() % 2
    r = 0
    for c in range(A.shape[1]):
        piv = np.nonzero(A[r:, c])[0]
        if piv.size == 0:
            continue
        p = r + piv[0]
        A[[r, p]] = A[[p, r]]
        for i in range(A.shape[0]):
            if i != r and A[i, c]:
                A[i] ^= A[r]
        r += 1
        if r == A.shape[0]:
            break
    return r


@pytest.mark.parametrize("nk", [(15, 7), (63, 45)])
def test_osd_mrb_is_greedy_generator_basis(nk):
    # Matroid duality: the complement of the least-reliable pivots on H is the greedy
    # most-reliable independent set of generator columns.
    n, k = nk
    G = O.encode(n, k, np.eye(k, dtype=np.uint8))
    _, llr = _frames(n, k, 10, 2.0, 61)
    _, _, mrb = O.osd(O.std_h(n, k), llr, order=0, return_mrb=True)
    for f in range(10):
        order = sorted(range(n), key=lambda i: (-abs(float(llr[f, i])), -i))
        chosen = []
        for i in order:
            if _gf2_rank(G[:, chosen + [i]].T.copy()) == len(chosen) + 1:
                chosen.append(i)
            if len(chosen) == k:
                break
        assert sorted(chosen) == sorted(mrb[f].tolist())


@pytest.mark.parametrize("nk", [(63, 36), (127, 99)])
def test_osd_outputs_codewords_and_beats_transmitted_when_listed(nk):
    n, k = nk
    H = O.std_h(n, k)
    cw, llr = _frames(n, k, 30, 2.0, 71)
    out, score, mrb = O.osd(H, llr, order=2, return_mrb=True)
    w = np.minimum(np.floor(np.abs(llr.astype(np.float64)) * 2.0**24), 2.0**40).astype(np.uint64)
    hard = (llr < 0).astype(np.uint8)
    for f in range(30):
        assert O.syndrome_weight(H, out[f]) == 0
        assert score[f] == w[f][out[f] != hard[f]].sum()
        # when the transmitted word has <= 2 errors on the MRB it is a candidate, so the
        # winner scores no worse than it
        if (cw[f][mrb[f]] != hard[f][mrb[f]]).sum() <= 2:
            assert score[f] <= w[f][cw[f] != hard[f]].sum()


def test_osd2_close_to_ml_on_bch15_7():
    n, k = 15, 7
    cw, llr = _frames(n, k, 3000, 2.0, 81)
    ml = O.ml(n, k, llr)
    o2, _ = O.osd(O.std_h(n, k), llr, order=2)
    fer_ml = np.any(ml != cw, axis=1).mean()
    fer_o2 = np.any(o2 != cw, axis=1).mean()
    assert fer_o2 >= fer_ml - 1e-12
    assert fer_o2 - fer_ml < 0.01


def test_hybrid_on_nms_reliabilities_is_ml_on_them_for_bch15_7():
    # With order k the OSD tries every word of the basis, so on BCH(15,7) it returns
    # the maximum-likelihood word for whatever reliabilities it is given: here the NMS
    # output y of the failed frames (ML is scale invariant, so y itself, unscaled,
    # serves as the reference metric).
    n, k = 15, 7
    Ho = O.build_ho(n, k)
    # 0 dB and 2 iterations leave about a sixth of the frames to the OSD
    _, llr = _frames(n, k, 600, 0.0, 101)
    aut = O.draw_autos(n, 3, 7, 0, 600)
    r = O.hybrid_nms_reliability(Ho, O.std_h(n, k), llr, aut, 2, 0.8, order=k)
    fail = r["osd_frames"]
    assert fail.size > 50
    nms = O.nms_enhanced(Ho, llr, aut, 2, 0.8)
    ml_y = O.ml(n, k, nms["y"][fail].astype(np.float32))
    assert np.array_equal(r["final"][fail], ml_y)
    # and the input really is y: ML on the channel LLR differs on some of those frames
    assert not np.array_equal(ml_y, O.ml(n, k, llr[fail]))


def test_hybrid_on_nms_reliabilities_is_scale_free():
    n, k = 63, 45
    Ho, Hs = O.build_ho(n, k), O.std_h(n, k)
    _, llr = _frames(n, k, 200, 2.0, 111)
    aut = O.draw_autos(n, 3, 9, 0, 200)
    a = O.hybrid_nms_reliability(Ho, Hs, llr, aut, 12, 0.78)
    b = O.hybrid_nms_reliability(Ho, Hs, (llr * 8.0).astype(np.float32), aut, 12, 0.78)
    assert a["osd_frames"].size > 10
    assert np.array_equal(a["final"], b["final"])
    # every output is a codeword
    assert all(O.syndrome_weight(Hs, w) == 0 for w in a["final"])


# ------------------------------------------------------------------ gradient
def test_train_grad_matches_central_differences():
    n, k = 63, 45
    Ho = O.build_ho(n, k)
    F, iters = 6, 3
    cw, llr = _frames(n, k, F, 3.0, 91)
    aut = O.draw_autos(n, 3, 5, 0, F)
    alpha = np.array([0.7, 0.8, 0.9])
    loss, da, dl, _ = O.train_grad(Ho, llr, aut, iters, alpha, cw)
    h = 1e-3
    for t in range(iters):
        ap, am = alpha.copy(), alpha.copy()
        ap[t] += h
        am[t] -= h
        fd = (O.train_grad(Ho, llr, aut, iters, ap, cw)[0] - O.train_grad(Ho, llr, aut, iters, am, cw)[0]) / (2 * h)
        assert da[t] == pytest.approx(fd, rel=1e-3, abs=1e-7)
    rng = np.random.default_rng(1)
    for _ in range(8):
        f, i = rng.integers(F), rng.integers(n)
        lp, lm = llr.copy(), llr.copy()
        lp[f, i] += np.float32(h)
        lm[f, i] -= np.float32(h)
        step = float(lp[f, i]) - float(lm[f, i])
        fd = (O.train_grad(Ho, lp, aut, iters, alpha, cw)[0] - O.train_grad(Ho, lm, aut, iters, alpha, cw)[0]) / step
        assert dl[f, i] == pytest.approx(fd, rel=2e-3, abs=1e-9)


# ------------------------------------------------------------------ precision formats
def test_q16_matches_ieee_binary16():
    rng = np.random.default_rng(3)
    xs = np.concatenate([rng.standard_normal(20000) * 10.0 ** rng.integers(-9, 5, 20000),
                         [0.0, 65504.0, -65504.0, 6.1e-5, 5.96e-8, 2049.0, 2051.0, 0.1]])
    for x in xs:
        exp = float(np.float16(x)) if abs(x) < 65504 else np.sign(x) * 65504.0
        assert O.q16(x) == exp, x


@pytest.mark.parametrize("fmt", [1, 2])
def test_quantised_decoder_equals_fp64_on_exact_inputs(fmt):
    # With alpha = 0.5 (P = 1, identity automorphism) and inputs that are multiples of
    # the format's step within range, every quantiser in the first iteration is exact
    # (minima of representable values times 1/2 stay representable, up to the integer
    # rounding of INT8 which is exact on even minima), so the quantised decoder must
    # reproduce the FP64 decoder.
    n, k = 15, 7
    Ho = O.build_ho(n, k)
    rng = np.random.default_rng(fmt)
    if fmt == 1:
        llr = rng.integers(-40, 41, (50, n)).astype(np.float32)
    else:
        llr = (rng.integers(-3, 4, (50, n)) * 2).astype(np.float32) / 4.0 * 2.0  # q even
    llr[llr == 0] = 1.0
    aut = np.zeros((50, 1), np.uint16)
    a = O.nms_enhanced_q(Ho, llr, aut, 1, 0.5, fmt, early_stop=False)
    b = O.nms_enhanced(Ho, llr, aut, 1, 0.5, early_stop=False)
    if fmt == 1:
        assert np.array_equal(a["y"], b["y"])
    else:
        # INT8 stores 4x clamped to +-31: compare where the FP64 result is in range
        inr = np.abs(b["y"]) * 4 <= 31
        assert np.array_equal(a["y"][inr], b["y"][inr])
    assert np.array_equal(a["hard"], b["hard"])


def test_osd2_matches_paper_printed_points():
    """The oracle's order-2 OSD reaches the error rates the paper prints for OSD(2)
    (Fig. 2, Fig. 3; golden tests/golden/osd2_printed_points.txt) within a band of
    three standard deviations of our estimate plus 10% for the paper's unknown sample."""
    rows = []
    with open(os.path.join(GOLD, "osd2_printed_points.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                n, k, e, meas, val = line.split()[:5]
                rows.append((int(n), int(k), float(e), meas, float(val)))
    frames_for = {(63, 36): 40000, (63, 45): 12000, (127, 99): 6000}
    for i, (n, k, e, meas, val) in enumerate(rows):
        F = frames_for[(n, k)]
        msg = synth.messages(F, k, 4300 + i)
        cw = O.encode(n, k, msg)
        llr = O.channel_llr(n, k, cw, synth.normals(F, n, 4300 + i), e)
        dec, _ = O.osd(O.std_h(n, k), llr, 2, threads=None)
        err = dec != cw
        fe = int(err.any(axis=1).sum())
        got = err.mean() if meas == "ber" else fe / F
        band = 3.0 / np.sqrt(max(fe, 1)) + 0.10
        assert fe >= 100, (n, k, e, fe)
        assert abs(got / val - 1.0) <= band, (n, k, e, meas, got, val, band)
