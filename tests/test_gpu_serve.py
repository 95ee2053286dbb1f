"""Continuous-batching server: results are the same alone and in a mixed stream, equal
to the batch hybrid decoder on the same frames and to the oracle's hybrid decoder on
every unambiguous frame, on both serving kernels (the one specialised to the server's
codes and the precompiled one), and the admission honours the HBM budget (queueing,
never dropping)."""
import numpy as np
import pytest

import oracle as O
from helpers import ambiguous_frames, autos_dev, frames, to_dev
from paper_2412_20828_gb300 import bchdec as B

pytestmark = pytest.mark.gpu

CODES = [(63, 36), (63, 45), (127, 64), (127, 99)]


@pytest.fixture(scope="module")
def setup():
    import torch
    from paper_2412_20828_gb300 import build
    build.build()
    codes = [B.Code(n, k) for n, k in CODES]
    stds = [B.Code(n, k, kind=B.PCM_STANDARD) for n, k in CODES]
    return torch, codes, stds


def _batch_reference(torch, monkeypatch, code, std, llr, seed, frame0):
    # the batch hybrid decoder on the precompiled kernel (bit-identical to the
    # specialised one: test_jit_and_generic_kernels_agree)
    monkeypatch.setenv("BCHDEC_NMS_KERNEL", "generic")
    F, ld = llr.shape
    aut = torch.zeros((F, 3), dtype=torch.int16, device="cuda")
    B.draw_automorphisms(code.n, 3, seed, frame0, aut)
    hard = torch.zeros((F, (code.n + 63) // 64), dtype=torch.int64, device="cuda")
    it = torch.zeros(F, dtype=torch.uint8, device="cuda")
    fl = torch.zeros(F, dtype=torch.uint8, device="cuda")
    B.hybrid_decode(code, std, B.params(12, 0.78, osd_order=2), to_dev(llr), aut, hard, it, fl)
    torch.cuda.synchronize()
    monkeypatch.delenv("BCHDEC_NMS_KERNEL")
    return hard.cpu().numpy(), it.cpu().numpy(), fl.cpu().numpy()


def _drain(srv, want):
    got = {}
    for _ in range(20000):
        for rid in srv.poll(timeout_us=2000):
            got[rid] = srv.fetch(rid)
        if all(w in got for w in want):
            return got
    raise AssertionError("server did not complete the requests")


@pytest.mark.parametrize("kernel", ["blocks", "warps", "generic"])
def test_results_alone_and_in_mix_match_batch_decoder(setup, monkeypatch, kernel):
    """blocks: the block-bound kernel (sessions per code with the batch mappings, the
    default); warps: the per-warp kernel with lane refill; generic: the precompiled one."""
    torch, codes, stds = setup
    if kernel == "generic":
        monkeypatch.setenv("BCHDEC_NMS_KERNEL", "generic")
    if kernel == "warps":
        monkeypatch.setenv("BCHDEC_SERVE_KERNEL", "warps")
    srv = B.Server(codes, stds, 12, 0.78, budget_bytes=1 << 30, max_requests=256)
    monkeypatch.delenv("BCHDEC_NMS_KERNEL", raising=False)
    monkeypatch.delenv("BCHDEC_SERVE_KERNEL", raising=False)
    try:
        info = srv.kernel_info()
        assert info == {"blocks": "jit-blocks", "warps": "jit"}.get(kernel, info) and (
            kernel != "generic" or info.startswith("generic"))
        reqs = []
        for i, (n, k) in enumerate(CODES):
            for j, (F, e) in enumerate([(37, 2.0), (300, 3.0), (1, 4.0)]):
                cw, llr = frames(n, k, F, e, 5000 + 10 * i + j, ld=(n + 3) & ~3)
                reqs.append((i, llr, 77 + j, 1000 * j))
        # alone, one at a time
        alone = []
        for code_id, llr, seed, f0 in reqs:
            rid = srv.submit(code_id, llr, seed, f0)
            alone.append(_drain(srv, [rid])[rid])
        # all at once, mixed
        rids = [srv.submit(code_id, llr, seed, f0) for code_id, llr, seed, f0 in reqs]
        mixed = _drain(srv, rids)
        checked = 0
        for (code_id, llr, seed, f0), a, rid in zip(reqs, alone, rids):
            m = mixed[rid]
            for x, y in zip(a, m):
                assert np.array_equal(x, y)
            ref = _batch_reference(torch, monkeypatch, codes[code_id], stds[code_id], llr, seed, f0)
            for x, y in zip(a, ref):
                assert np.array_equal(x, y)
            # and the oracle's hybrid decoder (Sec. IV) on every unambiguous frame
            n = codes[code_id].n
            autos = O.draw_autos(n, 3, seed, f0, llr.shape[0])
            tr = O.nms_enhanced(codes[code_id].dense(), llr, autos, 12, 0.78, trace=True)
            ok = ~ambiguous_frames(llr, tr, n)
            hyb = O.hybrid(codes[code_id].dense(), stds[code_id].dense(), llr, autos, 12, 0.78)
            assert np.array_equal(B.unpack_bits(a[0], n)[ok], hyb["final"][ok])
            assert np.array_equal(a[1][ok], tr["iters"][ok])
            assert np.array_equal((a[2] & B.FLAG_OSD)[ok] > 0, (tr["converged"][ok] == 0))
            checked += int(ok.sum())
        assert checked > 0.9 * sum(r[1].shape[0] for r in reqs)
        st = srv.stats()
        assert st["completed"] == 2 * len(reqs) and st["bytes_in_use"] == 0
    finally:
        srv.close()


def test_budget_admission_queues_and_rejects(setup):
    torch, codes, stds = setup
    # a budget that holds about two 500-frame (127,k) requests at a time
    srv = B.Server(codes, stds, 12, 0.78, budget_bytes=600_000, max_requests=8)
    try:
        n, k = 127, 64
        cw, llr = frames(n, k, 500, 3.0, 6000, ld=128)
        rids = [srv.submit(2, llr, 1, 0) for _ in range(6)]
        st = srv.stats()
        assert st["queued"] >= 3  # the rest waited for memory
        out = _drain(srv, rids)
        first = out[rids[0]]
        for r in rids[1:]:
            for x, y in zip(first, out[r]):
                assert np.array_equal(x, y)
        big = np.zeros((4096, 128), np.float32)
        with pytest.raises(B.BchError) as e:
            srv.submit(2, big, 1, 0)
        assert e.value.status == B.EBUDGET
    finally:
        srv.close()


def test_kernel_relaunches_after_idle_exit(setup):
    import time
    torch, codes, stds = setup
    srv = B.Server(codes, stds, 12, 0.78, budget_bytes=1 << 28, idle_exit_us=20000)
    try:
        n, k = 63, 45
        cw, llr = frames(n, k, 64, 3.0, 7000, ld=64)
        r1 = srv.submit(1, llr, 3, 0)
        a = _drain(srv, [r1])[r1]
        time.sleep(0.2)  # the persistent kernel has exited by now
        r2 = srv.submit(1, llr, 3, 0)
        b = _drain(srv, [r2])[r2]
        for x, y in zip(a, b):
            assert np.array_equal(x, y)
        assert srv.stats()["kernel_launches"] >= 2
    finally:
        srv.close()


def test_malformed_requests_are_rejected_and_the_server_keeps_serving(setup):
    """Host-injected malformed requests: unknown code, empty or oversized requests, a
    row stride shorter than the code and a null buffer fail with BCH_EINVAL before any
    device work; a valid request submitted afterwards decodes as before."""
    import ctypes as C
    torch, codes, stds = setup
    srv = B.Server(codes, stds, 12, 0.78, budget_bytes=1 << 28, max_requests=16, max_frames_per_request=512)
    try:
        n, k = 63, 45
        cw, llr = frames(n, k, 64, 3.0, 7100, ld=64)
        bad = [
            lambda: srv.submit(7, llr, 1, 0),                         # no such code
            lambda: srv.submit(1, llr[:0], 1, 0),                     # no frames
            lambda: srv.submit(1, np.zeros((513, 64), np.float32), 1, 0),  # above the per-request limit
            lambda: srv.submit(1, np.ascontiguousarray(llr[:, :32]), 1, 0),  # ld < n
        ]
        for f in bad:
            with pytest.raises(B.BchError) as e:
                f()
            assert e.value.status == B.EINVAL
        rid = C.c_uint64()
        rc = B.load().bch_server_submit(srv._h, 1, None, 64, 8, 1, 0, C.byref(rid))  # null llr
        assert rc == B.EINVAL
        assert srv.stats()["submitted"] == 0
        good = srv.submit(1, llr, 3, 0)
        out = _drain(srv, [good])[good]
        ref = O.hybrid(codes[1].dense(), stds[1].dense(), llr, O.draw_autos(n, 3, 3, 0, 64), 12, 0.78)
        tr = O.nms_enhanced(codes[1].dense(), llr, O.draw_autos(n, 3, 3, 0, 64), 12, 0.78, trace=True)
        ok = ~ambiguous_frames(llr, tr, n)
        assert np.array_equal(B.unpack_bits(out[0], n)[ok], ref["final"][ok])
    finally:
        srv.close()


def test_cancel_queued_in_flight_and_completed_requests(setup):
    """Cancel a request still queued for memory, one on the GPU and one completed but not
    fetched: none of them is reported or fetchable, their memory and slots come back,
    and the other requests' results are unchanged."""
    import time
    torch, codes, stds = setup
    # a budget of about two 500-frame (127,k) requests: the rest queue
    srv = B.Server(codes, stds, 12, 0.78, budget_bytes=600_000, max_requests=8)
    try:
        n, k = 127, 64
        cw, llr = frames(n, k, 500, 2.0, 7200, ld=128)
        rids = [srv.submit(2, llr, 1, 0) for _ in range(5)]
        assert srv.stats()["queued"] >= 2
        srv.cancel(rids[4])      # still queued
        srv.cancel(rids[0])      # admitted first: on the GPU (or already done)
        got = {}
        for _ in range(20000):
            for r in srv.poll(timeout_us=2000):
                got[r] = srv.fetch(r) if r != rids[2] else None
            if all(r in got for r in (rids[1], rids[2], rids[3])):
                break
        assert set(got) == {rids[1], rids[2], rids[3]}
        srv.cancel(rids[2])      # completed, never fetched
        for r in (rids[0], rids[2], rids[4]):
            with pytest.raises(B.BchError):
                srv.fetch(r)
        with pytest.raises(B.BchError):
            srv.cancel(rids[4])  # already cancelled
        # the cancelled in-flight request is released once its completion is seen
        for _ in range(200):
            srv.poll(timeout_us=1000)
            if srv.stats()["bytes_in_use"] == 0:
                break
            time.sleep(0.005)
        st = srv.stats()
        assert st["bytes_in_use"] == 0 and st["cancelled"] == 3 and st["in_flight"] == 0
        assert np.array_equal(got[rids[1]][0], got[rids[3]][0])
        ref = O.hybrid(codes[2].dense(), stds[2].dense(), llr, O.draw_autos(n, 3, 1, 0, 500), 12, 0.78,
                       threads=None)
        tr = O.nms_enhanced(codes[2].dense(), llr, O.draw_autos(n, 3, 1, 0, 500), 12, 0.78, trace=True,
                            threads=None)
        ok = ~ambiguous_frames(llr, tr, n)
        assert np.array_equal(B.unpack_bits(got[rids[1]][0], n)[ok], ref["final"][ok])
    finally:
        srv.close()
