"""Pre-enqueued row chunks (RTC_FLAG_PRELAUNCH) through the C ABI: the kernels of
a Shack-Hartmann chunk enqueued ahead of its arrival, waiting on a page-locked
mailbox.  They give the same bits as ordinary launches and match the FP64
oracle; a chunk that does not match the prediction, pixels that must be
copied, a wait that runs out and an abandoned frame all fall back to ordinary
launches, and the loop's counters say which happened."""
import time

import numpy as np
import pytest

from oracle import OracleLoop
from paper_1903_01852_gb300 import synth
from parity_util import TOL_F32, WAIT_US, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available()
    return torch


def sh_loop(seed=501, fmt="f32"):
    """Three SH cameras of different shapes (subaperture rows of 6 to 10 pixels)
    and one pyramid, which is never pre-enqueued."""
    rng = np.random.default_rng(seed)
    wfs = [synth.sh_wfs(rng, 12, 8, 104, 100, 0.2, nblocks=4),
           synth.sh_wfs(rng, 9, 10, 96, 94, 0.0, nblocks=3),
           synth.sh_wfs(rng, 16, 6, 100, 99, 0.0, nblocks=4),
           synth.pyramid_wfs(rng, 10, 26, 24, 0.0, nblocks=2)]
    ns = sum(2 * synth.num_valid(w) for w in wfs)
    na = 157
    cfg = dict(name="prelaunch", na=na, ns=ns, wfs=wfs, M=synth.control_matrix(rng, na, ns, sd=1e-2), M_scale=None,
               M_dtype="f32", P=synth.polc_matrix(rng, na), P_scale=None, P_dtype="f32", gain=0.4, leak=0.02,
               clip=None, a0=rng.normal(0, 0.05, na).astype(np.float32),
               ref_slopes=rng.normal(0, 0.1, ns).astype(np.float32))
    if fmt != "f32":
        from oracle import quantize_rows
        codes, scale = quantize_rows(cfg["M"], fmt)
        pc, ps = quantize_rows(cfg["P"], fmt)
        cfg.update(M=codes, M_scale=scale, M_dtype=fmt, P=pc, P_scale=ps, P_dtype=fmt)
    return cfg


def in_place_buffers(torch, frames, where):
    """Each frame's WFS images in page-locked host ("host") or device memory, rows
    16-byte aligned with a pitch that is a multiple of 16 bytes, so that chunks are
    read in place."""
    out = []
    for f in frames:
        bufs = []
        for x in f:
            h, wd = x.shape
            wp = (wd + 7) // 8 * 8
            src = torch.from_numpy(np.ascontiguousarray(x).view(np.int16))
            if where == "host":
                t = torch.zeros((h, wp), dtype=torch.int16, pin_memory=True)
            else:
                t = torch.zeros((h, wp), dtype=torch.int16, device="cuda")
            t[:, :wd] = src.to(t.device)
            bufs.append(t[:, :wd])
        out.append(bufs)
    return out


def submit(loop, fid, bufs, plans, upto=None):
    """Chunks of all cameras interleaved (chunk c of every WFS, then c + 1); upto
    stops after that many chunk rounds."""
    n = max(len(p) for p in plans)
    for c in range(n if upto is None else upto):
        for w, plan in enumerate(plans):
            if c < len(plan):
                r0, r1 = plan[c]
                loop.submit(fid, w, r0, r1, bufs[w][r0:r1])


def expected_prelaunches(cfg, plans, frames_after_first):
    return frames_after_first * sum(len(p) - 1 for w, p in zip(cfg["wfs"], plans) if w["kind"] == "sh")


@pytest.mark.parametrize("where,fmt", [("host", "f32"), ("device", "f32"), ("host", "bf16"), ("host", "e4m3")])
def test_prelaunched_chunks_match_ordinary_launches_and_the_oracle(rtc, torch_cuda, where, fmt):
    cfg = sh_loop(fmt=fmt)
    frames = synth.draw_frames(cfg, 5, seed=502)
    plans = [synth.chunk_plan(w, 4) for w in cfg["wfs"]]
    bufs = in_place_buffers(torch_cuda, frames, where)
    ref = OracleLoop(cfg)
    with rtc.Loop(cfg, telemetry=True, prelaunch=True) as pre, rtc.Loop(cfg, telemetry=True) as plain:
        for k, f in enumerate(frames):
            submit(pre, k + 1, bufs[k], plans)
            submit(plain, k + 1, bufs[k], plans)
            (fa, a), (fb, b) = pre.get_commands(timeout_us=WAIT_US), plain.get_commands(timeout_us=WAIT_US)
            sa, sb = pre.get_telemetry(fa, timeout_us=WAIT_US)[0], plain.get_telemetry(fb, timeout_us=WAIT_US)[0]
            assert fa == fb == k + 1
            assert np.array_equal(a, b) and np.array_equal(sa, sb)
            s_ref, a_ref = ref.step(f)
            assert rel(sa, s_ref) <= TOL_F32 and rel(a, a_ref) <= TOL_F32
        info = pre.info()
        assert info["prelaunch_used"] == expected_prelaunches(cfg, plans, len(frames) - 1)
        assert info["prelaunch_cancelled"] == 0 and info["prelaunch_expired"] == 0
        assert plain.info()["prelaunch_used"] == 0
        assert pre.check_guards() == 0


def test_other_chunk_rows_and_pageable_pixels_cancel_the_prediction(rtc, torch_cuda):
    cfg = sh_loop(seed=511)
    frames = synth.draw_frames(cfg, 6, seed=512)
    four = [synth.chunk_plan(w, 4) for w in cfg["wfs"]]
    three = [synth.chunk_plan(w, 3) for w in cfg["wfs"]]
    bufs = in_place_buffers(torch_cuda, frames, "host")
    # frames 1-2 four chunks; 3 three chunks (predictions from 2 miss); 4 three chunks
    # (predicted right); 5 four chunks from pageable memory (must be copied); 6 four chunks
    sched = [(four, True), (four, True), (three, True), (three, True), (four, False), (four, True)]
    ref = OracleLoop(cfg)
    with rtc.Loop(cfg, prelaunch=True) as pre, rtc.Loop(cfg) as plain:
        for k, (f, (plans, pinned)) in enumerate(zip(frames, sched)):
            src = bufs[k] if pinned else [np.ascontiguousarray(x) for x in f]
            submit(pre, k + 1, src, plans)
            submit(plain, k + 1, src, plans)
            a, b = pre.get_commands(timeout_us=WAIT_US)[1], plain.get_commands(timeout_us=WAIT_US)[1]
            assert np.array_equal(a, b)
            assert rel(a, ref.step(f)[1]) <= TOL_F32
        info = pre.info()
        assert info["prelaunch_cancelled"] > 0 and info["prelaunch_expired"] == 0
        n4 = expected_prelaunches(cfg, four, 1)
        n3 = expected_prelaunches(cfg, three, 1)
        # used: every chunk after the first of frame 2 (predicted from 1) and of frame 4
        # (from 3); in frame 3 the chunks that frame 2 also had (a boundary both plans
        # share); none in frame 5 (copied) nor 6 (its predictions come from frame 5)
        shared = sum(1 for w, p3, p4 in zip(cfg["wfs"], three, four) if w["kind"] == "sh"
                     for c in range(1, len(p3)) if p3[c] in p4)
        assert info["prelaunch_used"] == n4 + n3 + shared
        assert pre.check_guards() == 0


def test_a_wait_that_runs_out_falls_back_to_ordinary_launches(rtc, torch_cuda):
    # the pre-enqueued kernels give up after 2 ms; the chunk arrives 50 ms later
    cfg = dict(sh_loop(seed=521), prelaunch_wait_us=2000)
    frames = synth.draw_frames(cfg, 3, seed=522)
    plans = [synth.chunk_plan(w, 4) for w in cfg["wfs"]]
    bufs = in_place_buffers(torch_cuda, frames, "host")
    ref = OracleLoop(cfg)
    with rtc.Loop(cfg, prelaunch=True) as pre, rtc.Loop(cfg) as plain:
        for k, f in enumerate(frames):
            if k == 1:
                submit(pre, k + 1, bufs[k], plans, upto=1)
                time.sleep(0.05)
                n = max(len(p) for p in plans)
                for c in range(1, n):
                    for w, plan in enumerate(plans):
                        if c < len(plan):
                            pre.submit(k + 1, w, *plan[c], bufs[k][w][plan[c][0]:plan[c][1]])
            else:
                submit(pre, k + 1, bufs[k], plans)
            submit(plain, k + 1, bufs[k], plans)
            a, b = pre.get_commands(timeout_us=WAIT_US)[1], plain.get_commands(timeout_us=WAIT_US)[1]
            assert np.array_equal(a, b)
            assert rel(a, ref.step(f)[1]) <= TOL_F32
        info = pre.info()
        nsh = sum(1 for w in cfg["wfs"] if w["kind"] == "sh")
        assert info["prelaunch_expired"] == nsh               # chunk 1 of every SH camera in frame 2
        assert info["prelaunch_used"] == expected_prelaunches(cfg, plans, 2) - nsh


def test_an_abandoned_frame_cancels_its_pending_kernels(rtc, torch_cuda):
    # waits of up to 1 s: the drop and the destroy below come first and cancel them
    cfg = dict(sh_loop(seed=531), prelaunch_wait_us=1_000_000)
    frames = synth.draw_frames(cfg, 4, seed=532)
    plans = [synth.chunk_plan(w, 4) for w in cfg["wfs"]]
    bufs = in_place_buffers(torch_cuda, frames, "host")
    with rtc.Loop(cfg, prelaunch=True) as pre, rtc.Loop(cfg) as plain:
        for lp in (pre, plain):
            submit(lp, 1, bufs[0], plans)
            lp.get_commands(timeout_us=WAIT_US)
            submit(lp, 2, bufs[1], plans, upto=2)            # frame 2 never completes
        with pytest.raises(TimeoutError):                     # its pixels are not all in
            pre.get_commands(timeout_us=100_000)
        for lp in (pre, plain):
            assert lp.submit(3, 0, *plans[0][0], bufs[2][0][plans[0][0][0]:plans[0][0][1]]) == rtc.RTC_EDROPPED
            for c in range(max(len(p) for p in plans)):
                for w, plan in enumerate(plans):
                    if c < len(plan) and (c, w) != (0, 0):
                        lp.submit(3, w, *plan[c], bufs[2][w][plan[c][0]:plan[c][1]])
        a, b = pre.get_commands(timeout_us=WAIT_US), plain.get_commands(timeout_us=WAIT_US)
        assert a[0] == b[0] == 3 and np.array_equal(a[1], b[1])
        info = pre.info()
        nsh = sum(1 for w in cfg["wfs"] if w["kind"] == "sh")
        assert info["frames_dropped"] == 1 and info["prelaunch_cancelled"] == nsh
        # frame 4 goes half way; destroying the loop cancels what waits for the rest (before
        # the other loop is destroyed: its cudaFree waits for all work on the device)
        submit(pre, 4, bufs[3], plans, upto=2)
        assert pre.info()["prelaunch_expired"] == 0
        t0 = time.perf_counter()
        pre.close()
        assert time.perf_counter() - t0 < 0.5


@pytest.mark.parametrize("prelaunch", [False, True])
def test_batched_rounds_equal_chunk_by_chunk_submission(rtc, torch_cuda, prelaunch):
    # rtc_submit_pixels_n: one call per round of chunks (chunk c of every camera)
    cfg = sh_loop(seed=541)
    frames = synth.draw_frames(cfg, 4, seed=542)
    plans = [synth.chunk_plan(w, 4) for w in cfg["wfs"]]
    bufs = in_place_buffers(torch_cuda, frames, "host")
    n = max(len(p) for p in plans)
    with rtc.Loop(cfg, prelaunch=prelaunch) as batched, rtc.Loop(cfg) as single:
        for k in range(len(frames)):
            for c in range(n):
                items = [(w, *p[c], bufs[k][w][p[c][0]:p[c][1]]) for w, p in enumerate(plans) if c < len(p)]
                assert batched.submit_chunks(batched.chunks(k + 1, items)) == rtc.RTC_OK
            submit(single, k + 1, bufs[k], plans)
            a, b = batched.get_commands(timeout_us=WAIT_US), single.get_commands(timeout_us=WAIT_US)
            assert a[0] == b[0] == k + 1 and np.array_equal(a[1], b[1])
        if prelaunch:
            assert batched.info()["prelaunch_used"] == expected_prelaunches(cfg, plans, len(frames) - 1)


def test_a_batch_stops_at_its_first_bad_chunk(rtc, torch_cuda):
    import ctypes as C
    cfg = sh_loop(seed=551)
    frames = synth.draw_frames(cfg, 1, seed=552)
    plans = [synth.chunk_plan(w, 2) for w in cfg["wfs"]]
    bufs = in_place_buffers(torch_cuda, frames, "host")[0]
    with rtc.Loop(cfg) as lp:
        # WFS 0 chunk 0, WFS 0 chunk 0 again (rows out of order), WFS 1 chunk 0
        items = [(0, *plans[0][0], bufs[0][plans[0][0][0]:plans[0][0][1]]),
                 (0, *plans[0][0], bufs[0][plans[0][0][0]:plans[0][0][1]]),
                 (1, *plans[1][0], bufs[1][plans[1][0][0]:plans[1][0][1]])]
        arr = lp.chunks(1, items)
        acc = C.c_int32(-1)
        assert rtc.lib.rtc_submit_pixels_n(lp._h, arr, 3, C.byref(acc)) == rtc.RTC_EORDER
        assert acc.value == 1
        # the rest of the frame, then its commands are complete and correct
        rest = [(w, *p[c], bufs[w][p[c][0]:p[c][1]]) for c in range(2) for w, p in enumerate(plans)
                if c < len(p) and (w, c) != (0, 0)]
        assert lp.submit_chunks(lp.chunks(1, rest)) == rtc.RTC_OK
        fid, a = lp.get_commands(timeout_us=WAIT_US)
        assert fid == 1 and rel(a, OracleLoop(cfg).step(frames[0])[1]) <= TOL_F32


def test_prelaunch_across_a_parameter_swap(rtc, torch_cuda):
    # the swap applies at a frame boundary, where no pre-enqueued chunk is pending
    from oracle import stored_matrix
    cfg = sh_loop(seed=561)
    rng = np.random.default_rng(562)
    M2 = synth.control_matrix(rng, cfg["na"], cfg["ns"], sd=1e-2)
    frames = synth.draw_frames(cfg, 6, seed=563)
    plans = [synth.chunk_plan(w, 4) for w in cfg["wfs"]]
    bufs = in_place_buffers(torch_cuda, frames, "host")
    ref = OracleLoop(cfg)
    with rtc.Loop(cfg, updatable=True, prelaunch=True) as pre, rtc.Loop(cfg, updatable=True) as plain:
        for k, f in enumerate(frames):
            if k == 3:
                for lp in (pre, plain):
                    lp.update(M=M2, control=(0.3, 0.05, None))
                ref.cfg = dict(cfg, M=M2, gain=0.3, leak=0.05)
                ref.m = stored_matrix(M2, "f32", None)
            submit(pre, k + 1, bufs[k], plans)
            submit(plain, k + 1, bufs[k], plans)
            a, b = pre.get_commands(timeout_us=WAIT_US)[1], plain.get_commands(timeout_us=WAIT_US)[1]
            assert np.array_equal(a, b)
            assert rel(a, ref.step(f)[1]) <= TOL_F32
        assert pre.info()["swaps"] == 1
        assert pre.info()["prelaunch_used"] == expected_prelaunches(cfg, plans, len(frames) - 1)


def test_prelaunch_in_a_shard_loop(rtc, torch_cuda):
    # a RTC_FLAG_PARTIAL loop (one WFS group of a split loop): its partial reconstruction
    cfg = dict(sh_loop(seed=571), P=None, P_scale=None)
    frames = synth.draw_frames(cfg, 4, seed=572)
    plans = [synth.chunk_plan(w, 4) for w in cfg["wfs"]]
    bufs = in_place_buffers(torch_cuda, frames, "host")
    with rtc.Loop(cfg, partial=True, prelaunch=True) as pre, rtc.Loop(cfg, partial=True) as plain:
        for k in range(len(frames)):
            submit(pre, k + 1, bufs[k], plans)
            submit(plain, k + 1, bufs[k], plans)
            a, b = pre.get_commands(timeout_us=WAIT_US)[1], plain.get_commands(timeout_us=WAIT_US)[1]
            assert np.array_equal(a, b)
        assert pre.info()["prelaunch_used"] == expected_prelaunches(cfg, plans, len(frames) - 1)


def test_a_batch_that_starts_a_new_frame_drops_the_incomplete_one(rtc, torch_cuda):
    import ctypes as C
    cfg = dict(sh_loop(seed=581), prelaunch_wait_us=1_000_000)
    frames = synth.draw_frames(cfg, 3, seed=582)
    plans = [synth.chunk_plan(w, 3) for w in cfg["wfs"]]
    bufs = in_place_buffers(torch_cuda, frames, "host")
    n = max(len(p) for p in plans)
    rounds = lambda k, fid: [rtc.Loop.chunks(fid, [(w, *p[c], bufs[k][w][p[c][0]:p[c][1]])
                                                   for w, p in enumerate(plans) if c < len(p)]) for c in range(n)]
    with rtc.Loop(cfg, prelaunch=True) as pre, rtc.Loop(cfg) as plain:
        for lp in (pre, plain):
            for arr in rounds(0, 1):
                assert lp.submit_chunks(arr) == rtc.RTC_OK
            lp.get_commands(timeout_us=WAIT_US)
            assert lp.submit_chunks(rounds(1, 2)[0]) == rtc.RTC_OK        # frame 2: first round only
        # frame 3's first round drops frame 2 and is accepted whole
        for lp in (pre, plain):
            arr = rounds(2, 3)[0]
            acc = C.c_int32(-1)
            assert rtc.lib.rtc_submit_pixels_n(lp._h, arr, len(arr), C.byref(acc)) == rtc.RTC_EDROPPED
            assert acc.value == len(arr)
            for arr in rounds(2, 3)[1:]:
                assert lp.submit_chunks(arr) == rtc.RTC_OK
        a, b = pre.get_commands(timeout_us=WAIT_US), plain.get_commands(timeout_us=WAIT_US)
        assert a[0] == b[0] == 3 and np.array_equal(a[1], b[1])
        info = pre.info()
        nsh = sum(1 for w in cfg["wfs"] if w["kind"] == "sh")
        assert info["frames_dropped"] == 1 and info["prelaunch_cancelled"] == nsh and info["prelaunch_expired"] == 0


def test_prelaunch_with_explicit_polc(rtc, torch_cuda):
    # explicit POLC: the slope kernel adds u = D a to every slope, the pre-enqueued one too
    cfg = sh_loop(seed=591)
    rng = np.random.default_rng(592)
    cfg = dict(cfg, P=None, P_scale=None, polc="explicit",
               D=synth.interaction_matrix(rng, cfg["ns"], cfg["na"], m_sd=1e-2))   # M is N(0, 1e-4) here
    frames = synth.draw_frames(cfg, 4, seed=593)
    plans = [synth.chunk_plan(w, 4) for w in cfg["wfs"]]
    bufs = in_place_buffers(torch_cuda, frames, "host")
    ref = OracleLoop(cfg)
    with rtc.Loop(cfg, telemetry=True, prelaunch=True) as pre, rtc.Loop(cfg, telemetry=True) as plain:
        for k, f in enumerate(frames):
            submit(pre, k + 1, bufs[k], plans)
            submit(plain, k + 1, bufs[k], plans)
            (fa, a), (fb, b) = pre.get_commands(timeout_us=WAIT_US), plain.get_commands(timeout_us=WAIT_US)
            sa, sb = pre.get_telemetry(fa, timeout_us=WAIT_US)[0], plain.get_telemetry(fb, timeout_us=WAIT_US)[0]
            assert np.array_equal(a, b) and np.array_equal(sa, sb)
            s_ref, a_ref = ref.step(f)
            assert rel(sa, s_ref) <= TOL_F32 and rel(a, a_ref) <= TOL_F32
        assert pre.info()["prelaunch_used"] == expected_prelaunches(cfg, plans, len(frames) - 1)
