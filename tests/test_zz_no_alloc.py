"""rtc_reconstruct_noalloc through the C ABI, against the FP64 oracle and the loop.

That entry point is for callers that must not allocate device memory while they
run: a hard real-time control thread cannot afford a cudaMalloc inside its frame
(it may synchronise the device and has no latency bound), and code hosted in a
framework that owns every device allocation is not allowed to make one.  It
keeps its partial sums in a fixed array inside the library instead.

Here it is fed the slopes a loop measured, frame after frame, and must give the
oracle's commands for those slopes (and the loop's own commands) within the
float32 parity tolerance, on consecutive calls that carry the integrator state
from one call to the next; and, on a ragged size with row scales, a POLC term
and separate input and output state buffers, the float64 product of the
definition.

This file is named so that pytest collects it last.
"""
import ctypes as C

import numpy as np
import pytest

from oracle import control_step, mvm
from paper_1903_01852_gb300 import synth
from parity_util import TOL_F32, WAIT_US, rel

pytestmark = pytest.mark.gpu


def _ptr(t):
    return None if t is None else t.data_ptr()


def _call(rtc, torch, na, ns, M, ld, scale, s, q, a_in, a_out, gain, leak):
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return rtc.lib.rtc_reconstruct_noalloc(na, ns, M.data_ptr(), ld, _ptr(scale), s.data_ptr(), _ptr(q),
                                           a_in.data_ptr(), a_out.data_ptr(), gain, leak, stream)


def test_noalloc_step_matches_oracle_and_loop_on_consecutive_calls(rtc):
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available()
    cfg = synth.make_config("elt_scao_sh")          # 5316 x 8608: several column splits and a ragged last split
    na, ns = cfg["na"], cfg["ns"]
    frames = synth.draw_frames(cfg, 2, seed=7)
    measured = []
    with rtc.Loop(cfg, telemetry=True) as loop:
        for k, f in enumerate(frames):
            loop.submit_frame(k + 1, f)
            fid, a = loop.get_commands(timeout_us=WAIT_US)
            s, _ = loop.get_telemetry(fid, timeout_us=WAIT_US)
            measured.append((s, a))

    M = torch.from_numpy(cfg["M"]).cuda()
    m64 = cfg["M"].astype(np.float64)
    s_dev = torch.empty(ns, dtype=torch.float32, device="cuda")
    a_dev = torch.zeros(na, dtype=torch.float32, device="cuda")
    a_ref = np.zeros(na)
    for s, a_loop in measured:
        s_dev.copy_(torch.from_numpy(s))
        rc = _call(rtc, torch, na, ns, M, M.stride(0), None, s_dev, None, a_dev, a_dev, cfg["gain"], cfg["leak"])
        assert rc == rtc.RTC_OK
        torch.cuda.synchronize()
        got = a_dev.cpu().numpy()
        a_ref = control_step(a_ref, mvm(m64, s), np.zeros(na), cfg["gain"], cfg["leak"])
        assert rel(got, a_ref) <= TOL_F32
        assert rel(got, a_loop) <= TOL_F32


def test_noalloc_ragged_with_row_scale_polc_term_and_separate_state(rtc):
    # ns = 2053: three column splits of 688 columns, the last one 677 wide (not a
    # multiple of four: scalar tail); rows padded to ld = 2056 floats.
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(2053)
    na, ns, ld = 301, 2053, 2056
    Mp = np.zeros((na, ld), np.float32)
    Mp[:, :ns] = rng.standard_normal((na, ns)).astype(np.float32)
    scale = rng.uniform(0.5, 2.0, na).astype(np.float32) * np.float32(1e-3)
    q = [rng.normal(0, 0.05, na).astype(np.float32) for _ in range(2)]
    slopes = [rng.normal(0, 1.0, ns).astype(np.float32) for _ in range(2)]
    gain, leak = 0.4, 0.02
    a0 = rng.normal(0, 0.1, na).astype(np.float32)

    M = torch.from_numpy(Mp).cuda()
    sc = torch.from_numpy(scale).cuda()
    bufs = [torch.from_numpy(a0).cuda(), torch.zeros(na, dtype=torch.float32, device="cuda"),
            torch.zeros(na, dtype=torch.float32, device="cuda")]
    m64 = Mp[:, :ns].astype(np.float64) * scale.astype(np.float64)[:, None]
    a_ref = a0.astype(np.float64)
    for k in range(2):
        s_dev = torch.from_numpy(slopes[k]).cuda()
        q_dev = torch.from_numpy(q[k]).cuda()
        rc = _call(rtc, torch, na, ns, M, ld, sc, s_dev, q_dev, bufs[k], bufs[k + 1], gain, leak)
        assert rc == rtc.RTC_OK
        torch.cuda.synchronize()
        a_ref = control_step(a_ref, mvm(m64, slopes[k]), q[k], gain, leak)
        assert rel(bufs[k + 1].cpu().numpy(), a_ref) <= TOL_F32
    assert np.array_equal(bufs[0].cpu().numpy(), a0)      # the input state is only read


def test_noalloc_rejects_sizes_beyond_its_scratch_and_bad_pointers(rtc):
    torch = pytest.importorskip("torch")
    buf = torch.zeros(64, dtype=torch.float32, device="cuda")
    p = buf.data_ptr()
    too_many = 2097152 + 1                       # RTC_NOALLOC_MAX_FLOATS + 1 rows
    assert rtc.lib.rtc_reconstruct_noalloc(too_many, 4, p, 4, None, p, None, p, p, 0.5, 0.01, None) == rtc.RTC_EINVAL
    assert rtc.lib.rtc_reconstruct_noalloc(4, 4, p + 4, 4, None, p, None, p, p, 0.5, 0.01, None) == rtc.RTC_EINVAL
    assert rtc.lib.rtc_reconstruct_noalloc(4, 6, p, 6, None, p, None, p, p, 0.5, 0.01, None) == rtc.RTC_EINVAL
