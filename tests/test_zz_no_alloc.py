"""rtc_reconstruct_noalloc reproduces the loop's own commands, through the C ABI.

That entry point is for callers that must not allocate device memory while they
run: a hard real-time control thread cannot afford a cudaMalloc inside its frame
(it may synchronise the device and has no latency bound), and code hosted in a
framework that owns every device allocation is not allowed to make one.  It
keeps its partial sums in a fixed array inside the library instead.  Here it is
fed the slopes a loop measured, frame after frame, and must give the commands
that loop produced, within the float32 parity tolerance, on consecutive calls
that carry the integrator state from one call to the next.

This file is named so that pytest collects it last.
"""
import ctypes as C

import numpy as np
import pytest

from paper_1903_01852_gb300 import synth
from parity_util import TOL_F32, WAIT_US, rel

pytestmark = pytest.mark.gpu


def test_noalloc_step_matches_loop_commands_on_consecutive_calls(rtc):
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
    s_dev = torch.empty(ns, dtype=torch.float32, device="cuda")
    a_dev = torch.zeros(na, dtype=torch.float32, device="cuda")
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for s, a_loop in measured:
        s_dev.copy_(torch.from_numpy(s))
        rc = rtc.lib.rtc_reconstruct_noalloc(na, ns, M.data_ptr(), M.stride(0), None, s_dev.data_ptr(), None,
                                             a_dev.data_ptr(), a_dev.data_ptr(), cfg["gain"], cfg["leak"], stream)
        assert rc == rtc.RTC_OK
        torch.cuda.synchronize()
        assert rel(a_dev.cpu().numpy(), a_loop) <= TOL_F32


def test_noalloc_rejects_sizes_beyond_its_scratch_and_bad_pointers(rtc):
    torch = pytest.importorskip("torch")
    buf = torch.zeros(64, dtype=torch.float32, device="cuda")
    p = buf.data_ptr()
    too_many = 2097152 + 1                       # RTC_NOALLOC_MAX_FLOATS + 1 rows
    assert rtc.lib.rtc_reconstruct_noalloc(too_many, 4, p, 4, None, p, None, p, p, 0.5, 0.01, None) == rtc.RTC_EINVAL
    assert rtc.lib.rtc_reconstruct_noalloc(4, 4, p + 4, 4, None, p, None, p, p, 0.5, 0.01, None) == rtc.RTC_EINVAL
    assert rtc.lib.rtc_reconstruct_noalloc(4, 6, p, 6, None, p, None, p, p, 0.5, 0.01, None) == rtc.RTC_EINVAL
