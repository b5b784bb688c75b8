"""Edge cases of the CUDA path against the FP64 oracle, through the C ABI: the
largest WFS count, sensors with no valid unit, one column block per slope row,
a single actuator, frame ids at the top of their range."""
import numpy as np
import pytest

from oracle import OracleLoop
from paper_1903_01852_gb300 import synth
from parity_util import TOL_F32, WAIT_US, rel, run_pair

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available()
    return torch


def loop_config(wfs, na, seed, polc=True, ref=True):
    rng = np.random.default_rng(seed)
    ns = sum(2 * synth.num_valid(w) for w in wfs)
    return dict(name="edge", na=na, ns=ns, wfs=wfs, M=synth.control_matrix(rng, na, ns, sd=1e-2), M_scale=None,
                M_dtype="f32", P=synth.polc_matrix(rng, na) if polc else None, P_scale=None, P_dtype="f32",
                gain=0.45, leak=0.02, clip=None, a0=rng.normal(0, 0.1, na).astype(np.float32),
                ref_slopes=rng.normal(0, 0.1, ns).astype(np.float32) if ref else None)


def sixteen_wfs(seed=201):
    """The largest loop the ABI takes: 12 SH and 4 pyramid WFS of assorted shapes."""
    rng = np.random.default_rng(seed)
    wfs = []
    for k in range(12):
        n, npx = 3 + k % 5, 4 + k % 4
        wfs.append(synth.sh_wfs(rng, n, npx, n * npx + 3 + k, n * npx + 1 + k % 3, 0.0,
                                nblocks=1 + k % min(n, 3)))
    for k in range(4):
        p = 5 + 2 * k
        w = synth.pyramid_wfs(rng, p, 2 * p + 6, 2 * p + 4, 0.0, nblocks=1 + k % 3)
        if k % 2:
            w["norm"] = "global"
        wfs.append(w)
    return wfs


@pytest.mark.parametrize("nchunks", [1, 2, 5])
def test_sixteen_wfs_loop(rtc, torch_cuda, nchunks):
    cfg = loop_config(sixteen_wfs(), 43, seed=202)
    assert len(cfg["wfs"]) == 16
    frames = synth.draw_frames(cfg, 3, seed=203)
    with rtc.Loop(cfg, telemetry=True) as loop:
        run_pair(loop, cfg, frames, nchunks=nchunks)


def test_sensors_without_any_valid_unit(rtc, torch_cuda):
    rng = np.random.default_rng(211)
    dead_sh = synth.sh_wfs(rng, 4, 6, 24, 24, 0.0, nblocks=2)
    dead_sh["valid"][:] = 0
    dead_pyr = synth.pyramid_wfs(rng, 7, 18, 18, 0.0, nblocks=3)
    dead_pyr["valid"][:] = 0
    dead_pyr["norm"] = "global"
    live = synth.sh_wfs(rng, 5, 6, 31, 30, 0.0, nblocks=2)
    cfg = loop_config([dead_sh, live, dead_pyr], 19, seed=212)
    assert cfg["ns"] == 2 * synth.num_valid(live)
    frames = synth.draw_frames(cfg, 3, seed=213)
    for mode in ("chunked", "device"):
        with rtc.Loop(cfg, telemetry=True) as loop:
            run_pair(loop, cfg, frames, mode=mode, nchunks=3)


def test_one_column_block_per_slope_row(rtc, torch_cuda):
    rng = np.random.default_rng(221)
    sh = synth.sh_wfs(rng, 9, 6, 56, 55, 0.2, nblocks=9)
    pyr = synth.pyramid_wfs(rng, 11, 30, 28, 0.0, nblocks=11)
    pyr_g = synth.pyramid_wfs(rng, 6, 16, 16, 0.0, nblocks=6)
    pyr_g["norm"] = "global"
    cfg = loop_config([sh, pyr, pyr_g], 31, seed=222)
    frames = synth.draw_frames(cfg, 3, seed=223)
    outs = []
    for plans in ("rows", "whole"):
        with rtc.Loop(cfg, telemetry=True) as loop:
            ref = OracleLoop(cfg)
            cm = []
            for k, f in enumerate(frames):
                p = [[(r, r + 1) for r in range(x.shape[0])] for x in f] if plans == "rows" else None
                loop.submit_frame(k + 1, f, p)
                cm.append(loop.get_commands(timeout_us=WAIT_US)[1])
                s, _ = loop.get_telemetry(k + 1, timeout_us=WAIT_US)
                s_ref, a_ref = ref.step(f)
                assert rel(s, s_ref) <= TOL_F32 and rel(cm[-1], a_ref) <= TOL_F32
            outs.append(cm)
    assert all(np.array_equal(x, y) for x, y in zip(*outs))


def test_single_actuator_and_single_subaperture(rtc, torch_cuda):
    rng = np.random.default_rng(231)
    w = synth.sh_wfs(rng, 1, 7, 9, 8, 0.0, ox=1, oy=0)
    cfg = loop_config([w], 1, seed=232)
    frames = synth.draw_frames(cfg, 5, seed=233)
    for fmt in ("f32", "bf16", "e4m3"):
        c = dict(cfg)
        if fmt != "f32":
            from oracle import quantize_rows
            codes, scale = quantize_rows(cfg["M"], fmt)
            pc, ps = quantize_rows(cfg["P"], fmt)
            c.update(M=codes, M_scale=scale, M_dtype=fmt, P=pc, P_scale=ps, P_dtype=fmt)
        with rtc.Loop(c, telemetry=True) as loop:
            run_pair(loop, c, frames, nchunks=2)


def test_frame_ids_at_the_top_of_the_range(rtc, torch_cuda):
    cfg = synth.make_config("scao_small")
    frames = synth.draw_frames(cfg, 3, seed=241)
    top = (1 << 64) - 4
    with rtc.Loop(cfg, telemetry=True) as loop:
        run_pair(loop, cfg, frames, first_id=top)
        with pytest.raises(rtc.RtcError, match="EORDER"):
            loop.submit_frame(top, frames[0])          # not increasing


def test_graph_mode_frame_timing_spans_the_launch(rtc, torch_cuda):
    cfg = synth.make_config("scao_small", polc=True)
    frames = synth.draw_frames(cfg, 3, seed=261)
    with rtc.Loop(cfg, graphs=True, timing=True, telemetry=True, ring=2) as g, rtc.Loop(cfg) as d:
        for k, f in enumerate(frames):
            for b, x in zip(g.next_frame_buffers(), f):
                b[:] = x
            g.submit_graph(k + 1)
            d.submit_frame(k + 1, f)
            assert np.array_equal(g.get_commands(timeout_us=WAIT_US)[1], d.get_commands(timeout_us=WAIT_US)[1])
            t = g.get_timing(k + 1, timeout_us=WAIT_US)
            assert t["latency_us"] > 0 and t["frame_us"] >= t["latency_us"] and t["polc_us"] >= 0


def test_server_release_while_another_thread_submits(rtc, torch_cuda):
    import threading
    import time
    cfg = synth.make_config("scao_small")
    budget = 2 * rtc.footprint(cfg, flags=rtc.RTC_FLAG_GRAPHS)[0]
    with rtc.Server(budget) as srv:
        lid = srv.admit(cfg)
        errors, count = [], [0]

        def submitter():
            fid = 1
            while True:
                try:
                    srv.submit(lid, fid)
                except rtc.RtcError as e:
                    if "ENOENT" not in str(e):
                        errors.append(e)
                    return
                fid += 1
                count[0] += 1

        th = threading.Thread(target=submitter)
        th.start()
        time.sleep(0.05)
        srv.release(lid)                      # waits for a submit in progress, then destroys the loop
        th.join(timeout=30)
        assert not th.is_alive() and not errors and count[0] > 0
        assert srv.usage()["used"] == 0
