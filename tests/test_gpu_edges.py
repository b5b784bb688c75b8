"""Edge cases of the CUDA path against the FP64 oracle, through the C ABI: the
largest WFS count, sensors with no valid unit, one column block per slope row,
a single actuator, frame ids at the top of their range, slope threads with more
pixel rows than the host-pixel kernel keeps in flight."""
import os
import subprocess
import sys
import textwrap

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


ROWS_BEYOND_SCRIPT = textwrap.dedent("""
    import numpy as np, torch
    from oracle import OracleLoop
    from paper_1903_01852_gb300 import binding as rtc, synth
    rng = np.random.default_rng(211)
    w = synth.sh_wfs(rng, 24, 24, 600, 590, 0.0, nblocks=3)
    ns = 2 * synth.num_valid(w)
    na = 41
    cfg = dict(name="rows_beyond", na=na, ns=ns, wfs=[w], M=synth.control_matrix(rng, na, ns, sd=1e-2),
               M_scale=None, M_dtype="f32", P=synth.polc_matrix(rng, na), P_scale=None, P_dtype="f32", gain=0.4,
               leak=0.02, clip=None, a0=None, ref_slopes=rng.normal(0, 0.05, ns).astype(np.float32))
    frames = synth.draw_frames(cfg, 3, seed=212)
    plans = [synth.chunk_plan(w, 4)]
    ora = OracleLoop(cfg)
    worst = 0.0
    with rtc.Loop(cfg, telemetry=True) as a, rtc.Loop(cfg, telemetry=True) as c:
        for k, f in enumerate(frames):
            x = f[0]
            h, wd = x.shape
            t = torch.zeros((h, (wd + 7) // 8 * 8), dtype=torch.int16, pin_memory=True)
            t.numpy()[:, :wd] = x.view(np.int16)
            d = torch.zeros((h, (wd + 7) // 8 * 8), dtype=torch.int16, device="cuda")
            d[:, :wd] = torch.from_numpy(x.view(np.int16)).cuda()
            a.submit_frame(k + 1, [t[:, :wd]], plans)
            c.process_frame(k + 1, [d[:, :wd]])
            (fa, ca), (fc, cc) = a.get_commands(timeout_us=30_000_000), c.get_commands(timeout_us=30_000_000)
            sa, sc = a.get_telemetry(fa, timeout_us=30_000_000)[0], c.get_telemetry(fc, timeout_us=30_000_000)[0]
            assert fa == fc == k + 1 and np.array_equal(ca, cc) and np.array_equal(sa, sc)
            s_ref, a_ref = ora.step(f)
            rel = lambda u, v: float(np.max(np.abs(u - v)) / max(np.max(np.abs(v)), 1e-30))
            worst = max(worst, rel(sc, s_ref), rel(cc, a_ref))
    assert worst <= 1e-5, worst
    print("ok", worst)
""")


def test_host_pixel_rows_beyond_the_in_flight_window(torch_cuda, tmp_path):
    # The host-pixel slope kernel keeps at most 12 pixel rows of a thread in flight
    # and the default part split never gives a thread more; a build allowing 30
    # rows per thread runs the rest of that path: 24-pixel subapertures read in
    # place from page-locked row chunks (24 rows per thread) against device frames.
    from paper_1903_01852_gb300.build import build
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    lib = build(defines=["RTC_SLOPE_ROWS_PER_THREAD=30"], out=str(tmp_path / "librtc.so"))
    env = dict(os.environ, RTC_LIBRARY=lib, PYTHONPATH=root + os.pathsep + os.environ.get("PYTHONPATH", ""))
    r = subprocess.run([sys.executable, "-c", ROWS_BEYOND_SCRIPT], env=env, capture_output=True, text=True,
                       timeout=600, cwd=root)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-3000:]
    assert r.stdout.startswith("ok")


def test_lowest_stream_priority_gives_the_same_commands(rtc, torch_cuda):
    # priority only orders the scheduling of CTAs among loops; a loop at a priority
    # beyond the device's range (clamped to its lowest) computes the same bits
    cfg = synth.make_config("scao_small", polc=True)
    frames = synth.draw_frames(cfg, 3, seed=271)
    with rtc.Loop(dict(cfg, priority=100)) as low, rtc.Loop(cfg) as high:
        for k, f in enumerate(frames):
            low.submit_frame(k + 1, f)
            high.submit_frame(k + 1, f)
            assert np.array_equal(low.get_commands(timeout_us=WAIT_US)[1], high.get_commands(timeout_us=WAIT_US)[1])


GROUPED_SCRIPT = textwrap.dedent("""
    import sys, numpy as np
    sys.path.insert(0, "tests")
    from oracle import quantize_rows
    from paper_1903_01852_gb300 import binding as rtc, synth
    from parity_util import device_frames
    from test_gpu_parity import ragged_config
    out = {}
    for fmt in ("f32", "bf16", "e4m3"):
        cfg = ragged_config(seed=281)
        if fmt != "f32":
            codes, scale = quantize_rows(cfg["M"], fmt)
            pc, ps = quantize_rows(cfg["P"], fmt)
            cfg.update(M=codes, M_scale=scale, M_dtype=fmt, P=pc, P_scale=ps, P_dtype=fmt)
        frames = synth.draw_frames(cfg, 3, seed=282)
        with rtc.Loop(cfg) as whole, rtc.Loop(cfg) as chunked:
            for k, f in enumerate(frames):
                whole.process_frame(k + 1, device_frames(f))
                chunked.submit_frame(k + 1, f, [synth.chunk_plan(w, 3) for w in cfg["wfs"]])
                out[f"{fmt}_whole_{k}"] = whole.get_commands(timeout_us=30_000_000)[1]
                out[f"{fmt}_chunked_{k}"] = chunked.get_commands(timeout_us=30_000_000)[1]
    np.savez(sys.argv[1], **out)
""")


def test_grouped_mvm_gives_the_bits_of_one_block_per_cta(torch_cuda, tmp_path):
    # A build whose MVM CTAs always take several consecutive column blocks (2 for
    # float32, 3 for BF16, 4 for E4M3; the last group of a launch shorter) against
    # the default build, on a ragged loop submitted whole and in row chunks: the
    # per-block sums and the finalisation are the same, so the commands are too.
    from paper_1903_01852_gb300.build import build
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    lib = build(defines=["RTC_GEMV_GROUP_MIN_WAVES=0", "RTC_GEMV_GROUP_F32=2", "RTC_GEMV_GROUP_BF16=3",
                         "RTC_GEMV_GROUP_E4M3=4", "RTC_GEMV_MIN_WAVES=0"], out=str(tmp_path / "librtc.so"))
    res = {}
    for name, env_lib in (("grouped", lib), ("default", None)):
        env = dict(os.environ, PYTHONPATH=root + os.pathsep + os.environ.get("PYTHONPATH", ""))
        env.pop("RTC_LIBRARY", None)
        if env_lib:
            env["RTC_LIBRARY"] = env_lib
        path = str(tmp_path / f"{name}.npz")
        r = subprocess.run([sys.executable, "-c", GROUPED_SCRIPT, path], env=env, capture_output=True, text=True,
                           timeout=600, cwd=root)
        assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-3000:]
        res[name] = dict(np.load(path))
    assert res["grouped"].keys() == res["default"].keys() and len(res["default"]) == 18
    for k in res["default"]:
        assert np.array_equal(res["grouped"][k], res["default"][k]), k
