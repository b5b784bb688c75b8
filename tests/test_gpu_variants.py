"""Variants of the hot path against the FP64 oracle, through the C ABI: global
pyramid normalisation and explicit pseudo-open-loop control (Section 3.4)."""
import copy

import numpy as np
import pytest

from oracle import OracleLoop, quantize_rows
from paper_1903_01852_gb300 import synth
from parity_util import TOL_F32, WAIT_US, device_frames, rel, run_pair

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available()
    return torch


def ragged_global_config(seed=61):
    """Two pyramids (one normalised globally, ragged and split in 5 blocks) beside
    an SH WFS, with reference slopes and POLC."""
    rng = np.random.default_rng(seed)
    w1 = synth.pyramid_wfs(rng, 13, 37, 34, 0.0, qx=[1, 19, 2, 20], qy=[0, 1, 17, 18], nblocks=5)
    w1["norm"] = "global"
    w1["valid"][4, :] = 0                                                  # a pupil row with no valid pixel
    w2 = synth.sh_wfs(rng, 7, 5, 45, 39, 0.3, ox=3, oy=2, nblocks=3)
    w3 = synth.pyramid_wfs(rng, 9, 24, 24, 0.2, nblocks=2)
    wfs = [w1, w2, w3]
    ns = sum(2 * synth.num_valid(w) for w in wfs)
    na = 29
    return dict(name="ragged_global", na=na, ns=ns, wfs=wfs, M=synth.control_matrix(rng, na, ns, sd=1e-2),
                M_scale=None, M_dtype="f32", P=synth.polc_matrix(rng, na), P_scale=None, P_dtype="f32",
                gain=0.4, leak=0.02, clip=None, a0=rng.normal(0, 0.1, na).astype(np.float32),
                ref_slopes=rng.normal(0, 0.1, ns).astype(np.float32))


# ------------------------------------------------------------------ global pyramid normalisation

@pytest.mark.parametrize("nchunks", [1, 3, 8])
def test_global_norm_ragged_chunked(rtc, torch_cuda, nchunks):
    cfg = ragged_global_config()
    frames = synth.draw_frames(cfg, 4, seed=62)
    with rtc.Loop(cfg, telemetry=True) as loop:
        run_pair(loop, cfg, frames, nchunks=nchunks)


def test_global_norm_row_by_row_device_and_graph_equal_bitwise(rtc, torch_cuda):
    cfg = ragged_global_config(seed=63)
    frames = synth.draw_frames(cfg, 3, seed=64)
    outs = []
    with rtc.Loop(cfg, telemetry=True) as loop:
        cm = []
        for k, f in enumerate(frames):
            loop.submit_frame(k + 1, f, [[(r, r + 1) for r in range(x.shape[0])] for x in f])
            cm.append(loop.get_commands(timeout_us=WAIT_US)[1])
        outs.append(cm)
    with rtc.Loop(cfg, telemetry=True) as loop:
        outs.append(run_pair(loop, cfg, frames, mode="device")[1])
    with rtc.Loop(cfg, telemetry=True, graphs=True, ring=2) as g:
        cm = []
        for k, f in enumerate(frames):
            for b, x in zip(g.next_frame_buffers(), f):
                b[:] = x
            g.submit_graph(k + 1)
            cm.append(g.get_commands(timeout_us=WAIT_US)[1])
        outs.append(cm)
    for other in outs[1:]:
        assert all(np.array_equal(x, y) for x, y in zip(outs[0], other))


def test_global_norm_zero_flux_gives_minus_reference(rtc, torch_cuda):
    cfg = ragged_global_config(seed=65)
    dark = [np.zeros((w["height"], w["width"]), np.uint16) for w in cfg["wfs"]]
    with rtc.Loop(cfg, telemetry=True) as loop:
        loop.submit_frame(1, dark)
        fid, a = loop.get_commands(timeout_us=WAIT_US)
        s, _ = loop.get_telemetry(fid, timeout_us=WAIT_US)
    assert np.array_equal(s, -cfg["ref_slopes"]) and np.all(np.isfinite(a))


def test_global_norm_full_size_pyramid(rtc, torch_cuda):
    cfg = synth.make_config("elt_scao_pyramid", with_ref=True)
    cfg["wfs"][0]["norm"] = "global"
    frames = synth.draw_frames(cfg, 3, seed=66)
    with rtc.Loop(cfg, telemetry=True) as loop:
        run_pair(loop, cfg, frames, nchunks=8)
    # the two normalisations really differ on these frames
    loc = OracleLoop(dict(cfg, wfs=[dict(cfg["wfs"][0], norm="local")])).step(frames[0])[0]
    glo = OracleLoop(cfg).step(frames[0])[0]
    assert rel(glo, loc) > 1e-2


# ------------------------------------------------------------------ explicit POLC

def explicit_config(name="scao_small", seed=71, **kw):
    cfg = synth.make_config(name, **kw)
    rng = np.random.default_rng(seed)
    cfg = dict(cfg, P=None, polc="explicit", D=synth.interaction_matrix(rng, cfg["ns"], cfg["na"]),
               a0=rng.normal(0, 0.05, cfg["na"]).astype(np.float32))
    return cfg


@pytest.mark.parametrize("nchunks", [1, 4])
def test_explicit_polc_parity(rtc, torch_cuda, nchunks):
    cfg = explicit_config(with_ref=True, nblocks=4)
    frames = synth.draw_frames(cfg, 12, seed=72)
    with rtc.Loop(cfg, telemetry=True) as loop:
        errs, _ = run_pair(loop, cfg, frames, nchunks=nchunks)     # telemetry slopes are s + D a_{k-1}
    print("explicit POLC errors (slopes, commands):", errs[-1])


def test_explicit_equals_implicit_with_p_eq_md_minus_i(rtc, torch_cuda):
    cfg = explicit_config(seed=73)
    P = (cfg["M"].astype(np.float64) @ cfg["D"].astype(np.float64) - np.eye(cfg["na"])).astype(np.float32)
    imp = dict(cfg, polc="implicit", P=P, D=None)
    frames = synth.draw_frames(cfg, 10, seed=74)
    with rtc.Loop(cfg) as e, rtc.Loop(imp) as i:
        for k, f in enumerate(frames):
            e.submit_frame(k + 1, f)
            i.submit_frame(k + 1, f)
            ae = e.get_commands(timeout_us=WAIT_US)[1]
            ai = i.get_commands(timeout_us=WAIT_US)[1]
            assert rel(ae, ai) <= TOL_F32, k


@pytest.mark.parametrize("fmt", ["bf16", "e4m3"])
def test_explicit_polc_quantised_d_ragged(rtc, torch_cuda, fmt):
    base = ragged_global_config(seed=75)
    rng = np.random.default_rng(76)
    codes, scale = quantize_rows(synth.interaction_matrix(rng, base["ns"], base["na"], m_sd=1e-2), fmt)
    cfg = dict(base, P=None, polc="explicit", D=codes, D_scale=scale, D_dtype=fmt)
    frames = synth.draw_frames(cfg, 5, seed=77)
    with rtc.Loop(cfg, telemetry=True) as loop:
        run_pair(loop, cfg, frames, nchunks=3)


def test_explicit_polc_checkpoint_and_graph_mode(rtc, torch_cuda):
    cfg = explicit_config(seed=78)
    frames = synth.draw_frames(cfg, 6, seed=79)
    with rtc.Loop(cfg) as a:
        for k, f in enumerate(frames[:3]):
            a.submit_frame(k + 1, f)
            a.get_commands(timeout_us=WAIT_US)
        state = a.get_state()
        rest = []
        for k, f in enumerate(frames[3:]):
            a.submit_frame(k + 4, f)
            rest.append(a.get_commands(timeout_us=WAIT_US)[1])
    with rtc.Loop(cfg, graphs=True, ring=2) as g:
        g.set_state(state)                       # recomputes u = D a
        for k, f in enumerate(frames[3:]):
            for b, x in zip(g.next_frame_buffers(), f):
                b[:] = x
            g.submit_graph(k + 1)
            assert np.array_equal(g.get_commands(timeout_us=WAIT_US)[1], rest[k])


def test_explicit_polc_full_size_elt_scao(rtc, torch_cuda):
    cfg = explicit_config("elt_scao_sh", seed=80)
    frames = synth.draw_frames(cfg, 3, seed=81)
    with rtc.Loop(cfg, telemetry=True) as loop:
        assert loop.info()["p_bytes"] >= cfg["ns"] * cfg["na"] * 4
        run_pair(loop, cfg, frames, nchunks=8)


def test_explicit_polc_loop_in_the_server_mix(rtc, torch_cuda):
    cfgs = [explicit_config(seed=82), ragged_global_config(seed=83)]
    frames = [synth.draw_frames(c, 4, seed=84 + i) for i, c in enumerate(cfgs)]
    refs = [OracleLoop(c) for c in cfgs]
    budget = sum(rtc.footprint(c, flags=rtc.RTC_FLAG_GRAPHS)[0] for c in cfgs) + (64 << 20)
    with rtc.Server(budget) as srv:
        ids = [srv.admit(copy.deepcopy(c)) for c in cfgs]
        lps = [srv.loop(i) for i in ids]
        for k in range(4):
            for j in range(2):
                for b, x in zip(lps[j].next_frame_buffers(), frames[j][k]):
                    b[:] = x
                srv.submit(ids[j], k + 1)
            for j in range(2):
                a = lps[j].get_commands(timeout_us=WAIT_US)[1]
                assert rel(a, refs[j].step(frames[j][k])[1]) <= TOL_F32, (j, k)


# ------------------------------------------------------------------ telemetry circular buffer

ALL_TEL = 1 | 2 | 4      # RTC_TEL_SLOPES | RTC_TEL_COMMANDS | RTC_TEL_PARTIALS


def oracle_partials(cfg, s):
    """Per-WFS partial commands M~[:, cols_w] s[cols_w] in float64."""
    from oracle import rtc_oracle as orc
    m = orc.stored_matrix(cfg["M"], cfg.get("M_dtype", "f32"), cfg.get("M_scale"))
    out, c0 = [], 0
    for w in cfg["wfs"]:
        n = 2 * synth.num_valid(w)
        out.append(m[:, c0:c0 + n] @ s[c0:c0 + n])
        c0 += n
    return np.array(out)


def test_telemetry_buffer_entries_match_the_oracle(rtc, torch_cuda):
    cfg = ragged_global_config(seed=91)
    frames = synth.draw_frames(cfg, 6, seed=92)
    ref = OracleLoop(cfg)
    with rtc.Loop(cfg, tel_depth=16, tel_streams=ALL_TEL) as loop:
        for k, f in enumerate(frames):
            loop.submit_frame(k + 1, f, [synth.chunk_plan(w, 3) for w in cfg["wfs"]])
            loop.get_commands(timeout_us=WAIT_US)
        t_prev = 0
        for k, f in enumerate(frames):
            rec, s, a, p = loop.telemetry_read(timeout_us=WAIT_US, partials=True)
            s_ref, a_ref = ref.step(f)
            assert rec["index"] == k and rec["frame_id"] == k + 1 and rec["lost"] == 0
            assert rec["t_commands_ns"] > t_prev and rec["t_written_ns"] >= rec["t_commands_ns"]
            t_prev = rec["t_commands_ns"]
            assert rel(s, s_ref) <= TOL_F32 and rel(a, a_ref) <= TOL_F32
            p_ref = oracle_partials(cfg, s_ref)
            assert rel(p, p_ref) <= TOL_F32
            assert rel(p.sum(axis=0), p_ref.sum(axis=0)) <= TOL_F32
        with pytest.raises(rtc.RtcError, match="ETIMEDOUT"):
            loop.telemetry_read(timeout_us=0)


def test_telemetry_decimation_and_overrun_count_lost_entries(rtc, torch_cuda):
    cfg = synth.make_config("scao_small")
    frames = synth.draw_frames(cfg, 2, seed=93)
    with rtc.Loop(cfg, tel_depth=4, tel_streams=2, tel_decimate=3) as loop:
        cmds = {}
        for k in range(20):
            loop.submit_frame(k + 1, frames[k % 2])
            cmds[k + 1] = loop.get_commands(timeout_us=WAIT_US)[1]
        loop.sync()
        # frames 1, 4, ..., 19 were recorded as entries 0..6; a reader that fell behind a
        # depth-4 buffer gets the newest three and counts the four before them lost
        got = []
        for _ in range(3):
            rec, s, a, _ = loop.telemetry_read(timeout_us=WAIT_US, slopes=False)
            assert s is None and np.array_equal(a, cmds[rec["frame_id"]])
            got.append((rec["index"], rec["frame_id"], rec["lost"]))
        assert got == [(4, 13, 4), (5, 16, 0), (6, 19, 0)]
        with pytest.raises(rtc.RtcError, match="EINVAL"):
            loop.telemetry_read(timeout_us=0, slopes=True)          # slopes were not recorded


def test_telemetry_reader_thread_while_frames_run(rtc, torch_cuda):
    import threading
    cfg = synth.make_config("elt_scao_sh", polc=True)
    frames = synth.draw_frames(cfg, 2, seed=94)
    n = 150
    with rtc.Loop(cfg, tel_depth=32, tel_streams=ALL_TEL, graphs=True, ring=3) as loop:
        seen, lost = [], [0]

        def reader():
            while len(seen) + lost[0] < n:
                try:
                    rec, s, a, p = loop.telemetry_read(timeout_us=2_000_000, partials=True)
                except rtc.RtcError:
                    return
                lost[0] += rec["lost"]
                seen.append((rec["index"], rec["frame_id"], a))

        th = threading.Thread(target=reader)
        th.start()
        cmds = {}
        for k in range(n):
            for b, x in zip(loop.next_frame_buffers(), frames[k % 2]):
                b[:] = x
            loop.submit_graph(k + 1)
            fid, a = loop.get_commands(timeout_us=WAIT_US)
            cmds[fid] = a
        th.join(timeout=60)
        assert not th.is_alive()
    assert len(seen) + lost[0] == n and len(seen) > 0
    idx = [i for i, _, _ in seen]
    assert idx == sorted(idx) and len(set(idx)) == len(idx)
    for i, fid, a in seen:
        assert fid == i + 1 and np.array_equal(a, cmds[fid])


def test_loop_without_telemetry_buffer_rejects_reads(rtc, torch_cuda):
    cfg = synth.make_config("scao_small")
    with rtc.Loop(cfg) as loop:
        with pytest.raises(rtc.RtcError, match="no telemetry buffer"):
            loop.telemetry_read(timeout_us=0)


def test_telemetry_stream_to_a_file(rtc, torch_cuda, tmp_path):
    cfg = ragged_global_config(seed=95)
    frames = synth.draw_frames(cfg, 3, seed=96)
    n = 40
    path = tmp_path / "tel.bin"
    with open(path, "wb") as fh, rtc.Loop(cfg, tel_depth=64, tel_streams=ALL_TEL) as loop:
        loop.telemetry_stream_start(fh.fileno())
        with pytest.raises(rtc.RtcError, match="stream"):
            loop.telemetry_read(timeout_us=0)                  # the stream is the reader now
        cmds = {}
        for k in range(n):
            loop.submit_frame(k + 1, frames[k % 3])
            cmds[k + 1] = loop.get_commands(timeout_us=WAIT_US)[1]
        loop.sync()
        st = loop.telemetry_stream_stop()
    na, ns, nw = cfg["na"], cfg["ns"], len(cfg["wfs"])
    rec_bytes = 40 + 4 * (ns + na + nw * na)
    assert st["entries"] == n and st["lost"] == 0 and st["write_error"] == 0 and st["bytes"] == n * rec_bytes
    raw = path.read_bytes()
    assert len(raw) == n * rec_bytes
    ref = OracleLoop(cfg)
    for k in range(n):
        e = raw[k * rec_bytes:(k + 1) * rec_bytes]
        index, fid, t_cmd, t_wr, lost = np.frombuffer(e[:40], np.uint64)
        body = np.frombuffer(e[40:], np.float32)
        s, a, p = body[:ns], body[ns:ns + na], body[ns + na:].reshape(nw, na)
        s_ref, a_ref = ref.step(frames[k % 3])
        assert index == k and fid == k + 1 and lost == 0 and t_wr >= t_cmd
        assert np.array_equal(a, cmds[k + 1])
        assert rel(s, s_ref) <= TOL_F32 and rel(a, a_ref) <= TOL_F32
        assert rel(p, oracle_partials(cfg, s_ref)) <= TOL_F32
