"""Full-size configurations and matrix formats against the FP64 oracle, through the C ABI.

Every configuration of the benchmark set and every storage format the loop
offers is compared with the oracle element by element: on the stored matrix
(row scale times decoded code, as the reconstruction multiplies it) at the
float32 tolerance, and, for the low-precision formats, against the float32
matrix through an a-priori bound derived from the rounding of the format and
of the float32 sums.
"""
import copy

import numpy as np
import pytest

from oracle import OracleLoop, quantize_rows, stored_matrix
from paper_1903_01852_gb300 import synth
from parity_util import TOL_F32, WAIT_US, a_priori_bound, device_frames, rel, run_pair

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available()
    return torch


_codes = {}


def quantised(cfg, fmt, with_polc=True):
    """The configuration with M (and P) stored in fmt, codes and scales from the oracle's quantiser
    (kept per matrix for the module: the full-size quantisations take seconds)."""
    def q_rows(A):
        key = (id(A), fmt)
        if key not in _codes:
            _codes[key] = (A, quantize_rows(A, fmt))
        return _codes[key][1]
    q = copy.copy(cfg)
    codes, scale = q_rows(cfg["M"])
    q.update(M=codes, M_scale=scale, M_dtype=fmt)
    if with_polc and cfg.get("P") is not None:
        pc, ps = q_rows(cfg["P"])
        q.update(P=pc, P_scale=ps, P_dtype=fmt)
    return q


def pinned_frames(torch, frames):
    out = []
    for f in frames:
        per = []
        for x in f:
            t = torch.empty(x.shape, dtype=torch.int16, pin_memory=True)
            t.numpy()[:] = x.view(np.int16)
            per.append(t)
        out.append(per)
    return out


@pytest.fixture(scope="module")
def mcao():
    cfg = synth.make_config("mcao")
    return cfg, synth.draw_frames(cfg, 2, seed=211)


@pytest.fixture(scope="module")
def pyramid():
    cfg = synth.make_config("elt_scao_pyramid")
    return cfg, synth.draw_frames(cfg, 3, seed=212)


# ------------------------------------------------------------------ stored-matrix parity

@pytest.mark.parametrize("fmt", ["bf16", "e4m3"])
def test_full_size_pyramid_quantised_chunked(rtc, torch_cuda, pyramid, fmt):
    cfg, frames = pyramid
    q = quantised(cfg, fmt)
    with rtc.Loop(q, telemetry=True) as loop:
        errs, _ = run_pair(loop, q, frames, mode="chunked", nchunks=8)
    print(f"elt pyramid {fmt} (slopes, commands) vs the stored matrix:", errs)


def test_full_size_mcao_e4m3_device_frames(rtc, torch_cuda, mcao):
    cfg, frames = mcao
    q = quantised(cfg, "e4m3")
    with rtc.Loop(q, telemetry=True) as loop:
        errs, _ = run_pair(loop, q, frames, mode="device")
    print("mcao e4m3 (slopes, commands) vs the stored matrix:", errs)


@pytest.mark.parametrize("prelaunch", [False, True])
def test_full_size_mcao_fp32_row_chunks_read_in_place(rtc, torch_cuda, mcao, prelaunch):
    # The camera-paced path: each LGS frame in 8 row chunks of whole subaperture
    # rows, each NGS frame in one, submitted from page-locked host memory and
    # read in place (with prelaunch, each LGS chunk after the first of a frame
    # through kernels enqueued before it arrived); same bits as whole frames in
    # HBM, and the oracle's commands.
    torch = torch_cuda
    cfg, frames = mcao
    plans = [synth.chunk_plan(w, 8 if w["nsubx"] > 2 else 1) for w in cfg["wfs"]]
    host = pinned_frames(torch, frames)
    ref = OracleLoop(cfg)
    with rtc.Loop(cfg, telemetry=True, prelaunch=prelaunch) as chunked, rtc.Loop(cfg, telemetry=True) as whole:
        for k, f in enumerate(frames):
            for w, (plan, x) in enumerate(zip(plans, host[k])):
                for r0, r1 in plan:
                    chunked.submit(k + 1, w, r0, r1, x[r0:r1])
            whole.process_frame(k + 1, device_frames(f))
            fa, a = chunked.get_commands(timeout_us=WAIT_US)
            fb, b = whole.get_commands(timeout_us=WAIT_US)
            assert fa == fb == k + 1 and np.array_equal(a, b)
            s, _ = chunked.get_telemetry(fa, timeout_us=WAIT_US)
            s_ref, a_ref = ref.step(f)
            assert rel(s, s_ref) <= TOL_F32 and rel(a, a_ref) <= TOL_F32
        assert chunked.check_guards() == 0 and whole.check_guards() == 0
        if prelaunch:
            # submitted back to back, a camera can run ahead of the GPU by more chunks than it
            # has mailboxes (four): such a chunk takes ordinary launches (none is cancelled)
            lgs = sum(1 for w in cfg["wfs"] if w["nsubx"] > 2)
            info = chunked.info()
            assert 0 < info["prelaunch_used"] <= (len(frames) - 1) * lgs * 7
            assert info["prelaunch_cancelled"] == 0 and info["prelaunch_expired"] == 0


def test_full_size_serving_mix_each_loop_against_its_oracle(rtc, torch_cuda):
    # The serving mix: a HARMONI-like LTAO loop, the MAORY-like MCAO loop and two
    # ELT SCAO SH loops resident together, every matrix in BF16, graph mode; each
    # loop's frames overlap the others' on the GPU and each must give its own
    # oracle's slopes and commands.
    names = ["ltao", "mcao", "elt_scao_sh", "elt_scao_sh"]
    cfgs = [quantised(synth.make_config(n, seed=300 + i, polc=True), "bf16") for i, n in enumerate(names)]
    frames = [synth.draw_frames(c, 2, seed=310 + i) for i, c in enumerate(cfgs)]
    budget = sum(rtc.footprint(c, flags=rtc.RTC_FLAG_GRAPHS | rtc.RTC_FLAG_TELEMETRY)[0] for c in cfgs) + (64 << 20)
    refs = [OracleLoop(c) for c in cfgs]
    with rtc.Server(budget) as srv:
        ids = [srv.admit(c, telemetry=True) for c in cfgs]
        assert srv.usage()["admitted"] == 4
        lps = [srv.loop(i) for i in ids]
        for k in range(2):
            order = [(k + j) % 4 for j in range(4)]
            for j in order:
                for b, f in zip(lps[j].next_frame_buffers(), frames[j][k]):
                    b[:] = f
                srv.submit(ids[j], k + 1)
            for j in order:
                fid, a = lps[j].get_commands(timeout_us=WAIT_US)
                s, _ = lps[j].get_telemetry(fid, timeout_us=WAIT_US)
                s_ref, a_ref = refs[j].step(frames[j][k])
                assert fid == k + 1
                assert rel(s, s_ref) <= TOL_F32 and rel(a, a_ref) <= TOL_F32, (names[j], k)


# ------------------------------------------------------------------ a-priori bound against the float32 matrix

def gpu_reconstruction(rtc, cfg, frame):
    """The loop's float32 reconstruction y = M~ s of one frame, and the slopes it used.

    With zero initial state, no POLC term and gain 1/2, the first frame's
    commands are a = fma(1/2, y, 0) = y / 2 exactly, so y = 2 a."""
    c = dict(cfg, P=None, P_scale=None, a0=None, clip=None, gain=0.5)
    with rtc.Loop(c, telemetry=True) as loop:
        loop.process_frame(1, device_frames(frame))
        fid, a = loop.get_commands(timeout_us=WAIT_US)
        s, _ = loop.get_telemetry(fid, timeout_us=WAIT_US)
    return 2.0 * a.astype(np.float64), s


@pytest.mark.parametrize("name,fmt", [("mcao", "bf16"), ("mcao", "e4m3"),
                                      ("elt_scao_pyramid", "bf16"), ("elt_scao_pyramid", "e4m3")])
def test_format_error_within_a_priori_bound(rtc, torch_cuda, mcao, pyramid, name, fmt):
    cfg, frames = mcao if name == "mcao" else pyramid
    q = quantised(cfg, fmt, with_polc=False)
    y, s = gpu_reconstruction(rtc, q, frames[0])
    # the longest chain of roundings: every column of the widest sensor (a bound on
    # a column block's sum, whatever its split into lanes or tensor-core steps),
    # plus one addition per column block and the butterflies
    nblk = sum(int(w.get("nblocks", 1)) for w in cfg["wfs"])
    nterms = max(2 * synth.num_valid(w) for w in cfg["wfs"]) + nblk + 16
    bound = a_priori_bound(cfg["M"], q["M"], q["M_scale"], fmt, s, nterms)
    y_true = cfg["M"].astype(np.float64) @ s.astype(np.float64)
    err = np.abs(y - y_true)
    worst = float(np.max(err / bound))
    print(f"{name} {fmt}: normwise error vs the float32 matrix {rel(y, y_true):.3e}, "
          f"largest error / bound {worst:.3f}")
    assert np.all(err <= bound), worst
    # the same y against the stored matrix, at the float32 tolerance
    assert rel(y, stored_matrix(q["M"], fmt, q["M_scale"]) @ s.astype(np.float64)) <= TOL_F32
