"""The C ABI used from plain C (tests/c_caller/rtc_caller.c), without the Python
binding: it compiles as C11 against include/rtc.h and links against the library
(CPU); on a GPU its commands match the oracle and the binding's, bit for bit."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_1903_01852_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "c_caller", "rtc_caller.c")


def compile_caller(rtc, out_dir):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    lib_dir = os.path.dirname(os.path.abspath(rtc.LIB_PATH))
    exe = os.path.join(out_dir, "rtc_caller")
    subprocess.run(["gcc", "-std=c11", "-O2", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
                    SRC, "-o", exe, rtc.LIB_PATH, "-Wl,-rpath," + lib_dir], check=True)
    return exe


def test_c_caller_compiles_and_links(rtc, tmp_path):
    assert os.access(compile_caller(rtc, str(tmp_path)), os.X_OK)


def write_input(path, cfg, frames, nchunks):
    i32 = lambda *v: np.array(v, np.int32).tobytes()
    f32 = lambda a: np.ascontiguousarray(a, np.float32).tobytes()
    parts = [i32(len(cfg["wfs"]), cfg["na"], cfg["ns"], len(frames), nchunks, 0)]
    for w in cfg["wfs"]:
        sh = w["kind"] == "sh"
        parts.append(i32(0 if sh else 1, w["width"], w["height"], w.get("nsubx", 0), w.get("nsuby", 0),
                         w.get("npx", 0), w.get("ox", 0), w.get("oy", 0), w.get("pupil", 0),
                         *(w.get("qx") or [0] * 4), *(w.get("qy") or [0] * 4), w["nblocks"],
                         1 if w.get("norm") == "global" else 0, 1 if w["thresh_mode"] == "clip" else 0))
        parts.append(f32([w["threshold"]]))
        parts.append(np.ascontiguousarray(w["valid"], np.uint8).tobytes())
        parts += [f32(w["dark"]), f32(w["flat"])]
    parts.append(f32(cfg["M"]))
    if cfg.get("P") is not None:
        parts += [i32(1), f32(cfg["P"])]
    else:
        parts.append(i32(0))
    parts.append(f32([cfg["gain"], cfg["leak"]]))
    if cfg.get("ref_slopes") is not None:
        parts += [i32(1), f32(cfg["ref_slopes"])]
    else:
        parts.append(i32(0))
    for f in frames:
        parts += [np.ascontiguousarray(x, np.uint16).tobytes() for x in f]
    with open(path, "wb") as fh:
        fh.write(b"".join(parts))


@pytest.mark.gpu
def test_c_caller_matches_the_oracle_and_the_binding(rtc, tmp_path):
    from oracle import OracleLoop
    from parity_util import TOL_F32, WAIT_US, rel
    rng = np.random.default_rng(251)
    sh = synth.sh_wfs(rng, 12, 8, 100, 98, 0.2, nblocks=3)
    pyr = synth.pyramid_wfs(rng, 17, 44, 42, 0.1, nblocks=2)
    pyr["norm"] = "global"
    ns = 2 * (synth.num_valid(sh) + synth.num_valid(pyr))
    na = 53
    cfg = dict(name="c_caller", na=na, ns=ns, wfs=[sh, pyr], M=synth.control_matrix(rng, na, ns, sd=1e-2),
               M_scale=None, M_dtype="f32", P=synth.polc_matrix(rng, na), P_scale=None, P_dtype="f32", gain=0.4,
               leak=0.02, clip=None, a0=None, ref_slopes=rng.normal(0, 0.05, ns).astype(np.float32))
    frames = synth.draw_frames(cfg, 6, seed=252)
    exe = compile_caller(rtc, str(tmp_path))
    inp, out = str(tmp_path / "in.bin"), str(tmp_path / "out.bin")
    write_input(inp, cfg, frames, nchunks=4)
    r = subprocess.run([exe, inp, out], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    raw = np.fromfile(out, np.uint8)
    rec = 8 + 4 * na
    assert raw.size == rec * len(frames)
    ref = OracleLoop(cfg)
    plans = [[(c * x.shape[0] // 4, (c + 1) * x.shape[0] // 4) for c in range(4)] for x in frames[0]]
    with rtc.Loop(cfg) as loop:
        for k, f in enumerate(frames):
            e = raw[k * rec:(k + 1) * rec]
            fid = int(e[:8].view(np.uint64)[0])
            a = e[8:].view(np.float32)
            assert fid == k + 1
            assert rel(a, ref.step(f)[1]) <= TOL_F32
            loop.submit_frame(k + 1, f, plans)
            assert np.array_equal(loop.get_commands(timeout_us=WAIT_US)[1], a)
