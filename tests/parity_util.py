"""Shared helpers of the GPU parity tests: run the CUDA loop and the FP64 oracle
on the same seeded inputs and compare."""
import numpy as np

from oracle import OracleLoop
from paper_1903_01852_gb300 import synth

# Normwise relative tolerance for the float32 path (max |x - ref| / max |ref|).
TOL_F32 = 1e-5
WAIT_US = 60_000_000


def rel(x, ref):
    x = np.asarray(x, np.float64)
    ref = np.asarray(ref, np.float64)
    return float(np.max(np.abs(x - ref)) / max(float(np.max(np.abs(ref))), 1e-30)) if ref.size else 0.0


def device_frames(frames):
    """Copy uint16 frames to CUDA with a 16-byte-aligned row pitch (views keep the pitch)."""
    import torch
    out = []
    for f in frames:
        h, w = f.shape
        wp = (w + 7) // 8 * 8
        t = torch.zeros((h, wp), dtype=torch.int16, device="cuda")
        t[:, :w] = torch.from_numpy(np.ascontiguousarray(f).view(np.int16)).cuda()
        out.append(t[:, :w])
    return out


def run_pair(loop, cfg, frames, mode="chunked", nchunks=8, first_id=1, check=True, tol=TOL_F32):
    """Run frames through the GPU loop and the oracle; return per-frame errors
    (slopes, commands) and the GPU commands."""
    ref = OracleLoop(cfg)
    plans = [synth.chunk_plan(w, nchunks) for w in cfg["wfs"]]
    errs, cmds = [], []
    for k, f in enumerate(frames):
        fid = first_id + k
        if mode == "chunked":
            loop.submit_frame(fid, f, plans)
        else:
            loop.process_frame(fid, device_frames(f))
        got_id, a = loop.get_commands(timeout_us=WAIT_US)
        assert got_id == fid
        s, _ = loop.get_telemetry(fid, timeout_us=WAIT_US)
        s_ref, a_ref = ref.step(f)
        e = (rel(s, s_ref), rel(a, a_ref))
        if check:
            assert e[0] <= tol and e[1] <= tol, (k, e)
        errs.append(e)
        cmds.append(a)
    assert loop.check_guards() == 0          # no kernel wrote past any of the loop's buffers
    return errs, cmds
