"""Shared helpers of the GPU parity tests: run the CUDA loop and the FP64 oracle
on the same seeded inputs and compare."""
import numpy as np

from oracle import OracleLoop, stored_matrix
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


# Unit roundoff of a storage format relative to the scaled value, and the
# absolute rounding error of its subnormal range (half the subnormal spacing) in
# units of the row scale: BF16 keeps 8 significant bits; E4M3 keeps 4, and its
# subnormal spacing is 2^-9.
FORMAT_U = {"bf16": 2.0 ** -8, "e4m3": 2.0 ** -4}
FORMAT_SUB = {"bf16": 2.0 ** -134, "e4m3": 2.0 ** -10}
U32 = 2.0 ** -23          # one float32 rounding, to nearest or directed


def a_priori_bound(M, codes, scale, fmt, s, nterms):
    """Element-wise bound on |y - M s| when y is computed in float32 from the
    float32 matrix M stored as scale * code.

    Storage: code = RNE_fmt(fl(M / scale)), so |scale * code - M| <= (u + u32) |M|
    + scale * sub.  Arithmetic: float32 sums of the products code * s with at
    most nterms roundings on any path, then the row scale: gamma_K |M~| |s| with
    K = nterms + 1 and gamma_K = K u32 / (1 - K u32)."""
    K = nterms + 1
    gamma = K * U32 / (1.0 - K * U32)
    abs_s = np.abs(np.asarray(s, np.float64))
    Mabs = np.abs(np.asarray(M, np.float64))
    Mt = np.abs(stored_matrix(codes, fmt, scale))
    return ((FORMAT_U[fmt] + U32) * (Mabs @ abs_s)
            + np.asarray(scale, np.float64) * FORMAT_SUB[fmt] * abs_s.sum()
            + gamma * (Mt @ abs_s))
