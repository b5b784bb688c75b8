"""Seeded random configurations against the FP64 oracle, through the C ABI:
geometry (SH and pyramid sizes, origins, valid masks, block counts), frame
sizes, chunk plans, thresholds and modes, reference slopes, POLC form, clip and
matrix storage are all drawn per case.  Half of the chunked cases submit their
chunks from page-locked host memory, which the slope kernel reads in place."""
import numpy as np
import pytest

from oracle import OracleLoop, quantize_rows
from paper_1903_01852_gb300 import synth
from parity_util import TOL_F32, WAIT_US, device_frames, rel

pytestmark = pytest.mark.gpu

CASES = 48


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available()
    return torch


def random_wfs(rng):
    if rng.random() < 0.65:
        nsub = int(rng.integers(1, 13))
        npx = int(rng.integers(2, 13))
        w, h = nsub * npx + int(rng.integers(0, 9)), nsub * npx + int(rng.integers(0, 9))
        ox, oy = int(rng.integers(0, w - nsub * npx + 1)), int(rng.integers(0, h - nsub * npx + 1))
        wf = synth.sh_wfs(rng, nsub, npx, w, h, float(rng.choice([0.0, 0.2, 0.4])), ox=ox, oy=oy,
                          nblocks=int(rng.integers(1, nsub + 1)), threshold=float(rng.choice([0.0, 5.0, 40.0])),
                          thresh_mode=str(rng.choice(["subtract", "clip"])), sigma=float(rng.uniform(0.6, 2.0)),
                          max_offset=float(rng.uniform(0.0, npx / 3.0)))
    else:
        p = int(rng.integers(2, 17))
        w, h = 2 * p + int(rng.integers(0, 7)), 2 * p + int(rng.integers(0, 7))
        qx = [int(rng.integers(0, w // 2 - p + 1)), int(rng.integers(w // 2, w - p + 1)),
              int(rng.integers(0, w // 2 - p + 1)), int(rng.integers(w // 2, w - p + 1))]
        qy = [int(rng.integers(0, h // 2 - p + 1)), int(rng.integers(0, h // 2 - p + 1)),
              int(rng.integers(h // 2, h - p + 1)), int(rng.integers(h // 2, h - p + 1))]
        wf = synth.pyramid_wfs(rng, p, w, h, float(rng.choice([0.0, 0.3])), qx=qx, qy=qy,
                               nblocks=int(rng.integers(1, p + 1)), threshold=float(rng.choice([0.0, 3.0])))
        if rng.random() < 0.5:
            wf["norm"] = "global"
    if rng.random() < 0.15:                       # a ragged mask
        wf["valid"] = (rng.random(wf["valid"].shape) < 0.7).astype(np.uint8)
    return wf


def random_case(seed):
    rng = np.random.default_rng(seed)
    wfs = [random_wfs(rng) for _ in range(int(rng.integers(1, 5)))]
    ns = sum(2 * synth.num_valid(w) for w in wfs)
    na = int(rng.integers(1, 90))
    cfg = dict(name=f"random{seed}", na=na, ns=ns, wfs=wfs, M=synth.control_matrix(rng, na, ns, sd=1e-2),
               M_scale=None, M_dtype="f32", P=None, P_scale=None, P_dtype="f32", gain=float(rng.uniform(0.1, 0.6)),
               leak=float(rng.uniform(0.0, 0.05)), clip=None,
               a0=rng.normal(0, 0.1, na).astype(np.float32) if rng.random() < 0.5 else None,
               ref_slopes=rng.normal(0, 0.05, ns).astype(np.float32) if rng.random() < 0.5 else None)
    polc = rng.choice(["none", "implicit", "explicit"])
    if polc == "implicit":
        cfg["P"] = synth.polc_matrix(rng, na)
    elif polc == "explicit":
        cfg.update(polc="explicit", D=synth.interaction_matrix(rng, ns, na, m_sd=1e-2) if ns else
                   np.zeros((0, na), np.float32))
    if rng.random() < 0.2:
        cfg["clip"] = (-0.02, 0.03)
    fmt = str(rng.choice(["f32", "f32", "bf16", "e4m3"]))
    if fmt != "f32":
        codes, scale = quantize_rows(cfg["M"], fmt)
        cfg.update(M=codes, M_scale=scale, M_dtype=fmt)
        if cfg["P"] is not None:
            pc, ps = quantize_rows(cfg["P"], fmt)
            cfg.update(P=pc, P_scale=ps, P_dtype=fmt)
    mode = str(rng.choice(["chunked", "device", "rows"]))
    nchunks = int(rng.integers(1, 6))
    return cfg, mode, nchunks, rng


def pinned_frames(frames, torch):
    """Page-locked copies with a 16-byte row pitch, so whole-subaperture-row chunks are read in place."""
    out = []
    for x in frames:
        h, w = x.shape
        t = torch.zeros((h, (w + 7) // 8 * 8), dtype=torch.int16, pin_memory=True)
        t.numpy()[:, :w] = x.view(np.int16)
        out.append(t[:, :w])
    return out


@pytest.mark.parametrize("seed", range(CASES))
def test_random_configuration(rtc, torch_cuda, seed):
    cfg, mode, nchunks, rng = random_case(7000 + seed)
    if cfg["ns"] == 0:
        pytest.skip("no valid unit drawn")
    frames = synth.draw_frames(cfg, 3, seed=8000 + seed)
    ref = OracleLoop(cfg)
    with rtc.Loop(cfg, telemetry=True, ring=int(rng.integers(2, 6))) as loop:
        for k, f in enumerate(frames):
            fid = 1 + k
            if mode == "device":
                loop.process_frame(fid, device_frames(f))
            elif mode == "rows":
                loop.submit_frame(fid, f, [[(r, r + 1) for r in range(x.shape[0])] for x in f])
            else:
                loop.submit_frame(fid, pinned_frames(f, torch_cuda) if seed % 2 == 0 else f,
                                  [synth.chunk_plan(w, nchunks) for w in cfg["wfs"]])
            got, a = loop.get_commands(timeout_us=WAIT_US)
            s, _ = loop.get_telemetry(fid, timeout_us=WAIT_US)
            s_ref, a_ref = ref.step(f)
            assert got == fid
            assert rel(s, s_ref) <= TOL_F32, (seed, k, "slopes", rel(s, s_ref))
            assert rel(a, a_ref) <= TOL_F32, (seed, k, "commands", rel(a, a_ref))
        assert loop.check_guards() == 0          # no kernel wrote past any of the loop's buffers
