"""Benchmark of the AO RTC hot path on the MAORY-like MCAO loop.

One step = one frame through the whole hot path: calibration + slopes of all
9 WFS, the 7500 x 55608 reconstruction MVM, finalisation (partial sums +
implicit-POLC term + leaky integrator), the 7500 x 7500 POLC product for the
next frame and the slope/command telemetry to page-locked host memory.

Prints one JSON line.  ``value`` is the median per-frame latency (microseconds,
lower is better) of the float32 path with every frame already resident in
HBM, from CUDA events on the loop's stream (slope kernel start -> commands
written).  Beside it: p99/p99.9/jitter, the MVM's HBM bandwidth for FP32 and
BF16 matrices, BF16 latencies, camera-paced last-pixel latencies (the paper's
definition, Section 2.3), the end-to-end latency through rtc_submit_pixels
from page-locked host buffers, and the FP64 oracle on the host cores.

``--impl reference`` times the FP64 CPU oracle on the same workload instead.
"""
from __future__ import annotations

import os

# The CPU oracle is timed as it stands on one host thread: pin BLAS before numpy loads.
for _v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import argparse
import gc
import hashlib
import json
import platform
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MCAO frame latency p50/p99 µs + jitter RMS; MVM HBM GB/s, FP32 vs BF16"
WORKLOAD = ("MAORY-like MCAO: 6 LGS SH 80x80 subaps (obstruction 0.28 -> 4632 valid each, 10x10 px, 800x800, "
            "radially elongated spots) + 3 NGS SH 2x2 (100x100 px on 240x240); 55608 slopes; 7500 actuators; "
            "implicit POLC 7500x7500; telemetry of slopes+commands to page-locked host each frame")
FRAME_RING = 8          # distinct synthetic frames cycled through
PACED_HZ = 500.0        # MCAO frame rate (Table ao_compare)
READOUT_MS = 1.6        # camera readout spread over the row chunks
NCHUNKS = 8             # row chunks per LGS camera


def pct(xs, q):
    xs = sorted(xs)
    if not xs:
        return None
    k = (len(xs) - 1) * q / 100.0
    lo, hi = int(np.floor(k)), int(np.ceil(k))
    return float(xs[lo] + (xs[hi] - xs[lo]) * (k - lo))


def stats(xs, period_us=None):
    """Percentiles, mean, RMS jitter (standard deviation, the paper's "±") and max; with a
    frame period, also the deadline misses (frames whose latency exceeded it)."""
    out = {"p50": pct(xs, 50), "p99": pct(xs, 99), "p999": pct(xs, 99.9), "mean": float(np.mean(xs)),
           "jitter_rms": float(np.std(xs)), "max": float(np.max(xs)), "n": len(xs)}
    if period_us is not None:
        out["deadline_misses"] = int(np.count_nonzero(np.asarray(xs) > period_us))
    return out


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed regions."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None
        self.active = False
        self.lock = threading.Lock()

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        threading.Thread(target=self._read, daemon=True).start()

    def _read(self):
        for line in self.proc.stdout:
            with self.lock:
                if self.active:
                    self.rows.append([x.strip() for x in line.split(",")])

    def mark(self, on):
        with self.lock:
            self.active = on

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        with self.lock:
            rows = list(self.rows)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if len(r) > 5 + i and r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def code_text(src):
    """Source text without comments and whitespace: what the compiler sees of it."""
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    return re.sub(r"\s+", "", src)


KERNEL_SOURCES = ("rtc_kernels.cu", "rtc_internal.h", "rtc_runtime.cu")


def kernel_source_hash(texts=None):
    """Hash of what decides the kernels' memory traffic: the kernel and runtime sources
    (the runtime lays out the matrix blocks and picks the launches) and the build script
    with its compiler flags and tuning macros, comments and whitespace ignored; recorded
    beside the ncu figures so that they are reported only for the build they were taken
    on.  A library named by RTC_LIBRARY (another build) never matches."""
    default = texts is None
    if default:
        csrc = os.path.join(ROOT, "paper_1903_01852_gb300", "csrc")
        texts = {f: open(os.path.join(csrc, f)).read() for f in KERNEL_SOURCES}
        texts["build.py"] = open(os.path.join(ROOT, "paper_1903_01852_gb300", "build.py")).read()
    h = hashlib.sha256()
    for name in sorted(texts):
        h.update(name.encode())
        h.update(code_text(texts[name]).encode())
    if default and os.environ.get("RTC_LIBRARY"):
        h.update(("library:" + os.path.abspath(os.environ["RTC_LIBRARY"])).encode())
    return h.hexdigest()[:16]


def profiled_traffic():
    """DRAM bytes per launch of the FP32 MVM kernel from the committed ncu summary,
    if it was taken on the current kernel source (else None)."""
    p = os.path.join(ROOT, "profiles", "gemv_f32_mcao.md")
    if not os.path.exists(p):
        return None
    src, traffic = None, None
    for line in open(p):
        if line.startswith("kernel_source_sha256_16:"):
            src = line.split(":", 1)[1].strip()
        if line.startswith("dram_bytes_per_full_launch:"):
            traffic = float(line.split(":", 1)[1].strip())
    return traffic if src == kernel_source_hash() else None


# ---------------------------------------------------------------------------- workload

def make_workload(seed_frames=1, name="mcao"):
    from paper_1903_01852_gb300 import synth
    cfg = synth.make_config(name)
    frames = synth.draw_frames(cfg, FRAME_RING, seed=seed_frames)
    return cfg, frames


def quant_config(cfg, rtc, torch, fmt):
    """The same loop with M and P stored as per-row scaled BF16 / E4M3 codes
    (quantised on the GPU by rtc_quantize_rows)."""
    import copy
    q = copy.copy(cfg)
    view = np.uint16 if fmt == "bf16" else np.uint8
    codes, scale = rtc.quantize_rows(torch.from_numpy(cfg["M"]).cuda(), fmt)
    q.update(M=codes.cpu().numpy().view(view), M_scale=scale.cpu().numpy(), M_dtype=fmt)
    if cfg.get("P") is not None:
        pc, ps = rtc.quantize_rows(torch.from_numpy(cfg["P"]).cuda(), fmt)
        q.update(P=pc.cpu().numpy().view(view), P_scale=ps.cpu().numpy(), P_dtype=fmt)
    torch.cuda.synchronize()
    return q


def bf16_config(cfg, rtc, torch):
    return quant_config(cfg, rtc, torch, "bf16")


def mvm_bytes(info, cfg):
    """Algorithmic bytes of one reconstruction MVM launch with its fused finalisation:
    matrix (true size) and row scales, the slopes read, the per-block partial commands
    written and read back, and q, a (read and write) and the commands written."""
    b = {"f32": 4, "bf16": 2, "e4m3": 1}[cfg.get("M_dtype", "f32")]
    na, ns = info["na"], info["ns"]
    return (na * ns * b + (4 * na if cfg.get("M_scale") is not None else 0) + 4 * ns
            + 2 * 4 * na * info["nblocks"] + 4 * 4 * na)


def run_unpaced(loop, dev_frames, steps, warmup, torch, sampler, first_id):
    """Frames resident in HBM, back to back: returns per-frame timing dicts and the
    device time of the whole timed region."""
    ext = torch.cuda.ExternalStream(loop.stream())
    fid = first_id
    for k in range(warmup):
        loop.process_frame(fid, dev_frames[k % len(dev_frames)])
        loop.get_commands(timeout_us=10_000_000)
        fid += 1
    loop.sync()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ids = []
    gc.disable()
    sampler.mark(True)
    e0.record(ext)
    for k in range(steps):
        loop.process_frame(fid, dev_frames[k % len(dev_frames)])
        loop.get_commands(timeout_us=10_000_000)
        ids.append(fid)
        fid += 1
    e1.record(ext)
    loop.sync()
    torch.cuda.synchronize()
    sampler.mark(False)
    gc.enable()
    tim = [loop.get_timing(i) for i in ids[-min(len(ids), 4):]]
    return e0.elapsed_time(e1), ids, tim, fid


def run_unpaced_timed(loop, dev_frames, steps, warmup, sampler, first_id):
    """Same as run_unpaced but reads every frame's stage times (the ring holds only
    a few frames, so timing is read right after each frame)."""
    fid = first_id
    for k in range(warmup):
        loop.process_frame(fid, dev_frames[k % len(dev_frames)])
        loop.get_commands(timeout_us=10_000_000)
        fid += 1
    loop.sync()
    rows = []
    gc.disable()
    sampler.mark(True)
    for k in range(steps):
        loop.process_frame(fid, dev_frames[k % len(dev_frames)])
        loop.get_commands(timeout_us=10_000_000)
        rows.append(loop.get_timing(fid))
        fid += 1
    sampler.mark(False)
    gc.enable()
    return rows, fid


def run_host_path(loop, host_frames, plans, steps, warmup, sampler, first_id, paced, swap=None, arrival=None,
                  slowest=None, hz=PACED_HZ, readout_ms=READOUT_MS):
    """Frames from page-locked host memory through rtc_submit_pixels_n (each round of row
    chunks, chunk c of every camera, in one call) and rtc_get_commands.  Unpaced: latency =
    first submit -> commands returned.  Paced at the MCAO frame rate with the readout spread
    over the chunks: latency = last round submitted (last pixel in) -> commands returned; arrival (a list)
    also gets, per timed frame, the time from the arrival of the last row chunk of every
    camera (the start of the last round of submissions) -> commands returned, which
    includes the host's submission of every camera's last chunk.  slowest (a dict) receives
    the slowest timed frame's split: its index, the time spent in the submission calls of
    the frame, and the time rtc_get_commands waited.
    swap = (seconds, kwargs): a background thread calls loop.update(**kwargs) every that
    many seconds during the timed frames (the paper's parameter-swap experiment); the
    frames that applied a swap are reported apart."""
    upd_times, swap_lat, stop = [], [], threading.Event()

    def updater():
        while not stop.wait(swap[0]):
            t0 = time.perf_counter()
            loop.update(**swap[1])
            upd_times.append(time.perf_counter() - t0)

    th = threading.Thread(target=updater, daemon=True) if swap else None
    swaps_seen = loop.info()["swaps"] if swap else 0
    period = 1.0 / hz
    nch = max(len(p) for p in plans)
    dt = readout_ms * 1e-3 / nch
    lat = []
    fid = first_id
    rounds = {}     # (frame buffer, round) -> its chunk array; only the frame ids change
    gc.disable()
    t_next = time.perf_counter() + 0.002
    for k in range(warmup + steps):
        f = host_frames[k % len(host_frames)]
        timed = k >= warmup
        if timed and k == warmup:
            sampler.mark(True)
        if paced:
            while time.perf_counter() < t_next:
                pass
        t_first = time.perf_counter()
        t_last = t_round = t_first
        in_calls = 0.0
        for c in range(nch):
            if paced:
                tc = t_next + c * dt
                while time.perf_counter() < tc:
                    pass
            t_round = time.perf_counter()
            arr = rounds.get((k % len(host_frames), c))
            if arr is None:
                arr = loop.chunks(fid, [(w, *p[c], f[w][p[c][0]:p[c][1]]) for w, p in enumerate(plans) if c < len(p)])
                rounds[(k % len(host_frames), c)] = arr
            for ch in arr:
                ch.frame_id = fid
            t_last = time.perf_counter()
            loop.submit_chunks(arr)
            in_calls += time.perf_counter() - t_last
        t_wait = time.perf_counter()
        loop.get_commands(timeout_us=10_000_000)
        t_done = time.perf_counter()
        if timed:
            lat.append(((t_done - t_last) if paced else (t_done - t_first)) * 1e6)
            if slowest is not None and lat[-1] > slowest.get("latency_us", -1.0):
                slowest.update(frame=k - warmup, latency_us=lat[-1], submit_calls_us=in_calls * 1e6,
                               get_commands_wait_us=(t_done - t_wait) * 1e6)
            if arrival is not None:
                arrival.append((t_done - t_round) * 1e6)
            if th is not None:
                if k == warmup:
                    th.start()
                sw = loop.info()["swaps"]
                if sw != swaps_seen:
                    swap_lat.append(lat.pop())
                    swaps_seen = sw
        fid += 1
        t_next += period
        if paced and time.perf_counter() > t_next:
            t_next = time.perf_counter() + 0.0005
    sampler.mark(False)
    gc.enable()
    if th is not None:
        stop.set()
        th.join()
        return lat, fid, {"updates": len(upd_times), "swap_frames": len(swap_lat),
                          "upload_s_mean": float(np.mean(upd_times)) if upd_times else None,
                          "latency_us_swap_frames": stats(swap_lat, 1e6 / PACED_HZ) if swap_lat else None}
    return lat, fid


def run_graph_frames(loop, frames, steps, warmup, sampler, first_id):
    """Graph mode through the public API: the loop owns one page-locked input buffer set per
    ring slot (as many slots as distinct frames, each written once with its frame), and each
    step is one rtc_submit_frame_graph (slopes read the pixels in place over NVLink-C2C,
    MVM, POLC, telemetry) followed by rtc_get_commands; latency = submit entry -> commands
    returned, host clock."""
    from paper_1903_01852_gb300 import binding as rtc
    import ctypes as C
    for k, f in enumerate(frames):                  # stage frame k in slot k
        for b, x in zip(loop.next_frame_buffers(), f):
            b[:] = x
        loop.submit_graph(first_id + k)
        loop.get_commands(timeout_us=10_000_000)
    fid = first_id + len(frames)
    out = np.empty(loop.na, np.float32)
    outp = out.ctypes.data_as(rtc.f32p)
    got = C.c_uint64()
    h = loop._h
    lat = []
    gc.disable()
    for k in range(warmup + steps):
        if k == warmup:
            sampler.mark(True)
        t0 = time.perf_counter()
        rc = rtc.lib.rtc_submit_frame_graph(h, fid)
        rc2 = rtc.lib.rtc_get_commands(h, outp, loop.na, C.byref(got), 10_000_000)
        t1 = time.perf_counter()
        if rc or rc2:
            raise RuntimeError(f"graph frame failed: {rc} {rc2} {loop.last_error}")
        if k >= warmup:
            lat.append((t1 - t0) * 1e6)
        fid += 1
    sampler.mark(False)
    gc.enable()
    return lat, fid


def run_host_frames(loop, host_frames, steps, warmup, sampler, first_id):
    """Whole frames in page-locked host memory through rtc_process_frame (the slope
    kernel reads them in place over the CPU-GPU link) and rtc_get_commands; latency =
    call entry -> commands returned, host clock."""
    lat = []
    fid = first_id
    gc.disable()
    for k in range(warmup + steps):
        if k == warmup:
            sampler.mark(True)
        f = host_frames[k % len(host_frames)]
        t0 = time.perf_counter()
        loop.process_frame(fid, f)
        loop.get_commands(timeout_us=10_000_000)
        t1 = time.perf_counter()
        if k >= warmup:
            lat.append((t1 - t0) * 1e6)
        fid += 1
    sampler.mark(False)
    gc.enable()
    return lat, fid


def cpu_oracle(cfg, frames, nframes=3):
    """The oracle on the first nframes + 1 frames of the ring (the same frames, in the same
    order, as the parity loop): returns the per-frame times and commands of frames 2.."""
    from oracle import OracleLoop
    t0 = time.perf_counter()
    ref = OracleLoop(cfg)
    t_setup = time.perf_counter() - t0
    ref.step(frames[0])                       # warm-up frame (frame 1 of the parity loop)
    times, cmds = [], []
    for k in range(nframes):
        t0 = time.perf_counter()
        _, a = ref.step(frames[(k + 1) % len(frames)])
        times.append((time.perf_counter() - t0) * 1e6)
        cmds.append(a)
    return times, cmds, t_setup


def oracle_stages(cfg, frames, nframes=5):
    """Median per-frame time of each oracle step (the oracle's own functions, in the order
    OracleLoop.step applies them): calibration + slopes of all WFS, the MVM, the control
    law, the POLC product for the next frame."""
    from oracle import rtc_oracle as orc
    ref = orc.OracleLoop(cfg)
    ref.step(frames[0])
    rows = []
    for k in range(nframes):
        f = frames[(k + 1) % len(frames)]
        t0 = time.perf_counter()
        s = orc.frame_slopes(cfg, f)
        t1 = time.perf_counter()
        y = orc.mvm(ref.m, s)
        t2 = time.perf_counter()
        a = orc.control_step(ref.a, y, ref.q, cfg["gain"], cfg["leak"], cfg.get("clip"))
        t3 = time.perf_counter()
        q = ref.p @ a if ref.p is not None else ref.q
        t4 = time.perf_counter()
        ref.a, ref.q = a, q
        rows.append([(t1 - t0) * 1e6, (t2 - t1) * 1e6, (t3 - t2) * 1e6, (t4 - t3) * 1e6, (t4 - t0) * 1e6])
    med = np.median(np.array(rows), axis=0)
    return {"slopes_us": float(med[0]), "mvm_us": float(med[1]), "control_us": float(med[2]),
            "polc_us": float(med[3]), "frame_us": float(med[4]), "frames": nframes}


def host_cpu():
    """Host core count and model (x86 'model name'; on Arm the implementer/part codes,
    e.g. part 0xd4f is a Neoverse V2 core as in Grace)."""
    info = {}
    try:
        for line in open("/proc/cpuinfo"):
            key, _, val = line.partition(":")
            key = key.strip().lower()
            if key in ("model name", "cpu implementer", "cpu part") and key not in info:
                info[key] = val.strip()
    except OSError:
        pass
    model = info.get("model name") or " ".join(f"{k} {info[k]}" for k in ("cpu implementer", "cpu part") if k in info)
    return {"nproc": os.cpu_count(), "arch": platform.machine(), "model": model or None}


def oracle_stages_all_cores(nframes=5):
    """oracle_stages in a child process whose BLAS uses every host core (the matrix
    products parallelise over rows; the per-pixel steps stay on one thread)."""
    n = os.cpu_count() or 1
    env = dict(os.environ, OPENBLAS_NUM_THREADS=str(n), OMP_NUM_THREADS=str(n), MKL_NUM_THREADS=str(n))
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-stages", str(nframes)], env=env,
                       capture_output=True, text=True, timeout=900)
    if r.returncode != 0:
        return {"error": r.stderr.strip().splitlines()[-1] if r.stderr.strip() else str(r.returncode)}
    d = json.loads(r.stdout.strip().splitlines()[-1])
    d["threads"] = n
    return d


# ---------------------------------------------------------------------------- arms

def max_over_ranks(vals, world, device):
    """Element-wise maximum of a list of floats over all ranks (identity for one rank)."""
    if world <= 1:
        return list(vals)
    import torch
    import torch.distributed as dist
    t = torch.tensor(vals, device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if args.impl == "ours" else "gloo")
    return world, rank, local


def reference_arm(args, world, rank):
    if rank != 0:
        return
    cfg, frames = make_workload()
    # bound the CPU work: the oracle takes about a second per MCAO frame on one core
    from oracle import OracleLoop
    ref = OracleLoop(cfg)
    for k in range(max(1, min(args.warmup, 2))):
        ref.step(frames[k % len(frames)])
    t0 = time.perf_counter()
    ref.step(frames[0])
    est = time.perf_counter() - t0
    n = int(max(3, min(args.steps, 150.0 / max(est, 1e-3))))
    times = []
    for k in range(n):
        t0 = time.perf_counter()
        ref.step(frames[k % len(frames)])
        times.append((time.perf_counter() - t0) * 1e6)
    st = stats(times)
    sample = f"{n} full MCAO frames (all 9 WFS, full MVM + POLC) through the float64 numpy oracle, 1 BLAS thread"
    out = {"impl": "reference", "metric": METRIC, "value": st["p50"], "unit": "us", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": st["mean"] / 1e3,
           "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic (seeded)", "config": bench_config(cfg, world),
           "latency_us": st,
           "cpu_baseline": {"value": st["p50"], "unit": "us", "cores": 1, "kind": "oracle", "sample": sample},
           "e2e": {"value": st["p50"], "unit": "us", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def bench_config(cfg, world):
    """The workload's configuration as both arms report it."""
    return {"workload": WORKLOAD, "na": int(cfg["na"]), "ns": int(cfg["ns"]),
            "frames": f"{FRAME_RING} distinct frames resident in HBM, cycled",
            "l2": "inputs larger than L2: the 1.67 GB FP32 (0.83 GB BF16, 0.42 GB E4M3) matrix is streamed every frame",
            "replicas": world}


def ours_arm(args, world, rank, local):
    import torch
    from paper_1903_01852_gb300 import binding as rtc
    from paper_1903_01852_gb300 import synth

    torch.cuda.set_device(local)
    peak, peak_kind = peaks()
    cfg, frames = make_workload(name=args.workload)
    if args.quick:
        if args.dtype != "f32":
            cfg = quant_config(cfg, rtc, torch, args.dtype)
        return quick_arm(args, cfg, frames, rtc, torch, local)
    dev_frames = []
    for f in frames:
        per = []
        for x in f:
            h, w = x.shape
            t = torch.zeros((h, (w + 7) // 8 * 8), dtype=torch.int16, device="cuda")
            t[:, :w] = torch.from_numpy(x.view(np.int16)).cuda()
            per.append(t[:, :w])
        dev_frames.append(per)
    host_frames = []
    for f in frames:
        per = []
        for x in f:
            t = torch.empty(x.shape, dtype=torch.int16, pin_memory=True)
            t.numpy()[:] = x.view(np.int16)
            per.append(t)
        host_frames.append(per)
    plans = [synth.chunk_plan(w, NCHUNKS if w["nsubx"] > 2 else 1) for w in cfg["wfs"]]
    h2d = sum(int(np.prod(x.shape)) * 2 for x in frames[0])

    sampler = ClockSampler(local)
    sampler.start()
    loops = {}
    fmts = ("f32", "bf16", "e4m3")
    try:
        cfgs = {"f32": cfg, "bf16": quant_config(cfg, rtc, torch, "bf16"), "e4m3": quant_config(cfg, rtc, torch, "e4m3")}
        for name in fmts:
            # latency loops: the MVM starts while the slope kernel runs (frame-level events only)
            loops[name] = rtc.Loop(cfgs[name], device=local, timing=True, telemetry=True)
            # stage loops: slope and MVM kernels timed separately (serialised) for the MVM bandwidth
            loops[name + "_stage"] = rtc.Loop(cfgs[name], device=local, stage_timing=True, telemetry=True)
        for name in ("f32", "bf16"):
            # host-clock loops (paced and end-to-end): no CUDA events, whose records would add host
            # time before the launches that matter
            loops[name + "_host"] = rtc.Loop(cfgs[name], device=local, telemetry=True, updatable=(name == "f32"))
        # the same loops with each LGS chunk's kernels enqueued before the chunk arrives
        for name in ("f32", "bf16"):
            loops[name + "_pre"] = rtc.Loop(cfgs[name], device=local, telemetry=True, prelaunch=True)
        fid = 1
        # 1) timed region: K unpaced steps, frames resident in HBM (device events around the region)
        ms_total, ids, _, fid = run_unpaced(loops["f32"], dev_frames, args.steps, args.warmup, torch, sampler, fid)
        # per-frame latencies (event-timed, 2x10^4 frames each) and per-kernel stage times, every format
        per, stg = {}, {}
        for name in fmts:
            per[name], fid = run_unpaced_timed(loops[name], dev_frames, args.latency_frames, args.warmup, sampler, fid)
            stg[name], fid = run_unpaced_timed(loops[name + "_stage"], dev_frames, args.stage_frames, args.warmup,
                                               sampler, fid)
        # 2) end-to-end through the C ABI from page-locked host buffers (unpaced, whole frames):
        #    graph mode (the public path with the least host work), and rtc_process_frame
        with rtc.Loop(cfg, device=local, telemetry=True, graphs=True, ring=len(frames)) as gl:
            e2e_lat, _ = run_graph_frames(gl, frames, args.steps, args.warmup, sampler, 1)
        pf_lat, fid = run_host_frames(loops["f32_host"], host_frames, args.steps, args.warmup, sampler, fid)
        # 3) camera-paced last-pixel latency (the paper's definition), FP32 and BF16
        paced = {}
        for name, lp in (("f32", "f32_host"), ("bf16", "bf16_host"), ("f32_prelaunch", "f32_pre"),
                         ("bf16_prelaunch", "bf16_pre")):
            arr, slow = [], {}
            lat, fid = run_host_path(loops[lp], host_frames, plans, args.paced_frames, args.paced_warmup,
                                     sampler, fid, paced=True, arrival=arr, slowest=slow)
            paced[name] = stats(lat, 1e6 / PACED_HZ)
            paced[name]["slowest_frame"] = {k: (round(v, 1) if isinstance(v, float) else v) for k, v in slow.items()}
            a = stats(arr, 1e6 / PACED_HZ)
            paced[name]["from_arrival"] = {k: a[k] for k in ("p50", "p99", "p999", "jitter_rms", "deadline_misses")}
        for name in ("f32", "bf16"):
            paced[name + "_prelaunch"]["chunks"] = {k: loops[name + "_pre"].info()["prelaunch_" + k]
                                                    for k in ("used", "cancelled", "expired")}
        # 4) the same paced FP32 loop while the whole control matrix is re-uploaded and swapped every second
        lat, fid, swap_info = run_host_path(loops["f32_host"], host_frames, plans, args.swap_frames,
                                            args.paced_warmup, sampler, fid, paced=True, swap=(1.0, {"M": cfg["M"]}))
        swap_info["latency_us_other_frames"] = stats(lat, 1e6 / PACED_HZ)
        infos = {n: loops[n].info() for n in loops}
        for lp in loops.values():
            lp.close()
        loops = {}
        # 5) the serving mix (LTAO + MCAO + 2 ELT SCAO, BF16, graph mode), per-loop latency
        mix = None
        if rank == 0 and args.mix_seconds > 0:
            sampler.mark(True)
            mix = serving_mix(args.mix_seconds, with_alone=False)
            sampler.mark(False)
    finally:
        for lp in loops.values():
            lp.close()
        sampler.stop()
    lat = {n: stats([r["latency_us"] for r in per[n]]) for n in per}
    mvm_us = {n: statistics.median([r["mvm_us"] for r in stg[n]]) for n in stg}
    gbs = {n: mvm_bytes(infos[n], cfgs[n]) / (mvm_us[n] * 1e-6) / 1e9 for n in stg}
    stage = {n: {k: statistics.median([r[k] for r in stg[n]]) for k in ("slopes_us", "mvm_us", "polc_us")}
             for n in stg}

    # CPU oracle on the host cores (rank 0, N=1 only), plus parity of the first frames
    cpu = None
    parity = None
    if rank == 0 and world == 1 and not args.no_cpu:
        n_or = args.parity_frames
        times, cmds_ref, _ = cpu_oracle(cfg, frames, nframes=n_or)
        cpu = {"value": statistics.median(times), "unit": "us", "cores": 1, "kind": "oracle",
               "sample": f"{n_or} full MCAO frames (after 1 warm-up frame) through the float64 numpy oracle on 1 "
                         "host thread; same seeded frames and matrices"}
        with rtc.Loop(cfg, device=local) as chk:
            errs = []
            for k in range(n_or + 1):
                chk.process_frame(k + 1, dev_frames[k % len(dev_frames)])
                _, a = chk.get_commands(timeout_us=10_000_000)
                if k >= 1:
                    r = cmds_ref[k - 1]
                    errs.append(float(np.max(np.abs(a - r)) / np.max(np.abs(r))))
        parity = {"frames": len(errs), "max_rel_err_commands": max(errs), "tol": 1e-5}
        cpu["stages_1_thread"] = oracle_stages(cfg, frames)
        cpu["stages_all_cores"] = oracle_stages_all_cores()
        cpu["host"] = host_cpu()

    # max over ranks (replicas: the slowest replica's latencies)
    vals = max_over_ranks([lat["f32"]["p50"], ms_total / args.steps, float(np.median(e2e_lat))], world, "cuda")
    if rank != 0:
        return
    traffic = profiled_traffic()
    mb = mvm_bytes(infos["f32"], cfg)
    res = {
        "metric": METRIC, "value": vals[0], "unit": "us", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": vals[1], "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded frames, random-init matrices)",
        "config": bench_config(cfg, world),
        "latency_us": lat["f32"],
        "bf16": {"latency_us": lat["bf16"], "stage_us": stage["bf16"]},
        "e4m3": {"latency_us": lat["e4m3"], "stage_us": stage["e4m3"]},
        "stage_us": stage["f32"],
        "mvm_gbs": gbs,
        "mvm_frac_of_hbm": {n: gbs[n] / peak for n in gbs},
        "mvm_frames": args.stage_frames,
        "paced": paced,
        "swap": swap_info,
        "e2e": {"value": vals[2], "unit": "us", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": 4 * (infos["f32"]["na"] + infos["f32"]["ns"]),
                "latency_us": stats(e2e_lat), "process_frame_latency_us": stats(pf_lat)},
        "serving_mix": mix,
        "roofline": {"bound": "hbm", "achieved": gbs["f32"], "peak": peak, "unit": "GB/s",
                     "frac": gbs["f32"] / peak, "traffic": traffic, "kernel": "gemv_kernel<f32> (reconstruction MVM)",
                     "algorithmic_bytes_per_launch": mb, "peak_kind": peak_kind},
        "gpu_launches": 4 * args.steps,   # per frame: slopes, MVM (with finalisation), telemetry pack, POLC
        "clocks": sampler.summary(),
    }
    if cpu:
        res["cpu_baseline"] = cpu
    if parity:
        res["parity"] = parity
    print(json.dumps(res), flush=True)


def format_errors(args, frames, rtc, dev_frames, local, nframes=100):
    """Slope and command errors of the GPU loop against the FP64 oracle, per frame, for this
    configuration and matrix format: against the oracle on the stored matrix (the parity check)
    and against the oracle on the float32 matrix (the cost of the format)."""
    from oracle import OracleLoop, quantize_rows
    from paper_1903_01852_gb300 import synth
    base = synth.make_config(args.workload)
    cfg = dict(base)
    if args.dtype != "f32":      # codes and scales from the oracle's quantiser feed both sides
        codes, scale = quantize_rows(base["M"], args.dtype)
        cfg.update(M=codes, M_scale=scale, M_dtype=args.dtype)
        if base.get("P") is not None:
            pc, ps = quantize_rows(base["P"], args.dtype)
            cfg.update(P=pc, P_scale=ps, P_dtype=args.dtype)
    stored, true = OracleLoop(cfg), OracleLoop(base)
    out = {"frames": nframes, "slopes_vs_stored": 0.0, "cmds_vs_stored": 0.0, "cmds_vs_f32_matrix": 0.0}
    with rtc.Loop(cfg, device=local, telemetry=True) as loop:
        for k in range(nframes):
            f = frames[k % len(frames)]
            loop.process_frame(k + 1, dev_frames[k % len(dev_frames)])
            fid, a = loop.get_commands(timeout_us=10_000_000)
            s, _ = loop.get_telemetry(fid, timeout_us=10_000_000)
            s_ref, a_ref = stored.step(f)
            _, a_true = true.step(f)
            rel = lambda x, r: float(np.max(np.abs(x - r)) / max(np.max(np.abs(r)), 1e-30))
            out["slopes_vs_stored"] = max(out["slopes_vs_stored"], rel(s, s_ref))
            out["cmds_vs_stored"] = max(out["cmds_vs_stored"], rel(a, a_ref))
            out["cmds_vs_f32_matrix"] = max(out["cmds_vs_f32_matrix"], rel(a, a_true))
    out["norm"] = "max over frames of max|x - x_oracle| / max|x_oracle|"
    return out


def quick_arm(args, cfg, frames, rtc, torch, local):
    """Profiling aid: only the unpaced, HBM-resident float32 loop on the chosen workload
    (--chunked: the frames submitted instead as rounds of row chunks, 8 per camera with more
    than 2x2 subapertures, from page-locked memory read in place, unpaced, ordinary launches)."""
    if args.chunked:
        return quick_chunked(args, cfg, frames, rtc, torch, local)
    dev_frames = []
    for f in frames:
        per = []
        for x in f:
            h, w = x.shape
            t = torch.zeros((h, (w + 7) // 8 * 8), dtype=torch.int16, device="cuda")
            t[:, :w] = torch.from_numpy(x.view(np.int16)).cuda()
            per.append(t[:, :w])
        dev_frames.append(per)
    sampler = ClockSampler(local)
    with rtc.Loop(cfg, device=local, timing=True, telemetry=True) as loop:
        rows, _ = run_unpaced_timed(loop, dev_frames, args.steps, args.warmup, sampler, 1)
    with rtc.Loop(cfg, device=local, stage_timing=True, telemetry=True) as loop:
        srows, _ = run_unpaced_timed(loop, dev_frames, args.steps, args.warmup, sampler, 1)
        info = loop.info()
    lat = stats([r["latency_us"] for r in rows])
    errors = None
    if args.errors:
        errors = format_errors(args, frames, rtc, dev_frames, local, args.error_frames)
    mvm = statistics.median([r["mvm_us"] for r in srows])
    sl = statistics.median([r["slopes_us"] for r in srows])
    po = statistics.median([r["polc_us"] for r in srows])
    print(json.dumps({"workload": args.workload, "quick": True, "dtype": args.dtype, "latency_us": lat,
                      "slopes_us": sl, "polc_us": po, "mvm_us": mvm, "errors": errors,
                      "mvm_gbs": mvm_bytes(info, cfg) / (mvm * 1e-6) / 1e9}), flush=True)


def quick_chunked(args, cfg, frames, rtc, torch, local):
    from paper_1903_01852_gb300 import synth
    host = []
    for f in frames:
        per = []
        for x in f:
            h, w = x.shape
            t = torch.zeros((h, (w + 7) // 8 * 8), dtype=torch.int16, pin_memory=True)
            t.numpy()[:, :w] = x.view(np.int16)
            per.append(t[:, :w])
        host.append(per)
    plans = [synth.chunk_plan(w, NCHUNKS if w.get("nsubx", 0) > 2 else 1) for w in cfg["wfs"]]
    sampler = ClockSampler(local)
    with rtc.Loop(cfg, device=local, telemetry=True) as loop:
        lat, _ = run_host_path(loop, host, plans, args.steps, args.warmup, sampler, 1, paced=False)
    print(json.dumps({"workload": args.workload, "quick": True, "chunked": True, "dtype": args.dtype,
                      "latency_us": stats(lat)}), flush=True)


SERVING_LOOPS = (("ltao", "ltao", 500.0), ("mcao", "mcao", 500.0), ("scao_a", "elt_scao_sh", 1000.0),
                 ("scao_b", "elt_scao_sh", 1000.0))


def serving_mix(dur, with_alone=True, priorities=True):
    """Serving mix on one GPU: a HARMONI-like LTAO loop, the MAORY-like MCAO loop and two ELT SCAO SH
    loops resident at once (BF16 matrices, graph mode), admitted by HBM footprint into one server;
    frames arrive at 500 Hz (LTAO, MCAO) and 1 kHz (SCAO) with seeded staggered phases and +-20 us
    uniform jitter for dur seconds.  Latency per loop = rtc_server_submit -> commands written (the
    server's poller).  with_alone: each loop is also run alone with the same arrivals.
    priorities: the 1 kHz loops' streams one priority level above the 500 Hz loops'
    (rtc_geometry.priority), so their shorter frames get the SMs first."""
    import torch
    from paper_1903_01852_gb300 import binding as rtc
    from paper_1903_01852_gb300 import synth
    rng = np.random.default_rng(4242)
    cfgs, frames = {}, {}
    for name, conf, hz in SERVING_LOOPS:
        c = synth.make_config(conf, seed=5000 + len(cfgs))
        cfgs[name] = quant_config(c, rtc, torch, "bf16")
        cfgs[name]["priority"] = (0 if hz >= 1000.0 else 1) if priorities else 0
        frames[name] = synth.draw_frames(c, 2, seed=6000 + len(frames))
    foot = {n: rtc.footprint(cfgs[n], flags=rtc.RTC_FLAG_GRAPHS)[0] for n in cfgs}
    budget = int(sum(foot.values()) * 1.02)

    def schedule(names):
        ev = []
        for n, _, hz in SERVING_LOOPS:
            if n not in names:
                continue
            phase = rng.uniform(0, 1.0 / hz)
            t = 0.02 + phase
            while t < dur:
                ev.append((t + rng.uniform(-20e-6, 20e-6), n))
                t += 1.0 / hz
        return sorted(ev)

    def run(names):
        with rtc.Server(budget) as srv:
            ids = {n: srv.admit(cfgs[n]) for n in names}
            lps = {n: srv.loop(ids[n]) for n in names}
            for n in names:                       # stage two different frames in the ring's buffers
                for k in range(2):
                    for b, f in zip(lps[n].next_frame_buffers(), frames[n][k]):
                        b[:] = f
                    srv.submit(ids[n], k + 1)
                    lps[n].get_commands(timeout_us=10_000_000)
            for n in names:
                srv.stats(ids[n], reset=True)
            fid = {n: 10 for n in names}
            ev = schedule(names)
            gc.disable()
            t0 = time.perf_counter()
            for t, n in ev:
                while time.perf_counter() - t0 < t:
                    pass
                lps[n].next_frame_buffers()      # the slot is free (its previous frame is done)
                srv.submit(ids[n], fid[n])
                fid[n] += 1
                while True:                      # drain commands as they come (FIFO per loop)
                    try:
                        lps[n].get_commands(timeout_us=0)
                    except TimeoutError:
                        break
            elapsed = time.perf_counter() - t0
            gc.enable()
            for n in names:
                lps[n].sync()
            time.sleep(0.05)
            st = {n: srv.stats(ids[n]) for n in names}
            usage = srv.usage()
        return st, usage, len(ev) / elapsed

    names = [n for n, _, _ in SERVING_LOOPS]
    mix, usage, fps = run(names)
    alone = {n: run([n])[0][n] for n in names} if with_alone else None
    keys = ("p50_us", "p99_us", "p999_us", "mean_us", "jitter_rms_us", "max_us", "frames")
    loops = {}
    for n, conf, hz in SERVING_LOOPS:
        loops[n] = {"rate_hz": hz, "config": conf, "mix": {k: mix[n][k] for k in keys}}
        if alone:
            loops[n]["alone"] = {k: alone[n][k] for k in keys}
    return {"seconds": dur, "frames_per_s": fps, "budget_bytes": budget, "admitted_bytes": usage["used"],
            "priorities": "1 kHz loops above 500 Hz loops" if priorities else "all equal", "loops": loops}


def serving_arm(args):
    """The serving mix alone (--serving), each loop also run alone, one JSON line."""
    import torch
    torch.cuda.set_device(0)
    out = {"mode": "serving", "metric": "per-loop frame latency, serving mix on one GB300 (BF16 matrices, graphs)",
           "unit": "us", **serving_mix(args.serving_seconds, with_alone=True)}
    print(json.dumps(out), flush=True)


def variants_arm(args):
    """The hot path's variants, each against its baseline on the same loop:
    (1) implicit POLC (P, na x na, after the command) against explicit POLC (u = D a, ns x na, after the
        command; s + u formed in the slope kernel), MCAO FP32 (Section 3.4);
    (2) camera-paced MCAO FP32 latency while every frame's slopes, commands and per-WFS partial commands
        are recorded in the telemetry circular buffer and a library thread streams them to a file
        descriptor (Section 3.3), against the same loop without telemetry;
    (3) camera-paced MCAO latency against the number of row chunks (and column blocks) per LGS camera;
    (4) local against global normalisation of the ELT pyramid, FP32 and BF16."""
    import torch
    from paper_1903_01852_gb300 import binding as rtc
    from paper_1903_01852_gb300 import synth
    torch.cuda.set_device(0)
    sampler = ClockSampler(0)
    sampler.start()
    n_paced, n_warm = args.variant_frames, 300

    def dev_copy(frames):
        out = []
        for f in frames:
            per = []
            for x in f:
                h, w = x.shape
                t = torch.zeros((h, (w + 7) // 8 * 8), dtype=torch.int16, device="cuda")
                t[:, :w] = torch.from_numpy(x.view(np.int16)).cuda()
                per.append(t[:, :w])
            out.append(per)
        return out

    def pinned_copy(frames, pad=False):
        """Frames in page-locked memory; pad: rows padded to a multiple of 16 bytes (views keep
        the pitch), so that row chunks of any width are read in place."""
        out = []
        for f in frames:
            per = []
            for x in f:
                h, w = x.shape
                wp = (w + 7) // 8 * 8 if pad else w
                t = torch.zeros((h, wp), dtype=torch.int16, pin_memory=True)
                t.numpy()[:, :w] = x.view(np.int16)
                per.append(t[:, :w])
            out.append(per)
        return out

    out = {"mode": "variants", "unit": "us"}
    try:
        cfg, frames = make_workload()
        dev, host = dev_copy(frames), pinned_copy(frames)
        plans = [synth.chunk_plan(w, NCHUNKS if w["nsubx"] > 2 else 1) for w in cfg["wfs"]]
        # (1) POLC forms
        rng = np.random.default_rng(7)
        exp_cfg = dict(cfg, P=None, polc="explicit", D=synth.interaction_matrix(rng, cfg["ns"], cfg["na"]))
        polc = {}
        for name, c in (("implicit", cfg), ("explicit", exp_cfg)):
            with rtc.Loop(c, stage_timing=True) as sl:
                rows, _ = run_unpaced_timed(sl, dev, 200, 20, sampler, 1)
                pbytes = sl.info()["p_bytes"]
            with rtc.Loop(c, timing=True) as lp:
                ms, _, _, fid = run_unpaced(lp, dev, 300, 20, torch, sampler, 1)
            with rtc.Loop(c) as lp:
                lat, _ = run_host_path(lp, host, plans, n_paced, n_warm, sampler, 1, paced=True)
            polc_us = statistics.median([r["polc_us"] for r in rows])
            polc[name] = {"polc_product_us": polc_us, "polc_matrix_bytes": pbytes,
                          "polc_gbs": pbytes / (polc_us * 1e-6) / 1e9,
                          "unpaced_frame_period_us": ms * 1000.0 / 300, "paced_latency_us": stats(lat, 1e6 / PACED_HZ)}
        del exp_cfg
        out["polc"] = {"definition": "polc_product_us: the POLC kernel after the command (stage timing, "
                                     "serialised); unpaced_frame_period_us: back-to-back frames from HBM; "
                                     "paced_latency_us: last pixel in (the last round's one rtc_submit_pixels_n "
                                     f"call) -> commands returned at {PACED_HZ:.0f} Hz", **polc}
        # (2) telemetry streaming
        tel = {}
        all_streams = rtc.RTC_TEL_SLOPES | rtc.RTC_TEL_COMMANDS | rtc.RTC_TEL_PARTIALS
        with rtc.Loop(cfg) as lp:
            lat, _ = run_host_path(lp, host, plans, n_paced, n_warm, sampler, 1, paced=True)
            tel["without"] = stats(lat, 1e6 / PACED_HZ)
        with rtc.Loop(cfg, tel_depth=1000, tel_streams=all_streams) as lp, \
                open(os.devnull, "wb") as sink:
            lp.telemetry_stream_start(sink.fileno())
            lat, _ = run_host_path(lp, host, plans, n_paced, n_warm, sampler, 1, paced=True)
            lp.sync()
            st = lp.telemetry_stream_stop()
            tel["with"] = stats(lat, 1e6 / PACED_HZ)
            tel["stream"] = st
            tel["entry_bytes"] = st["bytes"] // max(st["entries"], 1)
        out["telemetry"] = {"definition": "paced MCAO FP32, last pixel in (the last round's one submission "
                                          "call) -> commands returned; 'with': every "
                                          "frame's slopes, commands and 9 per-WFS partial command vectors written "
                                          "by the GPU into a 1000-entry page-locked circular buffer, drained by the "
                                          "library's stream thread (copy out of the buffer, write() to /dev/null)",
                            **tel}
        # (3) pipelining depth: row chunks per LGS camera (= column blocks per LGS), FP32 and BF16
        chunks = {}
        bcfg = bf16_config(cfg, rtc, torch)
        for nch in (4, 8, 16, 40):
            for fmt, base in (("f32", cfg), ("bf16", bcfg)):
                if fmt == "bf16" and nch not in (8, 16):
                    continue
                c = dict(base, wfs=[dict(w, nblocks=nch) if w["nsubx"] > 2 else w for w in base["wfs"]])
                pl = [synth.chunk_plan(w, nch if w["nsubx"] > 2 else 1) for w in c["wfs"]]
                for pre in (False, True):
                    arr = []
                    with rtc.Loop(c, prelaunch=pre) as lp:
                        lat, _ = run_host_path(lp, host, pl, n_paced, n_warm, sampler, 1, paced=True, arrival=arr)
                    a = stats(arr, 1e6 / PACED_HZ)
                    chunks[f"{nch}_{fmt}{'_prelaunch' if pre else ''}"] = {
                        **{k: a[k] for k in ("p50", "p99", "p999", "jitter_rms", "deadline_misses", "n")},
                        "last_submission_p50": stats(lat)["p50"]}
        del bcfg
        out["chunks"] = {"definition": "paced MCAO latency (arrival of every camera's last rows -> commands "
                                       "returned, 500 Hz, 1.6 ms readout, one rtc_submit_pixels_n call per round) "
                                       "with each LGS camera's frame in N row chunks and its slopes in N column "
                                       "blocks, with and without RTC_FLAG_PRELAUNCH; key N_format[_prelaunch]",
                         **chunks}
        del cfg, frames, dev, host
        torch.cuda.empty_cache()
        # (5) the ELT SCAO Shack-Hartmann loop paced at its 1 kHz, its 740x740 frame read out in
        # 0.8 ms over 8 row chunks from page-locked memory, FP32 and BF16, with and without
        # pre-enqueued chunks
        scfg = synth.make_config("elt_scao_sh")
        sframes = synth.draw_frames(scfg, FRAME_RING, seed=5)
        shost = pinned_copy(sframes, pad=True)
        splans = [synth.chunk_plan(w, NCHUNKS) for w in scfg["wfs"]]
        scao = {}
        for fmt, c in (("f32", scfg), ("bf16", bf16_config(scfg, rtc, torch))):
            for pre in (False, True):
                arr = []
                with rtc.Loop(c, prelaunch=pre) as lp:
                    run_host_path(lp, shost, splans, 2 * n_paced, 2 * n_warm, sampler, 1, paced=True, arrival=arr,
                                  hz=1000.0, readout_ms=0.8)
                    used = lp.info()["prelaunch_used"]
                a = stats(arr, 1e3)
                scao[f"{fmt}{'_prelaunch' if pre else ''}"] = {
                    **{k: a[k] for k in ("p50", "p99", "p999", "jitter_rms", "deadline_misses", "n")},
                    "prelaunched_chunks": used}
        out["elt_scao_paced"] = {"definition": "ELT SCAO SH (74x74, 8608 slopes, 5316 actuators) paced at 1 kHz, "
                                               "0.8 ms readout over 8 row chunks from page-locked memory, one "
                                               "rtc_submit_pixels_n call per round; latency from the arrival of "
                                               "the last rows -> commands returned", **scao}
        del scfg, sframes, shost
        # (4) pyramid normalisation
        pcfg = synth.make_config("elt_scao_pyramid")
        pframes = synth.draw_frames(pcfg, FRAME_RING, seed=3)
        pdev = dev_copy(pframes)
        pyr = {}
        for norm in ("local", "global"):
            c = dict(pcfg, wfs=[dict(pcfg["wfs"][0], norm=norm)])
            for fmt, cc in (("f32", c), ("bf16", bf16_config(c, rtc, torch))):
                with rtc.Loop(cc, stage_timing=True) as sl:
                    rows, _ = run_unpaced_timed(sl, pdev, 500, 50, sampler, 1)
                with rtc.Loop(cc, timing=True) as lp:
                    rl, _ = run_unpaced_timed(lp, pdev, 1000, 50, sampler, 1)
                pyr[f"{norm}_{fmt}"] = {"slopes_us": statistics.median([r["slopes_us"] for r in rows]),
                                        "latency_us": stats([r["latency_us"] for r in rl])}
        out["pyramid_norm"] = {"definition": "ELT SCAO pyramid, frames from HBM, unpaced: slope-kernel time "
                                             "(stage timing) and frame latency (device events)", **pyr}
    finally:
        sampler.stop()
    out["clocks"] = sampler.summary()
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--paced-frames", type=int, default=20000, help="camera-paced frames per matrix format")
    ap.add_argument("--paced-warmup", type=int, default=500)
    ap.add_argument("--parity-frames", type=int, default=20, help="frames checked against the FP64 oracle")
    ap.add_argument("--swap-frames", type=int, default=2500, help="paced frames of the parameter-swap run")
    ap.add_argument("--serving", action="store_true", help="serving mix (LTAO + MCAO + 2 SCAO) instead")
    ap.add_argument("--serving-seconds", type=float, default=4.0)
    ap.add_argument("--latency-frames", type=int, default=20000,
                    help="event-timed frames per matrix format for the latency statistics")
    ap.add_argument("--stage-frames", type=int, default=300, help="stage-timed frames per format for the MVM GB/s")
    ap.add_argument("--mix-seconds", type=float, default=3.0,
                    help="seconds of the serving mix in the default run (0: leave it out)")
    ap.add_argument("--variants", action="store_true",
                    help="POLC forms, telemetry streaming, chunking depth, pyramid normalisation instead")
    ap.add_argument("--variant-frames", type=int, default=3000, help="paced frames per --variants case")
    ap.add_argument("--oracle-stages", type=int, default=0, help=argparse.SUPPRESS)
    ap.add_argument("--workload", default="mcao", help="configuration (profiling aid; the bench line is mcao)")
    ap.add_argument("--quick", action="store_true", help="profiling aid: only the unpaced loop")
    ap.add_argument("--dtype", default="f32", choices=["f32", "bf16", "e4m3"], help="matrix storage for --quick")
    ap.add_argument("--errors", action="store_true", help="--quick: also errors against the FP64 oracle")
    ap.add_argument("--chunked", action="store_true", help="--quick: rounds of row chunks from page-locked memory")
    ap.add_argument("--error-frames", type=int, default=100, help="--errors: frames compared with the oracle")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.oracle_stages:                    # child of oracle_stages_all_cores: host cores only, no GPU
        cfg, frames = make_workload()
        print(json.dumps(oracle_stages(cfg, frames, args.oracle_stages)), flush=True)
        return
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        reference_arm(args, world, rank)
    elif args.serving:
        if rank == 0:
            serving_arm(args)
    elif args.variants:
        if rank == 0:
            variants_arm(args)
    else:
        ours_arm(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
