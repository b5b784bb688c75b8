"""ctypes binding of ``librtc.so`` (include/rtc.h): argument marshalling only.

Every step of the hot path runs in the library's CUDA kernels; this module
only builds the C structs from a configuration dict, passes pointers (numpy
arrays for host data, torch tensors for device data) and turns status codes
into exceptions.  There is no fallback: if the library is missing or cannot
be loaded, importing this module raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# RTC_LIBRARY may name another build of the same library (e.g. one compiled with other tuning macros).
LIB_PATH = os.environ.get("RTC_LIBRARY") or os.path.join(HERE, "librtc.so")

RTC_OK, RTC_EINVAL, RTC_ENOMEM, RTC_ETIMEDOUT = 0, -1, -2, -3
RTC_EORDER, RTC_EDROPPED, RTC_ECUDA, RTC_ENOENT, RTC_ENOTSUP = -4, -5, -6, -7, -8
RTC_WFS_SH, RTC_WFS_PYRAMID = 0, 1
RTC_F32, RTC_BF16, RTC_E4M3 = 0, 1, 2
RTC_THRESH_SUBTRACT, RTC_THRESH_CLIP = 0, 1
RTC_NORM_LOCAL, RTC_NORM_GLOBAL = 0, 1
RTC_POLC_IMPLICIT, RTC_POLC_EXPLICIT = 0, 1
RTC_FLAG_TIMING, RTC_FLAG_TELEMETRY, RTC_FLAG_STAGE_TIMING, RTC_FLAG_UPDATABLE, RTC_FLAG_GRAPHS = 1, 2, 4, 8, 16
RTC_FLAG_PARTIAL, RTC_FLAG_PRELAUNCH = 32, 64
RTC_MAX_WFS = 16
RTC_TEL_SLOPES, RTC_TEL_COMMANDS, RTC_TEL_PARTIALS = 1, 2, 4
DTYPES = {"f32": RTC_F32, "bf16": RTC_BF16, "e4m3": RTC_E4M3}
CODE_NP = {RTC_F32: np.float32, RTC_BF16: np.uint16, RTC_E4M3: np.uint8}
STATUS = {0: "RTC_OK", -1: "RTC_EINVAL", -2: "RTC_ENOMEM", -3: "RTC_ETIMEDOUT", -4: "RTC_EORDER",
          -5: "RTC_EDROPPED", -6: "RTC_ECUDA", -7: "RTC_ENOENT", -8: "RTC_ENOTSUP"}

f32p = C.POINTER(C.c_float)


class rtc_wfs(C.Structure):
    _fields_ = [("kind", C.c_int32), ("width", C.c_int32), ("height", C.c_int32),
                ("nsubx", C.c_int32), ("nsuby", C.c_int32), ("npx", C.c_int32), ("ox", C.c_int32),
                ("oy", C.c_int32), ("pupil", C.c_int32), ("qx", C.c_int32 * 4), ("qy", C.c_int32 * 4),
                ("valid", C.POINTER(C.c_uint8)), ("nblocks", C.c_int32), ("norm", C.c_int32)]


class rtc_geometry(C.Structure):
    _fields_ = [("nwfs", C.c_int32), ("wfs", C.POINTER(rtc_wfs)), ("device", C.c_int32),
                ("flags", C.c_uint32), ("ring", C.c_int32), ("tel_depth", C.c_int32), ("tel_streams", C.c_uint32),
                ("tel_decimate", C.c_int32), ("priority", C.c_int32), ("prelaunch_wait_us", C.c_int32)]


class rtc_calib(C.Structure):
    _fields_ = [("dark", C.POINTER(f32p)), ("flat", C.POINTER(f32p)), ("threshold", f32p),
                ("thresh_mode", C.POINTER(C.c_int32)), ("ref_slopes", f32p)]


class rtc_cmat(C.Structure):
    _fields_ = [("na", C.c_int32), ("ns", C.c_int32), ("dtype", C.c_int32), ("data", C.c_void_p),
                ("row_scale", f32p)]


class rtc_polc(C.Structure):
    _fields_ = [("P", C.c_void_p), ("dtype", C.c_int32), ("row_scale", f32p), ("gain", C.c_float),
                ("leak", C.c_float), ("a0", f32p), ("clip", C.c_int32), ("amin", C.c_float),
                ("amax", C.c_float), ("mode", C.c_int32), ("D", C.c_void_p), ("d_dtype", C.c_int32),
                ("d_row_scale", f32p)]


class rtc_chunk(C.Structure):
    _fields_ = [("frame_id", C.c_uint64), ("wfs", C.c_int32), ("row_begin", C.c_int32),
                ("row_end", C.c_int32), ("px", C.c_void_p), ("pitch", C.c_size_t)]


class rtc_timing(C.Structure):
    _fields_ = [("frame_id", C.c_uint64), ("slopes_us", C.c_float), ("mvm_us", C.c_float),
                ("final_us", C.c_float), ("polc_us", C.c_float), ("latency_us", C.c_float),
                ("frame_us", C.c_float)]


class rtc_tel_record(C.Structure):
    _fields_ = [("index", C.c_uint64), ("frame_id", C.c_uint64), ("t_commands_ns", C.c_uint64),
                ("t_written_ns", C.c_uint64), ("lost", C.c_uint64)]


class rtc_tel_stream_stats(C.Structure):
    _fields_ = [("entries", C.c_uint64), ("lost", C.c_uint64), ("bytes", C.c_uint64), ("write_error", C.c_int32)]


class rtc_update_desc(C.Structure):
    _fields_ = [("M", C.c_void_p), ("M_scale", f32p), ("P", C.c_void_p), ("P_scale", f32p),
                ("dark", C.POINTER(f32p)), ("flat", C.POINTER(f32p)), ("threshold", f32p), ("ref_slopes", f32p),
                ("set_control", C.c_int32), ("gain", C.c_float), ("leak", C.c_float), ("clip", C.c_int32),
                ("amin", C.c_float), ("amax", C.c_float)]


class rtc_server_loop_info(C.Structure):
    _fields_ = [("admitted", C.c_int32), ("footprint_bytes", C.c_uint64), ("frames", C.c_uint64),
                ("p50_us", C.c_double), ("p99_us", C.c_double), ("p999_us", C.c_double), ("mean_us", C.c_double),
                ("jitter_rms_us", C.c_double), ("max_us", C.c_double)]


class rtc_info(C.Structure):
    _fields_ = [("na", C.c_int32), ("ns", C.c_int32), ("nwfs", C.c_int32), ("nblocks", C.c_int32),
                ("nrows", C.c_int32), ("m_dtype", C.c_int32), ("p_dtype", C.c_int32),
                ("m_bytes", C.c_uint64), ("p_bytes", C.c_uint64), ("pixel_bytes", C.c_uint64),
                ("device_bytes", C.c_uint64), ("frames_done", C.c_uint64), ("frames_dropped", C.c_uint64),
                ("frames_overrun", C.c_uint64), ("swaps", C.c_uint64), ("prelaunch_used", C.c_uint64),
                ("prelaunch_cancelled", C.c_uint64), ("prelaunch_expired", C.c_uint64)]


class rtc_master_desc(C.Structure):
    _fields_ = [("device", C.c_int32), ("na", C.c_int32), ("nshards", C.c_int32), ("polc", C.POINTER(rtc_polc))]


# (name, restype, argtypes) of every entry point declared in include/rtc.h
SIGNATURES = [
    ("rtc_create", C.c_int, [C.POINTER(rtc_geometry), C.POINTER(rtc_calib), C.POINTER(rtc_cmat),
                             C.POINTER(rtc_polc), C.POINTER(C.c_void_p)]),
    ("rtc_destroy", C.c_int, [C.c_void_p]),
    ("rtc_submit_pixels", C.c_int, [C.c_void_p, C.POINTER(rtc_chunk)]),
    ("rtc_submit_pixels_n", C.c_int, [C.c_void_p, C.POINTER(rtc_chunk), C.c_int32, C.POINTER(C.c_int32)]),
    ("rtc_process_frame", C.c_int, [C.c_void_p, C.c_uint64, C.POINTER(C.c_void_p), C.POINTER(C.c_size_t)]),
    ("rtc_next_frame_buffers", C.c_int, [C.c_void_p, C.POINTER(C.c_void_p), C.POINTER(C.c_size_t)]),
    ("rtc_submit_frame_graph", C.c_int, [C.c_void_p, C.c_uint64]),
    ("rtc_get_commands", C.c_int, [C.c_void_p, f32p, C.c_size_t, C.POINTER(C.c_uint64), C.c_int64]),
    ("rtc_get_telemetry", C.c_int, [C.c_void_p, C.c_uint64, f32p, C.c_size_t, f32p, C.c_size_t, C.c_int64]),
    ("rtc_get_timing", C.c_int, [C.c_void_p, C.c_uint64, C.POINTER(rtc_timing), C.c_int64]),
    ("rtc_telemetry_read", C.c_int, [C.c_void_p, C.POINTER(rtc_tel_record), f32p, C.c_size_t, f32p, C.c_size_t,
                                     f32p, C.c_size_t, C.c_int64]),
    ("rtc_telemetry_stream_start", C.c_int, [C.c_void_p, C.c_int]),
    ("rtc_telemetry_stream_stop", C.c_int, [C.c_void_p, C.POINTER(rtc_tel_stream_stats)]),
    ("rtc_update", C.c_int, [C.c_void_p, C.POINTER(rtc_update_desc)]),
    ("rtc_get_state", C.c_int, [C.c_void_p, f32p, C.c_size_t]),
    ("rtc_set_state", C.c_int, [C.c_void_p, f32p, C.c_size_t]),
    ("rtc_sync", C.c_int, [C.c_void_p]),
    ("rtc_check_guards", C.c_int, [C.c_void_p, C.POINTER(C.c_int32)]),
    ("rtc_get_stream", C.c_int, [C.c_void_p, C.POINTER(C.c_void_p)]),
    ("rtc_get_info", C.c_int, [C.c_void_p, C.POINTER(rtc_info)]),
    ("rtc_footprint", C.c_int, [C.POINTER(rtc_geometry), C.POINTER(rtc_calib), C.POINTER(rtc_cmat),
                                C.POINTER(rtc_polc), C.POINTER(C.c_uint64), C.POINTER(C.c_uint64)]),
    ("rtc_last_error", C.c_char_p, [C.c_void_p]),
    ("rtc_server_create", C.c_int, [C.c_int32, C.c_uint64, C.POINTER(C.c_void_p)]),
    ("rtc_server_destroy", C.c_int, [C.c_void_p]),
    ("rtc_server_admit", C.c_int, [C.c_void_p, C.POINTER(rtc_geometry), C.POINTER(rtc_calib), C.POINTER(rtc_cmat),
                                   C.POINTER(rtc_polc), C.POINTER(C.c_int32)]),
    ("rtc_server_release", C.c_int, [C.c_void_p, C.c_int32]),
    ("rtc_server_loop", C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_void_p)]),
    ("rtc_server_submit", C.c_int, [C.c_void_p, C.c_int32, C.c_uint64]),
    ("rtc_server_stats", C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.POINTER(rtc_server_loop_info)]),
    ("rtc_server_usage", C.c_int, [C.c_void_p, C.POINTER(C.c_uint64), C.POINTER(C.c_uint64), C.POINTER(C.c_int32),
                                   C.POINTER(C.c_int32)]),
    ("rtc_server_last_error", C.c_char_p, [C.c_void_p]),
    ("rtc_quantize_rows", C.c_int, [C.c_int32, C.c_int32, C.c_int32, C.c_void_p, C.c_size_t, C.c_void_p,
                                    C.c_void_p, C.c_void_p]),
    ("rtc_set_partial_output", C.c_int, [C.c_void_p, C.c_void_p]),
    ("rtc_master_create", C.c_int, [C.POINTER(rtc_master_desc), C.POINTER(C.c_void_p)]),
    ("rtc_master_input", C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_void_p)]),
    ("rtc_master_set_input", C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_size_t]),
    ("rtc_master_step", C.c_int, [C.c_void_p, C.c_uint64]),
    ("rtc_master_get_commands", C.c_int, [C.c_void_p, f32p, C.c_size_t, C.POINTER(C.c_uint64), C.c_int64]),
    ("rtc_master_destroy", C.c_int, [C.c_void_p]),
    ("rtc_master_last_error", C.c_char_p, [C.c_void_p]),
    ("rtc_reconstruct_noalloc", C.c_int, [C.c_int32, C.c_int32, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p,
                                          C.c_void_p, C.c_void_p, C.c_void_p, C.c_float, C.c_float, C.c_void_p]),
]


def load(path: str = LIB_PATH) -> C.CDLL:
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with `python -m paper_1903_01852_gb300.build`")
    lib = C.CDLL(path)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = load()


class RtcError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


def _err(loop_ptr=None):
    return lib.rtc_last_error(loop_ptr).decode(errors="replace")


def _check(rc, loop_ptr=None, allow=()):
    if rc != RTC_OK and rc not in allow:
        raise RtcError(rc, _err(loop_ptr))
    return rc


def _fptr(a):
    return None if a is None else a.ctypes.data_as(f32p)


def _f32(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float32)


def _ptr(x):
    """Address of a numpy array or torch tensor (host or device)."""
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    return x.ctypes.data


def _pitch(x):
    """Row pitch in bytes of a 2-D uint16 array or tensor."""
    if hasattr(x, "stride") and callable(x.stride):
        return x.stride(0) * x.element_size()
    return x.strides[0]


class _Described:
    """The C structs of one loop description, and the arrays they point into."""


def describe(cfg, device=0, flags=0, ring=4, tel=(0, 0, 1)):
    """Build rtc_geometry / rtc_calib / rtc_cmat / rtc_polc from a configuration dict.
    tel: (depth, RTC_TEL_* streams, decimate) of the telemetry circular buffer."""
    wl = cfg["wfs"]
    if len(wl) > RTC_MAX_WFS:
        raise ValueError("too many WFS")
    st = _Described()
    keep = []   # host arrays that must outlive the call that uses the structs
    warr = (rtc_wfs * len(wl))()
    darks = (f32p * len(wl))()
    flats = (f32p * len(wl))()
    thr = np.array([w.get("threshold", 0.0) for w in wl], np.float32)
    mode = np.array([RTC_THRESH_CLIP if w.get("thresh_mode") == "clip" else RTC_THRESH_SUBTRACT for w in wl],
                    np.int32)
    for k, w in enumerate(wl):
        s = warr[k]
        s.kind = RTC_WFS_SH if w["kind"] == "sh" else RTC_WFS_PYRAMID
        s.width, s.height = w["width"], w["height"]
        if w["kind"] == "sh":
            s.nsubx, s.nsuby, s.npx, s.ox, s.oy = w["nsubx"], w["nsuby"], w["npx"], w["ox"], w["oy"]
        else:
            s.pupil = w["pupil"]
            for q in range(4):
                s.qx[q], s.qy[q] = w["qx"][q], w["qy"][q]
            s.norm = RTC_NORM_GLOBAL if w.get("norm", "local") == "global" else RTC_NORM_LOCAL
        v = np.ascontiguousarray(w["valid"], dtype=np.uint8)
        keep.append(v)
        s.valid = v.ctypes.data_as(C.POINTER(C.c_uint8))
        s.nblocks = int(w.get("nblocks", 1))
        d, f = _f32(w.get("dark")), _f32(w.get("flat"))
        keep += [d, f]
        darks[k] = _fptr(d)
        flats[k] = _fptr(f)
    st.geo = rtc_geometry(len(wl), warr, device, flags, ring, int(tel[0]), int(tel[1]), int(tel[2]),
                          int(cfg.get("priority", 0)), int(cfg.get("prelaunch_wait_us", 0)))
    ref = _f32(cfg.get("ref_slopes"))
    st.cal = rtc_calib(darks, flats, thr.ctypes.data_as(f32p), mode.ctypes.data_as(C.POINTER(C.c_int32)), _fptr(ref))
    mdt = DTYPES[cfg.get("M_dtype", "f32")]
    M = np.ascontiguousarray(cfg["M"], dtype=CODE_NP[mdt])
    ms = _f32(cfg.get("M_scale"))
    st.cm = rtc_cmat(M.shape[0], M.shape[1], mdt, M.ctypes.data, _fptr(ms))
    P = cfg.get("P")
    pdt = DTYPES[cfg.get("P_dtype", "f32")]
    Pa = None if P is None else np.ascontiguousarray(P, dtype=CODE_NP[pdt])
    ps = _f32(cfg.get("P_scale"))
    a0 = _f32(cfg.get("a0"))
    clip = cfg.get("clip")
    explicit = cfg.get("polc", "implicit") == "explicit"
    if explicit:
        Pa = ps = None
    ddt = DTYPES[cfg.get("D_dtype", "f32")]
    Da = np.ascontiguousarray(cfg["D"], dtype=CODE_NP[ddt]) if explicit else None
    dsc = _f32(cfg.get("D_scale")) if explicit else None
    st.pol = rtc_polc(None if Pa is None else Pa.ctypes.data, pdt, _fptr(ps), float(cfg["gain"]), float(cfg["leak"]),
                      _fptr(a0), 1 if clip else 0, float(clip[0]) if clip else 0.0, float(clip[1]) if clip else 0.0,
                      RTC_POLC_EXPLICIT if explicit else RTC_POLC_IMPLICIT, None if Da is None else Da.ctypes.data,
                      ddt, _fptr(dsc))
    st.keep = keep + [warr, darks, flats, thr, mode, ref, M, ms, Pa, ps, a0, Da, dsc]
    return st


def footprint(cfg, flags=0):
    """rtc_footprint: (resident, peak) device bytes of a loop built from cfg."""
    st = describe(cfg, 0, flags)
    r, p = C.c_uint64(), C.c_uint64()
    _check(lib.rtc_footprint(C.byref(st.geo), C.byref(st.cal), C.byref(st.cm), C.byref(st.pol), C.byref(r),
                             C.byref(p)))
    return r.value, p.value


class Loop:
    """One AO loop on one GPU, built from a configuration dict (see synth)."""

    def __init__(self, cfg, device=0, timing=False, telemetry=False, ring=4, stage_timing=False, updatable=False,
                 graphs=False, tel_depth=0, tel_streams=RTC_TEL_SLOPES | RTC_TEL_COMMANDS, tel_decimate=1,
                 partial=False, prelaunch=False, _handle=None):
        self.cfg = cfg
        self.na = int(cfg["na"])
        self._owned = _handle is None
        if _handle is None:
            flags = ((RTC_FLAG_TIMING if timing or stage_timing else 0) | (RTC_FLAG_TELEMETRY if telemetry else 0)
                     | (RTC_FLAG_STAGE_TIMING if stage_timing else 0) | (RTC_FLAG_UPDATABLE if updatable else 0)
                     | (RTC_FLAG_GRAPHS if graphs else 0) | (RTC_FLAG_PARTIAL if partial else 0)
                     | (RTC_FLAG_PRELAUNCH if prelaunch else 0))
            st = describe(cfg, device, flags, ring, (tel_depth, tel_streams, tel_decimate))
            h = C.c_void_p()
            _check(lib.rtc_create(C.byref(st.geo), C.byref(st.cal), C.byref(st.cm), C.byref(st.pol), C.byref(h)))
            self._h = h
        else:
            self._h = C.c_void_p(_handle)
        inf = self.info()
        self.ns = inf["ns"]
        self._cmd = np.empty(self.na, np.float32)

    # -- lifetime ---------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None) and self._h.value and getattr(self, "_owned", True):
            lib.rtc_destroy(self._h)
        self._h = C.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- per frame --------------------------------------------------------
    def submit(self, frame_id, wfs, row_begin, row_end, px, pitch=None):
        """Submit rows [row_begin, row_end) of WFS ``wfs``; ``px`` is a 2-D uint16 array/tensor
        whose first row is row_begin.  Returns RTC_OK or RTC_EDROPPED."""
        ch = rtc_chunk(frame_id, wfs, row_begin, row_end, _ptr(px), _pitch(px) if pitch is None else pitch)
        return _check(lib.rtc_submit_pixels(self._h, C.byref(ch)), self._h, allow=(RTC_EDROPPED,))

    @staticmethod
    def chunks(frame_id, items):
        """A ctypes array of rtc_chunk for submit_chunks: items are (wfs, row_begin, row_end, px)
        with px as for submit.  Its frame_id fields may be rewritten for later frames."""
        arr = (rtc_chunk * len(items))()
        for i, (w, r0, r1, px) in enumerate(items):
            arr[i] = rtc_chunk(frame_id, w, r0, r1, _ptr(px), _pitch(px))
        return arr

    def submit_chunks(self, arr):
        """rtc_submit_pixels_n on a ctypes array of rtc_chunk (see chunks).  Returns RTC_OK
        or RTC_EDROPPED; raises on the first chunk that fails (those before it are accepted)."""
        acc = C.c_int32()
        return _check(lib.rtc_submit_pixels_n(self._h, arr, len(arr), C.byref(acc)), self._h, allow=(RTC_EDROPPED,))

    def submit_frame(self, frame_id, frames, plans=None):
        """Submit a whole frame as row chunks; ``plans[w]`` lists (row_begin, row_end) for WFS w
        (default: one chunk per WFS).  WFS are interleaved chunk by chunk, as parallel cameras
        would deliver them."""
        status = RTC_OK
        plans = plans or [[(0, f.shape[0])] for f in frames]
        n = max(len(p) for p in plans)
        for c in range(n):
            for w, plan in enumerate(plans):
                if c < len(plan):
                    r0, r1 = plan[c]
                    rc = self.submit(frame_id, w, r0, r1, frames[w][r0:r1])
                    status = rc if rc != RTC_OK else status
        return status

    def process_frame(self, frame_id, dev_frames):
        """Whole frame from device-resident uint16 tensors (one per WFS)."""
        n = len(dev_frames)
        px = (C.c_void_p * n)(*[t.data_ptr() for t in dev_frames])
        pitch = (C.c_size_t * n)(*[t.stride(0) * t.element_size() for t in dev_frames])
        return _check(lib.rtc_process_frame(self._h, frame_id, px, pitch), self._h, allow=(RTC_EDROPPED,))

    def next_frame_buffers(self):
        """Graph mode: numpy views (uint16, height x width) of the page-locked buffers the
        next frame is written into."""
        n = len(self.cfg["wfs"])
        px = (C.c_void_p * n)()
        pitch = (C.c_size_t * n)()
        _check(lib.rtc_next_frame_buffers(self._h, px, pitch), self._h)
        out = []
        for k, w in enumerate(self.cfg["wfs"]):
            buf = (C.c_uint16 * (w["height"] * pitch[k] // 2)).from_address(px[k])
            out.append(np.frombuffer(buf, dtype=np.uint16).reshape(w["height"], pitch[k] // 2)[:, :w["width"]])
        return out

    def submit_graph(self, frame_id):
        """Graph mode: launch the captured frame graph on the buffers last returned."""
        return _check(lib.rtc_submit_frame_graph(self._h, frame_id), self._h, allow=(RTC_EDROPPED,))

    def get_commands(self, timeout_us=-1, out=None):
        out = self._cmd.copy() if out is None else out
        fid = C.c_uint64()
        rc = lib.rtc_get_commands(self._h, out.ctypes.data_as(f32p), self.na, C.byref(fid), int(timeout_us))
        if rc == RTC_ETIMEDOUT:
            raise TimeoutError(_err(self._h))
        _check(rc, self._h)
        return fid.value, out

    def get_telemetry(self, frame_id, timeout_us=-1):
        s = np.empty(self.ns, np.float32)
        a = np.empty(self.na, np.float32)
        _check(lib.rtc_get_telemetry(self._h, frame_id, s.ctypes.data_as(f32p), self.ns,
                                     a.ctypes.data_as(f32p), self.na, int(timeout_us)), self._h)
        return s, a

    def telemetry_read(self, timeout_us=-1, slopes=True, cmds=True, partials=False):
        """rtc_telemetry_read: the oldest unread entry of the telemetry circular buffer, as
        (record dict, slopes, commands, partials [nwfs, na]); sections not asked for are None."""
        nw = len(self.cfg["wfs"])
        s = np.empty(self.ns, np.float32) if slopes else None
        a = np.empty(self.na, np.float32) if cmds else None
        p = np.empty((nw, self.na), np.float32) if partials else None
        r = rtc_tel_record()
        ptr = lambda x: None if x is None else x.ctypes.data_as(f32p)
        _check(lib.rtc_telemetry_read(self._h, C.byref(r), ptr(s), self.ns if slopes else 0, ptr(a),
                                      self.na if cmds else 0, ptr(p), nw * self.na if partials else 0,
                                      int(timeout_us)), self._h)
        return {k: getattr(r, k) for k, _ in rtc_tel_record._fields_}, s, a, p

    def telemetry_stream_start(self, fd):
        """rtc_telemetry_stream_start: a library thread writes every entry to the file descriptor fd."""
        _check(lib.rtc_telemetry_stream_start(self._h, int(fd)), self._h)

    def telemetry_stream_stop(self):
        st = rtc_tel_stream_stats()
        _check(lib.rtc_telemetry_stream_stop(self._h, C.byref(st)), self._h)
        return {k: getattr(st, k) for k, _ in rtc_tel_stream_stats._fields_}

    def get_timing(self, frame_id, timeout_us=-1):
        t = rtc_timing()
        _check(lib.rtc_get_timing(self._h, frame_id, C.byref(t), int(timeout_us)), self._h)
        return {k: getattr(t, k) for k, _ in rtc_timing._fields_}

    # -- parameter double buffer ---------------------------------------------
    def update(self, M=None, M_scale=None, P=None, P_scale=None, dark=None, flat=None, threshold=None,
               ref_slopes=None, control=None):
        """rtc_update: stage new parameters; the next frame to start uses them.
        dark / flat: dicts {wfs index: map}; control: (gain, leak, clip or None)."""
        keep = []

        def arr(x, dt):
            if x is None:
                return None
            a = np.ascontiguousarray(x, dtype=dt)
            keep.append(a)
            return a

        mdt = CODE_NP[DTYPES[self.cfg.get("M_dtype", "f32")]]
        pdt = CODE_NP[DTYPES[self.cfg.get("P_dtype", "f32")]]
        Ma, Pa = arr(M, mdt), arr(P, pdt)
        d = rtc_update_desc()
        d.M = None if Ma is None else Ma.ctypes.data
        d.M_scale = _fptr(arr(M_scale, np.float32))
        d.P = None if Pa is None else Pa.ctypes.data
        d.P_scale = _fptr(arr(P_scale, np.float32))
        nw = len(self.cfg["wfs"])
        for name, maps in (("dark", dark), ("flat", flat)):
            if maps:
                ptrs = (f32p * nw)()
                for k, m in maps.items():
                    ptrs[k] = _fptr(arr(m, np.float32))
                keep.append(ptrs)
                setattr(d, name, ptrs)
        d.threshold = _fptr(arr(threshold, np.float32))
        d.ref_slopes = _fptr(arr(ref_slopes, np.float32))
        if control is not None:
            g, l, clip = control
            d.set_control, d.gain, d.leak = 1, float(g), float(l)
            if clip:
                d.clip, d.amin, d.amax = 1, float(clip[0]), float(clip[1])
        _check(lib.rtc_update(self._h, C.byref(d)), self._h)

    # -- state ----------------------------------------------------------------
    def get_state(self):
        a = np.empty(self.na, np.float32)
        _check(lib.rtc_get_state(self._h, a.ctypes.data_as(f32p), self.na), self._h)
        return a

    def set_state(self, a):
        a = np.ascontiguousarray(a, dtype=np.float32)
        _check(lib.rtc_set_state(self._h, a.ctypes.data_as(f32p), self.na), self._h)

    def check_guards(self):
        """rtc_check_guards: number of buffer guard regions something overwrote (0 when intact)."""
        n = C.c_int32()
        _check(lib.rtc_check_guards(self._h, C.byref(n)), self._h)
        return n.value

    def sync(self):
        _check(lib.rtc_sync(self._h), self._h)

    def stream(self):
        """The loop's cudaStream_t as an integer handle."""
        h = C.c_void_p()
        _check(lib.rtc_get_stream(self._h, C.byref(h)), self._h)
        return h.value or 0

    def info(self):
        i = rtc_info()
        _check(lib.rtc_get_info(self._h, C.byref(i)), self._h)
        return {k: getattr(i, k) for k, _ in rtc_info._fields_}

    @property
    def last_error(self):
        return _err(self._h)


def set_partial_output(loop, ptr):
    """rtc_set_partial_output: a RTC_FLAG_PARTIAL loop also writes its partial
    reconstruction to device address ptr (int, or None to stop)."""
    _check(lib.rtc_set_partial_output(loop._h, ptr), loop._h)


class Master:
    """The control law of a loop split by WFS (rtc_master_*): adds the shards'
    partial reconstructions in shard order, POLC term, leaky integrator."""

    def __init__(self, cfg, nshards, device=0):
        self.na = int(cfg["na"])
        st = describe(dict(cfg, wfs=cfg.get("wfs") or [], M=np.zeros((self.na, 0), np.float32)), device)
        self._keep = st
        d = rtc_master_desc(device, self.na, int(nshards), C.pointer(st.pol))
        h = C.c_void_p()
        rc = lib.rtc_master_create(C.byref(d), C.byref(h))
        if rc != RTC_OK:
            raise RtcError(rc, lib.rtc_master_last_error(None).decode(errors="replace"))
        self._h = h
        self._cmd = np.empty(self.na, np.float32)

    def _err(self):
        return lib.rtc_master_last_error(self._h).decode(errors="replace")

    def input(self, shard):
        p = C.c_void_p()
        rc = lib.rtc_master_input(self._h, shard, C.byref(p))
        if rc != RTC_OK:
            raise RtcError(rc, self._err())
        return p.value

    def set_input(self, shard, y):
        """Copy a shard's partial (numpy float32 [na], or a device pointer) into input `shard`."""
        if isinstance(y, int):
            rc = lib.rtc_master_set_input(self._h, shard, y, self.na)
        else:
            y = np.ascontiguousarray(y, dtype=np.float32)
            rc = lib.rtc_master_set_input(self._h, shard, y.ctypes.data, y.size)
        if rc != RTC_OK:
            raise RtcError(rc, self._err())

    def step(self, frame_id):
        rc = lib.rtc_master_step(self._h, frame_id)
        if rc != RTC_OK:
            raise RtcError(rc, self._err())

    def get_commands(self, timeout_us=-1):
        fid = C.c_uint64()
        rc = lib.rtc_master_get_commands(self._h, self._cmd.ctypes.data_as(f32p), self.na, C.byref(fid), timeout_us)
        if rc == RTC_ETIMEDOUT:
            raise TimeoutError(self._err())
        if rc != RTC_OK:
            raise RtcError(rc, self._err())
        return fid.value, self._cmd.copy()

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib.rtc_master_destroy(self._h)
            self._h = C.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def quantize_rows(M, fmt, stream=None):
    """Per-row scaled BF16 / E4M3 quantisation of a float32 CUDA tensor [na, ns]
    (rtc_quantize_rows).  Returns (codes, scale) CUDA tensors."""
    import torch
    dt = DTYPES[fmt]
    na, ns = M.shape
    codes = torch.empty((na, ns), dtype=torch.int16 if dt == RTC_BF16 else torch.uint8, device=M.device)
    scale = torch.empty(na, dtype=torch.float32, device=M.device)
    st = stream if stream is not None else torch.cuda.current_stream(M.device).cuda_stream
    _check(lib.rtc_quantize_rows(dt, na, ns, M.data_ptr(), M.stride(0), codes.data_ptr(), scale.data_ptr(), st))
    return codes, scale


class Server:
    """Several loops resident on one GPU, admitted by device-memory footprint (rtc_server_*)."""

    def __init__(self, budget_bytes, device=0):
        h = C.c_void_p()
        _check(lib.rtc_server_create(device, int(budget_bytes), C.byref(h)))
        self._h = h
        self.cfgs = {}

    def _err(self):
        return lib.rtc_server_last_error(self._h).decode(errors="replace")

    def admit(self, cfg, telemetry=False, ring=4):
        st = describe(cfg, 0, RTC_FLAG_TELEMETRY if telemetry else 0, ring)
        lid = C.c_int32()
        rc = lib.rtc_server_admit(self._h, C.byref(st.geo), C.byref(st.cal), C.byref(st.cm), C.byref(st.pol),
                                  C.byref(lid))
        if rc != RTC_OK:
            raise RtcError(rc, self._err())
        self.cfgs[lid.value] = cfg
        return lid.value

    def loop(self, lid):
        """A non-owning Loop view of an admitted loop (None while queued)."""
        h = C.c_void_p()
        rc = lib.rtc_server_loop(self._h, lid, C.byref(h))
        if rc != RTC_OK:
            raise RtcError(rc, self._err())
        return None if not h.value else Loop(self.cfgs[lid], _handle=h.value)

    def submit(self, lid, frame_id):
        rc = lib.rtc_server_submit(self._h, lid, frame_id)
        if rc not in (RTC_OK, RTC_EDROPPED):
            raise RtcError(rc, self._err())
        return rc

    def stats(self, lid, reset=False):
        i = rtc_server_loop_info()
        rc = lib.rtc_server_stats(self._h, lid, 1 if reset else 0, C.byref(i))
        if rc != RTC_OK:
            raise RtcError(rc, self._err())
        return {k: getattr(i, k) for k, _ in rtc_server_loop_info._fields_}

    def usage(self):
        u, b, a, q = C.c_uint64(), C.c_uint64(), C.c_int32(), C.c_int32()
        _check(lib.rtc_server_usage(self._h, C.byref(u), C.byref(b), C.byref(a), C.byref(q)))
        return dict(used=u.value, budget=b.value, admitted=a.value, queued=q.value)

    def release(self, lid):
        rc = lib.rtc_server_release(self._h, lid)
        if rc != RTC_OK:
            raise RtcError(rc, self._err())
        self.cfgs.pop(lid, None)

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib.rtc_server_destroy(self._h)
            self._h = C.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
