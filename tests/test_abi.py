"""The C-ABI library loads and exports every entry point include/rtc.h declares
(CPU only: no call here reaches the GPU)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rtc.h")


def declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(rtc_\w+)\s*\(", text, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared()
    for n in ("rtc_create", "rtc_submit_pixels", "rtc_get_commands", "rtc_destroy", "rtc_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(rtc):
    missing = [n for n in declared() if not hasattr(rtc.lib, n)]
    assert not missing
    assert sorted(n for n, _, _ in rtc.SIGNATURES) == declared()


def test_create_rejects_null_and_bad_geometry_without_gpu(rtc):
    h = C.c_void_p()
    assert rtc.lib.rtc_create(None, None, None, None, C.byref(h)) == rtc.RTC_EINVAL
    assert h.value is None
    assert b"required" in rtc.lib.rtc_last_error(None)
    w = (rtc.rtc_wfs * 1)()
    w[0].kind, w[0].width, w[0].height = rtc.RTC_WFS_SH, 16, 16
    w[0].nsubx = w[0].nsuby = 3
    w[0].npx, w[0].nblocks = 8, 1          # 3 x 8 = 24 > 16: grid outside the frame
    geo = rtc.rtc_geometry(1, w, 0, 0, 4, 0, 0, 1)
    cm = rtc.rtc_cmat(1, 18, rtc.RTC_F32, C.c_void_p(1), None)
    pol = rtc.rtc_polc(None, 0, None, 0.5, 0.01, None, 0, 0.0, 0.0, 0, None, 0, None)
    assert rtc.lib.rtc_create(C.byref(geo), None, C.byref(cm), C.byref(pol), C.byref(h)) == rtc.RTC_EINVAL
    assert b"outside the frame" in rtc.lib.rtc_last_error(None)
    w[0].npx, w[0].nblocks = 4, 5          # more blocks than subaperture rows
    assert rtc.lib.rtc_create(C.byref(geo), None, C.byref(cm), C.byref(pol), C.byref(h)) == rtc.RTC_EINVAL


def test_quantize_rejects_bad_arguments_without_gpu(rtc):
    assert rtc.lib.rtc_quantize_rows(rtc.RTC_F32, 2, 2, None, 2, None, None, None) == rtc.RTC_EINVAL
    assert rtc.lib.rtc_quantize_rows(rtc.RTC_BF16, 2, 4, None, 2, None, None, None) == rtc.RTC_EINVAL
    assert rtc.lib.rtc_quantize_rows(rtc.RTC_BF16, 0, 4, None, 4, None, None, None) == rtc.RTC_OK


def test_null_loop_calls_are_rejected(rtc):
    assert rtc.lib.rtc_submit_pixels(None, None) == rtc.RTC_EINVAL
    assert rtc.lib.rtc_destroy(None) == rtc.RTC_OK
    assert rtc.lib.rtc_last_error(None) is not None


def test_footprint_is_computed_without_gpu_and_scales_with_storage(rtc):
    import numpy as np
    from paper_1903_01852_gb300 import synth
    cfg = synth.make_config("elt_scao_sh")
    r32, p32 = rtc.footprint(cfg)
    q = dict(cfg, M=np.zeros(cfg["M"].shape, np.uint16), M_dtype="bf16",
             M_scale=np.ones(cfg["na"], np.float32))
    r16, p16 = rtc.footprint(q)
    ru, _ = rtc.footprint(cfg, flags=rtc.RTC_FLAG_UPDATABLE)
    matrix = cfg["na"] * cfg["ns"] * 4
    assert r32 < p32 and r16 < p16
    assert matrix <= r32 < matrix * 1.1
    assert abs((r32 - r16) - matrix / 2) < 0.02 * matrix        # BF16 halves the matrix bytes
    assert abs((ru - r32) - matrix) < 0.05 * matrix             # the double buffer adds one matrix
    bad = dict(cfg, M=cfg["M"][:, :-2])
    import pytest
    with pytest.raises(rtc.RtcError):
        rtc.footprint(bad)


def test_structs_mirror_the_header_layout(rtc, tmp_path):
    """Every ctypes struct of the binding has the size and field offsets the C
    compiler gives the header's struct (checked with gcc on this host)."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    structs = [rtc.rtc_wfs, rtc.rtc_geometry, rtc.rtc_calib, rtc.rtc_cmat, rtc.rtc_polc, rtc.rtc_chunk,
               rtc.rtc_timing, rtc.rtc_tel_record, rtc.rtc_tel_stream_stats, rtc.rtc_update_desc, rtc.rtc_server_loop_info, rtc.rtc_info,
               rtc.rtc_master_desc]
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "rtc.h"', "int main(void) {"]
    for st in structs:
        n = st.__name__
        lines.append(f'printf("{n} %zu\\n", sizeof({n}));')
        for f, _ in st._fields_:
            lines.append(f'printf("{n}.{f} %zu\\n", offsetof({n}, {f}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], check=True, capture_output=True,
                                                 text=True).stdout.splitlines())
    for st in structs:
        n = st.__name__
        assert int(got[n]) == C.sizeof(st), n
        for f, _ in st._fields_:
            assert int(got[f"{n}.{f}"]) == getattr(st, f).offset, f"{n}.{f}"


def test_explicit_polc_and_norm_validation_without_gpu(rtc):
    import numpy as np
    from paper_1903_01852_gb300 import synth
    cfg = synth.make_config("scao_small")
    na, ns = cfg["na"], cfg["ns"]
    D = np.zeros((ns, na), np.float32)
    base = dict(cfg, P=None)
    r0, _ = rtc.footprint(base)
    r1, p1 = rtc.footprint(dict(base, polc="explicit", D=D))
    assert r1 - r0 >= ns * na * 4 and p1 > r1                 # D is resident, and uploaded through a temporary
    r, p = C.c_uint64(), C.c_uint64()
    P = np.zeros((na, na), np.float32)
    st = rtc.describe(dict(base, polc="explicit", D=D))
    st.pol.P = P.ctypes.data                                  # explicit mode with a P as well
    assert rtc.lib.rtc_footprint(C.byref(st.geo), C.byref(st.cal), C.byref(st.cm), C.byref(st.pol), C.byref(r),
                                 C.byref(p)) == rtc.RTC_EINVAL
    assert b"takes D, not P" in rtc.lib.rtc_last_error(None)
    st.pol.P = None
    st.pol.D = None
    assert rtc.lib.rtc_footprint(C.byref(st.geo), C.byref(st.cal), C.byref(st.cm), C.byref(st.pol), C.byref(r),
                                 C.byref(p)) == rtc.RTC_EINVAL
    assert b"needs D" in rtc.lib.rtc_last_error(None)
    st = rtc.describe(base)
    st.pol.D = D.ctypes.data                                  # D without explicit mode
    assert rtc.lib.rtc_footprint(C.byref(st.geo), C.byref(st.cal), C.byref(st.cm), C.byref(st.pol), C.byref(r),
                                 C.byref(p)) == rtc.RTC_EINVAL
    st = rtc.describe(base)
    st.pol.mode = 7
    assert rtc.lib.rtc_footprint(C.byref(st.geo), C.byref(st.cal), C.byref(st.cm), C.byref(st.pol), C.byref(r),
                                 C.byref(p)) == rtc.RTC_EINVAL
    st = rtc.describe(base)
    st.geo.wfs[0].norm = rtc.RTC_NORM_GLOBAL                  # SH WFS: no normalisation choice
    assert rtc.lib.rtc_footprint(C.byref(st.geo), C.byref(st.cal), C.byref(st.cm), C.byref(st.pol), C.byref(r),
                                 C.byref(p)) == rtc.RTC_EINVAL
    assert b"pyramid WFS only" in rtc.lib.rtc_last_error(None)
    pyr = synth.make_config("elt_scao_pyramid")
    assert rtc.footprint(dict(pyr, wfs=[dict(pyr["wfs"][0], norm="global")]))[0] > 0
    st = rtc.describe(pyr)
    st.geo.wfs[0].norm = 2
    assert rtc.lib.rtc_footprint(C.byref(st.geo), C.byref(st.cal), C.byref(st.cm), C.byref(st.pol), C.byref(r),
                                 C.byref(p)) == rtc.RTC_EINVAL


def test_wfs_count_limits_without_gpu(rtc):
    import numpy as np
    from paper_1903_01852_gb300 import synth
    rng = np.random.default_rng(5)
    wfs = [synth.sh_wfs(rng, 2, 4, 8, 8, 0.0) for _ in range(rtc.RTC_MAX_WFS)]
    ns = sum(2 * synth.num_valid(w) for w in wfs)
    cfg = dict(na=3, ns=ns, wfs=wfs, M=np.zeros((3, ns), np.float32), gain=0.5, leak=0.01)
    assert rtc.footprint(cfg)[0] > 0
    w17 = wfs + [synth.sh_wfs(rng, 2, 4, 8, 8, 0.0)]
    with pytest.raises(ValueError):
        rtc.footprint(dict(cfg, wfs=w17, M=np.zeros((3, ns + 8), np.float32)))
    st = rtc.describe(cfg)
    st.geo.nwfs = 0
    r, p = C.c_uint64(), C.c_uint64()
    assert rtc.lib.rtc_footprint(C.byref(st.geo), C.byref(st.cal), C.byref(st.cm), C.byref(st.pol), C.byref(r),
                                 C.byref(p)) == rtc.RTC_EINVAL


def test_graph_mode_excludes_stage_timing_without_gpu(rtc):
    from paper_1903_01852_gb300 import synth
    cfg = synth.make_config("scao_small")
    assert rtc.footprint(cfg, flags=rtc.RTC_FLAG_GRAPHS | rtc.RTC_FLAG_TIMING)[0] > 0
    with pytest.raises(rtc.RtcError, match="STAGE_TIMING"):
        rtc.footprint(cfg, flags=rtc.RTC_FLAG_GRAPHS | rtc.RTC_FLAG_STAGE_TIMING)


def test_partial_loops_and_master_validation_without_gpu(rtc):
    import numpy as np
    from paper_1903_01852_gb300 import synth
    cfg = synth.make_config("scao_small", polc=True)
    with pytest.raises(rtc.RtcError, match="no POLC matrix"):
        rtc.footprint(cfg, flags=rtc.RTC_FLAG_PARTIAL)            # a shard leaves POLC to the master
    assert rtc.footprint(dict(cfg, P=None), flags=rtc.RTC_FLAG_PARTIAL)[0] > 0
    assert rtc.lib.rtc_set_partial_output(None, None) == rtc.RTC_EINVAL
    h = C.c_void_p()
    assert rtc.lib.rtc_master_create(None, C.byref(h)) == rtc.RTC_EINVAL and h.value is None
    pol = rtc.rtc_polc(None, 0, None, 0.5, 0.01, None, 0, 0.0, 0.0, 0, None, 0, None)
    for na, nshards in ((0, 1), (4, 0), (4, rtc.RTC_MAX_WFS + 1)):
        d = rtc.rtc_master_desc(0, na, nshards, C.pointer(pol))
        assert rtc.lib.rtc_master_create(C.byref(d), C.byref(h)) == rtc.RTC_EINVAL
    pol.mode = rtc.RTC_POLC_EXPLICIT
    d = rtc.rtc_master_desc(0, 4, 2, C.pointer(pol))
    assert rtc.lib.rtc_master_create(C.byref(d), C.byref(h)) == rtc.RTC_EINVAL
    assert b"implicit POLC only" in rtc.lib.rtc_master_last_error(None)
    pol.mode = rtc.RTC_POLC_IMPLICIT
    P = np.full((4, 4), np.nan, np.float32)
    pol.P = P.ctypes.data
    assert rtc.lib.rtc_master_create(C.byref(d), C.byref(h)) == rtc.RTC_EINVAL
    assert b"NaN" in rtc.lib.rtc_master_last_error(None)
    assert rtc.lib.rtc_master_step(None, 1) == rtc.RTC_EINVAL
    assert rtc.lib.rtc_master_destroy(None) == rtc.RTC_OK


def test_negative_stream_priority_is_rejected_without_gpu(rtc):
    from paper_1903_01852_gb300 import synth
    cfg = synth.make_config("scao_small")
    assert rtc.footprint(dict(cfg, priority=3))[0] > 0
    with pytest.raises(rtc.RtcError, match="priority"):
        rtc.footprint(dict(cfg, priority=-1))


def test_prelaunch_flag_validation_without_gpu(rtc):
    from paper_1903_01852_gb300 import synth
    cfg = synth.make_config("scao_small")
    pre = rtc.RTC_FLAG_PRELAUNCH
    assert rtc.footprint(cfg, flags=pre)[0] > 0
    assert rtc.footprint(dict(cfg, prelaunch_wait_us=1_000_000), flags=pre)[0] > 0
    for timing in (rtc.RTC_FLAG_TIMING, rtc.RTC_FLAG_STAGE_TIMING):
        with pytest.raises(rtc.RtcError, match="PRELAUNCH excludes"):
            rtc.footprint(cfg, flags=pre | timing)      # events would be recorded out of order
    for bad in (-1, 1_000_001):
        with pytest.raises(rtc.RtcError, match="prelaunch_wait_us"):
            rtc.footprint(dict(cfg, prelaunch_wait_us=bad), flags=pre)


def test_batched_submission_validation_without_gpu(rtc):
    acc = C.c_int32(7)
    assert rtc.lib.rtc_submit_pixels_n(None, None, 0, C.byref(acc)) == rtc.RTC_EINVAL
    assert acc.value == 0                                     # zeroed whatever the outcome
