"""Pins of the FP64 oracle against facts fixed by mathematics, not by the oracle.

The paper prints no formula and no worked example (it gives shapes and latency
tables only), so each oracle step is pinned by closed forms, invariants,
special cases that reduce to a library routine, and brute force on tiny inputs,
chosen so that a dropped term, a wrong sign or index, or a transposed operand
fails at least one of them.
"""
import math
from fractions import Fraction

import numpy as np
import pytest
from scipy.special import ndtr

from oracle import rtc_oracle as orc


def sh_desc(n, nsub=1, valid=None, T=0.0, mode="subtract", dark=None, flat=None, ox=0, oy=0, h=None, w=None):
    h = h or oy + nsub * n
    w = w or ox + nsub * n
    return dict(kind="sh", width=w, height=h, nsubx=nsub, nsuby=nsub, npx=n, ox=ox, oy=oy,
                valid=np.ones((nsub, nsub), np.uint8) if valid is None else valid,
                dark=np.zeros((h, w), np.float32) if dark is None else dark,
                flat=np.ones((h, w), np.float32) if flat is None else flat,
                threshold=T, thresh_mode=mode)


def pyr_desc(p, T=0.0, valid=None):
    h = w = 2 * p + 4
    return dict(kind="pyramid", width=w, height=h, pupil=p, qx=[1, p + 3, 1, p + 3], qy=[1, 1, p + 3, p + 3],
                valid=np.ones((p, p), np.uint8) if valid is None else valid,
                dark=np.zeros((h, w), np.float32), flat=np.ones((h, w), np.float32),
                threshold=T, thresh_mode="subtract")


# ---------------------------------------------------------------- calibration

def test_calibration_identity_when_dark0_flat1_T0():
    raw = np.random.default_rng(0).integers(0, 65535, size=(7, 9)).astype(np.uint16)
    t, _ = orc.calibrate(raw, np.zeros((7, 9)), np.ones((7, 9)), 0.0)
    assert np.array_equal(t, raw.astype(float))


def test_calibration_dark_equal_raw_gives_zero():
    raw = np.random.default_rng(1).integers(50, 300, size=(5, 5)).astype(np.uint16)
    t, lit = orc.calibrate(raw, raw.astype(np.float32), np.full((5, 5), 1.3, np.float32), 0.0)
    assert not t.any() and not lit.any()


def test_calibration_hand_values_multiply_flat_subtract_dark():
    raw = np.array([[10, 4]], np.uint16)
    dark = np.array([[2, 2]], np.float32)
    flat = np.array([[2, 2]], np.float32)
    t_sub, _ = orc.calibrate(raw, dark, flat, 5.0, "subtract")   # (10-2)*2 = 16 -> 11 ; (4-2)*2 = 4 -> 0
    t_clip, _ = orc.calibrate(raw, dark, flat, 5.0, "clip")      # 16 kept whole ; 4 below T -> 0
    assert t_sub.tolist() == [[11.0, 0.0]]
    assert t_clip.tolist() == [[16.0, 0.0]]


def test_calibration_is_linear_in_flat():
    rng = np.random.default_rng(2)
    raw = rng.integers(90, 200, size=(6, 6)).astype(np.uint16)
    dark = rng.normal(100, 5, size=(6, 6)).astype(np.float32)
    flat = rng.normal(1, 0.02, size=(6, 6)).astype(np.float32)
    c1, _ = orc.calibrate(raw, dark, flat, -1e9)
    c2, _ = orc.calibrate(raw, dark, (2 * flat).astype(np.float32), -1e9)
    # with T far below, t = c + 1e9 ; remove the offset and compare the affine parts
    assert np.allclose((c2 - 1e9), 2 * (c1 - 1e9), rtol=0, atol=1e-6)


def test_lit_decision_is_single_precision():
    # a pixel whose float64 value is above T but whose float32 value equals T is not lit
    raw = np.array([[3]], np.uint16)
    dark = np.array([[0.0]], np.float32)
    flat = np.array([[np.float32(1.0)]], np.float32)
    t, lit = orc.calibrate(raw, dark, flat, 3.0)
    assert not lit.any() and t[0, 0] == 0.0


# ---------------------------------------------------------------- SH centre of gravity

@pytest.mark.parametrize("n", [2, 3, 8, 10])
def test_sh_uniform_frame_gives_zero(n):
    w = sh_desc(n, nsub=3, T=5.0)
    raw = np.full((3 * n, 3 * n), 40, np.uint16)
    assert np.array_equal(orc.sh_slopes(raw, w), np.zeros(18))


def test_sh_below_threshold_gives_zero_not_nan():
    w = sh_desc(8, nsub=2, T=5.0)
    raw = np.full((16, 16), 5, np.uint16)
    s = orc.sh_slopes(raw, w)
    assert np.all(np.isfinite(s)) and not s.any()


@pytest.mark.parametrize("n,i,j", [(8, 0, 0), (8, 7, 2), (10, 3, 9), (5, 4, 0)])
def test_sh_single_pixel_is_its_coordinate(n, i, j):
    w = sh_desc(n)
    raw = np.zeros((n, n), np.uint16)
    raw[i, j] = 1000
    sx, sy = orc.sh_slopes(raw, w)
    assert sx == j - (n - 1) / 2 and sy == i - (n - 1) / 2


def _gauss_tile(n, dx, dy, sigma, flux=1e6):
    # pixel-integrated circular Gaussian (separable), as float pixel values
    edges = np.arange(n + 1) - n / 2.0
    gx = ndtr((edges[1:] - dx) / sigma) - ndtr((edges[:-1] - dx) / sigma)
    gy = ndtr((edges[1:] - dy) / sigma) - ndtr((edges[:-1] - dy) / sigma)
    return flux * np.outer(gy, gx)


@pytest.mark.parametrize("dx,dy", [(0.0, 0.0), (0.7, -0.3), (-1.9, 1.25)])
def test_sh_gaussian_centroid_tends_to_offset(dx, dy):
    # closed form: the centroid of a pixel-integrated Gaussian spot that lies well
    # inside a large window equals its offset (tails beyond 16 sigma are < 1e-50)
    n = 40
    w = sh_desc(n)
    w["flat"] = _gauss_tile(n, dx, dy, 1.2)      # float64 pixel values carried by the flat map
    sx, sy = orc.sh_slopes(np.ones((n, n), np.uint16), w)
    assert abs(sx - dx) < 1e-12 and abs(sy - dy) < 1e-12


def test_sh_gaussian_small_window_matches_separable_marginals():
    # in an 8x8 window the centroid is the 1-D centroid of each marginal (separability)
    n, dx, dy, sig = 8, 0.8, -1.1, 1.2
    w = sh_desc(n)
    w["flat"] = _gauss_tile(n, dx, dy, sig)
    sx, sy = orc.sh_slopes(np.ones((n, n), np.uint16), w)
    edges = np.arange(n + 1) - n / 2.0
    c = np.arange(n) - (n - 1) / 2
    gx = ndtr((edges[1:] - dx) / sig) - ndtr((edges[:-1] - dx) / sig)
    gy = ndtr((edges[1:] - dy) / sig) - ndtr((edges[:-1] - dy) / sig)
    assert abs(sx - (gx @ c) / gx.sum()) < 1e-12 and abs(sy - (gy @ c) / gy.sum()) < 1e-12
    assert abs(sx - dx) > 1e-3        # truncation by the window is visible at this size


def test_sh_gaussian_centered_is_exactly_zero_by_symmetry():
    n = 8
    tile = _gauss_tile(n, 0.0, 0.0, 1.2)
    tile = np.maximum(tile, tile[::-1, :])
    tile = np.maximum(tile, tile[:, ::-1])
    w = sh_desc(n)
    w["flat"] = tile
    sx, sy = orc.sh_slopes(np.ones((n, n), np.uint16), w)
    assert abs(sx) < 1e-14 and abs(sy) < 1e-14      # zero up to float64 summation order


def test_sh_integer_translation_shifts_slope_exactly():
    n = 10
    blob = np.array([[1, 3, 1], [2, 9, 4], [1, 2, 1]], np.uint16) * 7
    base = np.zeros((n, n), np.uint16)
    base[2:5, 3:6] = blob
    s0 = orc.sh_slopes(base, sh_desc(n))
    for ky, kx in [(1, 0), (0, 2), (3, 4), (-2, -3)]:
        moved = np.roll(np.roll(base, ky, 0), kx, 1)
        s1 = orc.sh_slopes(moved, sh_desc(n))
        assert abs(s1[0] - s0[0] - kx) < 1e-12 and abs(s1[1] - s0[1] - ky) < 1e-12


def test_sh_mirror_and_transpose():
    rng = np.random.default_rng(3)
    n = 8
    raw = rng.integers(0, 500, size=(n, n)).astype(np.uint16)
    sx, sy = orc.sh_slopes(raw, sh_desc(n))
    fx, fy = orc.sh_slopes(raw[:, ::-1].copy(), sh_desc(n))
    tx, ty = orc.sh_slopes(raw.T.copy(), sh_desc(n))
    assert abs(fx + sx) < 1e-12 and abs(fy - sy) < 1e-12
    assert abs(tx - sy) < 1e-12 and abs(ty - sx) < 1e-12


def test_sh_scale_invariance():
    rng = np.random.default_rng(4)
    raw = rng.integers(0, 300, size=(16, 16)).astype(np.uint16)
    a = orc.sh_slopes(raw, sh_desc(8, nsub=2))
    b = orc.sh_slopes((raw * 3).astype(np.uint16), sh_desc(8, nsub=2))
    assert np.allclose(a, b, rtol=0, atol=1e-12)


def test_sh_order_is_row_major_interleaved_and_skips_invalid():
    n, nsub = 4, 3
    valid = np.array([[0, 1, 1], [1, 0, 1], [1, 1, 0]], np.uint8)
    raw = np.zeros((nsub * n, nsub * n), np.uint16)
    expect = []
    for i in range(nsub):
        for j in range(nsub):
            pi, pj = (i + j) % n, (2 * i + j) % n   # a distinct lit pixel in each subaperture
            raw[i * n + pi, j * n + pj] = 100
            if valid[i, j]:
                expect += [pj - (n - 1) / 2, pi - (n - 1) / 2]
    s = orc.sh_slopes(raw, sh_desc(n, nsub=nsub, valid=valid))
    assert s.tolist() == expect


def test_sh_grid_origin_offset():
    n = 4
    raw = np.zeros((9, 11), np.uint16)
    raw[2 + 3, 5 + 0] = 50   # grid at ox=5, oy=2: pixel (3,0) of the only subaperture
    s = orc.sh_slopes(raw, sh_desc(n, ox=5, oy=2, h=9, w=11))
    assert s.tolist() == [0 - 1.5, 3 - 1.5]


def test_reference_slopes_are_subtracted():
    n = 4
    raw = np.zeros((n, n), np.uint16)
    raw[0, 3] = 10
    cfg = dict(wfs=[sh_desc(n)], ref_slopes=np.array([0.25, -0.5], np.float32))
    assert orc.frame_slopes(cfg, [raw]).tolist() == [1.5 - 0.25, -1.5 + 0.5]


# ---------------------------------------------------------------- pyramid

def test_pyramid_recovers_slopes_from_closed_form_intensities():
    rng = np.random.default_rng(5)
    p = 6
    w = pyr_desc(p)
    sx = rng.uniform(-0.45, 0.45, size=(p, p))
    sy = rng.uniform(-0.45, 0.45, size=(p, p))
    n = 4.0 * 1024
    quads = [n / 4 * (1 + sx + sy), n / 4 * (1 - sx + sy), n / 4 * (1 + sx - sy), n / 4 * (1 - sx - sy)]
    # float intensities via the flat map on a raw of ones
    w["flat"] = np.zeros_like(w["flat"])
    for k in range(4):
        w["flat"][w["qy"][k]:w["qy"][k] + p, w["qx"][k]:w["qx"][k] + p] = quads[k]
    got = orc.pyramid_slopes(np.ones((w["height"], w["width"]), np.uint16), w).reshape(-1, 2)
    q32 = [w["flat"][w["qy"][k]:w["qy"][k] + p, w["qx"][k]:w["qx"][k] + p].astype(float) for k in range(4)]
    tot = sum(q32)
    ex = ((q32[0] + q32[2] - q32[1] - q32[3]) / tot).reshape(-1)
    assert np.allclose(got[:, 0], sx.reshape(-1), rtol=0, atol=2e-7)       # float32 storage of intensities
    assert np.allclose(got[:, 1], sy.reshape(-1), rtol=0, atol=2e-7)
    assert np.allclose(got[:, 0], ex, rtol=1e-15, atol=1e-15)


def test_pyramid_quadrant_signs():
    p = 3
    for k, (ex, ey) in enumerate([(1, 1), (-1, 1), (1, -1), (-1, -1)]):
        w = pyr_desc(p)
        raw = np.zeros((w["height"], w["width"]), np.uint16)
        raw[w["qy"][k] + 1, w["qx"][k] + 2] = 77
        s = orc.pyramid_slopes(raw, w).reshape(p, p, 2)
        assert s[1, 2].tolist() == [ex, ey]
        s[1, 2] = 0
        assert not s.any()


def test_pyramid_equal_quadrants_zero():
    p = 4
    w = pyr_desc(p)
    raw = np.full((w["height"], w["width"]), 9, np.uint16)
    assert not orc.pyramid_slopes(raw, w).any()


def test_pyramid_global_norm_hand_values():
    # one lit quadrant per pupil pixel: fluxes 8, 4, 2, 2 (mean 4)
    p = 2
    w = pyr_desc(p)
    w["norm"] = "global"
    raw = np.zeros((w["height"], w["width"]), np.uint16)
    for (i, j), k, v in [((0, 0), 0, 8), ((0, 1), 1, 4), ((1, 0), 2, 2), ((1, 1), 3, 2)]:
        raw[w["qy"][k] + i, w["qx"][k] + j] = v
    assert orc.pyramid_slopes(raw, w).tolist() == [2.0, 2.0, -1.0, 1.0, 0.5, -0.5, -0.5, -0.5]
    w["norm"] = "local"
    assert orc.pyramid_slopes(raw, w).tolist() == [1.0, 1.0, -1.0, 1.0, 1.0, -1.0, -1.0, -1.0]


def test_pyramid_global_norm_closed_form_with_varying_flux():
    # A = N_p/4 (1+sx+sy) etc.: local normalisation returns (sx, sy); global
    # normalisation returns (sx, sy) * N_p / mean(N) over the valid pixels.
    rng = np.random.default_rng(15)
    p = 6
    w = pyr_desc(p)
    valid = (rng.random((p, p)) > 0.25).astype(np.uint8)
    w["valid"] = valid
    w["norm"] = "global"
    sx = rng.uniform(-0.45, 0.45, size=(p, p))
    sy = rng.uniform(-0.45, 0.45, size=(p, p))
    n = rng.uniform(500.0, 3000.0, size=(p, p))
    quads = [n / 4 * (1 + sx + sy), n / 4 * (1 - sx + sy), n / 4 * (1 + sx - sy), n / 4 * (1 - sx - sy)]
    w["flat"] = np.zeros_like(w["flat"])
    for k in range(4):
        w["flat"][w["qy"][k]:w["qy"][k] + p, w["qx"][k]:w["qx"][k] + p] = quads[k]
    got = orc.pyramid_slopes(np.ones((w["height"], w["width"]), np.uint16), w).reshape(-1, 2)
    v = valid.astype(bool)
    factor = n[v] / n[v].mean()
    assert np.allclose(got[:, 0], sx[v] * factor, rtol=0, atol=1e-6)
    assert np.allclose(got[:, 1], sy[v] * factor, rtol=0, atol=1e-6)


def test_pyramid_global_norm_uniform_flux_equals_local_and_ignores_invalid_pixels():
    rng = np.random.default_rng(16)
    p = 5
    w = pyr_desc(p)
    valid = np.ones((p, p), np.uint8)
    valid[2, 3] = 0
    w["valid"] = valid
    sx = rng.integers(-25, 26, size=(p, p)) / 64.0          # dyadic: every intensity is exact in float32,
    sy = rng.integers(-25, 26, size=(p, p)) / 64.0          # so every pixel's flux is exactly 1024
    quads = [256 * (1 + sx + sy), 256 * (1 - sx + sy), 256 * (1 + sx - sy), 256 * (1 - sx - sy)]
    w["flat"] = np.zeros_like(w["flat"])
    for k in range(4):
        w["flat"][w["qy"][k]:w["qy"][k] + p, w["qx"][k]:w["qx"][k] + p] = quads[k]
    raw = np.ones((w["height"], w["width"]), np.uint16)
    loc = orc.pyramid_slopes(raw, dict(w, norm="local"))
    glo = orc.pyramid_slopes(raw, dict(w, norm="global"))
    assert np.allclose(glo, loc, rtol=0, atol=1e-15)
    # flux in the invalid pupil pixel does not enter the mean
    for k in range(4):
        w["flat"][w["qy"][k] + 2, w["qx"][k] + 3] = 5000.0
    assert np.allclose(orc.pyramid_slopes(raw, dict(w, norm="global")), loc, rtol=0, atol=1e-15)
    # a common factor on every intensity cancels
    w2 = dict(w, norm="global", flat=w["flat"] * 2)
    assert np.allclose(orc.pyramid_slopes(raw, w2), loc, rtol=0, atol=1e-15)


def test_pyramid_global_norm_zero_flux_gives_zero_slopes():
    w = pyr_desc(3)
    w["norm"] = "global"
    w["threshold"] = 10.0
    raw = np.full((w["height"], w["width"]), 10, np.uint16)
    out = orc.pyramid_slopes(raw, w)
    assert out.shape == (18,) and not out.any() and np.isfinite(out).all()


# ---------------------------------------------------------------- quantisation

torch = pytest.importorskip("torch")


def _edge_values():
    rng = np.random.default_rng(6)
    vals = [0.0, -0.0, 1.0, -1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, 1 - 2 ** -9, 3.0, 1e-30, -7.25e-12]
    vals += list(rng.standard_normal(4000) * 10.0 ** rng.uniform(-8, 3, 4000))
    return np.array(vals, np.float32)


def test_bf16_rne_matches_library_conversion():
    x = _edge_values()
    ours = orc.encode(orc.round_to_format(x, "bf16"), "bf16")
    ref = torch.from_numpy(x).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    assert np.array_equal(ours, ref)


def test_e4m3_rne_matches_library_conversion_in_range():
    x = _edge_values()
    x = x[np.abs(x) <= 448.0]
    ours = orc.encode(orc.round_to_format(x, "e4m3"), "e4m3")
    ref = torch.from_numpy(x).to(torch.float8_e4m3fn).view(torch.uint8).numpy()
    assert np.array_equal(ours, ref)


def test_rne_hand_cases_and_saturation():
    assert orc.round_to_format(np.float32(1 + 2 ** -8), "bf16") == 1.0            # tie -> even
    assert orc.round_to_format(np.float32(1 + 3 * 2 ** -8), "bf16") == 1 + 2 ** -6  # tie -> even (up)
    assert orc.round_to_format(np.float32(500.0), "e4m3") == 448.0
    assert orc.encode(orc.round_to_format(np.float32(-1000.0), "e4m3"), "e4m3") == 0xFE
    assert orc.round_to_format(np.float32(2 ** -10), "e4m3") == 0.0                # half of the smallest subnormal -> even (0)
    assert orc.round_to_format(np.float32(3 * 2 ** -10), "e4m3") == 2 ** -8         # 1.5 subnormal steps -> 2


def test_encode_decode_roundtrip():
    for fmt in ("bf16", "e4m3"):
        q = orc.round_to_format(_edge_values(), fmt)
        assert np.array_equal(orc.decode(orc.encode(q, fmt), fmt), q)


@pytest.mark.parametrize("fmt,u", [("bf16", 2.0 ** -8), ("e4m3", 2.0 ** -4)])
def test_quantize_rows_error_bound_and_scale(fmt, u):
    rng = np.random.default_rng(7)
    M = (rng.standard_normal((17, 301)) * 1e-3).astype(np.float32)
    M[3] = 0.0
    codes, scale = orc.quantize_rows(M, fmt)
    mt = orc.stored_matrix(codes, fmt, scale)
    err = np.abs(mt - M.astype(float))
    sub = scale.astype(float)[:, None] * (2.0 ** -10 if fmt == "e4m3" else 0.0)
    # RNE bound relative to the scaled value, plus the single-precision quotient's rounding
    assert np.all(err <= (u + 2 ** -23) * np.abs(M.astype(float)) + sub + 1e-30)
    assert scale[3] == 1.0 and not mt[3].any()
    top = np.abs(orc.decode(codes, fmt)).max(axis=1)
    assert np.all(top[np.arange(17) != 3] == (1.0 if fmt == "bf16" else 448.0))


# ---------------------------------------------------------------- MVM

def test_mvm_brute_force_integers():
    rng = np.random.default_rng(8)
    for na, ns in [(1, 1), (3, 5), (7, 13)]:
        M = rng.integers(-9, 10, size=(na, ns))
        s = rng.integers(-9, 10, size=ns)
        exact = [sum(int(M[i, j]) * int(s[j]) for j in range(ns)) for i in range(na)]
        assert orc.mvm(M.astype(float), s.astype(float)).tolist() == exact


def test_mvm_identity_onehot_and_block_partials():
    rng = np.random.default_rng(9)
    s = rng.standard_normal(12)
    assert np.array_equal(orc.mvm(np.eye(12), s), s)
    M = rng.standard_normal((5, 12))
    for j in (0, 7, 11):
        e = np.zeros(12)
        e[j] = 1.0
        assert np.array_equal(orc.mvm(M, e), M[:, j])
    parts = sum(orc.mvm(M[:, a:b], s[a:b]) for a, b in [(0, 3), (3, 8), (8, 12)])
    assert np.allclose(parts, orc.mvm(M, s), rtol=1e-14, atol=1e-14)


# ---------------------------------------------------------------- control law and POLC

def test_leaky_integrator_closed_form():
    g, leak, k = 0.5, 0.01, 37
    y = np.array([0.3, -1.2, 2.5])
    a = np.zeros(3)
    for _ in range(k):
        a = orc.control_step(a, y, np.zeros(3), g, leak)
    assert np.allclose(a, g * y * (1 - (1 - leak) ** k) / leak, rtol=1e-13, atol=0)


def test_leaky_integrator_exact_rational():
    # one step with dyadic values is exact in float64
    a = orc.control_step(np.array([0.5]), np.array([0.25]), np.array([0.125]), 0.5, 0.25)
    assert a[0] == float(Fraction(3, 4) * Fraction(1, 2) + Fraction(1, 2) * Fraction(3, 8))


def test_clip():
    a = orc.control_step(np.array([0.0, 0.0]), np.array([10.0, -10.0]), np.zeros(2), 1.0, 0.0, clip=(-1.0, 2.0))
    assert a.tolist() == [2.0, -1.0]


def test_implicit_polc_equals_explicit_polc():
    rng = np.random.default_rng(10)
    na, ns = 9, 14
    M = rng.standard_normal((na, ns)) * 0.1
    D = rng.standard_normal((ns, na)) * 0.1
    P = M @ D - np.eye(na)
    g, leak = 0.5, 0.01
    a_imp = np.zeros(na)
    a_exp = np.zeros(na)
    q = P @ a_imp
    for _ in range(10):
        s = rng.standard_normal(ns)
        a_imp = orc.control_step(a_imp, orc.mvm(M, s), q, g, leak)
        q = P @ a_imp
        a_exp = orc.explicit_polc_step(M, D, s, a_exp, g, leak)
        assert np.allclose(a_imp, a_exp, rtol=0, atol=1e-12)


def _polc_cfgs(rng, n=4, nsub=2, na=5):
    w = sh_desc(n, nsub=nsub)
    ns = 2 * nsub * nsub
    # small dyadic entries: P = M D - I is exact in float32, so both loops use the same matrices
    M = (rng.integers(-8, 9, size=(na, ns)) / 16.0).astype(np.float32)
    D = (rng.integers(-8, 9, size=(ns, na)) / 16.0).astype(np.float32)
    P = (M.astype(np.float64) @ D.astype(np.float64) - np.eye(na)).astype(np.float32)
    assert np.array_equal(P.astype(np.float64), M.astype(np.float64) @ D.astype(np.float64) - np.eye(na))
    base = dict(wfs=[w], M=M, gain=0.5, leak=0.01, ref_slopes=None)
    return dict(base, P=P), dict(base, polc="explicit", D=D), M, D


def test_oracle_loop_explicit_polc_equals_implicit_with_p_eq_md_minus_i():
    rng = np.random.default_rng(17)
    imp_cfg, exp_cfg, M, D = _polc_cfgs(rng)
    imp, exp = orc.OracleLoop(imp_cfg), orc.OracleLoop(exp_cfg)
    for _ in range(10):
        raw = rng.integers(0, 50, size=(8, 8)).astype(np.uint16)
        a_prev = exp.a.copy()
        s_i, a_i = imp.step([raw])
        s_e, a_e = exp.step([raw])
        assert np.allclose(s_e, s_i + D.astype(np.float64) @ a_prev, rtol=0, atol=1e-12)   # POL slopes
        assert np.allclose(a_e, a_i, rtol=0, atol=1e-12)


def test_oracle_loop_explicit_polc_with_d_zero_closed_form():
    # D = 0: a_k = (1 - leak - g) a_{k-1} + g y, so a_k = g y (1 - (1-leak-g)^k) / (leak + g)
    n = 4
    w = sh_desc(n)
    raw = np.zeros((n, n), np.uint16)
    raw[0, 3] = 10                        # slopes (1.5, -1.5)
    g, leak = 0.25, 0.125
    cfg = dict(wfs=[w], M=np.array([[2.0, 1.0], [0.0, -4.0]], np.float32), gain=g, leak=leak,
               ref_slopes=None, polc="explicit", D=np.zeros((2, 2), np.float32))
    loop = orc.OracleLoop(cfg)
    y = np.array([2.0 * 1.5 - 1.5, 6.0])
    for k in range(1, 8):
        s, a = loop.step([raw])
        assert s.tolist() == [1.5, -1.5]
        assert np.allclose(a, g * y * (1 - (1 - leak - g) ** k) / (leak + g), rtol=1e-14, atol=0)


def test_oracle_loop_one_frame_identity_matrix():
    n = 4
    w = sh_desc(n, nsub=2)
    raw = np.zeros((8, 8), np.uint16)
    raw[1, 2] = 9
    raw[5, 7] = 3
    cfg = dict(wfs=[w], M=np.eye(8, dtype=np.float32), P=None, gain=0.5, leak=0.01, ref_slopes=None)
    loop = orc.OracleLoop(cfg)
    s, a = loop.step([raw])
    assert np.array_equal(a, 0.5 * s)
    s2, a2 = loop.step([raw])
    assert np.allclose(a2, 0.99 * a + 0.5 * s2, rtol=1e-15, atol=0)


def test_two_sensor_frame_slopes_hand_values_in_configuration_order():
    # An SH sensor (2x2 subapertures of 2x2 px, subaperture (0, 1) invalid) and a
    # pyramid (2x2 pupil, pixel (1, 0) invalid), slopes worked out by hand: units
    # row-major within a sensor, x before y, sensors in configuration order, then
    # the reference slopes subtracted over the concatenation.
    sh = sh_desc(2, nsub=2, valid=np.array([[1, 0], [1, 1]], np.uint8))
    sh_raw = np.zeros((4, 4), np.uint16)
    sh_raw[0, 1], sh_raw[1, 1] = 3, 1               # subap (0,0): F 4, x (3+1)*0.5/4, y (-1.5+0.5)/4
    sh_raw[0, 3] = 7                                # subap (0,1): invalid, must not appear
    sh_raw[3, 0] = 2                                # subap (1,0): single pixel at (-0.5, +0.5)
    sh_raw[2, 2], sh_raw[2, 3], sh_raw[3, 3] = 1, 1, 2   # subap (1,1): x (-0.5+0.5+1)/4, y (-0.5-0.5+1)/4
    sh_expect = [0.5, -0.25, -0.5, 0.5, 0.25, 0.0]
    py = pyr_desc(2, valid=np.array([[1, 1], [0, 1]], np.uint8))
    py_raw = np.zeros((8, 8), np.uint16)
    A, B, C, D = (1, 1), (1, 5), (5, 1), (5, 5)     # (row, col) origins of the four pupil images
    py_raw[A[0], A[1]] = 4                          # pixel (0,0): A only -> (1, 1)
    py_raw[A[0], A[1] + 1], py_raw[B[0], B[1] + 1] = 1, 3   # pixel (0,1): A 1, B 3 -> ((1-3)/4, (1+3)/4)
    py_raw[A[0] + 1, A[1]] = 5                      # pixel (1,0): invalid
    py_raw[A[0] + 1, A[1] + 1], py_raw[C[0] + 1, C[1] + 1] = 1, 3   # pixel (1,1): A 1, C 3 -> (1, -0.5)
    py_expect = [1.0, 1.0, -0.5, 1.0, 1.0, -0.5]
    ref = np.arange(12) / 8.0
    s = orc.frame_slopes(dict(wfs=[sh, py], ref_slopes=ref), [sh_raw, py_raw])
    assert s.tolist() == (np.array(sh_expect + py_expect) - ref).tolist()
    s = orc.frame_slopes(dict(wfs=[py, sh], ref_slopes=None), [py_raw, sh_raw])
    assert s.tolist() == py_expect + sh_expect


def test_oracle_loop_explicit_polc_clip_hand_values():
    # D = 0, dyadic values: a_k = clip((1 - leak - g) a_{k-1} + g y) with (1 - leak - g) = 1/4
    n = 4
    raw = np.zeros((n, n), np.uint16)
    raw[0, 3] = 10                                   # slopes (1.5, -1.5)
    M = np.array([[4.0, -4.0], [-4.0, 4.0], [0.5, 0.5]], np.float32)   # y = M s = (12, -12, 0)
    cfg = dict(wfs=[sh_desc(n)], M=M, gain=0.5, leak=0.25, ref_slopes=None, polc="explicit",
               D=np.zeros((2, 3), np.float32), clip=(-2.0, 3.0))
    loop = orc.OracleLoop(cfg)
    for _ in range(2):                               # unclipped: (6, -6, 0) then (6.75, -6.5, 0)
        s, a = loop.step([raw])
        assert s.tolist() == [1.5, -1.5]
        assert a.tolist() == [3.0, -2.0, 0.0]
    # an all-zero frame gives y = 0: a = clip(a / 4), inside the bounds
    s, a = loop.step([np.zeros((n, n), np.uint16)])
    assert a.tolist() == [0.75, -0.5, 0.0]


def test_oracle_loop_explicit_polc_with_clip_equals_implicit_with_clip():
    # P = M D - I makes the two forms the same update; clipping the same quantity
    # and feeding the clipped state back (D a or P a) keeps them equal.
    rng = np.random.default_rng(23)
    imp_cfg, exp_cfg, M, D = _polc_cfgs(rng)
    imp_cfg["clip"] = exp_cfg["clip"] = (-0.3, 0.2)
    imp, exp = orc.OracleLoop(imp_cfg), orc.OracleLoop(exp_cfg)
    hit = 0
    for _ in range(10):
        raw = rng.integers(0, 50, size=(8, 8)).astype(np.uint16)
        _, a_i = imp.step([raw])
        _, a_e = exp.step([raw])
        assert np.allclose(a_e, a_i, rtol=0, atol=1e-12)
        assert a_e.min() >= -0.3 and a_e.max() <= 0.2
        hit += int(np.sum((a_e == -0.3) | (a_e == 0.2)))
    assert hit > 0                                    # the clip was active
