"""FP64 CPU oracle of the adaptive-optics real-time-control hot path.

TEST INFRASTRUCTURE ONLY.  This module is the independent reference that the
CUDA path is checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline / reference legs of ``bench.py`` may import it; the product
library never does, and the two share no code.

It follows the paper's per-frame pipeline (Fig. ao_diag, Section 2.2): pixel
calibration -> Shack-Hartmann centre-of-gravity or pyramid quad-difference
slopes -> reconstruction MVM -> (implicit POLC, Section 3.4) -> leaky
integrator -> DM commands.  The paper names these steps but prints no formula
for any of them, so each function below writes out the standard textbook
definition in float64, in the order the pipeline applies it:

* calibration   c = (raw - dark) * flat; threshold t = max(c - T, 0) ("subtract")
                or t = c if c > T else 0 ("clip")
* SH slopes     per valid subaperture, F = sum t, sx = sum t*x / F, sy = sum t*y / F
                with pixel-centre coordinates x = i - (n-1)/2, minus reference
                slopes; 0 when no pixel is lit
* pyramid       per valid pupil pixel with quadrant values A (top-left),
                B (top-right), C (bottom-left), D (bottom-right):
                N = A+B+C+D, sx = (A+C-B-D)/N, sy = (A+B-C-D)/N, minus reference;
                or, normalised globally, divided by the mean of N over valid pixels
* MVM           y = M~ s, M~ the matrix actually stored (row scale * code)
* control law   a_k = (1-leak) a_{k-1} + g (y_k + q_{k-1}), optional clip,
                q_k = P~ a_k computed after the command (implicit POLC, Section 3.4);
                or explicit POLC: s_ol = s + D~ a_{k-1}, a_k = (1-leak-g) a_{k-1} + g M~ s_ol

Slope order: interleaved (x, y) per valid unit, units in row-major order of the
subaperture grid (or pupil pixels), WFS after WFS in configuration order.

Readings where the paper is silent are listed with the project's design notes;
the one that touches precision is this: whether a pixel counts as lit (t > 0)
is an integer-valued decision, so it is taken on the single-precision value
fl(fl(raw - dark) * flat) exactly as the kernels compute it, while every value
that enters a sum is computed in float64.

Quantisation (per-row scales, BF16 and FP8-E4M3 codes) uses round-to-nearest-
even with saturation, written here from the formats' definitions; the scale and
the scaled value are single-precision quotients (IEEE round-to-nearest), as in
the kernels, because they decide the integer codes.
"""
from __future__ import annotations

import numpy as np

f64 = np.float64
f32 = np.float32

# ----------------------------------------------------------------------------
# Calibration (Section 2.2, "pixel handling"; Fig. ao_diag first process)
# ----------------------------------------------------------------------------


def lit_pixels(raw, dark, flat, threshold):
    """Boolean map of pixels whose calibrated value exceeds the threshold,
    decided in single precision: fl(fl(raw - dark) * flat) > T."""
    c32 = (np.asarray(raw).astype(f32) - np.asarray(dark, dtype=f32)) * np.asarray(flat, dtype=f32)
    return c32 > f32(threshold)


def calibrate(raw, dark, flat, threshold, mode="subtract"):
    """Calibrated, thresholded pixels in float64 and the lit-pixel map.

    c = (raw - dark) * flat.  mode "subtract": t = max(c - T, 0);
    mode "clip": t = c where c > T, else 0."""
    c = (np.asarray(raw).astype(f64) - np.asarray(dark, dtype=f64)) * np.asarray(flat, dtype=f64)
    lit = lit_pixels(raw, dark, flat, threshold)
    if mode == "subtract":
        t = np.where(lit, np.maximum(c - f64(threshold), 0.0), 0.0)
    elif mode == "clip":
        t = np.where(lit, c, 0.0)
    else:
        raise ValueError(mode)
    return t, lit


# ----------------------------------------------------------------------------
# Slopes (Section 2.2, Fig. wfs_slopes)
# ----------------------------------------------------------------------------


def sh_slopes(raw, w):
    """Centre-of-gravity slopes of one Shack-Hartmann WFS, interleaved x,y over
    its valid subapertures in row-major order (Fig. wfs_slopes: each slope is
    the centre of gravity of the pixel values in one subaperture)."""
    t, lit = calibrate(raw, w["dark"], w["flat"], w["threshold"], w["thresh_mode"])
    n, nx, ny, ox, oy = w["npx"], w["nsubx"], w["nsuby"], w["ox"], w["oy"]
    tiles = t[oy:oy + ny * n, ox:ox + nx * n].reshape(ny, n, nx, n)
    lit_tiles = lit[oy:oy + ny * n, ox:ox + nx * n].reshape(ny, n, nx, n)
    coord = np.arange(n, dtype=f64) - (n - 1) / 2.0     # pixel centres about the subaperture centre
    flux = tiles.sum(axis=(1, 3))
    sum_x = np.einsum("iajb,b->ij", tiles, coord)
    sum_y = np.einsum("iajb,a->ij", tiles, coord)
    any_lit = lit_tiles.any(axis=(1, 3)) & (flux > 0)
    safe = np.where(any_lit, flux, 1.0)
    sx = np.where(any_lit, sum_x / safe, 0.0)
    sy = np.where(any_lit, sum_y / safe, 0.0)
    v = w["valid"].astype(bool)
    return np.stack([sx[v], sy[v]], axis=1).reshape(-1)


def pyramid_slopes(raw, w):
    """Normalised quad-difference slopes of one pyramid WFS (Fig. wfs_slopes:
    relative x and y differences of corresponding pixels of the four pupil
    images), interleaved x,y over valid pupil pixels in row-major order.

    w["norm"] "local" (default): each pixel's differences are divided by its own
    flux N = A+B+C+D.  "global": they are divided by the mean of N over the
    valid pupil pixels; every slope is 0 when that mean is not positive."""
    t, lit = calibrate(raw, w["dark"], w["flat"], w["threshold"], w["thresh_mode"])
    p = w["pupil"]
    quad = [t[w["qy"][k]:w["qy"][k] + p, w["qx"][k]:w["qx"][k] + p] for k in range(4)]
    qlit = [lit[w["qy"][k]:w["qy"][k] + p, w["qx"][k]:w["qx"][k] + p] for k in range(4)]
    a, b, c, d = quad
    total = a + b + c + d
    v = w["valid"].astype(bool)
    norm = w.get("norm", "local")
    if norm == "local":
        any_lit = (qlit[0] | qlit[1] | qlit[2] | qlit[3]) & (total > 0)
        safe = np.where(any_lit, total, 1.0)
        sx = np.where(any_lit, (a + c - b - d) / safe, 0.0)
        sy = np.where(any_lit, (a + b - c - d) / safe, 0.0)
    elif norm == "global":
        mean_flux = total[v].mean() if v.any() else 0.0
        if mean_flux > 0:
            sx = (a + c - b - d) / mean_flux
            sy = (a + b - c - d) / mean_flux
        else:
            sx = sy = np.zeros_like(total)
    else:
        raise ValueError(norm)
    return np.stack([sx[v], sy[v]], axis=1).reshape(-1)


def wfs_slopes(raw, w):
    return sh_slopes(raw, w) if w["kind"] == "sh" else pyramid_slopes(raw, w)


def frame_slopes(cfg, frames):
    """All slopes of one frame: WFS after WFS, minus the reference slopes."""
    s = np.concatenate([wfs_slopes(frames[k], w) for k, w in enumerate(cfg["wfs"])])
    if cfg.get("ref_slopes") is not None:
        s = s - np.asarray(cfg["ref_slopes"], dtype=f64)
    return s


# ----------------------------------------------------------------------------
# Low-precision storage of the matrices (per-row scales, RNE with saturation)
# ----------------------------------------------------------------------------

FORMATS = {
    # name: (explicit mantissa bits, minimum normal exponent, largest finite, saturating)
    "bf16": (7, -126, float.fromhex("0x1.fep127"), False),
    "e4m3": (3, -6, 448.0, True),
}


def round_to_format(x32, fmt):
    """Round single-precision values to the nearest value of ``fmt`` (ties to
    even), saturating to the largest finite value for E4M3.  Returned as
    float64 holding the exact rounded value (sign of zero kept)."""
    mbits, emin, maxfin, saturate = FORMATS[fmt]
    x = np.asarray(x32, dtype=f32).astype(f64)
    _, e = np.frexp(x)                       # x = m * 2**e with 0.5 <= |m| < 1
    lead = np.maximum(e - 1, emin)           # exponent of the leading bit, subnormals pinned at emin
    quantum = np.ldexp(1.0, lead - mbits)    # spacing of representable values at that exponent
    q = np.rint(x / quantum) * quantum       # np.rint rounds half to even; x/quantum is exact
    q = np.copysign(q, x)
    if saturate:
        q = np.clip(q, -maxfin, maxfin)
    return q


def encode(q, fmt):
    """Bit pattern of exactly representable values ``q`` (from round_to_format)."""
    q = np.asarray(q, dtype=f64)
    if fmt == "bf16":
        return (q.astype(f32).view(np.uint32) >> 16).astype(np.uint16)
    mbits, emin, _, _ = FORMATS[fmt]
    sign = np.signbit(q).astype(np.uint8) << 7
    mag = np.abs(q)
    _, e = np.frexp(mag)
    lead = np.maximum(e - 1, emin)
    normal = mag >= np.ldexp(1.0, emin)
    expf = np.where(normal, lead - emin + 1, 0)       # biased exponent field (bias 7 for E4M3)
    mant = np.where(normal, mag / np.ldexp(1.0, lead) - 1.0, mag / np.ldexp(1.0, emin))
    mantf = np.rint(mant * (1 << mbits)).astype(np.int64)
    return (sign | (expf.astype(np.uint8) << mbits) | mantf.astype(np.uint8)).astype(np.uint8)


def decode(codes, fmt):
    """Values of BF16 / E4M3 bit patterns (float64, exact)."""
    codes = np.asarray(codes)
    if fmt == "bf16":
        return (codes.astype(np.uint32) << 16).view(f32).astype(f64)
    mbits, emin, _, _ = FORMATS[fmt]
    sign = np.where(codes & 0x80, -1.0, 1.0)
    expf = (codes >> mbits) & 0xF
    mant = (codes & ((1 << mbits) - 1)).astype(f64)
    val = np.where(expf == 0,
                   np.ldexp(mant / (1 << mbits), emin),
                   np.ldexp(1.0 + mant / (1 << mbits), expf.astype(np.int64) + emin - 1))
    return sign * val


def quantize_rows(M, fmt):
    """Per-row scaled quantisation of a float32 matrix.

    scale_r = max_j |M_rj| (BF16) or max_j |M_rj| / 448 (E4M3) in single
    precision, 1 for an all-zero row; code_rj = RNE(fl(M_rj / scale_r)).
    Returns (codes, scales) with codes as uint16 (BF16) or uint8 (E4M3)."""
    M = np.asarray(M, dtype=f32)
    amax = np.abs(M).max(axis=1) if M.shape[1] else np.zeros(M.shape[0], f32)
    if fmt == "bf16":
        scale = amax.astype(f32)
    elif fmt == "e4m3":
        scale = (amax / f32(448.0)).astype(f32)
    else:
        raise ValueError(fmt)
    scale = np.where(scale > 0, scale, f32(1.0)).astype(f32)
    x = (M / scale[:, None]).astype(f32)
    return encode(round_to_format(x, fmt), fmt), scale


def stored_matrix(data, dtype, scale):
    """The matrix the reconstruction actually multiplies by, in float64:
    row scale (if any) times the decoded entries."""
    if dtype == "f32":
        m = np.asarray(data, dtype=f32).astype(f64)
    else:
        m = decode(data, dtype)
    if scale is not None:
        m = m * np.asarray(scale, dtype=f32).astype(f64)[:, None]
    return m


# ----------------------------------------------------------------------------
# Reconstruction and control (Section 3, Section 3.4)
# ----------------------------------------------------------------------------


def mvm(m64, s):
    """Reconstruction matrix-vector multiply y = M~ s in float64."""
    return np.asarray(m64, dtype=f64) @ np.asarray(s, dtype=f64)


def control_step(a_prev, y, q_prev, gain, leak, clip=None):
    """Leaky integrator with the implicit-POLC term folded in:
    a_k = (1 - leak) a_{k-1} + gain (y_k + q_{k-1}), then optional clip."""
    a = (1.0 - leak) * np.asarray(a_prev, dtype=f64) + gain * (np.asarray(y, dtype=f64) + np.asarray(q_prev, dtype=f64))
    if clip is not None:
        a = np.clip(a, clip[0], clip[1])
    return a


def explicit_polc_step(m64, d64, s, a_prev, gain, leak):
    """Explicit pseudo-open-loop control (Section 3.4): form the POL slopes
    s_ol = s + D a_{k-1} first, then a_k = (1 - leak - gain) a_{k-1} + gain M s_ol.
    Used only to check that the implicit form with P = M D - I gives the same
    commands."""
    s_ol = np.asarray(s, dtype=f64) + d64 @ np.asarray(a_prev, dtype=f64)
    return (1.0 - leak - gain) * np.asarray(a_prev, dtype=f64) + gain * (m64 @ s_ol)


class OracleLoop:
    """One AO loop in float64: holds M~, P~ (or D~) and the integrator state.

    cfg["polc"] "implicit" (default): the control law above, with q = P~ a.
    "explicit": the pseudo-open-loop slopes s_ol = s + D~ a_{k-1} are formed
    first and a_k = (1 - leak - gain) a_{k-1} + gain M~ s_ol (Section 3.4's
    explicit form; D is the ns x na interaction matrix); step() then returns
    s_ol as the slopes, since they are what the reconstructor is applied to."""

    def __init__(self, cfg):
        self.cfg = cfg
        self.explicit = cfg.get("polc", "implicit") == "explicit"
        self.m = stored_matrix(cfg["M"], cfg.get("M_dtype", "f32"), cfg.get("M_scale"))
        self.p = (stored_matrix(cfg["P"], cfg.get("P_dtype", "f32"), cfg.get("P_scale"))
                  if cfg.get("P") is not None and not self.explicit else None)
        self.d = (stored_matrix(cfg["D"], cfg.get("D_dtype", "f32"), cfg.get("D_scale"))
                  if self.explicit else None)
        na = self.m.shape[0]
        a0 = cfg.get("a0")
        self.a = np.zeros(na) if a0 is None else np.asarray(a0, dtype=f64).copy()
        self.q = self.p @ self.a if self.p is not None else np.zeros(na)

    def step(self, frames):
        """One frame: returns (slopes, commands) and advances the state."""
        s = frame_slopes(self.cfg, frames)
        gain, leak, clip = self.cfg["gain"], self.cfg["leak"], self.cfg.get("clip")
        if self.explicit:
            s = s + self.d @ self.a           # pseudo-open-loop slopes
            self.a = (1.0 - leak - gain) * self.a + gain * mvm(self.m, s)
            if clip is not None:
                self.a = np.clip(self.a, clip[0], clip[1])
            return s, self.a.copy()
        y = mvm(self.m, s)
        self.a = control_step(self.a, y, self.q, gain, leak, clip)
        if self.p is not None:
            self.q = self.p @ self.a          # for the next frame, after the command is out
        return s, self.a.copy()
