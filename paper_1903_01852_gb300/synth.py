"""Seeded synthetic inputs shaped like the paper's AO set-ups (Table ao_compare, Section 3).

This module only *generates inputs*: pupil geometry, detector frames, calibration
maps, control and POLC matrices, and the camera's row-chunk plan.  It holds none
of the hot path's arithmetic (no calibration, no centroiding, no reconstruction,
no control law), so the FP64 oracle and the CUDA path can both consume exactly
the same arrays without sharing any code.

The paper streams images pre-computed by AO simulation from NVMe (Section 2.1);
those images are not available, so seeded frames with the paper's shapes stand
in for them.  Every generator takes an explicit ``numpy.random.Generator``
(PCG64) so that a (config, seed) pair fixes every byte.

A configuration is a plain dict::

    {"name", "na", "wfs": [wfs dicts], "M", "M_scale", "M_dtype",
     "P", "P_scale", "P_dtype", "gain", "leak", "clip", "a0", "ref_slopes"}

A Shack-Hartmann WFS dict has ``kind="sh"``, ``width``, ``height``, ``nsubx``,
``nsuby``, ``npx`` (pixels per subaperture side), ``ox``, ``oy`` (pixel origin
of the subaperture grid), ``valid`` (uint8 [nsuby, nsubx]).  A pyramid WFS dict
has ``kind="pyramid"``, ``width``, ``height``, ``pupil`` (pupil side in pixels),
``qx``, ``qy`` (pixel origins of the four pupil images A=top-left, B=top-right,
C=bottom-left, D=bottom-right) and ``valid`` (uint8 [pupil, pupil]).  Both carry
``dark``, ``flat`` (float32 [height, width]), ``threshold``, ``thresh_mode``
("subtract" or "clip"), ``nblocks`` (MVM column blocks) and the spot/flux model
parameters used to draw frames.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "annulus_mask", "sh_wfs", "pyramid_wfs", "control_matrix", "polc_matrix",
    "make_config", "draw_frames", "chunk_plan", "slope_row_bounds", "CONFIGS",
    "num_valid", "num_slopes",
]

# Configuration names, in the order the paper's set-ups are listed (Table ao_compare).
CONFIGS = ("scao_small", "elt_scao_sh", "elt_scao_pyramid", "mcao", "ltao")


def annulus_mask(n: int, obs: float) -> np.ndarray:
    """uint8 [n, n] mask: 1 where the cell centre lies in the annulus
    obs*n/2 <= r <= n/2 (a circular pupil with a central obstruction)."""
    c = np.arange(n) + 0.5 - n / 2.0
    r = np.hypot(c[None, :], c[:, None])
    return ((r <= n / 2.0) & (r >= obs * n / 2.0)).astype(np.uint8)


def _calib_maps(rng, width, height, dark_mean=100.0, dark_sd=5.0, flat_sd=0.02):
    dark = rng.normal(dark_mean, dark_sd, size=(height, width)).astype(np.float32)
    flat = rng.normal(1.0, flat_sd, size=(height, width)).astype(np.float32)
    return dark, flat


def sh_wfs(rng, nsub, npx, width, height, obs, *, ox=None, oy=None, nblocks=1,
           threshold=5.0, thresh_mode="subtract", photons=500.0, sigma=1.2,
           max_offset=2.0, read_noise=3.0, elongation=None, launch_angle=0.0):
    """Shack-Hartmann WFS description with seeded dark/flat maps.

    ``elongation`` (None or a float e) makes LGS-like spots whose major-axis
    sigma grows from ``sigma`` to ``sigma*(1+e)`` with distance from a launch
    point on the pupil edge at ``launch_angle`` (radians)."""
    if ox is None:
        ox = (width - nsub * npx) // 2
    if oy is None:
        oy = (height - nsub * npx) // 2
    dark, flat = _calib_maps(rng, width, height)
    return dict(kind="sh", width=width, height=height, nsubx=nsub, nsuby=nsub,
                npx=npx, ox=ox, oy=oy, valid=annulus_mask(nsub, obs),
                nblocks=nblocks, dark=dark, flat=flat, threshold=float(threshold),
                thresh_mode=thresh_mode, photons=photons, sigma=sigma,
                max_offset=max_offset, read_noise=read_noise,
                elongation=elongation, launch_angle=launch_angle)


def pyramid_wfs(rng, pupil, width, height, obs, *, qx=None, qy=None, nblocks=4,
                threshold=0.0, thresh_mode="subtract", photons=200.0,
                read_noise=3.0):
    """Pyramid WFS description: four pupil images of ``pupil`` px on a frame.

    Default pupil origins centre each image in one quarter of the frame
    (A top-left, B top-right, C bottom-left, D bottom-right)."""
    if qx is None:
        off = (width // 2 - pupil) // 2
        qx = [off, width // 2 + off, off, width // 2 + off]
    if qy is None:
        off = (height // 2 - pupil) // 2
        qy = [off, off, height // 2 + off, height // 2 + off]
    dark, flat = _calib_maps(rng, width, height)
    return dict(kind="pyramid", width=width, height=height, pupil=pupil,
                qx=list(map(int, qx)), qy=list(map(int, qy)),
                valid=annulus_mask(pupil, obs), nblocks=nblocks, dark=dark,
                flat=flat, threshold=float(threshold), thresh_mode=thresh_mode,
                photons=photons, read_noise=read_noise)


def num_valid(w) -> int:
    return int(np.count_nonzero(w["valid"]))


def num_slopes(cfg) -> int:
    return sum(2 * num_valid(w) for w in cfg["wfs"])


def control_matrix(rng, na, ns, sd=1e-3):
    """Dense control matrix, float32 [na, ns], entries N(0, sd^2)."""
    return rng.standard_normal((na, ns), dtype=np.float32) * np.float32(sd)


def polc_matrix(rng, na, rel_sd=0.2):
    """POLC matrix P = -I + E with E ~ N(0, (rel_sd/sqrt(na))^2), float32.

    This mimics P = M*D - I with M*D close to I, which keeps the leaky
    integrator with implicit POLC stable (spectral radius well below 1)."""
    p = rng.standard_normal((na, na), dtype=np.float32) * np.float32(rel_sd / math.sqrt(na))
    p[np.arange(na), np.arange(na)] -= np.float32(1.0)
    return p


def interaction_matrix(rng, ns, na, m_sd=1e-3, radius=0.2):
    """Interaction matrix D, float32 [ns, na], entries N(0, sd^2) with
    sd = radius / (m_sd * sqrt(na * ns)): with a control matrix of N(0, m_sd^2)
    entries, M*D then has spectral radius about `radius`, so the explicit POLC
    iteration (1 - leak - g) I + g M D stays well inside the unit circle."""
    sd = radius / (m_sd * math.sqrt(float(na) * float(ns)))
    return rng.standard_normal((ns, na), dtype=np.float32) * np.float32(sd)


def make_config(name: str, seed: int | None = None, *, polc=None, gain=0.5,
                leak=0.01, clip=None, with_ref=False, nblocks=None):
    """Build one of the named configurations with its seeded arrays.

    scao_small       16x16 SH, 8x8 px, 128x128 frame, no obstruction, na=289
    elt_scao_sh      74x74 SH, 10x10 px, 740x740 frame, no obstruction, na=5316, 8 blocks
    elt_scao_pyramid 4x92x92 pupils on 240x240, obstruction 0.28, na=5316
    mcao             6 LGS 80x80 SH (10x10 px, 800x800, elongated spots) + 3 NGS 2x2
                     (100x100 px on 240x240), na=7500, POLC 7500x7500
    ltao             6 LGS 68x68 SH (10x10 px, 800x800) + 1 NGS 2x2, na=5316
    """
    index = CONFIGS.index(name)
    rng = np.random.default_rng(1000 + index + 1 if seed is None else seed)
    wfs = []
    if name == "scao_small":
        na = 289
        wfs.append(sh_wfs(rng, 16, 8, 128, 128, 0.0, nblocks=nblocks or 1))
        polc = False if polc is None else polc
    elif name == "elt_scao_sh":
        na = 5316
        wfs.append(sh_wfs(rng, 74, 10, 740, 740, 0.0, nblocks=nblocks or 8))
        polc = False if polc is None else polc
    elif name == "elt_scao_pyramid":
        na = 5316
        wfs.append(pyramid_wfs(rng, 92, 240, 240, 0.28, nblocks=nblocks or 4))
        polc = False if polc is None else polc
    elif name in ("mcao", "ltao"):
        nlgs, nsub, nngs = (6, 80, 3) if name == "mcao" else (6, 68, 1)
        na = 7500 if name == "mcao" else 5316
        for k in range(nlgs):
            wfs.append(sh_wfs(rng, nsub, 10, 800, 800, 0.28, nblocks=nblocks or 8,
                              elongation=2.0, launch_angle=math.radians(60.0 * k)))
        for _ in range(nngs):
            wfs.append(sh_wfs(rng, 2, 100, 240, 240, 0.28, nblocks=1,
                              photons=5.0e4, sigma=6.0, max_offset=10.0))
        polc = True if polc is None else polc
    else:
        raise ValueError(name)
    ns = sum(2 * num_valid(w) for w in wfs)
    M = control_matrix(rng, na, ns)
    P = polc_matrix(rng, na) if polc else None
    ref = (rng.normal(0.0, 0.05, size=ns).astype(np.float32) if with_ref else None)
    return dict(name=name, na=na, ns=ns, wfs=wfs, M=M, M_scale=None, M_dtype="f32",
                P=P, P_scale=None, P_dtype="f32", gain=float(gain),
                leak=float(leak), clip=clip, a0=None, ref_slopes=ref)


def _sh_frame(rng, w):
    h, wd, n = w["height"], w["width"], w["npx"]
    sig = np.zeros((h, wd), dtype=np.float64)
    iy, ix = np.nonzero(w["valid"])
    nv = iy.size
    if nv:
        off = rng.uniform(-w["max_offset"], w["max_offset"], size=(nv, 2))
        c = np.arange(n) - (n - 1) / 2.0
        dx = c[None, None, :] - off[:, 0, None, None]   # [nv, 1, n]
        dy = c[None, :, None] - off[:, 1, None, None]   # [nv, n, 1]
        s0 = w["sigma"]
        if w["elongation"]:
            # radial elongation away from the launch point on the pupil edge
            nsub = w["nsubx"]
            rad = nsub / 2.0
            lx, ly = rad * math.cos(w["launch_angle"]), rad * math.sin(w["launch_angle"])
            cx = ix + 0.5 - nsub / 2.0
            cy = iy + 0.5 - nsub / 2.0
            rho = np.hypot(cx - lx, cy - ly)
            th = np.arctan2(cy - ly, cx - lx)
            smaj = s0 * (1.0 + w["elongation"] * rho / (2.0 * rad))
            smin = np.full(nv, s0)
            ct, st = np.cos(th)[:, None, None], np.sin(th)[:, None, None]
            u = ct * dx + st * dy
            v = -st * dx + ct * dy
            img = np.exp(-0.5 * ((u / smaj[:, None, None]) ** 2 + (v / smin[:, None, None]) ** 2))
        else:
            img = np.exp(-0.5 * (dx ** 2 + dy ** 2) / s0 ** 2)
        img *= w["photons"] / img.sum(axis=(1, 2), keepdims=True)
        img = rng.poisson(img).astype(np.float64)
        for k in range(nv):
            y0 = w["oy"] + iy[k] * n
            x0 = w["ox"] + ix[k] * n
            sig[y0:y0 + n, x0:x0 + n] = img[k]
    return sig


def _pyramid_frame(rng, w):
    h, wd, p = w["height"], w["width"], w["pupil"]
    sig = np.zeros((h, wd), dtype=np.float64)
    yy, xx = np.mgrid[0:p, 0:p] / float(p)
    mask = w["valid"].astype(bool)
    for k in range(4):
        # smooth positive pupil-image intensity: a few random low-order sinusoids
        f = np.ones((p, p))
        for _ in range(3):
            kx, ky = rng.uniform(0.5, 3.0, size=2)
            ph = rng.uniform(0, 2 * np.pi)
            f += 0.25 * rng.uniform(0.2, 1.0) * np.sin(2 * np.pi * (kx * xx + ky * yy) + ph)
        expected = np.where(mask, w["photons"] / 4.0 * np.clip(f, 0.05, None), 0.0)
        img = rng.poisson(expected).astype(np.float64)
        sig[w["qy"][k]:w["qy"][k] + p, w["qx"][k]:w["qx"][k] + p] += img
    return sig


def draw_frames(cfg, nframes: int, seed: int = 0):
    """Draw ``nframes`` frames; returns a list (per frame) of lists (per WFS) of
    uint16 [height, width] arrays.  Detector model: photon counts (Poisson) plus
    Gaussian read noise, then raw = signal/flat + dark, rounded and clipped to
    the uint16 range."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(nframes):
        per = []
        for w in cfg["wfs"]:
            sig = _sh_frame(rng, w) if w["kind"] == "sh" else _pyramid_frame(rng, w)
            sig += rng.normal(0.0, w["read_noise"], size=sig.shape)
            raw = sig / w["flat"].astype(np.float64) + w["dark"].astype(np.float64)
            per.append(np.clip(np.rint(raw), 0, 65535).astype(np.uint16))
        out.append(per)
    return out


def slope_row_bounds(w):
    """Pixel-row readiness of each slope row: for SH the subaperture rows, for a
    pyramid the pupil rows (which need the matching row of all four pupil
    images).  Returns a list of 'rows needed' (exclusive pixel-row bound)."""
    if w["kind"] == "sh":
        return [w["oy"] + (i + 1) * w["npx"] for i in range(w["nsuby"])]
    return [max(w["qy"]) + i + 1 for i in range(w["pupil"])]


def chunk_plan(w, nchunks: int):
    """Camera row-chunk boundaries for one WFS: ``nchunks`` chunks whose ends
    fall on slope-row readiness boundaries where possible (the paper streams
    rows and starts work as soon as a row of subapertures is complete,
    Section 2.2).  Returns a list of (row_begin, row_end)."""
    h = w["height"]
    if nchunks <= 1:
        return [(0, h)]
    ready = slope_row_bounds(w)
    nr = len(ready)
    if w["kind"] == "sh":
        ends = [ready[(k * nr) // nchunks - 1] for k in range(1, nchunks)]
    else:
        ends = [(k * h) // nchunks for k in range(1, nchunks)]
    ends = sorted(set(e for e in ends if 0 < e < h))
    bounds = [0] + ends + [h]
    return [(bounds[i], bounds[i + 1]) for i in range(len(bounds) - 1)]
