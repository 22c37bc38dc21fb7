"""Seeded synthetic images and binary masks.

Images are float32 arrays shaped (C, H, W) (planar channels); masks are uint8
arrays shaped (H, W) holding 0/1.  Everything is generated on the host with
numpy so that both evaluators read identical bytes.
"""
from __future__ import annotations

from typing import List, Sequence

import numpy as np


# ----------------------------------------------------------------- images ---

def _gauss_kernel(sigma: float, truncate: float = 3.0) -> np.ndarray:
    r = int(truncate * sigma + 0.5)
    x = np.arange(-r, r + 1, dtype=np.float64)
    k = np.exp(-0.5 * (x / sigma) ** 2)
    return k / k.sum()


def _blur_axis(a: np.ndarray, k: np.ndarray, axis: int) -> np.ndarray:
    r = (len(k) - 1) // 2
    pad = [(0, 0)] * a.ndim
    pad[axis] = (r, r)
    # "reflect about the edge" boundary: d c b a | a b c d | d c b a
    p = np.pad(a, pad, mode="symmetric")
    out = np.zeros_like(a)
    n = a.shape[axis]
    for i, w in enumerate(k):
        sl = [slice(None)] * a.ndim
        sl[axis] = slice(i, i + n)
        out += w * p[tuple(sl)]
    return out


def gaussian_blur(a: np.ndarray, sigma: float, truncate: float = 3.0) -> np.ndarray:
    k = _gauss_kernel(sigma, truncate)
    return _blur_axis(_blur_axis(np.asarray(a, np.float64), k, 0), k, 1)


def gaussian_field_image(h: int = 512, w: int = 512, sigma: float = 4.0,
                         seed: int = 0) -> np.ndarray:
    """White noise N(0,1), Gaussian blur (sigma px, truncated at 3 sigma,
    reflected border), min-max rescaled to [0, 1]; shape (1, h, w) float32."""
    rng = np.random.default_rng(seed)
    x = gaussian_blur(rng.standard_normal((h, w)), sigma)
    x = (x - x.min()) / (x.max() - x.min())
    return x.astype(np.float32)[None]


def uniform_image(h: int, w: int, channels: int = 1, seed: int = 0) -> np.ndarray:
    """i.i.d. U[0, 1) float32 pixels; shape (channels, h, w)."""
    rng = np.random.default_rng(seed)
    return rng.random((channels, h, w), dtype=np.float32)


# ------------------------------------------------------------------ masks ---

def bernoulli_mask(h: int, w: int, p: float, seed: int = 0) -> np.ndarray:
    """i.i.d. Bernoulli(p) foreground, drawn in float32 row blocks."""
    rng = np.random.default_rng(seed)
    out = np.empty((h, w), dtype=np.uint8)
    step = max(1, (1 << 24) // max(w, 1))
    pf = np.float32(p)
    for r in range(0, h, step):
        rr = min(h, r + step)
        out[r:rr] = rng.random((rr - r, w), dtype=np.float32) < pf
    return out


def seed_mask(h: int, w: int, p: float = 1e-4, seed: int = 1) -> np.ndarray:
    """Sparse seeds for reachability: Bernoulli(p) pixels."""
    return bernoulli_mask(h, w, p, seed)


def spiral_mask(h: int, w: int) -> np.ndarray:
    """A square spiral one pixel wide with one-pixel gaps between turns: a
    single path-shaped component under both 4- and 8-adjacency, the worst case
    for label propagation (its geodesic length is about h*w/2).

    A turtle starts at (0, 0) heading right and turns clockwise; after each
    stroke the wall it just drew moves two pixels inwards."""
    m = np.zeros((h, w), dtype=np.uint8)
    r = c = 0
    m[0, 0] = 1
    top, left, bottom, right = 0, 0, h - 1, w - 1
    d = 0
    while True:
        if d == 0:                      # right along the current row
            if right <= c:
                break
            m[r, c:right + 1] = 1
            c = right
            top += 2
        elif d == 1:                    # down along the current column
            if bottom <= r:
                break
            m[r:bottom + 1, c] = 1
            r = bottom
            right -= 2
        elif d == 2:                    # left
            if left >= c:
                break
            m[r, left:c + 1] = 1
            c = left
            bottom -= 2
        else:                           # up
            if top >= r:
                break
            m[top:r + 1, c] = 1
            r = top
            left += 2
        d = (d + 1) % 4
    return m


def checkerboard_mask(h: int, w: int) -> np.ndarray:
    """(y + x) even: one component under 8-adjacency, all singletons under
    4-adjacency."""
    y, x = np.indices((h, w))
    return ((y + x) % 2 == 0).astype(np.uint8)


def rings_mask(h: int, w: int) -> np.ndarray:
    """Concentric one-pixel square rings with one-pixel gaps: pixel (y, x) is
    foreground when its Chebyshev distance to the image border is even."""
    y, x = np.indices((h, w))
    d = np.minimum(np.minimum(y, x), np.minimum(h - 1 - y, w - 1 - x))
    return (d % 2 == 0).astype(np.uint8)


def rings_count(h: int, w: int) -> int:
    """Number of components of ``rings_mask`` (under 4- or 8-adjacency): one
    per even border distance that occurs."""
    dmax = (min(h, w) - 1) // 2
    return dmax // 2 + 1


# ----------------------------------------------------- MRI-shaped batches ---

def mri_side_lengths(n: int = 4096, seed: int = 0, median: float = 240.0,
                     sigma: float = 0.25, lo: int = 160, hi: int = 512):
    """Side lengths clip(round(median * exp(sigma z)), lo, hi), independently
    for height and width; returns an (n, 2) int array."""
    rng = np.random.default_rng(seed)
    z = rng.standard_normal((n, 2))
    s = np.clip(np.rint(median * np.exp(sigma * z)), lo, hi)
    return s.astype(np.int64)


def _smooth_ellipse(yy, xx, cy, cx, ry, rx, theta, soft):
    c, s = np.cos(theta), np.sin(theta)
    u = ((yy - cy) * c + (xx - cx) * s) / ry
    v = (-(yy - cy) * s + (xx - cx) * c) / rx
    r = np.sqrt(u * u + v * v)
    # logistic edge, width `soft` in units of the radius
    return 1.0 / (1.0 + np.exp((r - 1.0) / soft))


def mri_phantom(h: int, w: int, rng: np.random.Generator) -> np.ndarray:
    """One 4-channel MRI-slice-shaped phantom, shape (4, h, w) float32:
    a smooth brain ellipse, and a tumour made of a bright core ellipse, a rim
    annulus (bright in channel 1) and an oedema halo (bright in channel 0),
    plus N(0, 0.05) noise on every channel."""
    yy, xx = np.mgrid[0:h, 0:w].astype(np.float64)
    brain = _smooth_ellipse(yy, xx, h / 2 + rng.normal(0, h * 0.02),
                            w / 2 + rng.normal(0, w * 0.02),
                            h * rng.uniform(0.36, 0.44), w * rng.uniform(0.34, 0.42),
                            rng.uniform(-0.3, 0.3), 0.03)
    ty = h / 2 + rng.uniform(-0.18, 0.18) * h
    tx = w / 2 + rng.uniform(-0.18, 0.18) * w
    rc = min(h, w) * rng.uniform(0.05, 0.10)
    th = rng.uniform(0, np.pi)
    ell = rng.uniform(0.7, 1.0)
    core = _smooth_ellipse(yy, xx, ty, tx, rc, rc * ell, th, 0.08)
    outer = _smooth_ellipse(yy, xx, ty, tx, rc * 1.45, rc * 1.45 * ell, th, 0.06)
    rim = np.clip(outer - core, 0, 1)
    halo = _smooth_ellipse(yy, xx, ty, tx, rc * 2.6, rc * 2.6 * ell * 1.1, th, 0.15)
    halo = np.clip(halo - outer, 0, 1)
    base = 0.35 * brain
    ch = np.empty((4, h, w), dtype=np.float64)
    ch[0] = base + 0.45 * halo + 0.55 * core + 0.30 * rim
    ch[1] = base + 0.60 * rim
    ch[2] = base + 0.60 * core
    ch[3] = 0.30 + 0.40 * brain - 0.20 * (core + rim)
    ch += rng.normal(0.0, 0.05, size=ch.shape)
    return ch.astype(np.float32)


def mri_phantom_batch(sides: Sequence[Sequence[int]], seed: int = 0) -> List[np.ndarray]:
    """A list of 4-channel phantoms with the given (h, w) sides; image i is
    drawn from its own stream (seed, i) so any subset is reproducible."""
    out = []
    for i, (h, w) in enumerate(sides):
        rng = np.random.default_rng([seed, i])
        out.append(mri_phantom(int(h), int(w), rng))
    return out


def _phantom_chunk(args):
    sides, seed, first = args
    out = []
    for k, (h, w) in enumerate(sides):
        rng = np.random.default_rng([seed, first + k])
        out.append(mri_phantom(int(h), int(w), rng))
    return out


def mri_phantom_batch_parallel(sides: Sequence[Sequence[int]], seed: int = 0,
                               processes: int = 0) -> List[np.ndarray]:
    """``mri_phantom_batch`` computed by a pool of spawned processes (safe
    after a GPU context exists); identical output, image i from stream
    (seed, i)."""
    import concurrent.futures as cf
    import multiprocessing as mp
    import os
    n = len(sides)
    procs = processes or min(16, os.cpu_count() or 1)
    if procs <= 1 or n < 64:
        return mri_phantom_batch(sides, seed)
    step = (n + procs * 4 - 1) // (procs * 4)
    chunks = [([tuple(map(int, s)) for s in sides[i:i + step]], seed, i) for i in range(0, n, step)]
    with cf.ProcessPoolExecutor(max_workers=procs, mp_context=mp.get_context("spawn")) as ex:
        parts = list(ex.map(_phantom_chunk, chunks))
    return [im for part in parts for im in part]


def upscaled_slice(side: int = 7680, base: int = 240, seed: int = 0) -> np.ndarray:
    """One MRI-shaped slice (channel 0 of an MRI phantom, base x base)
    upscaled bilinearly to side x side: a stand-in for the paper's upscaled
    2D slice of its case-study timing (about 60 Mpx at 7680 x 7680).
    Returns a (1, side, side) float32 array."""
    from scipy import ndimage as nd
    ph = mri_phantom(base, base, np.random.default_rng([seed, 7680]))
    z = nd.zoom(ph[0].astype(np.float64), side / base, order=1, mode="nearest")
    return z[:side, :side].astype(np.float32)[None]


def to_u16(img: np.ndarray) -> np.ndarray:
    """A [0, 1] image as 16-bit pixels: round(v * 65535), clipped (the paper
    scales its normalised slices by 2^16 - 1, Sec. 4.2)."""
    return np.clip(np.rint(np.asarray(img, dtype=np.float64) * 65535.0), 0, 65535).astype(np.uint16)


def uniform_image_u16(h: int, w: int, channels: int = 1, seed: int = 0) -> np.ndarray:
    """(C, H, W) uint16 pixels, uniform over 0..65535."""
    rng = np.random.default_rng(seed)
    return rng.integers(0, 65536, size=(channels, h, w), dtype=np.uint16)


def _smooth_ellipsoid(zz, yy, xx, c, r, soft):
    """Logistic-edged axis-aligned ellipsoid, centre c = (z, y, x), radii r."""
    d = np.sqrt(((zz - c[0]) / r[0]) ** 2 + ((yy - c[1]) / r[1]) ** 2 + ((xx - c[2]) / r[2]) ** 2)
    return 1.0 / (1.0 + np.exp((d - 1.0) / soft))


def mri_phantom_volume(d: int, h: int, w: int, seed: int = 0) -> np.ndarray:
    """A 4-channel MRI-volume-shaped phantom (the paper's scans are 3D
    volumes of which it keeps one slice, Sec. 4.2), shape (4, d, h, w)
    float32: a brain ellipsoid and a tumour of core, rim shell and oedema
    halo as in the slice phantom, plus N(0, 0.05) noise on every channel."""
    rng = np.random.default_rng(seed)
    zz, yy, xx = np.mgrid[0:d, 0:h, 0:w].astype(np.float64)
    brain = _smooth_ellipsoid(zz, yy, xx, (d / 2, h / 2, w / 2),
                              (d * rng.uniform(0.36, 0.44), h * rng.uniform(0.36, 0.44),
                               w * rng.uniform(0.34, 0.42)), 0.03)
    c = (d / 2 + rng.uniform(-0.15, 0.15) * d, h / 2 + rng.uniform(-0.18, 0.18) * h,
         w / 2 + rng.uniform(-0.18, 0.18) * w)
    rc = min(d, h, w) * rng.uniform(0.07, 0.12)
    core = _smooth_ellipsoid(zz, yy, xx, c, (rc, rc, rc * rng.uniform(0.7, 1.0)), 0.08)
    outer = _smooth_ellipsoid(zz, yy, xx, c, (rc * 1.45, rc * 1.45, rc * 1.45), 0.06)
    rim = np.clip(outer - core, 0, 1)
    halo = np.clip(_smooth_ellipsoid(zz, yy, xx, c, (rc * 2.6, rc * 2.6, rc * 2.9), 0.15) - outer, 0, 1)
    base = 0.35 * brain
    ch = np.empty((4, d, h, w), dtype=np.float64)
    ch[0] = base + 0.45 * halo + 0.55 * core + 0.30 * rim
    ch[1] = base + 0.60 * rim
    ch[2] = base + 0.60 * core
    ch[3] = 0.30 + 0.40 * brain - 0.20 * (core + rim)
    ch += rng.normal(0.0, 0.05, size=ch.shape)
    return ch.astype(np.float32)
