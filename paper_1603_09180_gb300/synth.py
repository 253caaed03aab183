"""Seeded synthetic grayscale images for lambda-thinning workloads.

The paper measures on one 512x512 brain-MRI section (Sec. 5.2) that is not
available here, so every input is synthetic.  This module only makes
pixels: it holds none of the thinning arithmetic, and both the CPU oracle
tests and the CUDA path draw their inputs from it.

Recipe (fixed here, stated once):

1. three octaves of uniform noise U[0,1) at full resolution, drawn from
   numpy's PCG64 seeded with ``seed``;
2. each octave blurred by a Gaussian of sigma 2, 8 and 32 px (reflect
   boundary, kernel truncated at 4 sigma), done separably with real FFTs;
3. each blurred octave min-max normalised to [0, 1];
4. weighted sum with weights 0.2, 0.3, 0.5;
5. ``n_lines`` (20) dark line segments: endpoints uniform over the image,
   width uniform in {2, 3, 4} px, every pixel centre within width/2 of the
   segment lowered by ``depth`` (40/255 of the full range);
6. min-max rescale to [0, vmax] (255 for u8, 4095 for u16 by default),
   round half to even, cast.

Images are H x W numpy arrays (row = y, column = x), C-contiguous.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import fft

SIGMAS = (2.0, 8.0, 32.0)
WEIGHTS = (0.2, 0.3, 0.5)
BASE_SEED = 1603


def _blur1d(a: np.ndarray, sigma: float, axis: int) -> np.ndarray:
    """Gaussian blur along one axis: reflect boundary, radius int(4 sigma + 0.5)."""
    r = int(4.0 * sigma + 0.5)
    t = np.arange(-r, r + 1, dtype=np.float64)
    k = np.exp(-0.5 * (t / sigma) ** 2)
    k /= k.sum()
    a = np.moveaxis(a, axis, -1)
    n = a.shape[-1]
    pad = np.pad(a, [(0, 0)] * (a.ndim - 1) + [(r, r)], mode="symmetric")
    nf = fft.next_fast_len(pad.shape[-1] + 2 * r, real=True)
    out = fft.irfft(fft.rfft(pad, nf, axis=-1) * fft.rfft(k, nf), nf, axis=-1)
    return np.moveaxis(out[..., 2 * r: 2 * r + n], -1, axis)


def _blur(a: np.ndarray, sigma: float) -> np.ndarray:
    return _blur1d(_blur1d(a, sigma, 0), sigma, 1)


def _norm01(a: np.ndarray) -> np.ndarray:
    lo, hi = float(a.min()), float(a.max())
    if hi <= lo:
        return np.zeros_like(a)
    return (a - lo) / (hi - lo)


def _draw_lines(v: np.ndarray, rng: np.random.Generator, n_lines: int, depth: float) -> None:
    h, w = v.shape
    for _ in range(n_lines):
        x0, x1 = rng.uniform(0, w, 2)
        y0, y1 = rng.uniform(0, h, 2)
        width = int(rng.integers(2, 5))
        half = width / 2.0
        xa, xb = max(0, int(math.floor(min(x0, x1) - half))), min(w, int(math.ceil(max(x0, x1) + half)) + 1)
        ya, yb = max(0, int(math.floor(min(y0, y1) - half))), min(h, int(math.ceil(max(y0, y1) + half)) + 1)
        if xa >= xb or ya >= yb:
            continue
        yy, xx = np.mgrid[ya:yb, xa:xb].astype(np.float64)
        dx, dy = x1 - x0, y1 - y0
        L2 = dx * dx + dy * dy
        if L2 > 0:
            t = np.clip(((xx - x0) * dx + (yy - y0) * dy) / L2, 0.0, 1.0)
        else:
            t = np.zeros_like(xx)
        px, py = x0 + t * dx, y0 + t * dy
        d2 = (xx - px) ** 2 + (yy - py) ** 2
        v[ya:yb, xa:xb] -= depth * (d2 <= half * half)


def value_noise_image(h: int, w: int, dtype: str = "u8", seed: int = BASE_SEED,
                      vmax: int | None = None, n_lines: int = 20,
                      depth: float = 40.0 / 255.0) -> np.ndarray:
    """One seeded synthetic image, H x W, dtype 'u8' (uint8) or 'u16' (uint16)."""
    if dtype not in ("u8", "u16"):
        raise ValueError("dtype must be 'u8' or 'u16'")
    if vmax is None:
        vmax = 255 if dtype == "u8" else 4095
    rng = np.random.Generator(np.random.PCG64(seed))
    noise = rng.random((3, h, w))
    v = np.zeros((h, w), dtype=np.float64)
    for o in range(3):
        v += WEIGHTS[o] * _norm01(_blur(noise[o], SIGMAS[o]))
    _draw_lines(v, rng, n_lines, depth)
    v = _norm01(v) * vmax
    out = np.rint(v)
    return np.clip(out, 0, vmax).astype(np.uint8 if dtype == "u8" else np.uint16)


def uniform_noise_image(h: int, w: int, dtype: str = "u8", seed: int = 0, vmax: int | None = None) -> np.ndarray:
    """White noise in [0, vmax]: a worst case with many small basins (edge-case tests)."""
    if vmax is None:
        vmax = 255 if dtype == "u8" else 4095
    rng = np.random.Generator(np.random.PCG64(seed))
    a = rng.integers(0, vmax + 1, size=(h, w))
    return a.astype(np.uint8 if dtype == "u8" else np.uint16)


def uneven_batch_specs(n: int = 1024, seed: int = BASE_SEED, lo: int = 64, hi: int = 2048,
                       lambdas=(0, 10, 25)):
    """Job shapes for an uneven batch: w and h independently log-uniform in [lo, hi],
    lambda uniform over ``lambdas``.  Returns a list of (h, w, lam, image_seed)."""
    rng = np.random.Generator(np.random.PCG64(seed + 7))
    a, b = math.log(lo), math.log(hi)
    hs = np.rint(np.exp(rng.uniform(a, b, n))).astype(int)
    ws = np.rint(np.exp(rng.uniform(a, b, n))).astype(int)
    lams = rng.choice(np.asarray(lambdas), n)
    return [(int(hs[i]), int(ws[i]), int(lams[i]), seed * 10007 + i) for i in range(n)]


def serve_trace(rate_per_s: float, n: int, seed: int = BASE_SEED, lo: int = 128, hi: int = 4096,
                lambdas=(0, 10)):
    """Poisson request trace: arrival times (s), and per request (h, w, dtype, lam, image_seed).
    Sides log-uniform in [lo, hi], dtype u8/u16 with probability 1/2 each."""
    rng = np.random.Generator(np.random.PCG64(seed + 13))
    gaps = rng.exponential(1.0 / rate_per_s, n)
    t = np.cumsum(gaps)
    a, b = math.log(lo), math.log(hi)
    hs = np.rint(np.exp(rng.uniform(a, b, n))).astype(int)
    ws = np.rint(np.exp(rng.uniform(a, b, n))).astype(int)
    dts = np.where(rng.random(n) < 0.5, "u8", "u16")
    lams = rng.choice(np.asarray(lambdas), n)
    reqs = [(int(hs[i]), int(ws[i]), str(dts[i]), int(lams[i]), seed * 7919 + i) for i in range(n)]
    return t, reqs
