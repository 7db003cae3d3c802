"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds no arithmetic of the transform.  It only draws images and
residual planes so that the CUDA path and the CPU oracle can be fed the same
bytes.

* Natural-image stand-in (Sec. 4 uses 45 512x512 8-bit grayscale images from a
  public bank, not available here): a separable, stationary first-order Markov
  (AR(1)) Gaussian field -- the covariance model ``rho^|i-j|`` of Sec. 3.2 in
  both directions -- affinely mapped to ``128 + 40 f`` (optionally plus white
  Gaussian noise) and rounded/clipped to 0..255.
* Video-residual stand-in (Sec. 5.3 uses HEVC sequences, not available here):
  int16 residuals, 30 % exact zeros, otherwise a Laplacian of scale 6 rounded
  half away from zero and clipped to [-255, 255].
* Image sides for mixed-size batches: log-uniform on [lo, hi], rounded to the
  nearest multiple of 16 inside [lo, hi].
"""

from __future__ import annotations

import numpy as np
from scipy.signal import lfilter


def ar1_field(h: int, w: int, rho: float, rng: np.random.Generator) -> np.ndarray:
    """Unit-variance separable AR(1) field of shape (h, w), float64.

    ``x_0 ~ N(0, 1)``, ``x_n = rho x_{n-1} + sqrt(1 - rho^2) e_n`` along the
    columns of white noise, then the same recursion along the rows of the
    result; the covariance is ``rho^(|di| + |dj|)``.
    """
    e = rng.standard_normal((h, w))
    g = np.sqrt(1.0 - rho * rho)
    # y[n] = rho y[n-1] + g e[n] with y[0] = e[0] (stationary start).
    a = lfilter([g], [1.0, -rho], e, axis=0, zi=((1.0 - g) * e[:1, :]))[0]
    b = lfilter([g], [1.0, -rho], a, axis=1, zi=((1.0 - g) * a[:, :1]))[0]
    return b


def ar1_image(h: int, w: int, rho: float, seed: int, noise_sigma: float = 0.0,
              scale: float = 40.0, mean: float = 128.0) -> np.ndarray:
    """uint8 image ``clip(round_half_even(mean + scale f + noise), 0, 255)``."""
    rng = np.random.default_rng(seed)
    f = ar1_field(h, w, rho, rng)
    v = mean + scale * f
    if noise_sigma > 0:
        v = v + noise_sigma * rng.standard_normal((h, w))
    return np.clip(np.rint(v), 0, 255).astype(np.uint8)


def laplacian_residual(h: int, w: int, seed: int, scale: float = 6.0,
                       p_zero: float = 0.3) -> np.ndarray:
    """int16 residual plane: 30 % exact zeros, else a rounded Laplacian."""
    rng = np.random.default_rng(seed)
    lap = rng.laplace(0.0, scale, size=(h, w))
    r = np.sign(lap) * np.floor(np.abs(lap) + 0.5)
    r = np.clip(r, -255, 255)
    zero = rng.random((h, w)) < p_zero
    r[zero] = 0
    return r.astype(np.int16)


def log_uniform_side(rng: np.random.Generator, lo: int, hi: int) -> int:
    v = float(np.exp(rng.uniform(np.log(lo), np.log(hi))))
    s = int(round(v / 16.0)) * 16
    return int(min(max(s, lo), hi))


# ---------------------------------------------------------------------------
# Workload recipes (sizes and seeds are part of the recipe).
# ---------------------------------------------------------------------------
ZONAL_R_SWEEP = (1, 6, 16, 36, 64, 100, 150, 256)
QUANT_QP_SWEEP = (22, 27, 32, 37)


def single_image_256(seed: int = 1) -> np.ndarray:
    """One 256x256 uint8 AR(1) image, rho = 0.95 (256 blocks)."""
    return ar1_image(256, 256, 0.95, seed)


def batch_image(i: int, n: int = 64, side: int = 512, first_seed: int = 100) -> np.ndarray:
    """Image ``i`` of the ``n``-image batch: the first half AR(1) rho=0.95,
    the second half AR(1) rho=0.80 plus N(0, 8^2) noise; seed first_seed + i."""
    if i < n // 2:
        return ar1_image(side, side, 0.95, first_seed + i)
    return ar1_image(side, side, 0.80, first_seed + i, noise_sigma=8.0)


def image_batch_512(n: int = 64, side: int = 512, first_seed: int = 100, indices=None) -> np.ndarray:
    """The images ``indices`` (default: all) of the ``n``-image batch of
    :func:`batch_image`.  Shape (len(indices), side, side)."""
    idx = list(range(n)) if indices is None else list(indices)
    out = np.empty((len(idx), side, side), dtype=np.uint8)
    for k, i in enumerate(idx):
        out[k] = batch_image(i, n, side, first_seed)
    return out


N_VIDEO_FRAMES = 240


def residual_frame(index: int, luma=(1088, 1920), seed: int = 3):
    """Frame ``index`` of the 4:2:0 int16 residual sequence: (Y, Cb, Cr)."""
    ly, lx = luma
    s = seed * 1000003 + 3 * index
    return (laplacian_residual(ly, lx, s),
            laplacian_residual(ly // 2, lx // 2, s + 1),
            laplacian_residual(ly // 2, lx // 2, s + 2))


def residual_frames(n_frames: int, luma=(1088, 1920), seed: int = 3, first: int = 0):
    """Frames ``first .. first + n_frames - 1`` of the residual sequence."""
    return [residual_frame(f, luma, seed) for f in range(first, first + n_frames)]


def mixed_sizes(n: int, lo: int, hi: int, seed: int) -> list:
    """``n`` (height, width) pairs, sides independently log-uniform."""
    rng = np.random.default_rng(seed)
    return [(log_uniform_side(rng, lo, hi), log_uniform_side(rng, lo, hi)) for _ in range(n)]


def mixed_batch(n: int, lo: int = 128, hi: int = 4096, seed: int = 4,
                max_pixels: int | None = None) -> list:
    """Mixed-size uint8 AR(1) images, rho ~ U[0.8, 0.97] per image.

    ``max_pixels`` truncates the list once the running pixel total would pass
    it (for CPU-side tests)."""
    rng = np.random.default_rng(seed)
    sizes = mixed_sizes(n, lo, hi, seed + 7)
    imgs, total = [], 0
    for i, (h, w) in enumerate(sizes):
        if max_pixels is not None and total + h * w > max_pixels:
            break
        rho = float(rng.uniform(0.8, 0.97))
        imgs.append(ar1_image(h, w, rho, seed * 100003 + i))
        total += h * w
    return imgs


def poisson_arrivals(n: int, rate: float, seed: int) -> np.ndarray:
    """Arrival times (seconds) of a Poisson process of the given rate."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, size=n))
