"""Seeded synthetic images shared by the tests, the benchmark and the oracle.

The paper's own test images ("Isha", "Greekdome", "Tulip", the 720 x 540
timing image) are not available; these generators stand in for them with the
shapes, value ranges and structure of the paper's workloads: piecewise-constant
regions with edges (what the bilateral filter must preserve), smooth shading,
and additive Gaussian noise, on the [0, 255] gray scale.

This module holds no arithmetic of the filter itself, so both the CUDA path
and the oracle may use it.  Every generator takes a seed and uses
``numpy.random.default_rng(seed)``.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "rectangles", "smooth_field", "rect_disk_u8", "batch_specs", "batch_images",
    "upstream", "sample_indices", "radius_map",
]


def rectangles(H: int, W: int, n_rect: int = 12, noise: float = 10.0, seed: int = 0,
               dtype=np.float32) -> np.ndarray:
    """Uniform gray background plus ``n_rect`` axis-aligned rectangles of
    uniform gray in [0, 255] (later ones overwrite earlier ones), plus
    N(0, noise^2) noise, clamped to [0, 255]."""
    rng = np.random.default_rng(seed)
    img = np.full((H, W), rng.uniform(0, 255), dtype=np.float64)
    for _ in range(n_rect):
        y0, y1 = np.sort(rng.integers(0, H + 1, size=2))
        x0, x1 = np.sort(rng.integers(0, W + 1, size=2))
        img[y0:y1, x0:x1] = rng.uniform(0, 255)
    img += rng.normal(0.0, noise, size=(H, W))
    return np.clip(img, 0.0, 255.0).astype(dtype)


def smooth_field(H: int, W: int, n_waves: int = 20, n_regions: int = 16,
                 noise: float = 5.0, seed: int = 0, dtype=np.float32) -> np.ndarray:
    """Sum of ``n_waves`` random 2-D sinusoids, plus piecewise-constant
    rectangular regions, plus N(0, noise^2) noise, rescaled into [0, 255]."""
    rng = np.random.default_rng(seed)
    yy = np.arange(H, dtype=np.float64)[:, None]
    xx = np.arange(W, dtype=np.float64)[None, :]
    img = np.zeros((H, W), dtype=np.float64)
    for _ in range(n_waves):
        ky, kx = rng.uniform(-0.05, 0.05, size=2)
        ph = rng.uniform(0, 2 * np.pi)
        amp = rng.uniform(5.0, 25.0)
        img += amp * np.sin(ky * yy + kx * xx + ph)
    for _ in range(n_regions):
        y0, y1 = np.sort(rng.integers(0, H + 1, size=2))
        x0, x1 = np.sort(rng.integers(0, W + 1, size=2))
        img[y0:y1, x0:x1] += rng.uniform(-60, 60)
    lo, hi = img.min(), img.max()
    img = (img - lo) / max(hi - lo, 1e-9) * 235.0 + 10.0
    img += rng.normal(0.0, noise, size=(H, W))
    return np.clip(img, 0.0, 255.0).astype(dtype)


def rect_disk_u8(H: int, W: int, C: int = 3, n_shapes: int = 40, noise: float = 8.0,
                 seed: int = 0) -> np.ndarray:
    """H x W x C interleaved uint8 texture: random rectangles and disks of
    random colour on a random background, plus N(0, noise^2) noise, rounded
    and clamped to [0, 255]."""
    rng = np.random.default_rng(seed)
    img = np.empty((H, W, C), dtype=np.float32)
    img[:] = rng.uniform(0, 255, size=C).astype(np.float32)
    yy = np.arange(H, dtype=np.float32)[:, None]
    xx = np.arange(W, dtype=np.float32)[None, :]
    for k in range(n_shapes):
        col = rng.uniform(0, 255, size=C).astype(np.float32)
        if k % 2 == 0:
            y0, y1 = np.sort(rng.integers(0, H + 1, size=2))
            x0, x1 = np.sort(rng.integers(0, W + 1, size=2))
            img[y0:y1, x0:x1, :] = col
        else:
            cy, cx = rng.uniform(0, H), rng.uniform(0, W)
            rad = rng.uniform(0.02, 0.25) * min(H, W)
            m = (yy - cy) ** 2 + (xx - cx) ** 2 <= rad * rad
            img[m] = col
    # add noise plane by plane to bound peak memory at 4096 x 4096 x 3
    for c in range(C):
        img[:, :, c] += rng.normal(0.0, noise, size=(H, W)).astype(np.float32)
    return np.clip(np.rint(img), 0, 255).astype(np.uint8)


def batch_specs(count: int = 64, seed: int = 0, w_range=(128, 1920), h_range=(128, 1080),
                sigma_s_range=(2.0, 16.0), sigma_r_range=(15.0, 60.0)):
    """Per-image (H, W, sigma_s, sigma_r) for a batch of uneven images:
    W ~ U[128, 1920], H ~ U[128, 1080] (integers), sigma_s ~ U[2, 16],
    sigma_r ~ U[15, 60]."""
    rng = np.random.default_rng(seed)
    specs = []
    for _ in range(count):
        W = int(rng.integers(w_range[0], w_range[1] + 1))
        H = int(rng.integers(h_range[0], h_range[1] + 1))
        ss = float(rng.uniform(*sigma_s_range))
        sr = float(rng.uniform(*sigma_r_range))
        specs.append((H, W, ss, sr))
    return specs


def batch_images(specs, noise: float = 10.0, seed: int = 0):
    """One rectangles-plus-noise image per spec."""
    return [rectangles(H, W, noise=noise, seed=seed * 100003 + i)
            for i, (H, W, _, _) in enumerate(specs)]


def upstream(shape, seed: int = 0, dtype=np.float32) -> np.ndarray:
    """Random-normal upstream gradient."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal(size=shape).astype(dtype)


def sample_indices(H: int, W: int, n_interior: int, seed: int = 0,
                   border: bool = True) -> np.ndarray:
    """Flat pixel indices: every border pixel (if ``border``) plus
    ``n_interior`` distinct seeded pixels."""
    rng = np.random.default_rng(seed)
    idx = set()
    if border:
        for j in range(W):
            idx.add(j)
            idx.add((H - 1) * W + j)
        for i in range(H):
            idx.add(i * W)
            idx.add(i * W + W - 1)
    n_interior = min(n_interior, H * W)
    picks = rng.choice(H * W, size=n_interior, replace=False)
    idx.update(int(p) for p in picks)
    return np.array(sorted(idx), dtype=np.int64)


def radius_map(H: int, W: int, r_max: int, seed: int = 0, smooth: bool = True) -> np.ndarray:
    """int32 H x W map of box half-widths in [0, r_max] for the space-variant
    filter: a seeded smooth field (a few random 2-D sinusoids) quantised to
    the integers 0 .. r_max, or (``smooth=False``) independent uniform draws."""
    rng = np.random.default_rng(seed)
    if not smooth:
        return rng.integers(0, r_max + 1, size=(H, W)).astype(np.int32)
    yy = np.arange(H, dtype=np.float64)[:, None]
    xx = np.arange(W, dtype=np.float64)[None, :]
    v = np.zeros((H, W), dtype=np.float64)
    for _ in range(4):
        ky, kx = rng.uniform(-0.02, 0.02, size=2)
        v += np.sin(ky * yy + kx * xx + rng.uniform(0, 2 * np.pi))
    v = (v - v.min()) / max(v.max() - v.min(), 1e-9)
    return np.rint(v * r_max).astype(np.int32)
