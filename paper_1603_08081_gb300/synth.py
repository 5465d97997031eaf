"""Seeded synthetic test images (shared input generator; holds none of the filter's arithmetic).

The paper measures on the 512x512 *Barbara* image (Sec. V, T = 217).  That image
is not available here and is not recreated; these images stand in for it.  They
have the structure a bilateral filter is meant for: piecewise-constant regions
separated by step edges at every orientation, a slow linear ramp, and additive
Gaussian noise.

Recipe (numpy ``default_rng(seed)``, PCG64):

* Voronoi partition with ``R = clamp(H*W / 96**2, 8, 4096)`` seed points drawn
  uniformly in the image; every cell gets an integer level uniform in [20, 235].
* Linear gradient ``+ 40*x/W - 20*y/H``.
* Noise ``+ N(0, 10**2)``.
* ``rint`` (ties to even), clamp to [0, 255], cast to uint8.  T = 255.

Both the CUDA path (through the tests and the bench) and the oracle receive the
same arrays from here; neither generates its own.
"""
from __future__ import annotations

import numpy as np

__all__ = ["make_image", "make_image_f32", "make_batch_specs", "make_grad"]


def _voronoi_labels(H: int, W: int, pts: np.ndarray) -> np.ndarray:
    """Index of the nearest seed for every pixel centre (exact nearest neighbour)."""
    try:
        from scipy.spatial import cKDTree

        tree = cKDTree(pts)
        yy, xx = np.mgrid[0:H, 0:W]
        q = np.stack([yy.ravel().astype(np.float64), xx.ravel().astype(np.float64)], 1)
        _, idx = tree.query(q, k=1)
        return idx.reshape(H, W)
    except ImportError:  # pragma: no cover - scipy is present on both machines
        lab = np.empty((H, W), np.int64)
        xx = np.arange(W, dtype=np.float64)
        for y in range(H):
            d = (pts[:, 0:1] - y) ** 2 + (pts[:, 1:2] - xx[None, :]) ** 2
            lab[y] = np.argmin(d, axis=0)
        return lab


def make_image(H: int, W: int, seed: int) -> np.ndarray:
    """uint8 (H, W) synthetic image, values in [0, 255] (T = 255)."""
    H, W = int(H), int(W)
    if H <= 0 or W <= 0:
        return np.zeros((max(H, 0), max(W, 0)), np.uint8)
    rng = np.random.default_rng(seed)
    R = int(min(max(H * W // (96 * 96), 8), 4096))
    pts = np.stack([rng.uniform(0, H, R), rng.uniform(0, W, R)], 1)
    levels = rng.integers(20, 236, size=R).astype(np.float64)
    img = levels[_voronoi_labels(H, W, pts)]
    yy, xx = np.mgrid[0:H, 0:W]
    img = img + 40.0 * xx / W - 20.0 * yy / H
    img = img + rng.normal(0.0, 10.0, size=(H, W))
    return np.clip(np.rint(img), 0, 255).astype(np.uint8)


def make_image_f32(H: int, W: int, seed: int) -> np.ndarray:
    """The same construction scaled to [0, 1] as float32 (T = 1)."""
    return (make_image(H, W, seed).astype(np.float32) / np.float32(255.0)).astype(np.float32)


def make_grad(H: int, W: int, seed: int) -> np.ndarray:
    """Upstream gradient g ~ N(0, 1), float32."""
    return np.random.default_rng(seed).normal(0.0, 1.0, size=(H, W)).astype(np.float32)


def make_batch_specs(n: int = 64, seed: int = 1399, lo: int = 256, hi: int = 2048):
    """Per-image (H, W, sigma_s, sigma_r, image_seed) for a batch of uneven images.

    H and W are independent uniform integers in [lo, hi]; sigma_s ~ U[2, 10],
    sigma_r ~ U[10, 60]; image i uses seed 1300 + i.
    """
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        H = int(rng.integers(lo, hi + 1))
        W = int(rng.integers(lo, hi + 1))
        ss = float(rng.uniform(2.0, 10.0))
        sr = float(rng.uniform(10.0, 60.0))
        out.append((H, W, ss, sr, 1300 + i))
    return out
