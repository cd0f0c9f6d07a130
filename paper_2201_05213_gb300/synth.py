"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This module holds no arithmetic of the compression method itself: it only
draws images, image-size lists and initial network weights from seeded numpy
generators (PCG64).  The paper measures on ImageNet photographs with weights
pre-trained on CIFAR10 (Section 4); neither is available, so these images stand
in for them with natural-image-like statistics:

* a Gaussian random field per channel whose power spectrum falls as 1/f^2
  (amplitude 1/f, zero DC), standardised;
* the three channels mixed by a random 3x3 matrix (inter-channel correlation),
  re-standardised and scaled to mean 128, std 40;
* ``n_poly`` constant-colour polygons (3-6 vertices, even-odd fill at pixel
  centres) giving hard edges;
* additive N(0, 2^2) noise, rounded to the nearest integer and clipped to
  [0, 255].
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "make_image",
    "make_batch",
    "random_crops",
    "uneven_sizes",
    "xavier_weights",
    "num_weights",
    "weight_shapes",
]


def _rng(seed, *stream):
    return np.random.default_rng([int(seed), *[int(s) for s in stream]])


def _field(rng, H, W):
    """One channel of a 1/f-amplitude Gaussian random field, standardised."""
    white = rng.standard_normal((H, W))
    spec = np.fft.rfft2(white)
    fy = np.fft.fftfreq(H)[:, None]
    fx = np.fft.rfftfreq(W)[None, :]
    f = np.sqrt(fx * fx + fy * fy)
    amp = np.zeros_like(f)
    nz = f > 0
    amp[nz] = 1.0 / f[nz]
    out = np.fft.irfft2(spec * amp, s=(H, W))
    out -= out.mean()
    sd = out.std()
    return out / (sd if sd > 0 else 1.0)


def _fill_polygon(img, verts, colour):
    """Even-odd fill of a polygon, sampled at pixel centres, restricted to its bbox."""
    H, W, _ = img.shape
    xs, ys = verts[:, 0], verts[:, 1]
    x0 = max(int(np.floor(xs.min())), 0)
    x1 = min(int(np.ceil(xs.max())) + 1, W)
    y0 = max(int(np.floor(ys.min())), 0)
    y1 = min(int(np.ceil(ys.max())) + 1, H)
    if x0 >= x1 or y0 >= y1:
        return
    py, px = np.mgrid[y0:y1, x0:x1]
    cy = py + 0.5
    cx = px + 0.5
    inside = np.zeros(cy.shape, dtype=bool)
    n = len(verts)
    for a in range(n):
        xa, ya = verts[a]
        xb, yb = verts[(a + 1) % n]
        cond = (ya > cy) != (yb > cy)
        with np.errstate(divide="ignore", invalid="ignore"):
            xint = xa + (cy - ya) * (xb - xa) / (yb - ya)
        inside ^= cond & (cx < xint)
    img[y0:y1, x0:x1][inside] = colour


def make_image(seed: int, H: int, W: int, n_poly: int = 4, index: int = 0) -> np.ndarray:
    """One H x W x 3 uint8 image (HWC, C-contiguous) from ``seed`` and ``index``."""
    rng = _rng(seed, index)
    chans = np.stack([_field(rng, H, W) for _ in range(3)], axis=-1)  # H,W,3
    A = rng.standard_normal((3, 3))
    mixed = chans @ A.T
    mixed -= mixed.mean(axis=(0, 1), keepdims=True)
    sd = mixed.std(axis=(0, 1), keepdims=True)
    sd[sd == 0] = 1.0
    img = 128.0 + 40.0 * (mixed / sd)
    for _ in range(n_poly):
        nv = int(rng.integers(3, 7))
        verts = np.stack([rng.uniform(0, W, nv), rng.uniform(0, H, nv)], axis=1)
        colour = rng.integers(0, 256, 3).astype(np.float64)
        _fill_polygon(img, verts, colour)
    img = img + rng.normal(0.0, 2.0, img.shape)
    return np.clip(np.rint(img), 0, 255).astype(np.uint8)


def make_batch(seed: int, sizes, n_poly: int = 4):
    """A list of images; image k has shape ``sizes[k]`` = (H, W) and stream index k."""
    return [make_image(seed, int(H), int(W), n_poly, index=k) for k, (H, W) in enumerate(sizes)]


def uneven_sizes(seed: int, n: int, lo: int = 32, hi: int = 512, step: int = 16):
    """``n`` (H, W) pairs, each side drawn independently and uniformly from lo..hi by step."""
    rng = _rng(seed, 10_000)
    choices = np.arange(lo, hi + 1, step)
    return [(int(rng.choice(choices)), int(rng.choice(choices))) for _ in range(n)]


def random_crops(seed: int, n: int, size: int = 32, source: int = 256, per_source: int = 16,
                 n_poly: int = 4) -> np.ndarray:
    """``n`` random size x size crops (N,H,W,3 uint8) cut from fresh source images."""
    rng = _rng(seed, 20_000)
    out = np.empty((n, size, size, 3), dtype=np.uint8)
    k = 0
    src_idx = 0
    while k < n:
        img = make_image(seed, source, source, n_poly, index=100_000 + src_idx)
        src_idx += 1
        for _ in range(min(per_source, n - k)):
            y = int(rng.integers(0, source - size + 1))
            x = int(rng.integers(0, source - size + 1))
            out[k] = img[y:y + size, x:x + size]
            k += 1
    return out


def weight_shapes(h: int, C: int, R: int, K: int):
    """(name, shape) of every tensor of the flat weight vector, in storage order.

    W0 is [C][F] with F = 6h(h+1) context features; residual block r has
    W1_r, b1_r, W2_r, b2_r ([C][C] and [C]); the head WH is [10K][C].
    """
    F = 6 * h * (h + 1)
    shapes = [("W0", (C, F)), ("b0", (C,))]
    for r in range(R):
        shapes += [(f"W1_{r}", (C, C)), (f"b1_{r}", (C,)), (f"W2_{r}", (C, C)), (f"b2_{r}", (C,))]
    shapes += [("WH", (10 * K, C)), ("bH", (10 * K,))]
    return shapes


def num_weights(h: int, C: int, R: int, K: int) -> int:
    return int(sum(int(np.prod(s)) for _, s in weight_shapes(h, C, R, K)))


def xavier_weights(h: int, C: int, R: int, K: int, seed: int = 0) -> np.ndarray:
    """Flat float32 weights: Xavier-uniform matrices (fan_in + fan_out), zero biases."""
    rng = _rng(seed, 30_000)
    parts = []
    for name, shp in weight_shapes(h, C, R, K):
        if len(shp) == 2:
            fan_out, fan_in = shp
            a = np.sqrt(6.0 / (fan_in + fan_out))
            parts.append(rng.uniform(-a, a, shp).ravel())
        else:
            parts.append(np.zeros(shp).ravel())
    return np.concatenate(parts).astype(np.float32)
