"""Seeded synthetic inputs for lattice information-theoretic clustering.

This module only draws inputs: binary silhouettes, weight images, gray images and initial
codebooks.  It holds none of the clustering arithmetic, so the FP64 oracle and the CUDA path
can both be fed from it without sharing any part of the method.

Every generator is deterministic: image ``i`` of workload ``c`` is drawn from
``numpy.random.PCG64(c * 1000 + i)``.

Workloads (the paper's own data, the MPEG-7 shapes and the lizard image of its figures, are not
available, so these stand in for them; the shapes follow the paper's binary-silhouette setting,
Sec. 3.2 and Sec. 4, and its weighted and gray-value variants, Sec. 5 and Sec. 1):

* ``c1``: one 64x64 binary image, union of 5 random ellipses, 10-20 % on; M=8, sigma=2.
* ``c2``: one 1024x1024 binary image, 200 random ellipses plus 20 thin random polylines,
  about 10 % on; M=64, sigma=4.
* ``c3``: 4096 binary blob-union silhouettes with independent sides U{64..512}, on-fraction
  target U[5 %, 40 %]; per-image M from {16, 32, 64, 128}, sigma from {2, 3, 4}.
* ``c4``: 512x512 float32 weights, Gaussian-smoothed white noise (sigma 8, reflect padding)
  mapped to clip(0.5 + 0.25 z / std(z), 0, 1); M=32 seeds with h > 0.5; sigma=3.
* ``c5``: 256x256 8-bit gray image, smoothed noise (sigma 6) min-max scaled to [0, 255], plus
  5 % salt-and-pepper; lattice [u, v, g] with 256 gray levels; M=64; sigma=(3, 3, 8).
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "rng_for", "draw_ellipse", "draw_polyline", "c1_image", "c2_image", "c3_batch", "c3_shape", "c3_codebook",
    "c4_weights", "c5_gray", "init_codebook", "init_codebook_gray", "blob_silhouette",
]


def rng_for(config: int, index: int) -> np.random.Generator:
    """Generator for image ``index`` of workload ``config`` (PCG64, seed config*1000+index)."""
    return np.random.Generator(np.random.PCG64(config * 1000 + index))


def draw_ellipse(img: np.ndarray, cu: float, cv: float, a: float, b: float, theta: float) -> int:
    """Set the pixels of a filled rotated ellipse to 1; return how many pixels were newly set."""
    H, W = img.shape
    r = int(np.ceil(max(a, b))) + 1
    u0, u1 = max(0, int(cu) - r), min(H, int(cu) + r + 1)
    v0, v1 = max(0, int(cv) - r), min(W, int(cv) + r + 1)
    if u0 >= u1 or v0 >= v1:
        return 0
    uu, vv = np.meshgrid(np.arange(u0, u1) - cu, np.arange(v0, v1) - cv, indexing="ij")
    c, s = np.cos(theta), np.sin(theta)
    p = (uu * c + vv * s) / a
    q = (-uu * s + vv * c) / b
    inside = (p * p + q * q) <= 1.0
    sub = img[u0:u1, v0:v1]
    new = int(np.count_nonzero(inside & (sub == 0)))
    sub[inside] = 1
    return new


def draw_polyline(img: np.ndarray, pts: np.ndarray) -> None:
    """Rasterise a 1-px-thick polyline with Bresenham segments between successive vertices."""
    H, W = img.shape
    for (u0, v0), (u1, v1) in zip(pts[:-1], pts[1:]):
        u0, v0, u1, v1 = int(u0), int(v0), int(u1), int(v1)
        du, dv = abs(u1 - u0), -abs(v1 - v0)
        su, sv = (1 if u0 < u1 else -1), (1 if v0 < v1 else -1)
        err = du + dv
        while True:
            if 0 <= u0 < H and 0 <= v0 < W:
                img[u0, v0] = 1
            if u0 == u1 and v0 == v1:
                break
            e2 = 2 * err
            if e2 >= dv:
                err += dv
                u0 += su
            if e2 <= du:
                err += du
                v0 += sv


def c1_image(index: int = 0) -> np.ndarray:
    """64x64 uint8 union of 5 ellipses (semi-axes U[4,16], angle U[0,pi)); redrawn until 10-20 % on."""
    rng = rng_for(1, index)
    while True:
        img = np.zeros((64, 64), np.uint8)
        for _ in range(5):
            draw_ellipse(img, rng.uniform(0, 64), rng.uniform(0, 64), rng.uniform(4, 16),
                         rng.uniform(4, 16), rng.uniform(0, np.pi))
        if 0.10 <= img.mean() <= 0.20:
            return img


def c2_image(index: int = 0, size: int = 1024) -> np.ndarray:
    """size^2 uint8: 200 ellipses (semi-axes U[4,22]) and 20 polylines of 3-8 local vertices."""
    rng = rng_for(2, index)
    img = np.zeros((size, size), np.uint8)
    scale = size / 1024.0
    for _ in range(200):
        draw_ellipse(img, rng.uniform(0, size), rng.uniform(0, size), rng.uniform(4, 22) * scale,
                     rng.uniform(4, 22) * scale, rng.uniform(0, np.pi))
    for _ in range(20):
        n = int(rng.integers(3, 9))
        p = [rng.uniform(0, size, 2)]
        for _ in range(n - 1):
            p.append(np.clip(p[-1] + rng.uniform(-128, 128, 2) * scale, 0, size - 1))
        draw_polyline(img, np.array(p))
    return img


def blob_silhouette(rng: np.random.Generator, H: int, W: int, target: float) -> np.ndarray:
    """Union of disks and ellipses added until the on-fraction reaches ``target``."""
    img = np.zeros((H, W), np.uint8)
    on, need = 0, int(np.ceil(target * H * W))
    side = min(H, W)
    while on < need:
        a = rng.uniform(0.04, 0.16) * side
        b = a if rng.random() < 0.5 else rng.uniform(0.04, 0.16) * side
        on += draw_ellipse(img, rng.uniform(0, H), rng.uniform(0, W), max(a, 1.5), max(b, 1.5),
                           rng.uniform(0, np.pi))
    return img


def _c3_draw(i: int):
    rng = rng_for(3, i)
    H, W = int(rng.integers(64, 513)), int(rng.integers(64, 513))
    target = rng.uniform(0.05, 0.40)
    M = int(rng.choice([16, 32, 64, 128]))
    s = float(rng.choice([2.0, 3.0, 4.0]))
    return rng, H, W, target, M, s


def c3_shape(i: int):
    """``(H, W, M, sigma)`` of image ``i`` of the ragged batch, without drawing its pixels."""
    _, H, W, _, M, s = _c3_draw(i)
    return H, W, M, s


def c3_batch(n: int = 4096, start: int = 0, indices=None):
    """Ragged batch of binary silhouettes (images ``start .. start+n-1``, or the listed ``indices``).

    Returns ``(images, M, sigma)``: a list of uint8 arrays with sides drawn from U{64..512},
    per-image codebook sizes from {16, 32, 64, 128} and kernel widths from {2, 3, 4}.
    """
    images, Ms, sigmas = [], [], []
    for i in (range(start, start + n) if indices is None else indices):
        rng, H, W, target, M, s = _c3_draw(int(i))
        images.append(blob_silhouette(rng, H, W, target))
        Ms.append(M)
        sigmas.append(s)
    return images, np.array(Ms, np.int32), np.array(sigmas, np.float32)


def c3_codebook(i: int, img: np.ndarray, M: int) -> np.ndarray:
    """Initial codebook of image ``i`` of the ragged batch as the benchmark draws it: M distinct
    foreground pixels (PCG64 seed 3 * 1000 + 500000 + i)."""
    return init_codebook(rng_for(3, 500_000 + i), img.astype(np.float32), int(M))


def _smooth_noise(rng: np.random.Generator, shape, sigma: float) -> np.ndarray:
    from scipy.ndimage import gaussian_filter  # input recipe only (not the method)
    z = rng.standard_normal(shape)
    return gaussian_filter(z, sigma, mode="reflect", truncate=4.0)


def c4_weights(index: int = 0, size: int = 512) -> np.ndarray:
    """size^2 float32 weights clip(0.5 + 0.25 z/std(z), 0, 1), z smoothed white noise (sigma 8)."""
    rng = rng_for(4, index)
    z = _smooth_noise(rng, (size, size), 8.0)
    return np.clip(0.5 + 0.25 * z / z.std(), 0.0, 1.0).astype(np.float32)


def c5_gray(index: int = 0, size: int = 256) -> np.ndarray:
    """size^2 uint8 gray image: smoothed noise (sigma 6) scaled to [0,255] + 5 % salt-and-pepper."""
    rng = rng_for(5, index)
    z = _smooth_noise(rng, (size, size), 6.0)
    g = np.rint(255.0 * (z - z.min()) / (z.max() - z.min()))
    sp = rng.random((size, size)) < 0.05
    g[sp] = np.where(rng.random(int(sp.sum())) < 0.5, 0.0, 255.0)
    return g.astype(np.uint8)


def init_codebook(rng: np.random.Generator, weights: np.ndarray, M: int, thresh: float = 0.0) -> np.ndarray:
    """M distinct lattice sites drawn uniformly among pixels with weight > thresh; float32 [M, 2] (u, v)."""
    idx = np.flatnonzero(weights.reshape(-1) > thresh)
    if idx.size < M:
        raise ValueError(f"only {idx.size} candidate pixels for M={M}")
    pick = rng.choice(idx, size=M, replace=False)
    W = weights.shape[1]
    return np.stack([pick // W, pick % W], axis=1).astype(np.float32)


def init_codebook_gray(rng: np.random.Generator, gray: np.ndarray, M: int) -> np.ndarray:
    """M distinct occupied voxels (u, v, gray(u, v)) of a gray image's [u, v, g] lattice; float32 [M, 3]."""
    uv = init_codebook(rng, np.ones_like(gray, dtype=np.float32), M)
    g = gray[uv[:, 0].astype(int), uv[:, 1].astype(int)].astype(np.float32)
    return np.concatenate([uv, g[:, None]], axis=1)
