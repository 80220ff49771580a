"""Seeded synthetic inputs for the vector-valued Allen-Cahn segmentation.

This module holds no arithmetic of the method. It only draws images, initial
phase fields and target label maps from seeded generators (numpy PCG64), so
that the CUDA path and the CPU oracle can be fed identical inputs.

Images are float32 arrays of shape (H, W, 3), row index = y, values in [0, 1];
the paper treats the image as piecewise constant per pixel (Sec. 4.1) with
colour channels handled jointly (Sec. 4.4). The paper's own test images
(concentric circles, geometric composite, "Flowers", "Lena") are not
available; the generators below stand in for them with the same structure:
a few flat-coloured regions plus i.i.d. Gaussian noise.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "palette", "shapes_image", "disks_polygons_image", "voronoi_ramp_image",
    "stripes_image", "dirichlet_init", "voronoi_labels", "batch_specs",
    "round_bf16", "CONFIGS", "config_image",
]


def palette(rng: np.random.Generator, k: int, min_dist: float = 0.2) -> np.ndarray:
    """k colours uniform in [0,1]^3, redrawn until all pairwise distances >= min_dist."""
    for _ in range(10000):
        cols = rng.uniform(0.0, 1.0, size=(k, 3))
        d = np.linalg.norm(cols[:, None, :] - cols[None, :, :], axis=-1)
        d[np.arange(k), np.arange(k)] = np.inf
        if d.min() >= min_dist:
            return cols
    raise RuntimeError("palette: could not satisfy the distance constraint")


def _noise_clip(rng, img, sigma):
    if sigma > 0:
        img = img + rng.normal(0.0, sigma, size=img.shape)
    return np.clip(img, 0.0, 1.0).astype(np.float32)


def _pixel_centres(W, H):
    ys, xs = np.mgrid[0:H, 0:W]
    return xs + 0.5, ys + 0.5


def shapes_image(seed: int, W: int = 64, H: int = 64, n_rect: int = 4, n_disk: int = 3,
                 n_colours: int = 4, sigma: float = 0.05,
                 rect_side=(8, 32), disk_r=(4, 16)) -> np.ndarray:
    """Axis-aligned rectangles and disks painted with palette colours on a
    background of palette colour 0, plus clipped Gaussian noise.

    Defaults are the 64x64, 4-rectangle / 3-disk, 4-colour, sigma=0.05 image;
    rect_side and disk_r are in pixels and are scaled by W/64 by callers that
    want the same look at another size."""
    rng = np.random.default_rng(seed)
    cols = palette(rng, n_colours)
    img = np.empty((H, W, 3), np.float64)
    img[:] = cols[0]
    xc, yc = _pixel_centres(W, H)
    for _ in range(n_rect):
        w = rng.integers(rect_side[0], rect_side[1] + 1)
        h = rng.integers(rect_side[0], rect_side[1] + 1)
        x0 = rng.integers(0, max(1, W - w + 1))
        y0 = rng.integers(0, max(1, H - h + 1))
        img[y0:y0 + h, x0:x0 + w] = cols[rng.integers(0, n_colours)]
    for _ in range(n_disk):
        r = rng.uniform(*disk_r)
        cx, cy = rng.uniform(0, W), rng.uniform(0, H)
        inside = (xc - cx) ** 2 + (yc - cy) ** 2 <= r * r
        img[inside] = cols[rng.integers(0, n_colours)]
    return _noise_clip(rng, img, sigma)


def disks_polygons_image(seed: int, W: int = 1024, H: int = 1024, n_shapes: int = 64,
                         n_colours: int = 4, sigma: float = 0.1,
                         r_range=(16, 96)) -> np.ndarray:
    """Random disks and random convex 3..8-gons (vertices on a circle) in
    n_colours palette colours on palette colour 0, plus clipped noise."""
    rng = np.random.default_rng(seed)
    cols = palette(rng, n_colours)
    img = np.empty((H, W, 3), np.float64)
    img[:] = cols[0]
    for _ in range(n_shapes):
        r = rng.uniform(*r_range)
        cx, cy = rng.uniform(0, W), rng.uniform(0, H)
        colour = cols[rng.integers(0, n_colours)]
        x0, x1 = max(0, int(cx - r) - 1), min(W, int(cx + r) + 2)
        y0, y1 = max(0, int(cy - r) - 1), min(H, int(cy + r) + 2)
        if x0 >= x1 or y0 >= y1:
            continue
        ys, xs = np.mgrid[y0:y1, x0:x1]
        px, py = xs + 0.5, ys + 0.5
        if rng.uniform() < 0.5:
            inside = (px - cx) ** 2 + (py - cy) ** 2 <= r * r
        else:
            k = int(rng.integers(3, 9))
            ang = np.sort(rng.uniform(0, 2 * np.pi, size=k))
            vx, vy = cx + r * np.cos(ang), cy + r * np.sin(ang)
            inside = np.ones(px.shape, bool)
            for j in range(k):  # counter-clockwise vertices: interior on the left
                ax, ay = vx[j], vy[j]
                bx, by = vx[(j + 1) % k], vy[(j + 1) % k]
                inside &= (bx - ax) * (py - ay) - (by - ay) * (px - ax) >= 0
        img[y0:y1, x0:x1][inside] = colour
    return _noise_clip(rng, img, sigma)


def voronoi_ramp_image(seed: int, W: int = 4096, H: int = 4096, n_regions: int = 8,
                       sigma: float = 0.05, max_ramp: float = 0.2) -> np.ndarray:
    """Voronoi partition of n_regions uniform seeds; each region has a base
    colour U[0,1]^3 plus a linear ramp whose total change across the image is
    at most max_ramp per channel; clipped Gaussian noise on top."""
    rng = np.random.default_rng(seed)
    sx, sy = rng.uniform(0, W, n_regions), rng.uniform(0, H, n_regions)
    base = rng.uniform(0, 1, (n_regions, 3))
    amp = rng.uniform(0, max_ramp, (n_regions, 3))
    ang = rng.uniform(0, 2 * np.pi, (n_regions, 3))
    dx, dy = np.cos(ang), np.sin(ang)
    norm = np.abs(dx) + np.abs(dy)
    img = np.empty((H, W, 3), np.float32)
    xs = np.arange(W) + 0.5
    chunk = 256
    for y0 in range(0, H, chunk):
        y1 = min(H, y0 + chunk)
        ys = (np.arange(y0, y1) + 0.5)[:, None]
        best = np.full((y1 - y0, W), np.inf)
        lab = np.zeros((y1 - y0, W), np.int64)
        for k in range(n_regions):
            d = (xs[None, :] - sx[k]) ** 2 + (ys - sy[k]) ** 2
            m = d < best
            best[m] = d[m]
            lab[m] = k
        X, Y = xs[None, :] / W, ys / H
        out = base[lab] + amp[lab] * (dx[lab] * X[..., None] + dy[lab] * Y[..., None]) / norm[lab]
        noise = rng.normal(0.0, sigma, size=out.shape) if sigma > 0 else 0.0
        img[y0:y1] = np.clip(out + noise, 0, 1)
    return img


def stripes_image(W: int, H: int, widths, colours, axis: int = 0) -> np.ndarray:
    """Noise-free image of full-length axis-aligned stripes.

    axis=0: vertical stripes (columns), widths sum to W; axis=1: horizontal
    stripes, widths sum to H. colours[k % len(colours)] paints stripe k."""
    img = np.empty((H, W, 3), np.float32)
    pos = 0
    for k, w in enumerate(widths):
        c = np.asarray(colours[k % len(colours)], np.float32)
        if axis == 0:
            img[:, pos:pos + w] = c
        else:
            img[pos:pos + w, :] = c
        pos += w
    if pos != (W if axis == 0 else H):
        raise ValueError("stripe widths must cover the image")
    return img


def dirichlet_init(seed: int, n_nodes: int, N: int) -> np.ndarray:
    """Random point of the Gibbs simplex per node: Dirichlet(1,...,1) drawn
    as normalised standard exponentials. Shape (n_nodes, N), float64."""
    rng = np.random.default_rng(seed)
    e = rng.standard_exponential(size=(n_nodes, N))
    return e / e.sum(axis=1, keepdims=True)


def voronoi_labels(seed: int, Wn: int, Hn: int, n_seeds: int = 6, n_labels: int = 4) -> np.ndarray:
    """Piecewise-constant target label map on an Hn x Wn grid: a Voronoi
    partition of n_seeds points, each cell labelled uniformly in 0..n_labels-1."""
    rng = np.random.default_rng(seed)
    sx, sy = rng.uniform(0, Wn, n_seeds), rng.uniform(0, Hn, n_seeds)
    lab_of = rng.integers(0, n_labels, n_seeds)
    ys, xs = np.mgrid[0:Hn, 0:Wn]
    d = (xs[None] - sx[:, None, None]) ** 2 + (ys[None] - sy[:, None, None]) ** 2
    return lab_of[np.argmin(d, axis=0)].astype(np.int8)


def batch_specs(seed: int, count: int = 256):
    """Uneven batch: sizes uniform over {128^2, 256^2, 512^2, 1024^2, 768x512},
    N uniform over {2, 4, 6}, noise sigma U[0.02, 0.15]. Returns a list of dicts
    with keys W, H, N, sigma, seed."""
    rng = np.random.default_rng(seed)
    sizes = [(128, 128), (256, 256), (512, 512), (1024, 1024), (768, 512)]
    out = []
    for k in range(count):
        W, H = sizes[rng.integers(0, len(sizes))]
        out.append(dict(W=W, H=H, N=int(rng.choice([2, 4, 6])),
                        sigma=float(rng.uniform(0.02, 0.15)), seed=int(seed * 100003 + k)))
    return out


def round_bf16(x: np.ndarray) -> np.ndarray:
    """Round float32 values to the nearest bfloat16 (ties to even), returned as
    float32. Written from the IEEE-754 binary32 layout: keep the top 16 bits,
    rounding on the lower 16. Inputs here are finite values in [0, 1]."""
    b = np.ascontiguousarray(x, np.float32).view(np.uint32).astype(np.uint64)
    lsb = (b >> 16) & 1
    r = ((b + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


# The five workloads. eps, tau are in pixel units (pixel side h = 1); tau = eps^2.
CONFIGS = {
    "c1_64_n4_fp64": dict(W=64, H=64, N=4, eps=2.0, lam=1.0, tau=4.0, steps=20, tol=1e-10,
                          precision="fp64", image="shapes", sigma=0.05),
    "c2_1024_n4": dict(W=1024, H=1024, N=4, eps=2.0, lam=1.0, tau=4.0, steps=50, tol=1e-8,
                       tol_mixed=1e-6, precision="fp64", image="disks_polygons", sigma=0.1),
    "c3_4096_n8_mixed": dict(W=4096, H=4096, N=8, eps=3.0, lam=2.0, tau=9.0, steps=100, tol=1e-6,
                             precision="mixed", image="voronoi_ramp", sigma=0.05),
    "c5_512_n4_adjoint": dict(W=512, H=512, N=4, eps=2.0, lam=1.0, tau=4.0, steps=64, tol=1e-10,
                              precision="fp64", image="disks", sigma=0.08),
}


def config_image(name: str, seed: int = 0, W: int | None = None, H: int | None = None) -> np.ndarray:
    """The synthetic image of a named workload (optionally at another size)."""
    cfg = CONFIGS[name]
    W = W or cfg["W"]
    H = H or cfg["H"]
    kind = cfg["image"]
    if kind == "shapes":
        s = W / 64.0
        return shapes_image(seed, W, H, sigma=cfg["sigma"], rect_side=(max(1, int(8 * s)), max(1, int(32 * s))),
                            disk_r=(4 * s, 16 * s))
    if kind == "disks_polygons":
        s = W / 1024.0
        return disks_polygons_image(seed, W, H, sigma=cfg["sigma"], r_range=(16 * s, 96 * s))
    if kind == "voronoi_ramp":
        return voronoi_ramp_image(seed, W, H, sigma=cfg["sigma"])
    if kind == "disks":
        s = W / 512.0
        return shapes_image(seed, W, H, n_rect=0, n_disk=12, sigma=cfg["sigma"], disk_r=(16 * s, 64 * s))
    raise KeyError(kind)
