"""Seeded synthetic inputs for the FOEED / EED inpainting workloads.

This module only draws images and masks. It holds none of the inpainting
method's arithmetic (no pre-smoothing, no tensors, no stencils of the method,
no time stepping), so both the FP64 oracle tests and the CUDA path may use it.

Every generator takes a ``numpy.random.Generator`` (PCG64) or a seed and is
fully deterministic. The recipes stand in for the paper's natural and medical
test images (lena, peppers, t1slice, Sec. 4.1), which are not available: grey
values in [0, 1], random masks of a few percent density (Sec. 4.1 uses 2-30%).

Workloads (sizes and parameters):
  W1  64 x 64 FP64, ramps + disks + noise, 5% uniform mask, sigma=1, lambda=0.05,
      FSI cycle length 20, 40 cycles.
  W2  512 x 512 FP32, 20 star polygons + 1/f noise, 4% mask, sigma=1,
      lambda=0.03, cycle length 30, run to relative residual < 1e-6.
  W3  2048 x 2048 FP32, 40 additive ellipses, Rician-like noise, 12-bit
      quantised, 3% mask (half uniform, half |Laplacian|-weighted), sigma=1.5,
      lambda=0.02, 100 cycles of length 40.
  W4  256 instances, sides in {128,...,1024}, square and 2:1, W2 generator,
      density U[2%,10%], lambda U[0.01,0.1], sigma=1, 50 cycles of length 25.
  W5  1024 x 1024 FP32, W2 generator, 4% mask, 30 cycles of length 20.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "rng_for", "ramps_disks", "piecewise_smooth", "ellipse_phantom",
    "uniform_mask", "laplacian_weighted_mask", "workload",
    "batched_workload", "WORKLOADS",
]


def rng_for(workload_index: int, instance: int = 0) -> np.random.Generator:
    """PCG64 stream for (workload, instance): seed = 1000 * workload + instance."""
    return np.random.Generator(np.random.PCG64(1000 * int(workload_index) + int(instance)))


def _grid(h: int, w: int):
    y, x = np.mgrid[0:h, 0:w].astype(np.float64)
    return x, y


def ramps_disks(h: int, w: int, rng: np.random.Generator, n_ramps: int = 3,
                n_disks: int = 6, noise: float = 0.01) -> np.ndarray:
    """Sum of smooth linear/quadratic ramps, constant disks and Gaussian noise, in [0,1]."""
    x, y = _grid(h, w)
    xn = x / max(w - 1, 1)
    yn = y / max(h - 1, 1)
    img = np.zeros((h, w))
    for _ in range(n_ramps):
        a, b, c, d = rng.uniform(-1.0, 1.0, size=4)
        img += a * xn + b * yn + c * xn * xn + d * yn * yn
    lo, hi = img.min(), img.max()
    img = 0.2 + 0.6 * (img - lo) / (hi - lo) if hi > lo else np.full((h, w), 0.5)
    for _ in range(n_disks):
        r = rng.uniform(4.0, 12.0)
        cx, cy = rng.uniform(0, w), rng.uniform(0, h)
        val = rng.uniform(0.0, 1.0)
        img[(x - cx) ** 2 + (y - cy) ** 2 <= r * r] = val
    img = img + rng.normal(0.0, noise, size=(h, w))
    return np.clip(img, 0.0, 1.0)


def _star_polygon_inside(x, y, cx, cy, angles, radii):
    """Even-odd point-in-polygon test for the polygon with the given polar vertices."""
    vx = cx + radii * np.cos(angles)
    vy = cy + radii * np.sin(angles)
    inside = np.zeros(x.shape, dtype=bool)
    k = len(vx)
    for i in range(k):
        x1, y1 = vx[i], vy[i]
        x2, y2 = vx[(i + 1) % k], vy[(i + 1) % k]
        if y1 == y2:
            continue
        cond = (y1 > y) != (y2 > y)
        xc = x1 + (y - y1) * (x2 - x1) / (y2 - y1)
        inside ^= cond & (x < xc)
    return inside


def _pink_noise(h: int, w: int, rng: np.random.Generator, amp: float) -> np.ndarray:
    """White noise shaped to a 1/f amplitude spectrum, scaled to standard deviation amp."""
    white = rng.normal(0.0, 1.0, size=(h, w))
    spec = np.fft.fft2(white)
    fy = np.fft.fftfreq(h)[:, None]
    fx = np.fft.fftfreq(w)[None, :]
    f = np.sqrt(fx * fx + fy * fy)
    f[0, 0] = np.inf
    noise = np.real(np.fft.ifft2(spec / f))
    s = noise.std()
    return noise * (amp / s) if s > 0 else noise


def piecewise_smooth(h: int, w: int, rng: np.random.Generator, n_polys: int = 20,
                     noise_amp: float = 0.02) -> np.ndarray:
    """Random star-shaped polygons (3-9 vertices) with constant or linear-ramp
    interiors, painted in order over a ramp background, plus 1/f noise, in [0,1]."""
    x, y = _grid(h, w)
    g = rng.uniform(-0.5, 0.5, size=2)
    img = 0.5 + g[0] * (x / max(w, 1) - 0.5) * 0.4 + g[1] * (y / max(h, 1) - 0.5) * 0.4
    scale = min(h, w)
    for _ in range(n_polys):
        k = int(rng.integers(3, 10))
        cx, cy = rng.uniform(0, w), rng.uniform(0, h)
        angles = np.sort(rng.uniform(0.0, 2.0 * np.pi, size=k))
        radii = rng.uniform(0.05, 0.3, size=k) * scale
        rmax = radii.max()
        x0, x1 = int(max(0, np.floor(cx - rmax))), int(min(w, np.ceil(cx + rmax) + 1))
        y0, y1 = int(max(0, np.floor(cy - rmax))), int(min(h, np.ceil(cy + rmax) + 1))
        if x0 >= x1 or y0 >= y1:
            continue
        xs, ys = x[y0:y1, x0:x1], y[y0:y1, x0:x1]
        inside = _star_polygon_inside(xs, ys, cx, cy, angles, radii)
        base = rng.uniform(0.0, 1.0)
        if rng.uniform() < 0.5:
            val = np.full(xs.shape, base)
        else:
            gx, gy = rng.uniform(-1.0, 1.0, size=2) / scale
            val = base + gx * (xs - cx) + gy * (ys - cy)
        blk = img[y0:y1, x0:x1]
        blk[inside] = val[inside]
    img = img + _pink_noise(h, w, rng, noise_amp)
    return np.clip(img, 0.0, 1.0)


def ellipse_phantom(h: int, w: int, rng: np.random.Generator, n_ellipses: int = 40,
                    noise: float = 0.005, levels: int = 4095) -> np.ndarray:
    """Medical-like phantom: additive ellipses (axes U[20,400] px, angle U[0,pi),
    intensity U[-0.3,0.6]) normalised to [0,1], Rician-like noise
    sqrt((u+n1)^2+n2^2), then quantised to 12 bits and rescaled to [0,1]."""
    x, y = _grid(h, w)
    img = np.zeros((h, w))
    for _ in range(n_ellipses):
        a, b = rng.uniform(20.0, 400.0, size=2)
        th = rng.uniform(0.0, np.pi)
        cx, cy = rng.uniform(0, w), rng.uniform(0, h)
        val = rng.uniform(-0.3, 0.6)
        r = max(a, b)
        x0, x1 = int(max(0, np.floor(cx - r))), int(min(w, np.ceil(cx + r) + 1))
        y0, y1 = int(max(0, np.floor(cy - r))), int(min(h, np.ceil(cy + r) + 1))
        if x0 >= x1 or y0 >= y1:
            continue
        dx = x[y0:y1, x0:x1] - cx
        dy = y[y0:y1, x0:x1] - cy
        c, s = np.cos(th), np.sin(th)
        xr = c * dx + s * dy
        yr = -s * dx + c * dy
        inside = (xr / a) ** 2 + (yr / b) ** 2 <= 1.0
        img[y0:y1, x0:x1] += val * inside
    lo, hi = img.min(), img.max()
    img = (img - lo) / (hi - lo) if hi > lo else np.zeros((h, w))
    n1 = rng.normal(0.0, noise, size=(h, w))
    n2 = rng.normal(0.0, noise, size=(h, w))
    img = np.sqrt((img + n1) ** 2 + n2 ** 2)
    img = np.clip(img, 0.0, 1.0)
    return np.round(img * levels) / levels


def uniform_mask(h: int, w: int, density: float, rng: np.random.Generator,
                 exclude: np.ndarray | None = None) -> np.ndarray:
    """uint8 mask with round(density*h*w) known pixels drawn uniformly without replacement."""
    n = h * w
    k = int(round(density * n))
    mask = np.zeros(n, dtype=np.uint8)
    pool = np.arange(n) if exclude is None else np.flatnonzero(exclude.ravel() == 0)
    k = min(k, len(pool))
    if k > 0:
        mask[rng.choice(pool, size=k, replace=False)] = 1
    return mask.reshape(h, w)


def laplacian_weighted_mask(img: np.ndarray, density: float, rng: np.random.Generator) -> np.ndarray:
    """Half the known pixels uniform, half drawn (without replacement, disjoint)
    with probability proportional to the absolute 5-point Laplacian of img
    (edge-replicated border). Total count round(density*h*w)."""
    h, w = img.shape
    n = h * w
    k = int(round(density * n))
    k_uni = k // 2
    mask = uniform_mask(h, w, k_uni / n, rng)
    p = np.pad(img, 1, mode="edge")
    lap = np.abs(p[:-2, 1:-1] + p[2:, 1:-1] + p[1:-1, :-2] + p[1:-1, 2:] - 4.0 * img)
    weight = lap.ravel().copy()
    weight[mask.ravel() != 0] = 0.0
    k_rest = k - int(mask.sum())
    if k_rest > 0:
        nz = np.count_nonzero(weight)
        if nz < k_rest:  # too few edge pixels: top up uniformly
            weight = weight + (mask.ravel() == 0) * (weight.max() * 1e-6 + 1e-300)
        weight /= weight.sum()
        idx = rng.choice(n, size=k_rest, replace=False, p=weight)
        flat = mask.ravel()
        flat[idx] = 1
        mask = flat.reshape(h, w)
    return mask


# Solver parameters of each workload. tau = None means the method default
# (0.05 for FOEED, 0.25 for EED; Sec. 3.1).
WORKLOADS = {
    1: dict(name="ramps-disks-64x64-fp64", h=64, w=64, dtype="f64", density=0.05,
            sigma=1.0, lam=0.05, cycle_len=20, max_cycles=40, tol=0.0),
    2: dict(name="polygons-512x512-fp32", h=512, w=512, dtype="f32", density=0.04,
            sigma=1.0, lam=0.03, cycle_len=30, max_cycles=20000, tol=1e-6),
    3: dict(name="phantom-2048x2048-fp32", h=2048, w=2048, dtype="f32", density=0.03,
            sigma=1.5, lam=0.02, cycle_len=40, max_cycles=100, tol=0.0),
    5: dict(name="polygons-1024x1024-fp32-adjoint", h=1024, w=1024, dtype="f32",
            density=0.04, sigma=1.0, lam=0.03, cycle_len=20, max_cycles=30, tol=0.0),
}


def workload(index: int, h: int | None = None, w: int | None = None, instance: int = 0):
    """Image, mask and parameters of workload `index` (1, 2, 3 or 5).

    h, w override the size (same recipe, smaller grid) for quick tests.
    Returns (image float64 [h,w], mask uint8 [h,w], params dict)."""
    p = dict(WORKLOADS[index])
    hh = p["h"] if h is None else int(h)
    ww = p["w"] if w is None else int(w)
    p["h"], p["w"] = hh, ww
    rng = rng_for(index, instance)
    if index == 1:
        img = ramps_disks(hh, ww, rng)
        mask = uniform_mask(hh, ww, p["density"], rng)
    elif index in (2, 5):
        img = piecewise_smooth(hh, ww, rng)
        mask = uniform_mask(hh, ww, p["density"], rng)
    elif index == 3:
        img = ellipse_phantom(hh, ww, rng)
        mask = laplacian_weighted_mask(img, p["density"], rng)
    else:
        raise ValueError(f"no single-image workload {index}")
    return img, mask, p


def batched_workload(n_instances: int = 256, seed_base: int = 4000, sides=(128, 256, 384, 512, 768, 1024)):
    """W4: list of (image, mask, lambda) with uneven sizes; half square, half 2:1 (w = 2h)."""
    out = []
    for i in range(n_instances):
        rng = np.random.Generator(np.random.PCG64(seed_base + i))
        s = int(rng.choice(sides))
        if i % 2 == 0:
            h, w = s, s
        else:
            h, w = max(s // 2, 1), s
        density = rng.uniform(0.02, 0.10)
        lam = rng.uniform(0.01, 0.1)
        img = piecewise_smooth(h, w, rng)
        mask = uniform_mask(h, w, density, rng)
        out.append((img, mask, lam))
    return out
