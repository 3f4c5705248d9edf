"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench.

This module only draws and renders pixels.  It holds none of the detector's
arithmetic (no FAST test, no Sobel, no resize), so the oracle and the CUDA path
can both consume its frames without sharing any of the method's code.

The paper measures on photos and videos that are not distributed with it
(Sec. 6, Fig. 5 and Fig. 14).  Scenes here stand in for them:

* ``scene``: flat (128) or 1/f-noise background, 200 filled rectangles (half of
  them rotated), 30 checkerboard patches, Gaussian blur sigma=1 (radius 3),
  additive Gaussian noise sigma=3, round-half-even and clamp to uint8.
* ``fig6_pattern_image``: the five FAST ring test cases of Fig. 6, each tiled
  625 times (25 x 25, 40 px pitch) into a 1024 x 1024 image (Sec. 6.1).

Everything is rendered in float64 from a ``numpy.random.Generator`` seeded by
the caller, so a (size, seed) pair always gives the same frame on one numpy.
"""

from __future__ import annotations

import numpy as np

__all__ = ["scene", "pink_background", "fig6_ring_states", "fig6_patch",
           "fig6_pattern_image", "RING_OFFSETS"]

# The 16 pixels of the radius-3 Bresenham circle of Fig. 2(a), clockwise from
# the top (dx, dy), y pointing down.  Only used here to place test-pattern
# pixels; the oracle and the kernels each hold their own copy.
RING_OFFSETS = ((0, -3), (1, -3), (2, -2), (3, -1), (3, 0), (3, 1), (2, 2), (1, 3),
                (0, 3), (-1, 3), (-2, 2), (-3, 1), (-3, 0), (-3, -1), (-2, -2), (-1, -3))


def _gauss_kernel(sigma: float, radius: int) -> np.ndarray:
    t = np.arange(-radius, radius + 1, dtype=np.float64)
    k = np.exp(-0.5 * (t / sigma) ** 2)
    return k / k.sum()


def _blur(img: np.ndarray, sigma: float, radius: int = 3) -> np.ndarray:
    """Separable Gaussian blur with edge replication (float64)."""
    k = _gauss_kernel(sigma, radius)
    p = np.pad(img, radius, mode="edge")
    h, w = img.shape
    tmp = np.zeros((h + 2 * radius, w), dtype=np.float64)
    for i, c in enumerate(k):
        tmp += c * p[:, i:i + w]
    out = np.zeros((h, w), dtype=np.float64)
    for i, c in enumerate(k):
        out += c * tmp[i:i + h, :]
    return out


def _value_noise(h: int, w: int, cells: int, rng: np.random.Generator) -> np.ndarray:
    """Bilinearly interpolated lattice noise with about ``cells`` lattice cells across."""
    gh = max(2, int(round(cells * h / max(w, 1))) + 2)
    gw = cells + 2
    grid = rng.uniform(-1.0, 1.0, size=(gh, gw))
    ys = np.linspace(0.0, gh - 1.001, h)
    xs = np.linspace(0.0, gw - 1.001, w)
    y0 = np.floor(ys).astype(np.int64)
    x0 = np.floor(xs).astype(np.int64)
    fy = (ys - y0)[:, None]
    fx = (xs - x0)[None, :]
    g00 = grid[y0][:, x0]
    g01 = grid[y0][:, x0 + 1]
    g10 = grid[y0 + 1][:, x0]
    g11 = grid[y0 + 1][:, x0 + 1]
    return (1 - fy) * ((1 - fx) * g00 + fx * g01) + fy * ((1 - fx) * g10 + fx * g11)


def pink_background(h: int, w: int, rng: np.random.Generator, octaves: int = 6,
                    amplitude: float = 40.0) -> np.ndarray:
    """128 plus a 1/f texture: octave o has 4*2^o cells across and weight 2^-o."""
    acc = np.zeros((h, w), dtype=np.float64)
    for o in range(octaves):
        acc += (0.5 ** o) * _value_noise(h, w, 4 * (2 ** o), rng)
    peak = np.abs(acc).max()
    if peak > 0:
        acc *= amplitude / peak
    return 128.0 + acc


def scene(w: int, h: int, seed: int, *, background: str = "flat", n_rect: int = 200,
          n_checker: int = 30, blur_sigma: float = 1.0, noise_sigma: float = 3.0) -> np.ndarray:
    """One seeded synthetic grayscale frame, shape (h, w), dtype uint8."""
    rng = np.random.default_rng(seed)
    if background == "flat":
        img = np.full((h, w), 128.0, dtype=np.float64)
    elif background == "pink":
        img = pink_background(h, w, rng)
    else:
        raise ValueError(f"unknown background {background!r}")

    # Filled rectangles, painted in draw order; every other one rotated.
    for i in range(n_rect):
        cx, cy = rng.uniform(0, w), rng.uniform(0, h)
        sx, sy = rng.uniform(0.015, 0.2, size=2) * w
        ang = rng.uniform(0.0, np.pi) if (i % 2 == 1) else 0.0
        val = rng.uniform(0.0, 255.0)
        ca, sa = np.cos(ang), np.sin(ang)
        ex = 0.5 * (abs(sx * ca) + abs(sy * sa))
        ey = 0.5 * (abs(sx * sa) + abs(sy * ca))
        x0, x1 = max(0, int(np.floor(cx - ex))), min(w, int(np.ceil(cx + ex)) + 1)
        y0, y1 = max(0, int(np.floor(cy - ey))), min(h, int(np.ceil(cy + ey)) + 1)
        if x0 >= x1 or y0 >= y1:
            continue
        yy, xx = np.mgrid[y0:y1, x0:x1]
        dx = xx + 0.5 - cx
        dy = yy + 0.5 - cy
        u = dx * ca + dy * sa
        v = -dx * sa + dy * ca
        m = (np.abs(u) <= 0.5 * sx) & (np.abs(v) <= 0.5 * sy)
        img[y0:y1, x0:x1][m] = val

    # Axis-aligned checkerboard patches.
    for _ in range(n_checker):
        side = int(round(rng.uniform(0.04, 0.15) * w))
        sq = int(rng.integers(4, 13))
        a, b = rng.uniform(0.0, 255.0, size=2)
        px = int(rng.integers(0, max(1, w - side)))
        py = int(rng.integers(0, max(1, h - side)))
        x1, y1 = min(w, px + side), min(h, py + side)
        if x1 <= px or y1 <= py:
            continue
        yy, xx = np.mgrid[0:y1 - py, 0:x1 - px]
        board = ((yy // sq) + (xx // sq)) % 2 == 0
        img[py:y1, px:x1] = np.where(board, a, b)

    if blur_sigma > 0:
        img = _blur(img, blur_sigma)
    if noise_sigma > 0:
        img = img + rng.normal(0.0, noise_sigma, size=img.shape)
    return np.clip(np.rint(img), 0, 255).astype(np.uint8)


# Fig. 6: which ring positions (1-based, as in the figure) are bright in each case.
def fig6_ring_states(case: str) -> list[int]:
    """Bright ring positions (1..16) for the five test cases of Fig. 6.

    (a) nine contiguous bright points from the first pixel;
    (b) more than nine contiguous bright points, running from pixel 6 round to pixel 1;
    (c) nine contiguous bright points that wrap past pixel 16;
    (d) many contiguous bright points, but fewer than nine;
    (e) no contiguous bright points.
    """
    if case == "a":
        return list(range(1, 10))
    if case == "b":
        return list(range(6, 17)) + [1]
    if case == "c":
        return [12, 13, 14, 15, 16, 1, 2, 3, 4]
    if case == "d":
        return list(range(1, 9))
    if case == "e":
        return list(range(1, 17, 2))
    raise ValueError(case)


def fig6_patch(case: str, center: int = 100, delta: int = 40) -> np.ndarray:
    """7x7 patch: center value ``center``, the Fig. 6 bright ring pixels at ``center+delta``."""
    p = np.full((7, 7), center, dtype=np.uint8)
    for pos in fig6_ring_states(case):
        dx, dy = RING_OFFSETS[pos - 1]
        p[3 + dy, 3 + dx] = center + delta
    return p


def fig6_pattern_image(case: str, size: int = 1024, reps: int = 25, pitch: int = 40,
                       center: int = 100, delta: int = 40) -> tuple[np.ndarray, list[tuple[int, int]]]:
    """The Fig. 6 pattern tiled reps x reps times; returns (image, list of pattern centres (x, y))."""
    img = np.full((size, size), center, dtype=np.uint8)
    patch = fig6_patch(case, center, delta)
    off = (size - reps * pitch) // 2 + pitch // 2
    centres = []
    for j in range(reps):
        for i in range(reps):
            cx, cy = off + i * pitch, off + j * pitch
            img[cy - 3:cy + 4, cx - 3:cx + 4] = patch
            centres.append((cx, cy))
    return img, centres
