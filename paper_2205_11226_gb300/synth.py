"""Seeded synthetic frames and block-loss masks.

The paper measures on Kodak, Tecnick and HEVC ClassB/ClassC sequences; none of those
is available here, so every input is generated from a seed: 8-bit luma frames built
from piecewise-constant polygonal regions (Voronoi cells, straight edges), sinusoidal
gratings and sensor-like noise, and the paper's two loss families (dispersed isolated
blocks and consecutive/slice loss).  This module holds no part of the concealment
arithmetic; it serves the library, the benchmark and the tests alike.
"""
from __future__ import annotations

import numpy as np

MB = 16


def _gauss_blur(img: np.ndarray, sigma: float) -> np.ndarray:
    r = int(np.ceil(3 * sigma))
    t = np.arange(-r, r + 1, dtype=np.float64)
    k = np.exp(-0.5 * (t / sigma) ** 2)
    k /= k.sum()
    pad = np.pad(img, r, mode="reflect")
    tmp = np.zeros((pad.shape[0], img.shape[1]))
    for i, w in enumerate(k):
        tmp += w * pad[:, i:i + img.shape[1]]
    out = np.zeros(img.shape)
    for i, w in enumerate(k):
        out += w * tmp[i:i + img.shape[0], :]
    return out


def make_frame(width: int, height: int, seed: int, fine_texture: bool = False) -> np.ndarray:
    """One uint8 [height, width] frame.

    6 Voronoi regions with levels U[30, 225]; gratings A*sin(2*pi*(x cos t + y sin t)/P + psi)
    with t ~ U[0, pi), P ~ U[8, 64], A ~ U[20, 60], psi ~ U[0, 2*pi) added inside regions
    0, 1 and 2 (regions 3-5 stay flat); Gaussian noise sigma = 2.  With ``fine_texture``,
    uniform noise band-passed to 2-4 px (difference of Gaussian blurs, sigma 1 and 2) and
    scaled to standard deviation 6 is added everywhere.  Rounded and clipped to [0, 255].
    """
    rng = np.random.default_rng(seed)
    yy, xx = np.mgrid[0:height, 0:width].astype(np.float64)
    pts = rng.uniform([0, 0], [width, height], size=(6, 2))
    levels = rng.uniform(30, 225, size=6)
    d2 = np.stack([(xx - px) ** 2 + (yy - py) ** 2 for px, py in pts])
    region = np.argmin(d2, axis=0)
    img = levels[region]
    for g in range(3):
        th = rng.uniform(0, np.pi)
        per = rng.uniform(8, 64)
        amp = rng.uniform(20, 60)
        psi = rng.uniform(0, 2 * np.pi)
        wave = amp * np.sin(2 * np.pi * (xx * np.cos(th) + yy * np.sin(th)) / per + psi)
        img = img + np.where(region == g, wave, 0.0)
    img = img + rng.normal(0.0, 2.0, size=img.shape)
    if fine_texture:
        u = rng.uniform(-1.0, 1.0, size=img.shape)
        band = _gauss_blur(u, 1.0) - _gauss_blur(u, 2.0)
        band *= 6.0 / max(band.std(), 1e-12)
        img = img + band
    return np.clip(np.rint(img), 0, 255).astype(np.uint8)


def mb_grid(width: int, height: int) -> tuple[int, int]:
    """(rows, cols) of the 16x16 block grid; partial blocks at the edges count."""
    return (height + MB - 1) // MB, (width + MB - 1) // MB


def loss_single(width: int, height: int, row: int, col: int) -> np.ndarray:
    m = np.zeros(mb_grid(width, height), dtype=np.uint8)
    m[row, col] = 1
    return m


def loss_checkerboard(width: int, height: int) -> np.ndarray:
    """Dispersed pattern: a block is lost iff its row and column are both odd (~25 %)."""
    r, c = mb_grid(width, height)
    m = np.zeros((r, c), dtype=np.uint8)
    m[1::2, 1::2] = 1
    return m


def loss_runs(width: int, height: int, seed: int, target: float = 0.20,
              run_min: int = 4, run_max: int = 20) -> np.ndarray:
    """Slice loss: runs of U{run_min..run_max} consecutive blocks in raster order at random
    starts (runs may wrap rows, never overlap) until at least ``target`` of blocks are lost."""
    rng = np.random.default_rng(seed)
    r, c = mb_grid(width, height)
    n = r * c
    flat = np.zeros(n, dtype=np.uint8)
    need = int(np.ceil(target * n))
    tries = 0
    while flat.sum() < need and tries < 100000:
        tries += 1
        ln = int(rng.integers(run_min, run_max + 1))
        s = int(rng.integers(0, n))
        e = min(n, s + ln)
        if flat[s:e].any():
            continue
        flat[s:e] = 1
    return flat.reshape(r, c)


def loss_isolated(width: int, height: int, seed: int, count: int) -> np.ndarray:
    """``count`` lost blocks, each with all 8 neighbours received (when possible)."""
    rng = np.random.default_rng(seed)
    r, c = mb_grid(width, height)
    m = np.zeros((r, c), dtype=np.uint8)
    order = rng.permutation(r * c)
    placed = 0
    for idx in order:
        if placed >= count:
            break
        y, x = divmod(int(idx), c)
        if m[max(0, y - 1):y + 2, max(0, x - 1):x + 2].any():
            continue
        m[y, x] = 1
        placed += 1
    return m


def loss_mixed(width: int, height: int, seed: int, rate_lo: float, rate_hi: float) -> np.ndarray:
    """Loss rate ~ U[rate_lo, rate_hi]; half of the lost blocks isolated, half in runs."""
    rng = np.random.default_rng(seed)
    r, c = mb_grid(width, height)
    rate = float(rng.uniform(rate_lo, rate_hi))
    n_target = max(1, int(round(rate * r * c)))
    m = loss_isolated(width, height, seed + 1, n_target // 2)
    flat = m.reshape(-1)
    tries = 0
    while flat.sum() < n_target and tries < 100000:
        tries += 1
        ln = int(rng.integers(4, 21))
        s = int(rng.integers(0, r * c))
        e = min(r * c, s + ln)
        if flat[max(0, s - 1):min(r * c, e + 1)].any():
            continue
        flat[s:e] = 1
    return flat.reshape(r, c)


def loss_shapes(width: int, height: int, seed: int, target: float = 0.10) -> np.ndarray:
    """Arbitrarily shaped loss, per pixel (uint8 [height, width], 1 = lost): filled ellipses
    (semi-axes U[2, 20] px, random orientation) and straight strokes (width U{1..6} px,
    length U[16, 160] px, random direction), half of the shapes each, at uniform random
    positions, until at least ``target`` of the pixels are lost.  Shapes may overlap and
    cross block borders; odd widths and offsets leave 2x2 patches partly lost."""
    rng = np.random.default_rng(seed)
    m = np.zeros((height, width), dtype=bool)
    need = int(np.ceil(target * width * height))
    while int(m.sum()) < need:
        cy, cx = rng.uniform(0, height), rng.uniform(0, width)
        th = rng.uniform(0, np.pi)
        ct, st = np.cos(th), np.sin(th)
        if rng.uniform() < 0.5:
            a, b = rng.uniform(2, 20), rng.uniform(2, 20)
            r = int(np.ceil(max(a, b))) + 1
            half_u, half_v = a, b
            ellipse = True
        else:
            ln, wd = rng.uniform(16, 160), int(rng.integers(1, 7))
            r = int(np.ceil(ln / 2 + wd)) + 1
            half_u, half_v = ln / 2, wd / 2
            ellipse = False
        y0, y1 = max(0, int(cy) - r), min(height, int(cy) + r + 1)
        x0, x1 = max(0, int(cx) - r), min(width, int(cx) + r + 1)
        if y0 >= y1 or x0 >= x1:
            continue
        yy, xx = np.mgrid[y0:y1, x0:x1].astype(np.float64)
        u = (xx + 0.5 - cx) * ct + (yy + 0.5 - cy) * st
        v = -(xx + 0.5 - cx) * st + (yy + 0.5 - cy) * ct
        if ellipse:
            inside = (u / half_u) ** 2 + (v / half_v) ** 2 <= 1.0
        else:
            inside = (np.abs(u) <= half_u) & (np.abs(v) <= half_v)
        m[y0:y1, x0:x1] |= inside
    return m.astype(np.uint8)


def blocks_of(px_lost: np.ndarray) -> np.ndarray:
    """Block flags of a per-pixel loss mask: 1 where the 16x16 block holds a lost pixel."""
    px = np.asarray(px_lost) != 0
    h, w = px.shape
    r, c = mb_grid(w, h)
    pad = np.zeros((r * MB, c * MB), dtype=bool)
    pad[:h, :w] = px
    return pad.reshape(r, MB, c, MB).any(axis=(1, 3)).astype(np.uint8)


# --------------------------------------------------------------------------------------
# the five workloads: one 256x256 frame with one lost block; the 512x512 checkerboard; a
# 1920x1080 frame with runs of lost blocks; the 64-frame batch of mixed sizes; the stream

def workload_single(seed: int = 0):
    """256x256 frame, one lost block at pixel (112, 112) = block (7, 7)."""
    f = make_frame(256, 256, seed)
    return f, loss_single(256, 256, 7, 7)


def workload_checkerboard(seed: int = 0, width: int = 512, height: int = 512):
    """512x512 frame, checkerboard over alternate block rows (256 of 1024 blocks)."""
    f = make_frame(width, height, seed)
    return f, loss_checkerboard(width, height)


def workload_slice_1080p(seed: int = 0):
    """1920x1080 with fine texture, runs of 4-20 blocks to >= 20 % loss."""
    f = make_frame(1920, 1080, seed, fine_texture=True)
    return f, loss_runs(1920, 1080, seed + 7, 0.20)


def workload_shapes_1080p(seed: int = 0, target: float = 0.10):
    """1920x1080 with fine texture; arbitrarily shaped loss (ellipses and strokes) to
    >= ``target`` of the pixels.  Returns (frame, per-pixel mask)."""
    f = make_frame(1920, 1080, seed, fine_texture=True)
    return f, loss_shapes(1920, 1080, seed + 11, target)


BATCH_SIZES = [(352, 288)] * 24 + [(1280, 720)] * 24 + [(1920, 1080)] * 16


def workload_batch(seed: int = 0, sizes=None):
    """64 frames of mixed sizes, per-frame loss U[5, 30] %, isolated + runs."""
    sizes = BATCH_SIZES if sizes is None else sizes
    frames, masks = [], []
    for i, (w, h) in enumerate(sizes):
        frames.append(make_frame(w, h, seed * 1000 + i))
        masks.append(loss_mixed(w, h, seed * 1000 + 500 + i, 0.05, 0.30))
    return frames, masks


STREAM_SIZES = [(352, 288), (1280, 720), (1920, 1080)]


def stream_requests(seed: int = 0, n: int = 20000, rate_hz: float = 600.0):
    """Serving stream: Poisson arrivals at ``rate_hz``; each request's size drawn 1/3 each
    from the three resolutions; loss U[2, 30] %.  Returns a list of (t_arrival_s, w, h,
    frame_seed, mask_seed); frames are generated lazily by the caller."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate_hz, size=n))
    sz = rng.integers(0, 3, size=n)
    out = []
    for i in range(n):
        w, h = STREAM_SIZES[int(sz[i])]
        out.append((float(t[i]), w, h, seed * 100000 + i, seed * 100000 + 50000 + i))
    return out


def psnr(a: np.ndarray, b: np.ndarray, mask: np.ndarray | None = None) -> float:
    """PSNR in dB between two 8-bit images (optionally over a boolean pixel mask)."""
    d = a.astype(np.float64) - b.astype(np.float64)
    if mask is not None:
        d = d[mask]
    mse = float(np.mean(d * d)) if d.size else 0.0
    return float("inf") if mse == 0 else 10.0 * np.log10(255.0 ** 2 / mse)


def lost_pixel_mask(mb_lost: np.ndarray, width: int, height: int) -> np.ndarray:
    m = np.kron(mb_lost.astype(bool), np.ones((MB, MB), dtype=bool))
    return m[:height, :width]
