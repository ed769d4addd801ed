"""Seeded synthetic inputs shaped like the colour-image workloads of the
bilateral-filter experiments (Section 4: 256x256, 512x512 and 876x584 RGB
images filtered with sigma_s in [1, 10] and sigma_r in [30, 90]).

The natural images used there are not available, so every image here is drawn
from a seeded generator with the structure that matters to an edge-preserving
filter: flat regions, smooth shading, hard edges and i.i.d. noise.

This module holds no part of the filter's arithmetic: it only draws images,
covariance matrices and request mixes.  Both the CPU oracle tests and the CUDA
path use it, so it must stay free of anything either side computes.

Images are float32, planar ``(d, H, W)``, clipped to [0, 255].
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "voronoi_image",
    "value_noise_polygon_image",
    "haar_orthogonal",
    "spd_from_eigs",
    "spd_eig_range",
    "spd_cond",
    "Workload",
    "WORKLOADS",
    "batch_items",
    "serving_trace",
    "crop_origins",
]


def _rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(np.uint64(seed & 0xFFFFFFFFFFFFFFFF))


def voronoi_image(H: int, W: int, d: int = 3, n_cells: int = 16,
                  noise_sigma: float = 10.0, seed: int = 0) -> np.ndarray:
    """Piecewise-constant image: ``n_cells`` Voronoi cells with uniform random
    sites and uniform random colours in [0, 255]^d, plus i.i.d. N(0, sigma^2)
    noise, clipped to [0, 255]."""
    rng = _rng(seed)
    sites_x = rng.uniform(0, W, n_cells)
    sites_y = rng.uniform(0, H, n_cells)
    colours = rng.uniform(0, 255, (n_cells, d))
    out = np.empty((d, H, W), np.float32)
    xs = np.arange(W, dtype=np.float64)
    rows_per = max(1, (1 << 22) // max(1, W * n_cells))
    for y0 in range(0, H, rows_per):
        ys = np.arange(y0, min(H, y0 + rows_per), dtype=np.float64)
        dy = (ys[:, None, None] - sites_y[None, None, :]) ** 2
        dx = (xs[None, :, None] - sites_x[None, None, :]) ** 2
        lab = np.argmin(dy + dx, axis=2)                     # (rows, W)
        out[:, y0:y0 + len(ys), :] = colours[lab].transpose(2, 0, 1)
    if noise_sigma > 0:
        out += rng.normal(0.0, noise_sigma, out.shape).astype(np.float32)
    np.clip(out, 0.0, 255.0, out=out)
    return out


def _value_noise(H: int, W: int, cells: int, rng: np.random.Generator) -> np.ndarray:
    """Bilinear value noise on a (cells+1)^2 lattice of uniform [0,1] values,
    with a smoothstep fade between lattice points."""
    lat = rng.uniform(0, 1, (cells + 1, cells + 1))
    gy = np.linspace(0, cells, H, endpoint=False)
    gx = np.linspace(0, cells, W, endpoint=False)
    iy = np.floor(gy).astype(np.int64)
    ix = np.floor(gx).astype(np.int64)
    fy = gy - iy
    fx = gx - ix
    fy = fy * fy * (3 - 2 * fy)
    fx = fx * fx * (3 - 2 * fx)
    a = lat[iy][:, ix]
    b = lat[iy][:, ix + 1]
    c = lat[iy + 1][:, ix]
    e = lat[iy + 1][:, ix + 1]
    top = a + (b - a) * fx[None, :]
    bot = c + (e - c) * fx[None, :]
    return top + (bot - top) * fy[:, None]


def _fill_polygon(mask_shape, verts: np.ndarray) -> tuple[slice, slice, np.ndarray]:
    """Even-odd rule point-in-polygon test on pixel centres, restricted to the
    polygon's bounding box.  Returns (row slice, col slice, boolean mask)."""
    H, W = mask_shape
    x0 = max(0, int(math.floor(verts[:, 0].min())))
    x1 = min(W, int(math.ceil(verts[:, 0].max())) + 1)
    y0 = max(0, int(math.floor(verts[:, 1].min())))
    y1 = min(H, int(math.ceil(verts[:, 1].max())) + 1)
    if x0 >= x1 or y0 >= y1:
        return slice(0, 0), slice(0, 0), np.zeros((0, 0), bool)
    px = np.arange(x0, x1, dtype=np.float64)[None, :] + 0.5
    py = np.arange(y0, y1, dtype=np.float64)[:, None] + 0.5
    inside = np.zeros((y1 - y0, x1 - x0), bool)
    n = len(verts)
    for k in range(n):
        xa, ya = verts[k]
        xb, yb = verts[(k + 1) % n]
        if ya == yb:
            continue
        crosses = (ya > py) != (yb > py)
        xint = xa + (py - ya) * (xb - xa) / (yb - ya)
        inside ^= crosses & (px < xint)
    return slice(y0, y1), slice(x0, x1), inside


def value_noise_polygon_image(H: int, W: int, d: int = 3, octaves=(8, 16, 32, 64),
                              n_polygons: int = 64, noise_sigma: float = 15.0,
                              seed: int = 0) -> np.ndarray:
    """Smooth value noise (``octaves`` lattice sizes, amplitude halving per
    octave, rescaled to [0, 255]) with ``n_polygons`` filled random polygons
    (3-8 vertices, uniform colour) on top, plus N(0, sigma^2) noise, clipped."""
    rng = _rng(seed)
    out = np.empty((d, H, W), np.float32)
    for c in range(d):
        acc = np.zeros((H, W))
        amp = 1.0
        for cells in octaves:
            acc += amp * _value_noise(H, W, cells, rng)
            amp *= 0.5
        lo, hi = acc.min(), acc.max()
        out[c] = (255.0 * (acc - lo) / max(hi - lo, 1e-12)).astype(np.float32)
    scale = min(H, W)
    for _ in range(n_polygons):
        nv = int(rng.integers(3, 9))
        cx, cy = rng.uniform(0, W), rng.uniform(0, H)
        rad = rng.uniform(0.03, 0.15) * scale
        ang = np.sort(rng.uniform(0, 2 * math.pi, nv))
        rr = rad * rng.uniform(0.5, 1.0, nv)
        verts = np.stack([cx + rr * np.cos(ang), cy + rr * np.sin(ang)], axis=1)
        colour = rng.uniform(0, 255, d).astype(np.float32)
        ys, xs, m = _fill_polygon((H, W), verts)
        if m.size:
            for c in range(d):
                blk = out[c, ys, xs]
                blk[m] = colour[c]
    if noise_sigma > 0:
        out += rng.normal(0.0, noise_sigma, out.shape).astype(np.float32)
    np.clip(out, 0.0, 255.0, out=out)
    return out


def haar_orthogonal(d: int, rng: np.random.Generator) -> np.ndarray:
    """Haar-distributed orthogonal matrix: QR of a Gaussian matrix with the
    signs of R's diagonal moved into Q (Mezzadri 2007)."""
    A = rng.normal(size=(d, d))
    Q, R = np.linalg.qr(A)
    return Q * np.sign(np.diag(R))[None, :]


def spd_from_eigs(eigs, Q) -> np.ndarray:
    C = (Q * np.asarray(eigs, np.float64)[None, :]) @ Q.T
    return 0.5 * (C + C.T)


def spd_eig_range(d: int, lo: float, hi: float, seed: int) -> np.ndarray:
    """C = Q diag(lambda) Q^T with lambda ~ U[lo, hi] and Q Haar-random."""
    rng = _rng(seed)
    Q = haar_orthogonal(d, rng)
    return spd_from_eigs(rng.uniform(lo, hi, d), Q)


def spd_cond(d: int, seed: int, lam_min_range=(20.0 ** 2, 40.0 ** 2), cond: float = 10.0) -> np.ndarray:
    """C with lambda_min ~ U[lam_min_range] and the other eigenvalues
    ~ U[lambda_min, cond * lambda_min] (condition number <= cond)."""
    rng = _rng(seed)
    Q = haar_orthogonal(d, rng)
    lmin = rng.uniform(*lam_min_range)
    eigs = np.concatenate([[lmin], rng.uniform(lmin, cond * lmin, d - 1)])
    return spd_from_eigs(eigs, Q)


@dataclass
class Workload:
    """One filtering problem: image generator, size, channel count, spatial
    scale, range covariance, raised-cosine order and number of samples."""
    name: str
    H: int
    W: int
    d: int
    sigma_s: float
    C: np.ndarray
    N: int
    K: int
    gen: str = "voronoi"          # "voronoi" | "noise_polygons"
    noise: float = 10.0
    seed: int = 0
    extra: dict = field(default_factory=dict)

    def image(self) -> np.ndarray:
        if self.gen == "voronoi":
            return voronoi_image(self.H, self.W, self.d, 16, self.noise, self.seed)
        return value_noise_polygon_image(self.H, self.W, self.d, noise_sigma=self.noise, seed=self.seed)


def _w_small() -> Workload:
    return Workload("rgb256_voronoi_s3_K32", 256, 256, 3, 3.0, np.diag([30.0 ** 2] * 3), 10, 32,
                    "voronoi", 10.0, seed=1000)


def _w_mid() -> Workload:
    return Workload("rgb1024_noisepoly_s5_K64_fullC", 1024, 1024, 3, 5.0,
                    spd_eig_range(3, 20.0 ** 2, 50.0 ** 2, seed=2000), 10, 64,
                    "noise_polygons", 15.0, seed=2000)


def _w_4k() -> Workload:
    return Workload("rgb3840x2160_voronoi_s8_K128", 2160, 3840, 3, 8.0, np.diag([40.0 ** 2] * 3), 10, 128,
                    "voronoi", 10.0, seed=3000)


def _w_d6() -> Workload:
    # six channels (the uneven batch's d = 6 images, e.g. two RGB frames stacked)
    return Workload("d6_1024_voronoi_s5_K32", 1024, 1024, 6, 5.0,
                    spd_cond(6, seed=4, lam_min_range=(30.0 ** 2, 40.0 ** 2), cond=5.0), 10, 32,
                    "voronoi", 10.0, seed=3300)


WORKLOADS = {"small": _w_small, "mid": _w_mid, "4k": _w_4k, "d6": _w_d6}


def crop_origins(H: int, W: int, size: int = 256, n: int = 4, seed: int = 3100) -> list[tuple[int, int]]:
    """Fixed crop origins for checking a large image on smaller windows:
    the four corners' neighbourhoods are covered by the first and last crops."""
    rng = _rng(seed)
    pts = [(0, 0), (H - size, W - size)]
    while len(pts) < n:
        pts.append((int(rng.integers(0, H - size + 1)), int(rng.integers(0, W - size + 1))))
    return pts


def batch_items(n: int = 64, seed: int = 4000, max_hw=(1536, 2048), min_hw=(256, 256)) -> list[Workload]:
    """Uneven batch: sizes uniform in [256, 2048] x [256, 1536], d in {3, 6},
    sigma_s ~ U[2, 10], per-image C with condition number <= 10,
    K in {32, 64, 128}, N = 10."""
    rng = _rng(seed)
    out = []
    for i in range(n):
        W = int(rng.integers(min_hw[1], max_hw[1] + 1))
        H = int(rng.integers(min_hw[0], max_hw[0] + 1))
        d = int(rng.choice([3, 6]))
        s = float(rng.uniform(2.0, 10.0))
        K = int(rng.choice([32, 64, 128]))
        C = spd_cond(d, seed=seed * 7 + i)
        out.append(Workload(f"batch{i}", H, W, d, s, C, 10, K, "voronoi", 10.0, seed=seed + i))
    return out


def serving_trace(duration_s: float = 10.0, rate: float = 2000.0, seed: int = 5000,
                  min_side: int = 512, max_side: int = 4096):
    """Poisson arrivals (exponential gaps at ``rate``/s) of RGB requests with
    area log-uniform in [min_side^2, max_side^2] (square), sigma_s ~ U[2, 10],
    C = sigma_r^2 I with sigma_r ~ U[20, 60], K = 64, N = 10.
    Returns a list of (arrival_time_s, Workload)."""
    rng = _rng(seed)
    t = 0.0
    out = []
    i = 0
    while True:
        t += float(rng.exponential(1.0 / rate))
        if t >= duration_s:
            break
        la = rng.uniform(2 * math.log(min_side), 2 * math.log(max_side))
        side = int(round(math.exp(la / 2)))
        s = float(rng.uniform(2.0, 10.0))
        sr = float(rng.uniform(20.0, 60.0))
        out.append((t, Workload(f"req{i}", side, side, 3, s, np.diag([sr * sr] * 3), 10, 64,
                                "voronoi", 10.0, seed=seed + i)))
        i += 1
    return out
