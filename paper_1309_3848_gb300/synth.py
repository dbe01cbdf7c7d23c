"""Seeded synthetic inputs: Voronoi colour images and the workload lists.

The paper evaluates on the Berkeley Segmentation Dataset (Sec. 6); these
synthetic images stand in for it.  This module draws random numbers and
paints pictures; it holds none of the superpixel method's arithmetic (no
binning, no grid geometry, no energy), so both the GPU path and the oracle
can take their inputs from it.

Image recipe: M seed points uniform over the image; every pixel takes the
colour of the nearest seed (squared Euclidean distance between the pixel's
integer coordinates and the seed's real coordinates); every cell has a
uniform random RGB colour.  Optional per-image linear gradient, optional
per-cell sinusoidal texture (same on all channels), then N(0, sigma^2)
noise, then clip(rint(v), 0, 255) to uint8.  Seeds are real-valued, so exact
distance ties have probability zero.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np

IMAGE_SIZES_BATCH = [(320, 240), (481, 321), (640, 480), (1280, 720), (1920, 1080)]
IMAGE_SIZES_SERVE = IMAGE_SIZES_BATCH + [(3840, 2160)]


@dataclasses.dataclass(frozen=True)
class ImageSpec:
    width: int
    height: int
    seed: int
    cells: int
    sigma: float
    texture: bool = False
    gradient: bool = False


@dataclasses.dataclass(frozen=True)
class JobSpec:
    """One image plus the method's parameters for it.  `levels` is the
    requested number of block levels; callers clamp it to what the grid
    geometry allows (each side with its own geometry code)."""
    image: ImageSpec
    num_superpixels: int
    bins_per_channel: int
    levels: int
    iters_per_level: int
    patch: int = 3
    gamma: Tuple[int, int] = (1, 1)
    clamp_levels: bool = False
    color_space: int = 0  # 0 = RGB bytes, 1 = CIE L*a*b* codes
    means_iters: int = 0  # means-based pixel iterations after the histogram ones
    compactness: int = 0  # SLIC's m in those iterations
    edge_threshold: int = 0  # edge snapping, 0 = off
    compact_prior: int = 0  # the compactness prior in the histogram pixel phases, 0 = off

    @property
    def pixels(self) -> int:
        return self.image.width * self.image.height


def _nearest_seed(W: int, H: int, pts: np.ndarray) -> np.ndarray:
    """Index of the nearest seed for every pixel, shape (H, W)."""
    M = len(pts)
    ys, xs = np.mgrid[0:H, 0:W]
    if M <= 64 or W * H <= 4096:
        best = np.full((H, W), np.inf)
        idx = np.zeros((H, W), np.int64)
        for m in range(M):  # ascending index: strict < keeps the lower index on ties
            d = (xs - pts[m, 0]) ** 2 + (ys - pts[m, 1]) ** 2
            closer = d < best
            best = np.where(closer, d, best)
            idx = np.where(closer, m, idx)
        return idx
    from scipy.spatial import cKDTree  # the box image ships scipy

    tree = cKDTree(pts)
    q = np.stack([xs.ravel(), ys.ravel()], axis=1).astype(np.float64)
    _, idx = tree.query(q, k=1, workers=-1)
    return idx.reshape(H, W)


def make_image(spec: ImageSpec) -> np.ndarray:
    """HxWx3 uint8 image for a spec (deterministic in the spec)."""
    W, H = spec.width, spec.height
    rng = np.random.default_rng(spec.seed)
    M = max(1, spec.cells)
    pts = np.stack([rng.uniform(0, W, M), rng.uniform(0, H, M)], axis=1)
    colours = rng.integers(0, 256, size=(M, 3)).astype(np.float64)
    cell = _nearest_seed(W, H, pts)
    img = colours[cell]
    ys, xs = np.mgrid[0:H, 0:W].astype(np.float64)
    if spec.gradient:
        g = rng.uniform(-40.0, 40.0, 3)
        h = rng.uniform(-40.0, 40.0, 3)
        img += (xs / W)[..., None] * g + (ys / H)[..., None] * h
    if spec.texture:
        period = rng.uniform(8.0, 32.0, M)
        theta = rng.uniform(0.0, 2.0 * math.pi, M)
        phi = rng.uniform(0.0, 2.0 * math.pi, M)
        fx = np.cos(theta) / period
        fy = np.sin(theta) / period
        tex = 20.0 * np.sin(2.0 * math.pi * (fx[cell] * xs + fy[cell] * ys) + phi[cell])
        img += tex[..., None]
    if spec.sigma > 0:
        img += rng.normal(0.0, spec.sigma, size=img.shape)
    return np.clip(np.rint(img), 0, 255).astype(np.uint8)


def voronoi_truth(spec: ImageSpec) -> np.ndarray:
    """The Voronoi cell index of every pixel (ground truth for quality checks)."""
    rng = np.random.default_rng(spec.seed)
    M = max(1, spec.cells)
    pts = np.stack([rng.uniform(0, spec.width, M), rng.uniform(0, spec.height, M)], axis=1)
    return _nearest_seed(spec.width, spec.height, pts).astype(np.int32)


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------

def plain_481() -> List[JobSpec]:
    """One 481x321 image: 12 cells, gradient, noise sigma 8; 5 bins/channel,
    ~200 superpixels, 4 block levels, 2 iterations per level, 3x3 patch."""
    img = ImageSpec(481, 321, seed=0, cells=12, sigma=8.0, gradient=True)
    return [JobSpec(img, 200, 5, 4, 2)]


def plain_1080() -> List[JobSpec]:
    """One 1920x1080 image: 200 textured cells, noise sigma 6; 5 bins/channel,
    1000 superpixels, 4 block levels, 4 iterations per level."""
    img = ImageSpec(1920, 1080, seed=1, cells=200, sigma=6.0, texture=True)
    return [JobSpec(img, 1000, 5, 4, 4)]


def batch_64(count: int = 64) -> List[JobSpec]:
    """64 images of mixed sizes, cells = pixels/2000, noise sigma 8,
    400..1500 superpixels, 5 bins/channel, up to 4 block levels, 2 iterations."""
    rng = np.random.default_rng(2)
    jobs = []
    for i in range(count):
        W, H = IMAGE_SIZES_BATCH[int(rng.integers(0, len(IMAGE_SIZES_BATCH)))]
        K = int(rng.integers(400, 1501))
        img = ImageSpec(W, H, seed=2_000_000 + i, cells=(W * H) // 2000, sigma=8.0)
        jobs.append(JobSpec(img, K, 5, 4, 2, clamp_levels=True))
    return jobs


def batch_4k(count: int = 16) -> List[JobSpec]:
    """16 images 3840x2160, 1000 cells, noise sigma 5; 5000 superpixels,
    8 bins/channel (512 bins), 5 block levels, 4 iterations per level."""
    return [JobSpec(ImageSpec(3840, 2160, seed=3_000_000 + i, cells=1000, sigma=5.0), 5000, 8, 5, 4)
            for i in range(count)]


WORKLOADS = {
    "plain_481x321": plain_481,
    "plain_1920x1080": plain_1080,
    "batch64_mixed": batch_64,
    "batch16_3840x2160": batch_4k,
}


def serve_requests(rate: float, duration: float, seed: int, max_requests: int = 4000,
                   sizes: Optional[Sequence[Tuple[int, int]]] = None) -> List[Tuple[float, JobSpec]]:
    """Poisson arrivals at `rate` req/s for `duration` s (at most
    `max_requests`): (arrival time in s, job).  Sizes uniform over `sizes`,
    200..5000 superpixels, 5 bins/channel, up to 4 levels, 2 iterations,
    cells = pixels/2000, noise sigma 8, one image seed per request."""
    sizes = list(sizes or IMAGE_SIZES_SERVE)
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    while len(out) < max_requests:
        t += float(rng.exponential(1.0 / rate))
        if t > duration:
            break
        W, H = sizes[int(rng.integers(0, len(sizes)))]
        K = int(rng.integers(200, 5001))
        img = ImageSpec(W, H, seed=int(rng.integers(0, 2**31)), cells=max(1, (W * H) // 2000), sigma=8.0)
        out.append((t, JobSpec(img, K, 5, 4, 2, clamp_levels=True)))
    return out


def random_small_jobs(seed: int, count: int, max_side: int = 64) -> List[JobSpec]:
    """Small random jobs for fuzzing: sizes, superpixel counts, bins, levels,
    iterations, patch and gamma all drawn from `seed`."""
    rng = np.random.default_rng(seed)
    jobs = []
    for i in range(count):
        W = int(rng.integers(4, max_side + 1))
        H = int(rng.integers(4, max_side + 1))
        K = int(rng.integers(1, max(2, (W * H) // 12)))
        B = int(rng.integers(1, 9))
        L = int(rng.integers(0, 5))
        iters = int(rng.integers(1, 4))
        patch = int(rng.choice([0, 3]))
        gamma = (int(rng.integers(0, 4)), int(rng.integers(1, 4)))
        img = ImageSpec(W, H, seed=int(rng.integers(0, 2**31)), cells=int(rng.integers(1, 12)),
                        sigma=float(rng.choice([0.0, 4.0, 12.0])), gradient=bool(rng.integers(0, 2)))
        jobs.append(JobSpec(img, K, B, L, iters, patch, gamma, clamp_levels=True))
    return jobs
