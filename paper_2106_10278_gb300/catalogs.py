"""Seeded synthetic particle catalogues and the named workloads.

This module only draws inputs (positions, weights, bin edges); it holds none of
the estimator's arithmetic, so both the CUDA path and the FP64 oracle may use
it.  Every position lies in [0, L) on every axis.  By default positions and
weights are rounded to FP32, so that an FP32 device copy and the FP64 host copy
describe the same points; ``fp32=False`` keeps the full FP64 mantissa, the
inputs that FP64 plans are tested on (a stage that silently narrowed them to
float would then show).

Workloads (all periodic boxes, linear radial bins):

=========  =====================================================================
name       recipe
=========  =====================================================================
d3n3_fp64  D=3, N=3, lmax=5, FP64. n=2000 uniform in a cube of side 250
           (full FP64 mantissa), w=1, 10 bins over [0, 100].
d2         D=2, N=3 and N=4, lmax=10. n=200k in the unit square: 100k uniform
           plus 100k in 400 Gaussian blobs (centres uniform, members
           multinomial, sigma=0.005, wrapped), w ~ N(1, 0.1), 16 bins over
           [0.002, 0.05].
d3n4       D=3, N=4, lmax=5, data minus randoms: ~1M Poisson draws from a
           lognormal field on a 256^3 grid (P(k) ~ k^-1.5, Gaussian variance 1,
           rho = exp(G - 1/2)) in a box of side 1000, w=+1, plus 1M uniform
           randoms with w=-1; 10 bins over [20, 160].
d4n3       D=4, N=3, lmax=4. n=100k in the unit 4-cube: 50k uniform plus 50k
           in 200 Gaussian blobs (sigma=0.01, wrapped), w ~ N(1, 0.1), 8 bins
           over [0.01, 0.12].
=========  =====================================================================
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _fp32_in_box(x: np.ndarray, L: np.ndarray, fp32: bool = True) -> np.ndarray:
    """Wrap into [0, L), round to FP32 (unless fp32 is False), and re-wrap values that rounded up to L."""
    x = np.mod(x, L)
    L64 = np.asarray(L, dtype=np.float64)
    if fp32:
        x = x.astype(np.float32).astype(np.float64)
    return np.where(x >= L64, 0.0, x)


def uniform(n: int, D: int, L, seed: int, fp32: bool = True) -> np.ndarray:
    """n points uniform in the periodic box [0, L)^D (FP32-representable unless fp32 is False)."""
    L = np.broadcast_to(np.asarray(L, dtype=np.float64), (D,))
    return _fp32_in_box(_rng(seed).random((n, D)) * L, L, fp32)


def sphere_uniform(n: int, seed: int) -> np.ndarray:
    """n directions uniform on the unit 2-sphere (normalised Gaussian 3-vectors), rounded to
    FP32 so that an FP32 device copy holds the same vectors; their length is 1 up to FP32
    rounding, and consumers normalise them."""
    v = _rng(seed).normal(size=(n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return v.astype(np.float32).astype(np.float64)


def gaussian_blobs(n: int, D: int, L, n_centres: int, sigma: float, seed: int, fp32: bool = True) -> np.ndarray:
    """n points in Gaussian blobs: centres uniform, membership multinomial, wrapped (FP32-representable
    unless fp32 is False)."""
    L = np.broadcast_to(np.asarray(L, dtype=np.float64), (D,))
    g = _rng(seed)
    centres = g.random((n_centres, D)) * L
    counts = g.multinomial(n, np.full(n_centres, 1.0 / n_centres))
    members = np.repeat(np.arange(n_centres), counts)
    x = centres[members] + g.normal(0.0, sigma, (n, D))
    return _fp32_in_box(x, L, fp32)


def _rfftn(x):
    try:
        import scipy.fft as sf
        return sf.rfftn(x, workers=-1)
    except ImportError:
        return np.fft.rfftn(x)


def _irfftn(x, shape):
    try:
        import scipy.fft as sf
        return sf.irfftn(x, s=shape, workers=-1)
    except ImportError:
        return np.fft.irfftn(x, s=shape, axes=(0, 1, 2))


def lognormal_poisson(n_mean: float, L: float, seed: int, grid: int = 256, slope: float = -1.5) -> np.ndarray:
    """Poisson draws from a lognormal density on a grid^3 mesh of a periodic cube.

    G is a Gaussian field with power spectrum P(k) ~ k^slope (k != 0), scaled to
    unit variance; the density is rho = exp(G - 1/2); each cell holds a Poisson
    number of points with mean n_mean * rho / sum(rho), placed uniformly in it.
    """
    g = _rng(seed)
    white = g.standard_normal((grid, grid, grid))
    fk = _rfftn(white)
    kx = np.fft.fftfreq(grid)[:, None, None]
    ky = np.fft.fftfreq(grid)[None, :, None]
    kz = np.fft.rfftfreq(grid)[None, None, :]
    k2 = kx * kx + ky * ky + kz * kz
    k2[0, 0, 0] = 1.0
    amp = k2 ** (slope / 4.0)  # sqrt(P(k)) with P ~ k^slope
    amp[0, 0, 0] = 0.0
    G = _irfftn(fk * amp, (grid, grid, grid))
    G /= G.std()
    rho = np.exp(G - 0.5)
    lam = n_mean * rho / rho.sum()
    counts = g.poisson(lam).ravel()
    cells = np.repeat(np.arange(grid ** 3), counts)
    ix, iy, iz = np.unravel_index(cells, (grid, grid, grid))
    cell = L / grid
    base = np.stack([ix, iy, iz], axis=1).astype(np.float64) * cell
    x = base + g.random((cells.size, 3)) * cell
    return _fp32_in_box(x, np.full(3, float(L)))


def lognormal_field(shape, seed: int, slope: float = -1.5, sigma: float = 1.0, fp32: bool = True) -> np.ndarray:
    """A density field on a periodic grid of the given shape (any number of axes): rho = exp(G - s^2/2)
    with G Gaussian, power spectrum ~ k^slope (k != 0) and standard deviation s = sigma, so rho has
    mean 1 (FP32-representable unless fp32 is False)."""
    g = _rng(seed)
    shape = tuple(int(m) for m in shape)
    fk = np.fft.fftn(g.standard_normal(shape))
    k2 = np.zeros(shape)
    for a, m in enumerate(shape):
        f = np.fft.fftfreq(m).reshape([-1 if b == a else 1 for b in range(len(shape))])
        k2 = k2 + f * f
    k2.flat[0] = 1.0
    amp = k2 ** (slope / 4.0)
    amp.flat[0] = 0.0
    G = np.fft.ifftn(fk * amp).real
    G *= sigma / G.std()
    rho = np.exp(G - 0.5 * sigma * sigma)
    return rho.astype(np.float32).astype(np.float64) if fp32 else rho


def normal_weights(n: int, mean: float, sd: float, seed: int, fp32: bool = True) -> np.ndarray:
    """n weights drawn from N(mean, sd^2) (FP32-representable unless fp32 is False)."""
    w = _rng(seed).normal(mean, sd, n)
    return w.astype(np.float32).astype(np.float64) if fp32 else w


def linear_edges(lo: float, hi: float, nbins: int) -> np.ndarray:
    return np.linspace(lo, hi, nbins + 1)


@dataclass
class Workload:
    name: str
    D: int
    N: int
    lmax: int
    edges: np.ndarray
    box: np.ndarray
    pos: np.ndarray
    w: np.ndarray
    precision: str = "fp32"
    periodic: bool = True
    extra: dict = field(default_factory=dict)
    geometry: str = "box"  # "sphere": pos are directions on S^2, edges in cos theta, box unused

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])


@dataclass
class Batch:
    """Several catalogues concatenated: catalogue i is rows offsets[i]:offsets[i+1] in its box boxes[i]."""
    name: str
    D: int
    edges: np.ndarray
    boxes: np.ndarray   # (ncat, D)
    offsets: np.ndarray  # (ncat + 1,) int64
    pos: np.ndarray
    w: np.ndarray

    @property
    def ncat(self) -> int:
        return len(self.offsets) - 1

    def catalogue(self, i: int):
        a, b = int(self.offsets[i]), int(self.offsets[i + 1])
        return self.pos[a:b], self.w[a:b], self.boxes[i]


def batch64(ncat: int = 64, scale: float = 1.0, grid: int = 128) -> Batch:
    """The batched D=3 workload: ncat catalogues with n_i log-uniform in [5e4, 5e5] (times
    `scale`) and periodic cubes of side L_i uniform in [500, 1000] (both drawn with seed 3);
    catalogue i (seed 1000 + i) is half uniform, half Poisson draws from a lognormal field
    (P(k) ~ k^-1.5, sigma_ln = 1) on a grid^3 mesh of its box; weights 1; 8 bins over [10, 120]."""
    g = _rng(3)
    sizes = np.round(np.exp(g.uniform(np.log(5e4), np.log(5e5), ncat)) * scale).astype(np.int64)
    sides = g.uniform(500.0, 1000.0, ncat)
    parts = []
    for i in range(ncat):
        L = float(sides[i])
        half = int(sizes[i]) // 2
        uni = uniform(half, 3, L, 1000 + i)
        ln = lognormal_poisson(float(sizes[i] - half), L, 1000 + i, grid=grid)
        parts.append(np.concatenate([uni, ln]))
    offsets = np.zeros(ncat + 1, dtype=np.int64)
    offsets[1:] = np.cumsum([len(p) for p in parts])
    pos = np.concatenate(parts)
    boxes = np.repeat(sides[:, None], 3, axis=1)
    return Batch("batch64", 3, linear_edges(10.0, 120.0, 8), boxes, offsets, pos, np.ones(len(pos)))


def workload(name: str, seed: int | None = None, scale: float = 1.0) -> Workload:
    """Build a named workload.  ``scale`` < 1 shrinks the particle count (and,
    for the lognormal box, the volume) at fixed density, for tests."""
    if name == "d3n3_fp64":
        s = 0 if seed is None else seed
        n = max(8, int(round(2000 * scale)))
        pos = uniform(n, 3, 250.0, s, fp32=False)
        return Workload(name, 3, 3, 5, linear_edges(0.0, 100.0, 10), np.full(3, 250.0), pos, np.ones(n), "fp64")
    if name in ("d2", "d2n3", "d2n4"):
        s = 1 if seed is None else seed
        n_half = max(4, int(round(100_000 * scale)))
        nc = max(1, int(round(400 * scale)))
        pos = np.concatenate([uniform(n_half, 2, 1.0, s), gaussian_blobs(n_half, 2, 1.0, nc, 0.005, s + 500)])
        w = normal_weights(2 * n_half, 1.0, 0.1, s + 900)
        N = 4 if name == "d2n4" else 3
        return Workload(name, 2, N, 10, linear_edges(0.002, 0.05, 16), np.full(2, 1.0), pos, w)
    if name == "d3n4":
        s = 2 if seed is None else seed
        L = 1000.0 * scale ** (1.0 / 3.0)
        grid = max(16, int(round(256 * scale ** (1.0 / 3.0))))
        data = lognormal_poisson(1e6 * scale, L, s, grid=grid)
        nr = max(4, int(round(1e6 * scale)))
        rand = uniform(nr, 3, L, s + 500)
        pos = np.concatenate([data, rand])
        w = np.concatenate([np.ones(data.shape[0]), -np.ones(nr)])
        return Workload(name, 3, 4, 5, linear_edges(20.0, 160.0, 10), np.full(3, L), pos, w)
    if name == "d3n5":
        # the paper's 5PCF example: uniform points in the periodic unit cube, ten bins in [0.1, 0.4], lmax 4
        s = 5 if seed is None else seed
        n = max(8, int(round(10_000 * scale)))
        return Workload(name, 3, 5, 4, linear_edges(0.1, 0.4, 10), np.full(3, 1.0), uniform(n, 3, 1.0, s), np.ones(n))
    if name == "d4n3":
        s = 4 if seed is None else seed
        n_half = max(4, int(round(50_000 * scale)))
        nc = max(1, int(round(200 * scale)))
        pos = np.concatenate([uniform(n_half, 4, 1.0, s), gaussian_blobs(n_half, 4, 1.0, nc, 0.01, s + 500)])
        w = normal_weights(2 * n_half, 1.0, 0.1, s + 900)
        return Workload(name, 4, 3, 4, linear_edges(0.01, 0.12, 8), np.full(4, 1.0), pos, w)
    if name == "s2n4":
        # the paper's 2-sphere 4PCF example (evenly distributed points, ten bins over cos theta in
        # [-0.5, 0.5), lmax 4) at n = 100k
        s = 6 if seed is None else seed
        n = max(8, int(round(100_000 * scale)))
        return Workload(name, 2, 4, 4, linear_edges(-0.5, 0.5, 10), np.ones(2), sphere_uniform(n, s), np.ones(n),
                        periodic=False, geometry="sphere")
    raise KeyError(name)
