"""Seeded synthetic inputs for the Lippmann-Schwinger solves.

This module only draws random media, incident directions and receiver
positions.  It contains none of the solver's arithmetic, so both the CUDA
path's tests/benchmarks and the CPU oracle's tests can take their inputs from
it without sharing any method code.

The paper's own velocity fields (Sec. 2.5 fields (i)-(iv), Sec. 3.2) come
without seeds or exact widths; the recipes below are synthetic stand-ins with
the same structure: Gaussian bumps / a band-limited random field, c = Theta(1),
c = 1 near the boundary of the unit box, m = 1 - 1/c^2 (Sec. 1).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "Workload",
    "WORKLOADS",
    "grid_points",
    "taper",
    "gaussian_medium",
    "bandlimited_medium",
    "plane_wave_directions",
    "make_workload",
    "ragged_sizes",
    "ragged_instances",
    "RAGGED_32",
]


def grid_points(n: int, d: int) -> list[np.ndarray]:
    """Coordinates p_i = i h, i = 1..n, h = 1/(n+1) along each axis (Sec. 2.1)."""
    h = 1.0 / (n + 1)
    x = np.arange(1, n + 1, dtype=np.float64) * h
    return np.meshgrid(*([x] * d), indexing="ij")


def taper(xs: list[np.ndarray], inner: float = 0.1) -> np.ndarray:
    """C^1 window: 1 on [inner, 1-inner]^d, cos^2 ramp to 0 on the box boundary."""
    w = np.ones_like(xs[0])
    for x in xs:
        t = np.minimum(x, 1.0 - x)
        r = np.where(t >= inner, 1.0, np.cos(0.5 * math.pi * (inner - t) / inner) ** 2)
        w = w * r
    return w


def gaussian_medium(n: int, d: int, n_gauss: int, width: float,
                    c_range: tuple[float, float], seed: int) -> np.ndarray:
    """m = 1 - 1/c^2 with c = 1 + W(x) sum_k (c_k - 1) exp(-|x-x_k|^2 / (2 width^2)).

    Centres x_k ~ U[0.2, 0.8]^d, c_k ~ U[c_min, c_max], c clipped to the range.
    Returns a float64 array of shape (n,)*d, axis 0 = x1 (slowest).
    """
    rng = np.random.default_rng(seed)
    centres = rng.uniform(0.2, 0.8, size=(n_gauss, d))
    ck = rng.uniform(c_range[0], c_range[1], size=n_gauss)
    xs = grid_points(n, d)
    bump = np.zeros_like(xs[0])
    for k in range(n_gauss):
        r2 = sum((x - centres[k, a]) ** 2 for a, x in enumerate(xs))
        bump += (ck[k] - 1.0) * np.exp(-r2 / (2.0 * width * width))
    c = 1.0 + taper(xs) * bump
    c = np.clip(c, c_range[0], c_range[1])
    return 1.0 - 1.0 / (c * c)


def bandlimited_medium(n: int, d: int, corr_len: float, amplitude: float,
                       seed: int) -> np.ndarray:
    """Smooth random field: white noise through a Gaussian spectral filter of
    correlation length corr_len, scaled to [-1, 1]; c = 1 + amplitude*W*field."""
    rng = np.random.default_rng(seed)
    noise = rng.standard_normal((n,) * d)
    h = 1.0 / (n + 1)
    freqs = np.meshgrid(*([np.fft.fftfreq(n, d=h)] * d), indexing="ij")
    k2 = sum(f * f for f in freqs)
    filt = np.exp(-0.5 * (2.0 * math.pi) ** 2 * k2 * corr_len ** 2)
    field = np.real(np.fft.ifftn(np.fft.fftn(noise) * filt))
    field = field / np.max(np.abs(field))
    c = 1.0 + amplitude * taper(grid_points(n, d)) * field
    return 1.0 - 1.0 / (c * c)


def plane_wave_directions(d: int, count: int, seed: int | None = None,
                          fixed: tuple[float, ...] | None = None) -> np.ndarray:
    """Unit incident directions, shape (count, d).

    fixed: one given direction (normalised);  seed with count == 1: one
    seeded angle;  otherwise (2D) uniform angles 2 pi k / count.
    """
    if fixed is not None:
        v = np.asarray(fixed, dtype=np.float64)
        return (v / np.linalg.norm(v))[None, :].repeat(count, axis=0)
    if d != 2:
        raise ValueError("angle sets are defined for 2D only")
    if count == 1 and seed is not None:
        th = np.random.default_rng(seed).uniform(0.0, 2.0 * math.pi, size=1)
    else:
        th = 2.0 * math.pi * np.arange(count) / count
    return np.stack([np.cos(th), np.sin(th)], axis=1)


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    dim: int
    n: int
    freq: float          # omega / (2 pi)
    b_pml: int
    b_slab: int
    medium: str          # "gauss" | "band"
    n_gauss: int = 0
    width: float = 0.0
    c_range: tuple[float, float] = (0.8, 1.2)
    n_rhs: int = 1
    seed: int = 0
    direction: tuple[float, ...] | None = None

    @property
    def omega(self) -> float:
        return 2.0 * math.pi * self.freq


# The five workloads: sizes, frequencies, media and directions as specified;
# seeds are 1705 + workload index.
WORKLOADS = {
    "2d_n64": Workload("2d_n64", 2, 64, 8.0, 12, 4, "gauss", 4, 0.08, (0.8, 1.2),
                       1, 1706, (1.0, 0.0)),
    "2d_n256": Workload("2d_n256", 2, 256, 32.0, 12, 4, "gauss", 16, 0.05, (0.75, 1.25),
                        1, 1707, None),
    "2d_n512_r64": Workload("2d_n512_r64", 2, 512, 64.0, 12, 4, "band", 0, 0.05,
                            (0.8, 1.2), 64, 1708, None),
    "3d_n64": Workload("3d_n64", 3, 64, 16.0, 8, 4, "gauss", 8, 0.1, (0.8, 1.2),
                       1, 1709, (1.0, 1.0, 1.0)),
    "2d_n256_r16": Workload("2d_n256_r16", 2, 256, 32.0, 12, 4, "gauss", 16, 0.05,
                            (0.75, 1.25), 16, 1707, None),
    # the 3D workload at n = 32 (same medium recipe, seed and points per
    # wavelength): a small case for profiler captures of the 3D kernels
    "3d_n32": Workload("3d_n32", 3, 32, 33.0 / 8.0, 8, 4, "gauss", 8, 0.1, (0.8, 1.2),
                       1, 1709, (1.0, 1.0, 1.0)),
}


def make_workload(w: Workload | str, n: int | None = None):
    """Return (m, directions) for a workload; n overrides the grid size
    (frequency scaled to keep the points per wavelength)."""
    if isinstance(w, str):
        w = WORKLOADS[w]
    nn = w.n if n is None else n
    if w.medium == "gauss":
        m = gaussian_medium(nn, w.dim, w.n_gauss, w.width, w.c_range, w.seed)
    else:
        m = bandlimited_medium(nn, w.dim, w.width, 0.2, w.seed)
    if w.direction is not None:
        dirs = plane_wave_directions(w.dim, w.n_rhs, fixed=w.direction)
    elif w.n_rhs == 1:
        dirs = plane_wave_directions(w.dim, 1, seed=w.seed)
    else:
        dirs = plane_wave_directions(w.dim, w.n_rhs)
    return m, dirs


# The ragged-instance batch: 32 independent problems, n uniform on
# {128, ..., 384}, omega/2pi = n/8 (8 points per wavelength), band-limited
# media with c in [0.8, 1.2], one plane wave each at a seeded angle.
RAGGED_32 = dict(count=32, n_lo=128, n_hi=384, seed=1710)


def ragged_sizes(count: int, n_lo: int, n_hi: int, seed: int) -> list[int]:
    """Grid sizes drawn uniformly from {n_lo, ..., n_hi}."""
    rng = np.random.default_rng(seed)
    return [int(v) for v in rng.integers(n_lo, n_hi + 1, size=count)]


def ragged_instances(ns, seed: int, corr_len: float = 0.05, amplitude: float = 0.2):
    """For each n: (freq = n/8, band-limited medium m, one seeded direction).
    Instance q uses seed + q."""
    out = []
    for q, n in enumerate(ns):
        m = bandlimited_medium(int(n), 2, corr_len, amplitude, seed + q)
        d = plane_wave_directions(2, 1, seed=seed + 1000 + q)
        out.append((n / 8.0, m, d))
    return out
