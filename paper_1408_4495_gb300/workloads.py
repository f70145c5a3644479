"""Seeded synthetic inputs: media m(x) and incident directions for the solver's workloads.

This module holds no arithmetic of the method.  It only draws the inputs (the medium
sampled on the grid and the plane-wave directions) from seeded generators, so that the
CUDA library and the CPU checker receive identical arrays.

Grid convention: n points per dimension at x = i h, i = 1..n, h = 1/(n+1).

The paper's media (Sec. 3.3: Gaussian bumps and smoothed cavities with the velocity
c = (1-m)^(-1/2) between 2/3 and 1) do not have printed parameters; these recipes are
stand-ins of the same shape:

* ``cutoff``: C-infinity step so that m vanishes within 0.1 of the boundary of the unit cube.
* ``bumps``: sum of Gaussian bumps A exp(-|x-c|^2 / (2 w^2)) times the cutoff.
* ``smooth_noise``: white noise convolved with a Gaussian of width 4h, scaled to a given
  max |m|, times the cutoff.
* ``box_cavity``: the smoothed square (2D) and cubic (3D) cavities of Sec. 3.3.
* ``cavity``: the media of Sec. 4 (general domains): a smoothed cavity of an l2 or l1 ball,
  m = A s((rho - |x - c|_p) / delta) with the C-infinity step s, so that supp(m) is the open
  ball of radius rho (the unknowns of the general-domain method) and m = A inside rho - delta.
* ``serving_stream``: a seeded Poisson stream of requests of the serving mix: 2D and 3D grids,
  omega / 2 pi = n / 8, 4-8 Gaussian bumps per medium rescaled to max|m| <= 0.3, 1..k plane
  waves per request; media drawn from a pool so that some requests share a medium.
* ``laplace_3d``: the potentials of Sec. 5 (a negative Gaussian, or a smoothed indicator of
  a ball, scaled so that max |V| = 1/h^2 as in the paper's tables) times the cutoff, and
  delta sources near the top-left corner of the middle cross-section x_1 = 1/2.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


def grid_x(n: int) -> np.ndarray:
    return (np.arange(n, dtype=np.float64) + 1.0) / (n + 1)


def _smooth_step(t: np.ndarray) -> np.ndarray:
    """0 for t <= 0, 1 for t >= 1, e^{-1/t} / (e^{-1/t} + e^{-1/(1-t)}) in between."""
    t = np.asarray(t, dtype=np.float64)
    out = np.where(t >= 1.0, 1.0, 0.0)
    mid = (t > 0.0) & (t < 1.0)
    tm = t[mid]
    a = np.exp(-1.0 / tm)
    b = np.exp(-1.0 / (1.0 - tm))
    out[mid] = a / (a + b)
    return out


def cutoff(n: int, d: int, width: float = 0.1) -> np.ndarray:
    x = grid_x(n)
    c1 = _smooth_step((x - width) / width) * _smooth_step((1.0 - width - x) / width)
    out = c1
    for _ in range(d - 1):
        out = np.multiply.outer(out, c1)
    return out


def bumps(n: int, d: int, amps, widths, centres) -> np.ndarray:
    X = np.meshgrid(*([grid_x(n)] * d), indexing="ij")
    m = np.zeros((n,) * d)
    for A, w, c in zip(amps, widths, centres):
        r2 = sum((X[a] - c[a]) ** 2 for a in range(d))
        m += A * np.exp(-r2 / (2.0 * w * w))
    return m * cutoff(n, d)


def smooth_noise(n: int, d: int, seed: int, sigma_h: float = 4.0, max_abs: float = 0.2) -> np.ndarray:
    rng = np.random.default_rng(seed)
    noise = rng.standard_normal((n,) * d)
    # zero-padded (linear) convolution with a Gaussian of width sigma_h grid steps
    L = 2 * n
    k1 = np.fft.fftfreq(L) * L
    g1 = np.exp(-0.5 * (k1 / sigma_h) ** 2)
    ker = g1
    for _ in range(d - 1):
        ker = np.multiply.outer(ker, g1)
    pad = np.zeros((L,) * d)
    pad[(slice(0, n),) * d] = noise
    sm = np.real(np.fft.ifftn(np.fft.fftn(pad) * np.fft.fftn(ker)))[(slice(0, n),) * d]
    sm *= max_abs / np.max(np.abs(sm))
    return sm * cutoff(n, d)


def directions_circle(count: int) -> np.ndarray:
    a = 2.0 * np.pi * np.arange(count) / count
    return np.stack([np.cos(a), np.sin(a)], axis=1)


def directions_sphere(count: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    v = rng.standard_normal((count, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


@dataclass
class Workload:
    name: str
    d: int
    n: int
    omega: float
    m: np.ndarray = field(repr=False)
    directions: np.ndarray = field(repr=False)
    mixed: bool = True
    buffer_b: int = 2
    restart: int = 50
    tol: float = 1e-6

    @property
    def nrhs(self) -> int:
        return len(self.directions)


def plain_2d(n: int = 32) -> Workload:
    """2D plain FP64: one bump A=-0.2, w=0.1 at (0.5,0.5); omega/2pi = 4; d = (1,0)."""
    m = bumps(n, 2, [-0.2], [0.1], [(0.5, 0.5)])
    return Workload(f"2d_plain_n{n}", 2, n, 2 * math.pi * 4, m, np.array([[1.0, 0.0]]), mixed=False)


def bumps_2d(n: int = 256, freq: float = 32.0, nb: int = 8, nrhs: int = 16, seed: int = 1002) -> Workload:
    """2D batched: nb seeded bumps, A ~ U[-0.3,0.3], w ~ U[0.03,0.1], c ~ U[0.2,0.8]^2."""
    rng = np.random.default_rng(seed)
    amps = rng.uniform(-0.3, 0.3, nb)
    widths = rng.uniform(0.03, 0.1, nb)
    centres = rng.uniform(0.2, 0.8, (nb, 2))
    m = bumps(n, 2, amps, widths, centres)
    return Workload(f"2d_bumps_n{n}", 2, n, 2 * math.pi * freq, m, directions_circle(nrhs))


def noise_2d(n: int = 1024, freq: float = 128.0, nrhs: int = 64, seed: int = 1003) -> Workload:
    """2D large: white noise * Gaussian(4h), max|m| = 0.2, times the cutoff."""
    m = smooth_noise(n, 2, seed, 4.0, 0.2)
    return Workload(f"2d_noise_n{n}", 2, n, 2 * math.pi * freq, m, directions_circle(nrhs))


def bumps_3d(n: int = 64, freq: float = 8.0, nb: int = 6, nrhs: int = 8, seed: int = 1004) -> Workload:
    """3D batched: nb seeded bumps, A ~ U[-0.2,0.2], w ~ U[0.05,0.12], c ~ U[0.2,0.8]^3."""
    rng = np.random.default_rng(seed)
    amps = rng.uniform(-0.2, 0.2, nb)
    widths = rng.uniform(0.05, 0.12, nb)
    centres = rng.uniform(0.2, 0.8, (nb, 3))
    m = bumps(n, 3, amps, widths, centres)
    return Workload(f"3d_bumps_n{n}", 3, n, 2 * math.pi * freq, m, directions_sphere(nrhs, seed))


def enforce_buffer(m: np.ndarray, b: int) -> np.ndarray:
    """Zero the b+1 outermost layers exactly (the cutoff already makes them ~0 there)."""
    m = m.copy()
    n, d = m.shape[0], m.ndim
    w = b + 1
    for a in range(d):
        sl = [slice(None)] * d
        sl[a] = slice(0, w)
        m[tuple(sl)] = 0.0
        sl[a] = slice(n - w, n)
        m[tuple(sl)] = 0.0
    return m


@dataclass
class LaplaceWorkload:
    name: str
    n: int
    V: np.ndarray = field(repr=False)
    points: np.ndarray = field(repr=False)  # (nsrc, 3) 0-based grid indices of the sources
    mixed: bool = True
    buffer_b: int = 2
    restart: int = 50
    tol: float = 1e-6

    @property
    def nrhs(self) -> int:
        return len(self.points)


def laplace_3d(n: int = 64, nsrc: int = 8, shape: str = "gaussian", seed: int = 1005) -> LaplaceWorkload:
    """Sec. 5 stand-in: V = -(1/h^2) S(x) times the cutoff with S a Gaussian bump
    exp(-|x-c|^2 / (2 w^2)), w = 0.1, or a ball indicator smoothed over 0.05 (radius 0.25),
    c = (1/2, 1/2, 1/2); sources: the first at the grid point nearest (1/2, 1/4, 3/4), the
    others at seeded offsets of up to 4 grid steps in the cross-section, all distinct."""
    X = np.meshgrid(*([grid_x(n)] * 3), indexing="ij")
    r = np.sqrt(sum((X[a] - 0.5) ** 2 for a in range(3)))
    if shape == "gaussian":
        S = np.exp(-r * r / (2 * 0.1 * 0.1))
    elif shape == "ball":
        S = _smooth_step((0.25 - r) / 0.05 + 0.5)
    else:
        raise ValueError("shape must be 'gaussian' or 'ball'")
    h = 1.0 / (n + 1)
    V = -(1.0 / (h * h)) * S * cutoff(n, 3)
    base = np.array([round(0.5 / h) - 1, round(0.25 / h) - 1, round(0.75 / h) - 1])
    rng = np.random.default_rng(seed)
    pts = [base]
    seen = {tuple(base)}
    while len(pts) < nsrc:
        q = base + np.concatenate([[0], rng.integers(-4, 5, 2)])
        q = np.clip(q, 0, n - 1)
        if tuple(q) not in seen:
            seen.add(tuple(q))
            pts.append(q)
    return LaplaceWorkload(f"3d_laplace_{shape}_n{n}", n, V, np.array(pts, dtype=np.int64))


def cavity(n: int, d: int, norm: str = "l2", rho: float = 0.4, delta: float = 0.1, amp: float = -0.3,
           centre=None) -> np.ndarray:
    """Sec. 4 stand-in: smoothed cavity of an l2 (norm="l2") or l1 (norm="l1") ball."""
    X = np.meshgrid(*([grid_x(n)] * d), indexing="ij")
    c = centre if centre is not None else [0.5] * d
    if norm == "l2":
        r = np.sqrt(sum((X[a] - c[a]) ** 2 for a in range(d)))
    elif norm == "l1":
        r = sum(np.abs(X[a] - c[a]) for a in range(d))
    else:
        raise ValueError("norm must be 'l2' or 'l1'")
    return amp * _smooth_step((rho - r) / delta)


# the serving mix: 70 % 2D n in {128, 256, 512}, 30 % 3D n in {32, 48}
SERVING_GRIDS = ((2, 128), (2, 256), (2, 512), (3, 32), (3, 48))
SERVING_WEIGHTS = (0.7 / 3, 0.7 / 3, 0.7 / 3, 0.15, 0.15)


def box_cavity(n: int, d: int, amp: float = -1.25, half: float = 0.2, delta: float = 0.1) -> np.ndarray:
    """Secs. 3.3 stand-in for the smoothed square (2D, Fig. R22) and cubic (3D, Fig. R32)
    cavities: amp times a smoothed indicator of the box |x_a - 1/2| < half on every axis,
    product over the axes of s((half - |x_a - 1/2|) / delta + 1/2) with the C-infinity step s
    (so m = amp on |x_a - 1/2| < half - delta/2 and 0 beyond half + delta/2), times the cutoff.
    amp = -1.25 gives the velocity c = (1 - m)^(-1/2) = 2/3 inside and 1 outside, the range
    the paper states for its examples."""
    x = grid_x(n)
    s1 = _smooth_step((half - np.abs(x - 0.5)) / delta + 0.5)
    out = s1
    for _ in range(d - 1):
        out = np.multiply.outer(out, s1)
    return amp * out * cutoff(n, d)


def serving_stream(count: int, rate: float, seed: int = 1006, grids=SERVING_GRIDS, weights=SERVING_WEIGHTS,
                   max_dirs: int = 32, pool: int | None = None):
    """Seeded serving mix: ``count`` requests with exponential inter-arrival times of mean
    1 / rate seconds.  Each entry is (d, n, omega, m, directions, arrival).  With ``pool`` set,
    each grid draws its medium from ``pool`` seeded media, so requests can share a medium."""
    rng = np.random.default_rng(seed)
    media = {}
    out = []
    t = 0.0
    for _ in range(count):
        t += rng.exponential(1.0 / rate)
        d, n = grids[rng.choice(len(grids), p=np.asarray(weights) / np.sum(weights))]
        mseed = int(rng.integers(0, pool)) if pool else int(rng.integers(0, 2**31))
        key = (d, n, mseed)
        if key not in media:
            mr = np.random.default_rng(mseed)
            nb = int(mr.integers(4, 9))
            m = bumps(n, d, mr.uniform(-0.3, 0.3, nb), mr.uniform(0.05, 0.12, nb), mr.uniform(0.25, 0.75, (nb, d)))
            peak = np.max(np.abs(m))
            if peak > 0.3:
                m *= 0.3 / peak
            media[key] = enforce_buffer(m, 2)
        k = int(rng.integers(1, max_dirs + 1))
        dirs = directions_circle(k) if d == 2 else directions_sphere(k, int(rng.integers(0, 2**31)))
        out.append((d, n, 2 * math.pi * n / 8, media[key], dirs, t))
    return out
