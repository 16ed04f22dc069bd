"""Seeded synthetic inputs for the EXACT hot path.

This module only draws random numbers and builds the *inputs* of a
reconstruction: a random-ellipse phantom, an energy grid, a smooth source
spectrum, detector windows, attenuation coefficients, a Poisson sampler that
turns given mean counts into counts, and the Gaussian measurement case of
Sec. 3.2.  It contains none of the method's arithmetic: no projector, no link
function, no operator, no solver.  Mean photon counts are computed by each
consumer with its own projector and link (the oracle in tests, the CUDA path in
the benchmark) and then handed to ``poisson_counts``.

The paper's own phantom (a PMMA disc), measured spectra and sensitivities
(Sec. 3.1, Fig. 2) are not available; these seeded stand-ins take the shapes
the paper uses (image sizes, number of windows, number of energies, views and
detector cells) and the value ranges a CT phantom has (densities in [0, 1]).
"""
from __future__ import annotations

import hashlib
from dataclasses import dataclass

import numpy as np

__all__ = [
    "case_seed", "Ellipse", "random_ellipses", "rasterize_ellipses",
    "ellipse_phantom", "energy_grid", "smooth_spectrum", "window_partition",
    "window_trapezoids", "power_law_mu", "poisson_counts", "gaussian_case",
    "random_image", "random_sinogram",
]


def case_seed(config_id: str, job_id: int = 0) -> int:
    """Deterministic 63-bit seed from a configuration name and a job index."""
    h = hashlib.sha256(f"{config_id}/{job_id}".encode()).digest()
    return int.from_bytes(h[:8], "little") & ((1 << 63) - 1)


@dataclass(frozen=True)
class Ellipse:
    """An ellipse in pixel units, centred at (cx, cy), semi-axes (a, b),
    rotated by ``phi`` radians, adding ``rho`` to the density inside."""
    cx: float
    cy: float
    a: float
    b: float
    phi: float
    rho: float


def random_ellipses(n: int, n_ellipses: int, seed: int) -> list[Ellipse]:
    """Draw ``n_ellipses`` ellipses for an ``n`` x ``n`` image.

    Centres are uniform in the disc of radius 0.6 * n/2, semi-axes uniform in
    [0.05, 0.35] * n/2, rotations uniform in [0, pi) and density increments
    uniform in [0.1, 0.6].
    """
    rng = np.random.default_rng(seed)
    half = 0.5 * n
    out = []
    for _ in range(n_ellipses):
        r = 0.6 * half * np.sqrt(rng.uniform())
        ang = rng.uniform(0.0, 2.0 * np.pi)
        a, b = rng.uniform(0.05, 0.35, size=2) * half
        out.append(Ellipse(float(r * np.cos(ang)), float(r * np.sin(ang)),
                           float(a), float(b), float(rng.uniform(0.0, np.pi)),
                           float(rng.uniform(0.1, 0.6))))
    return out


def rasterize_ellipses(ellipses, nx: int, ny: int, pixel: float = 1.0,
                       supersample: int = 1, clip: bool = True) -> np.ndarray:
    """Rasterise ellipses onto a ``[ny][nx]`` grid (row-major, float64).

    Pixel (ix, iy) has its centre at ((ix-(nx-1)/2)*pixel, (iy-(ny-1)/2)*pixel);
    ellipse coordinates are in the same physical units.  With
    ``supersample`` = s each pixel is the mean of s*s sub-samples.  Densities
    are summed and, if ``clip``, clipped to [0, 1].
    """
    s = int(supersample)
    offs = (np.arange(s) + 0.5) / s - 0.5
    xs = ((np.arange(nx) - 0.5 * (nx - 1))[:, None] + offs[None, :]).reshape(-1) * pixel
    ys = ((np.arange(ny) - 0.5 * (ny - 1))[:, None] + offs[None, :]).reshape(-1) * pixel
    X, Y = np.meshgrid(xs, ys)
    img = np.zeros_like(X)
    for e in ellipses:
        c, sn = np.cos(e.phi), np.sin(e.phi)
        u = (X - e.cx) * c + (Y - e.cy) * sn
        v = -(X - e.cx) * sn + (Y - e.cy) * c
        img += e.rho * ((u / e.a) ** 2 + (v / e.b) ** 2 <= 1.0)
    if clip:
        img = np.clip(img, 0.0, 1.0)
    return img.reshape(ny, s, nx, s).mean(axis=(1, 3))


def ellipse_phantom(n: int, n_ellipses: int, seed: int, supersample: int = 1) -> np.ndarray:
    """Random-ellipse phantom on an n x n grid with unit pixels, in [0, 1]."""
    return rasterize_ellipses(random_ellipses(n, n_ellipses, seed), n, n, 1.0, supersample)


def energy_grid(n_energy: int, e_lo: float = 20.0, e_hi: float = 120.0) -> np.ndarray:
    """Centres of ``n_energy`` equal bins spanning [e_lo, e_hi] keV."""
    return e_lo + (np.arange(n_energy) + 0.5) * (e_hi - e_lo) / n_energy


def smooth_spectrum(energies: np.ndarray, seed: int, e_max: float = 120.0) -> np.ndarray:
    """Smooth seeded source spectrum phi_k >= 0 with sum 1.

    phi(E) ~ E (E_max - E) (1 + 0.2 sin(2 pi f E / E_max + p0)), f ~ U[0.5, 2],
    p0 ~ U[0, 2 pi).
    """
    rng = np.random.default_rng(seed)
    f = rng.uniform(0.5, 2.0)
    p0 = rng.uniform(0.0, 2.0 * np.pi)
    e = np.asarray(energies, dtype=np.float64)
    phi = e * np.maximum(e_max - e, 0.0) * (1.0 + 0.2 * np.sin(2.0 * np.pi * f * e / e_max + p0))
    phi = np.maximum(phi, 0.0)
    return phi / phi.sum()


def window_partition(n_energy: int, n_windows: int) -> np.ndarray:
    """0/1 matrix D[w][k]: the energy bins split into contiguous, nearly equal groups."""
    edges = np.linspace(0, n_energy, n_windows + 1).round().astype(int)
    D = np.zeros((n_windows, n_energy))
    for w in range(n_windows):
        D[w, edges[w]:edges[w + 1]] = 1.0
    return D


def window_trapezoids(n_energy: int, n_windows: int, seed: int) -> np.ndarray:
    """Overlapping trapezoidal detector sensitivities D[w][k] in [0, 1]."""
    rng = np.random.default_rng(seed)
    centers = (np.arange(n_windows) + 0.5) / n_windows * n_energy
    width = n_energy / n_windows
    k = np.arange(n_energy) + 0.5
    D = np.zeros((n_windows, n_energy))
    for w in range(n_windows):
        c = centers[w] + rng.uniform(-0.1, 0.1) * width
        dist = np.abs(k - c) / width
        D[w] = np.clip(1.5 - 2.0 * dist, 0.0, 1.0)
    return D


def power_law_mu(energies: np.ndarray, c: float, e_ref: float = 60.0) -> np.ndarray:
    """Attenuation per unit length and density, mu_k = c (E_k / e_ref)^-3."""
    return c * (np.asarray(energies, dtype=np.float64) / e_ref) ** -3.0


def poisson_counts(mean: np.ndarray, seed: int) -> np.ndarray:
    """Independent Poisson draws with the given means (float64 array of counts)."""
    rng = np.random.default_rng(seed)
    return rng.poisson(np.asarray(mean, dtype=np.float64)).astype(np.float64)


def gaussian_case(n: int, d: int, norm: float, seed: int):
    """Gaussian measurement vectors a_i ~ N(0, I_d) (Sec. 2.2) and a signal of
    Euclidean norm ``norm`` with a uniformly random direction.  Returns (A, x)."""
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, d))
    x = rng.standard_normal(d)
    return A, x * (norm / np.linalg.norm(x))


def random_image(nx: int, ny: int, seed: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    """Uniform random ``[ny][nx]`` image."""
    return np.random.default_rng(seed).uniform(lo, hi, size=(ny, nx))


def random_sinogram(n_views: int, n_bins: int, seed: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """Uniform random ``[views][bins]`` array (adjoint test inputs)."""
    return np.random.default_rng(seed).uniform(lo, hi, size=(n_views, n_bins))
