"""Seeded synthetic workloads for the IFGF operator apply.

This module only draws inputs: surface point clouds, complex densities and
target samples.  It holds none of the method's arithmetic, and it is the one
module that both the CPU oracle tests and the GPU path use.

Geometries follow the test surfaces of the paper's numerical section
(Sec. 4: a sphere and spheroids x^2 + y^2 + (z/e)^2 = a^2).  The paper
discretises them with equispaced parametric patches; here the sphere uses a
Fibonacci lattice and the spheroids an area-uniform random sample, both at a
unit diameter.  The wavenumber of a body that is ``L`` wavelengths across is
``kappa = 2*pi*L`` (unit diameter).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "fibonacci_sphere",
    "spheroid",
    "densities",
    "targets",
    "Workload",
    "WORKLOADS",
    "make",
    "batch_problems",
]


def fibonacci_sphere(n: int, diameter: float = 1.0) -> np.ndarray:
    """Fibonacci-lattice nodes on a sphere of the given diameter, shape (3, n), float64.

    z_i = 1 - (2i+1)/n, rho_i = sqrt(1 - z_i^2), phi_i = i*pi*(3 - sqrt(5)) mod 2*pi.
    """
    i = np.arange(n, dtype=np.float64)
    z = 1.0 - (2.0 * i + 1.0) / n
    rho = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    phi = np.mod(i * (math.pi * (3.0 - math.sqrt(5.0))), 2.0 * math.pi)
    r = 0.5 * diameter
    return np.stack([r * rho * np.cos(phi), r * rho * np.sin(phi), r * z]).astype(np.float64)


def spheroid(n: int, a: float, c: float, seed: int) -> np.ndarray:
    """Area-uniform random points on the spheroid (x/a)^2 + (y/a)^2 + (z/c)^2 = 1, shape (3, n).

    Standard rejection method: a Gaussian triple gives a uniform direction u on
    the unit sphere; the map u -> (a ux, a uy, c uz) scales the area element by
    a*sqrt(c^2 (ux^2 + uy^2) + a^2 uz^2), so u is kept with probability
    sqrt(c^2 (ux^2+uy^2) + a^2 uz^2) / max(a, c).
    """
    rng = np.random.default_rng(seed)
    out = np.empty((3, 0), dtype=np.float64)
    m = max(a, c)
    while out.shape[1] < n:
        want = int((n - out.shape[1]) * 1.6) + 1024
        g = rng.standard_normal((3, want))
        u = g / np.linalg.norm(g, axis=0)
        w = np.sqrt(c * c * (u[0] ** 2 + u[1] ** 2) + a * a * u[2] ** 2) / m
        keep = rng.random(want) < w
        u = u[:, keep]
        out = np.concatenate([out, np.stack([a * u[0], a * u[1], c * u[2]])], axis=1)
    return np.ascontiguousarray(out[:, :n])


def densities(n: int, nrhs: int, seed: int, dtype=np.complex128) -> np.ndarray:
    """Complex densities a_m with real and imaginary parts iid U[-1, 1], shape (nrhs, n)."""
    rng = np.random.default_rng(seed)
    re = rng.uniform(-1.0, 1.0, size=(nrhs, n))
    im = rng.uniform(-1.0, 1.0, size=(nrhs, n))
    return np.ascontiguousarray((re + 1j * im).astype(dtype))


def targets(n: int, m: int, seed: int) -> np.ndarray:
    """m distinct seeded-random target indices in [0, n), sorted, int64 (all n if m >= n)."""
    if m >= n:
        return np.arange(n, dtype=np.int64)
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(n, size=m, replace=False)).astype(np.int64)


def random_cloud(n: int, seed: int, scale: float = 1.0) -> np.ndarray:
    """Uniform random points in a cube (used for small ragged tree tests), shape (3, n)."""
    rng = np.random.default_rng(seed)
    return np.ascontiguousarray(rng.uniform(-0.5 * scale, 0.5 * scale, size=(3, n)))


@dataclass
class Workload:
    """One named benchmark problem: a body, its sampling and the sampled error targets."""

    name: str
    geometry: str  # "sphere" or "spheroid"
    n: int
    wavelengths: float  # diameter in wavelengths; 0 means the Laplace kernel
    nrhs: int = 1
    seed: int = 1
    n_targets: int = 2000
    axes: tuple = (0.5, 0.5)  # (a, c) for spheroids, unit diameter
    extra: dict = field(default_factory=dict)

    @property
    def kappa(self) -> float:
        return 2.0 * math.pi * self.wavelengths

    def points(self) -> np.ndarray:
        if self.geometry == "sphere":
            return fibonacci_sphere(self.n)
        a, c = self.axes
        return spheroid(self.n, a, c, self.seed)

    def densities(self, dtype=np.complex128) -> np.ndarray:
        return densities(self.n, self.nrhs, self.seed + 100, dtype)

    def targets(self) -> np.ndarray:
        return targets(self.n, self.n_targets, self.seed + 200)


WORKLOADS = {
    # Plain FP64 case: 4-wavelength sphere, every point is a target.
    "sphere4": Workload("sphere4", "sphere", 24_576, 4.0, 1, 1, 24_576),
    # Same sampling density at a quarter of the points (profiling-sized case).
    "sphere32": Workload("sphere32", "sphere", 393_216, 32.0, 1, 6, 2000),
    # Headline case: 64-wavelength sphere, single density.
    "sphere64": Workload("sphere64", "sphere", 1_572_864, 64.0, 1, 2, 2000),
    # Oblate spheroid (a, a, a/4), 128 wavelengths, 32 densities.
    "oblate128": Workload("oblate128", "spheroid", 6_291_456, 128.0, 32, 3, 2000, (0.5, 0.125)),
    # 512-wavelength sphere; the Laplace repeat uses wavelengths = 0.
    "sphere512": Workload("sphere512", "sphere", 25_165_824, 512.0, 1, 5, 2000),
    "sphere512_laplace": Workload("sphere512_laplace", "sphere", 25_165_824, 0.0, 1, 5, 2000),
    # Prolate spheroid (a, a, 10a) of unit length, the paper's third geometry.
    "prolate128": Workload("prolate128", "spheroid", 6_291_456, 128.0, 1, 7, 2000, (0.05, 0.5)),
}


def linearithmic_series(geometry: str = "sphere") -> list:
    """Four problems at a fixed sampling density (about 122 points per square wavelength on the
    sphere): each doubles the wavelengths across the body and quadruples N, from 393,216 points
    at 32 wavelengths to 25,165,824 at 256 (sphere; the prolate spheroid (a, a, 10a) keeps the same
    N and its length in wavelengths)."""
    axes = (0.5, 0.5) if geometry == "sphere" else (0.05, 0.5)
    return [Workload(f"{geometry}_n{n}", geometry, n, lam, 1, 11 + i, 200, axes)
            for i, (n, lam) in enumerate(((393_216, 32.0), (1_572_864, 64.0), (6_291_456, 128.0),
                                          (25_165_824, 256.0)))]


def make(name: str) -> Workload:
    return WORKLOADS[name]


def batch_problems(count: int = 64, seed: int = 4) -> list:
    """Uneven batch: spheres or (a, a, a/2) spheroids, diameters log-uniform in [2, 32] wavelengths.

    The point count follows about 100 points per square wavelength of area,
    rounded up to a multiple of 6144 and clamped to [6144, 393216].
    """
    rng = np.random.default_rng(seed)
    probs = []
    for p in range(count):
        is_sphere = bool(rng.random() < 0.5)
        diam = float(np.exp(rng.uniform(math.log(2.0), math.log(32.0))))
        if is_sphere:
            area = math.pi * diam * diam
            axes = (0.5, 0.5)
        else:
            # Spheroid (a, a, a/2) with a = 1/2 (unit diameter); area in units of diameter^2.
            a, c = 0.5, 0.25
            e = math.sqrt(1.0 - (c * c) / (a * a))
            area_unit = 2.0 * math.pi * a * a * (1.0 + (1.0 - e * e) / e * math.atanh(e))
            area = area_unit * diam * diam
            axes = (a, c)
        n = int(min(393_216, max(6_144, 6_144 * math.ceil(100.0 * area / 6_144))))
        probs.append(
            Workload(
                f"batch{p}",
                "sphere" if is_sphere else "spheroid",
                n,
                diam,
                1,
                4000 + p,
                500,
                axes,
            )
        )
    return probs
