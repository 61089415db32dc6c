"""Seeded synthetic inputs: lattice sizes, body placements, initial fields and
request streams.  This module holds no arithmetic of the lattice Boltzmann
method; the CUDA library and the oracle both receive what it produces.

The paper measures on no dataset: every workload is a periodic box with
spheres (and walls), generated here from a seed.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Body:
    pos: tuple
    e: tuple
    R: float
    B1: float
    beta: float
    mobile: bool = True


@dataclass
class Workload:
    name: str
    shape: tuple
    collision: str
    lambda_e: float
    steps: int
    bodies: list = field(default_factory=list)
    walls: list = field(default_factory=list)  # (axis, index, vel)
    obstacles: list = field(default_factory=list)  # (pos, radius)
    tube: bool = False
    contact: tuple | None = None  # (sigma, eps)

    @property
    def cells(self) -> int:
        return int(np.prod(self.shape))


def c1_fixed_squirmer() -> Workload:
    """32^3 periodic, BGK tau = 1, one fixed squirmer R = 4 at the node (16,16,16),
    e = +z, B1 = 0.01, beta = 0, fluid at rest, 500 steps."""
    return Workload("c1_fixed_squirmer_32", (32, 32, 32), "bgk", 1.0, 500,
                    [Body((16.0, 16.0, 16.0), (0.0, 0.0, 1.0), 4.0, 0.01, 0.0, False)])


def c2_free_swimmer(beta: float = 0.0, n: int = 128, R: float = 8.0, steps: int = 20000) -> Workload:
    """128^3 periodic, TRT (lambda_e = 1, magic 3/16), one free squirmer R = 8,
    B1 = 0.005 at the box centre, e = +z."""
    c = n / 2.0
    return Workload(f"c2_free_swimmer_{n}_beta{beta:+g}", (n, n, n), "trt", 1.0, steps,
                    [Body((c, c, c), (0.0, 0.0, 1.0), R, 0.005, beta, True)])


def c3_pusher(n: int = 256, steps: int = 10000) -> Workload:
    """256^3 periodic, TRT, one pusher R = 16, beta = -3, B1 = 0.002."""
    c = n / 2.0
    return Workload(f"c3_pusher_{n}", (n, n, n), "trt", 1.0, steps,
                    [Body((c, c, c), (0.0, 0.0, 1.0), 16.0, 0.002, -3.0, True)])


def random_unit(rng) -> tuple:
    v = rng.standard_normal(3)
    v /= np.linalg.norm(v)
    return tuple(float(a) for a in v)


def c4_suspension(n: int = 256, count: int = 200, R: float = 6.0, min_dist: float = 34.0,
                  seed: int = 1903, steps: int = 5000) -> Workload:
    """256^3 periodic, 200 squirmers R = 6 placed by random sequential addition
    with minimum-image centre distance >= 34, random unit orientations,
    beta ~ U[-5, 5], B1 = 0.003."""
    rng = np.random.default_rng(seed)
    pts = []
    bodies = []
    tries = 0
    while len(pts) < count:
        tries += 1
        if tries > 200000:
            raise RuntimeError("placement failed")
        p = rng.uniform(0, n, 3)
        ok = True
        for q in pts:
            d = p - q
            d -= n * np.round(d / n)
            if d @ d < min_dist * min_dist:
                ok = False
                break
        if not ok:
            continue
        pts.append(p)
        bodies.append(Body(tuple(float(a) for a in p), random_unit(rng), R, 0.003,
                           float(rng.uniform(-5, 5)), True))
    return Workload(f"c4_suspension_{n}_{count}", (n, n, n), "trt", 1.0, steps, bodies)


def smooth_fields(shape, seed: int, drho: float = 0.01, umax: float = 0.02):
    """Smooth periodic random density and velocity fields (x-fastest, flattened):
    rho = 1 + drho * (sum of a few low Fourier modes), u likewise."""
    nx, ny, nz = shape
    rng = np.random.default_rng(seed)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")

    def mode():
        kx, ky, kz = rng.integers(0, 3, 3)
        ph = rng.uniform(0, 2 * math.pi)
        return np.sin(2 * math.pi * (kx * x / nx + ky * y / ny + kz * z / nz) + ph)

    rho = 1.0 + drho * (mode() + 0.5 * mode())
    u = np.stack([umax * (mode() + 0.5 * mode()) / 1.5 for _ in range(3)])
    return rho.reshape(-1), u.reshape(3, -1)


def random_populations(N: int, seed: int, base, spread: float = 0.1):
    """Random positive populations: base_i * (1 + spread * U[-1, 1]) per cell."""
    rng = np.random.default_rng(seed)
    base = np.asarray(base, dtype=np.float64).reshape(19, 1)
    return base * (1.0 + spread * rng.uniform(-1, 1, (19, N)))
