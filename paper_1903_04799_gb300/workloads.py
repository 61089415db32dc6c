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


def two_squirmers_passing(d: float = 27.0, n: int = 250, R: float = 9.0, beta: float = 5.0,
                          B1: float = 0.003, steps: int = 60000) -> Workload:
    """Two pullers (beta = 5, R = 9) in a 250^3 periodic box, facing each other
    12R apart along z with lateral offset d along y: centres
    (c, c + d/2, c - 6R) with e = +z and (c, c - d/2, c + 6R) with e = -z,
    c = n/2.  The pair is symmetric under the half turn about the x axis
    through (c, c), which maps the lattice onto itself.  B1 = 0.003 gives
    v0 = 0.002 and a Reynolds number 2 v0 R / nu of 0.22; 60 000 steps carry
    each sphere about 120 lattice units, past the other."""
    c = n / 2.0
    return Workload(f"two_squirmers_passing_{n}_d{d:g}", (n, n, n), "trt", 1.0, steps,
                    [Body((c, c + d / 2, c - 6 * R), (0.0, 0.0, 1.0), R, B1, beta, True),
                     Body((c, c - d / 2, c + 6 * R), (0.0, 0.0, -1.0), R, B1, beta, True)])


@dataclass
class TubeRun:
    """A squirmer in a round tube (Sec. V, "Squirmer in a Round Tube")."""
    name: str
    shape: tuple
    axis: tuple      # (cx, cy) of the tube axis (along z)
    radius: float    # nodes at distance >= radius from the axis are wall
    body: Body
    steps: int
    contact: tuple   # (sigma, eps) of the WCA contact force

    @property
    def cells(self) -> int:
        return int(np.prod(self.shape))


def tube_oscillation(y0_over_R: float = -1.0, R: float = 9.0, B1: float = 0.01, steps: int = 200000) -> TubeRun:
    """Sec. V tube flow: a neutral squirmer (beta = 0, R = 9) in a round tube of
    diameter D = 20R/3 = 60 and length 3 pi R = 85 (periodic along the
    axis), starting parallel to the axis at a lateral displacement y0 (in
    units of R) from it.  The fluid nodes are those within D/2 of the axis
    (the tube wall is bounced back half-way, so the wall sits near D/2 + 1/2);
    the box is D + 4 cells wide with the axis at its centre (31.5, 31.5), the
    midpoint between two nodes, so that a squirmer on the axis is
    mirror-symmetric.  B1 (not printed in the paper) = 0.01: Reynolds number
    2 v0 R / nu = 0.72; the WCA contact force (sigma = 1, eps = 0.01) keeps
    the squirmer off the wall."""
    D = 20.0 * R / 3.0
    n = int(round(D)) + 4
    L = int(round(3.0 * math.pi * R))
    c = (n - 1) / 2.0
    z0 = L / 2.0 + 0.3
    return TubeRun(f"tube_R{R:g}_y0{y0_over_R:+g}", (n, n, L), (c, c), D / 2.0,
                   Body((c, c + y0_over_R * R, z0), (0.0, 0.0, 1.0), R, B1, 0.0, True), steps, (1.0, 0.01))


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


@dataclass
class ServeRequest:
    """One request of the serving mix (a dict of lb_request fields)."""
    arrival: float
    geometry: int
    shape: tuple
    storage: str
    R: float
    beta: float
    B1: float
    steps: int
    pos: tuple
    e: tuple
    obstacle: tuple = (0.0, 0.0, 0.0, 0.0)
    wca: tuple = (1.0, 0.0)

    @property
    def cells(self) -> int:
        return int(np.prod(self.shape))


def serving_mix(n: int = 256, seed: int = 190304799, rate: float = 4.0, steps_range=(2000, 20000),
                edge_range=(32, 160)) -> list:
    """The serving mix: n requests with exponential inter-arrival times (mean
    1/rate s); geometry uniform over {periodic box, square tube, box with a
    fixed obstacle}; squirmer R ~ U[3, 12], beta ~ U[-5, 5], B1 = 0.004,
    steps ~ U[steps_range]; storage FP16-deviation or FP32 by a fair coin.
      box:      cubic, edge ~ U[edge_range] (raised to 2R + 8 if smaller),
                squirmer at the centre, random orientation;
      tube:     (4R + 2)^2 cross-section (walls at 0 and 4R + 1), length 16R,
                squirmer on the axis tilted by at most 0.2 rad;
      obstacle: cubic box of edge max(8R + 8, U[edge_range]), obstacle of
                radius 2R at the centre, squirmer 2R + R + 4 away on a random
                axis, aimed at the obstacle with a small offset angle; WCA
                contact force (sigma 1, eps 0.01) on."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for _ in range(n):
        t += float(rng.exponential(1.0 / rate))
        geo = int(rng.integers(0, 3))
        R = float(rng.uniform(3.0, 12.0))
        beta = float(rng.uniform(-5.0, 5.0))
        steps = int(rng.integers(steps_range[0], steps_range[1] + 1))
        steps += steps % 2
        storage = "f16dev" if rng.random() < 0.5 else "f32"
        if geo == 0:
            L = max(int(rng.integers(edge_range[0], edge_range[1] + 1)), int(math.ceil(2 * R)) + 8)
            shape = (L, L, L)
            pos = (L / 2 + 0.25, L / 2 - 0.15, L / 2 + 0.05)
            out.append(ServeRequest(t, 0, shape, storage, R, beta, 0.004, steps, pos, random_unit(rng)))
        elif geo == 1:
            w = int(math.ceil(4 * R)) + 2
            length = int(math.ceil(16 * R))
            tilt = float(rng.uniform(0.0, 0.2))
            phi = float(rng.uniform(0.0, 2 * math.pi))
            e = (math.sin(tilt) * math.cos(phi), math.sin(tilt) * math.sin(phi), math.cos(tilt))
            pos = (w / 2 - 0.5 + 0.1, w / 2 - 0.5 - 0.1, length / 2)
            out.append(ServeRequest(t, 1, (w, w, length), storage, R, beta, 0.004, steps, pos, e,
                                    wca=(1.0, 0.01)))
        else:
            A = 2 * R
            L = max(int(math.ceil(8 * R)) + 8, int(rng.integers(edge_range[0], edge_range[1] + 1)))
            c = L / 2
            axis = int(rng.integers(0, 3))
            gap = A + R + 4.0
            pos = [c, c, c]
            pos[axis] -= gap
            off = float(rng.uniform(0.02, 0.1))
            e = [0.0, 0.0, 0.0]
            e[axis] = 1.0
            e[(axis + 1) % 3] = off
            out.append(ServeRequest(t, 2, (L, L, L), storage, R, beta, 0.004, steps, tuple(pos), tuple(e),
                                    obstacle=(c, c, c, A), wca=(1.0, 0.01)))
    return out
