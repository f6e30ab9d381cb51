"""Seeded synthetic inputs: dielectric media, pulse parameters and workload configs.

This module holds no step of the method. It only builds the index fields
n_x, n_y, n_z (float64, shape (Ny, Nx)) and the parameters that the method is
run with, so that the CUDA path and the CPU oracle are fed identical inputs.

The paper's own medium (a cone in n_z and a cylinder in n_x = n_y with
n_max = 3 in vacuum, Sec. 4, Fig. 2) is not specified beyond that, so the
workloads use smooth tanh-edged ellipses/cylinders in vacuum:

    n_i(x, y) = 1 + max_obj (n_i,obj - 1) * (1 - tanh(d / w)) / 2
    d = (rho - 1) * sqrt(a b),  rho = sqrt((x'/a)^2 + (y'/b)^2)

with (x', y') the site position in the object's rotated frame (for a circle of
radius R this is d = r - R). Sites sit at integer coordinates.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Sequence, Tuple

import numpy as np

POL_EZ = 0
POL_EY = 1


@dataclasses.dataclass(frozen=True)
class Ellipse:
    cx: float
    cy: float
    a: float
    b: float
    angle: float  # radians, rotation of the a-axis from +x
    n: Tuple[float, float, float]  # (n_x, n_y, n_z) inside
    w: float  # tanh edge width in cells


@dataclasses.dataclass(frozen=True)
class Pulse:
    pol: int  # POL_EZ or POL_EY
    x0: float
    sigma: float
    amp: float = 1.0


@dataclasses.dataclass
class Workload:
    name: str
    Nx: int
    Ny: int
    delta: float
    steps: int
    objects: List[Ellipse]
    pulse: Pulse
    precision: str = "fp32"

    def medium(self) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
        return medium(self.Nx, self.Ny, self.objects)

    @property
    def sites(self) -> int:
        return self.Nx * self.Ny


def medium(Nx: int, Ny: int, objects: Sequence[Ellipse]) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Index fields (n_x, n_y, n_z) of tanh-edged ellipses in vacuum (n = 1)."""
    y, x = np.meshgrid(np.arange(Ny, dtype=np.float64), np.arange(Nx, dtype=np.float64), indexing="ij")
    excess = np.zeros((3, Ny, Nx))
    for ob in objects:
        ca, sa = math.cos(ob.angle), math.sin(ob.angle)
        dx, dy = x - ob.cx, y - ob.cy
        xr = ca * dx + sa * dy
        yr = -sa * dx + ca * dy
        rho = np.sqrt((xr / ob.a) ** 2 + (yr / ob.b) ** 2)
        d = (rho - 1.0) * math.sqrt(ob.a * ob.b)
        prof = 0.5 * (1.0 - np.tanh(d / ob.w))
        for i in range(3):
            excess[i] = np.maximum(excess[i], (ob.n[i] - 1.0) * prof)
    n = 1.0 + excess
    return np.ascontiguousarray(n[0]), np.ascontiguousarray(n[1]), np.ascontiguousarray(n[2])


def cone_cylinder_medium(N: int, r_cone: float, r_cyl: float, n_max: float = 3.0, w: float = 8.0):
    """The anisotropic object of the paper's scattering runs (Sec. 4, Fig. 2),
    centred on an N x N lattice in vacuum: n_z conical (n_max at the centre,
    falling linearly to 1 at radius r_cone), n_x = n_y cylindrical (n_max
    inside radius r_cyl, a tanh edge of width w). The radii are not given in
    the paper; callers choose and record them."""
    y, x = np.meshgrid(np.arange(N, dtype=np.float64), np.arange(N, dtype=np.float64), indexing="ij")
    r = np.hypot(x - N / 2, y - N / 2)
    n_z = 1.0 + (n_max - 1.0) * np.clip(1.0 - r / r_cone, 0.0, None)
    n_xy = 1.0 + (n_max - 1.0) * 0.5 * (1.0 - np.tanh((r - r_cyl) / w))
    return np.ascontiguousarray(n_xy), np.ascontiguousarray(n_xy.copy()), np.ascontiguousarray(n_z)


def uniform_medium(Nx: int, Ny: int, n: Tuple[float, float, float]):
    return tuple(np.full((Ny, Nx), float(v)) for v in n)


def smooth_periodic_field(Nx: int, Ny: int, seed: int, kmax: int = 3, ncomp: int = 6) -> np.ndarray:
    """Random smooth periodic fields (a few low Fourier modes per component)."""
    rng = np.random.default_rng(seed)
    y, x = np.meshgrid(np.arange(Ny) / Ny, np.arange(Nx) / Nx, indexing="ij")
    out = np.zeros((ncomp, Ny, Nx))
    for c in range(ncomp):
        for kx in range(0, kmax + 1):
            for ky in range(-kmax, kmax + 1):
                if kx == 0 and ky <= 0:
                    continue
                amp = rng.normal() / (1.0 + kx * kx + ky * ky)
                ph = rng.uniform(0, 2 * math.pi)
                out[c] += amp * np.cos(2 * math.pi * (kx * x + ky * y) + ph)
    return out


def smooth_periodic_medium(Nx: int, Ny: int, seed: int, base=(1.5, 1.3, 1.8), amp=0.3, kmax: int = 2):
    """Smooth periodic anisotropic medium n_i = base_i (1 + amp * f_i), f_i of unit scale."""
    f = smooth_periodic_field(Nx, Ny, seed, kmax=kmax, ncomp=3)
    out = []
    for i in range(3):
        fi = f[i] / max(1e-12, np.abs(f[i]).max())
        out.append(np.ascontiguousarray(base[i] * (1.0 + amp * fi)))
    return tuple(out)


# ---------------------------------------------------------------------------
# Workloads (lattice sizes, delta, step counts and media of the five configs).
# ---------------------------------------------------------------------------

def workload_cylinder_256() -> Workload:
    """256^2, FP64, delta 0.1, 400 steps; one cylinder R 30 at the centre, edge 4,
    (n_x, n_y, n_z) = (1.5, 1.2, 2.0); E_z pulse at x0 60, sigma 8, amplitude 1."""
    return Workload("cylinder256_fp64", 256, 256, 0.1, 400,
                    [Ellipse(128.0, 128.0, 30.0, 30.0, 0.0, (1.5, 1.2, 2.0), 4.0)],
                    Pulse(POL_EZ, 60.0, 8.0, 1.0), precision="fp64")


def workload_ellipse_2048() -> Workload:
    """2048^2, FP32, delta 0.05, 10000 steps; ellipse semi-axes 200 x 120 rotated
    30 deg at the centre, edge 8, (2.0, 1.4, 1.1); E_y pulse sigma 40 at x0 512."""
    return Workload("ellipse2048_fp32", 2048, 2048, 0.05, 10000,
                    [Ellipse(1024.0, 1024.0, 200.0, 120.0, math.radians(30.0), (2.0, 1.4, 1.1), 8.0)],
                    Pulse(POL_EY, 512.0, 40.0, 1.0))


def workload_cylinders_8192(seed: int = 3, N: int = 8192) -> Workload:
    """8192^2, FP32, delta 0.02, 20000 steps; three seeded cylinders R in [100, 400],
    n_i uniform in [1.1, 3.0], edge 8; E_z pulse sigma 100 at x0 1024. With N < 8192
    the same recipe with every length (radii, margins, pulse position and width)
    scaled by N/8192 (a smaller case of the same kernel configuration)."""
    rng = np.random.default_rng(seed)
    f = N / 8192.0
    x0, sigma = 1024.0 * f, 100.0 * f
    objs = []
    for _ in range(3):
        R = float(rng.uniform(100.0, 400.0)) * f
        n = tuple(float(v) for v in rng.uniform(1.1, 3.0, size=3))
        yc = float(rng.uniform(R + 64.0 * f, N - R - 64.0 * f))
        xc = float(rng.uniform(x0 + 3 * sigma, x0 + 3 * sigma + 400.0 * f)) + R
        objs.append(Ellipse(xc, yc, R, R, 0.0, n, 8.0))
    return Workload(f"cylinders{N}_fp32", N, N, 0.02, 20000, objs, Pulse(POL_EZ, x0, sigma, 1.0))


BATCH_SIDES = (256, 384, 512, 768, 1024, 1536, 2048)


def random_ellipse_workload(rng: np.random.Generator, side: int, name: str, delta: float,
                            steps: int) -> Workload:
    """One instance: 1-3 ellipses with semi-axes 5-25% of the side, n_i in [1.0, 3.0],
    random polarisation, sigma 2-5% of the side, pulse at x0 = side/8."""
    nobj = int(rng.integers(1, 4))
    objs = []
    for _ in range(nobj):
        a = float(rng.uniform(0.05, 0.25)) * side
        b = float(rng.uniform(0.05, 0.25)) * side
        cx = float(rng.uniform(0.45, 0.75)) * side
        cy = float(rng.uniform(0.3, 0.7)) * side
        ang = float(rng.uniform(0.0, math.pi))
        n = tuple(float(v) for v in rng.uniform(1.0, 3.0, size=3))
        objs.append(Ellipse(cx, cy, a, b, ang, n, max(2.0, side / 256.0)))
    pol = int(rng.integers(0, 2))
    sigma = float(rng.uniform(0.02, 0.05)) * side
    return Workload(name, side, side, delta, steps, objs, Pulse(pol, side / 8.0, sigma, 1.0))


def workload_batch64(seed: int = 4, n: int = 64, delta: float = 0.05,
                     steps_range=(2000, 8000)) -> List[Workload]:
    """64 instances, sides from {256, ..., 2048}, 2000-8000 steps each."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        side = int(rng.choice(BATCH_SIDES))
        steps = int(rng.integers(steps_range[0], steps_range[1] + 1))
        out.append(random_ellipse_workload(rng, side, f"batch{i:02d}_{side}", delta, steps))
    return out


def workload_surrogate_1024(seed: int) -> Workload:
    """1024^2, delta 0.05; 1-3 ellipses, n_i in [1.0, 3.0], random polarisation,
    sigma in [20, 60], pulse at x0 128 (training / evaluation trajectories)."""
    rng = np.random.default_rng(seed)
    w = random_ellipse_workload(rng, 1024, f"surrogate_{seed}", 0.05, 4000)
    sigma = float(rng.uniform(20.0, 60.0))
    w.pulse = Pulse(w.pulse.pol, 128.0, sigma, 1.0)
    return w
