"""Workload definitions (grid, physics, boundary types, geometry) and seeded initial fields.

Every length is in grid units (dx = 1) unless a config says otherwise; the reference velocity is 1,
so nu = L_ref / Re and dt = CFL * dx / U.

Boundary-type codes (one per domain face, order x-, x+, y-, y+, z-, z+):
  0 periodic, 1 inflow (Dirichlet u_in), 2 outflow (zero normal gradient, p = 0), 3 slip wall,
  4 no-slip wall.
"""
from dataclasses import dataclass
from typing import Callable, Optional
import numpy as np

from . import soups

PERIODIC, INFLOW, OUTFLOW, SLIP, NOSLIP = 0, 1, 2, 3, 4
FP64, FP32_REFINE64 = 0, 1


@dataclass
class Config:
    name: str
    nx: int
    ny: int
    nz: int
    nu: float
    dt: float
    steps: int
    tol: float
    precision: int
    bc: tuple
    u_in: tuple = (1.0, 0.0, 0.0)
    dx: float = 1.0
    csm_on: int = 1
    forcing_on: int = 1
    deadend_on: int = 0
    soup: Optional[Callable] = None
    seed: int = 0
    a_ref: float = 1.0
    quick: float = 0.0
    integrator: int = 0          # 0 Adams-Bashforth 2, 1 Crank-Nicolson
    note: str = ""

    @property
    def ncell(self):
        return self.nx * self.ny * self.nz


CHANNEL = (INFLOW, OUTFLOW, SLIP, SLIP, SLIP, SLIP)
GROUND = (INFLOW, OUTFLOW, SLIP, SLIP, NOSLIP, SLIP)

CONFIGS = {
    "sphere_64x32x32": Config(
        "sphere_64x32x32", 64, 32, 32, nu=8.0 / 100.0, dt=0.2, steps=50, tol=1e-10,
        precision=FP64, bc=CHANNEL,
        soup=lambda: soups.icosphere(3, 4.0, (16.0, 16.0, 16.0)), seed=1,
        a_ref=np.pi * 8.0 ** 2 / 4.0,
        note="clean icosphere D=8 (1280 triangles), Re=100 on D, FP64"),
    "dirty_sphere_256x128x128": Config(
        "dirty_sphere_256x128x128", 256, 128, 128, nu=32.0 / 1e4, dt=0.2, steps=500, tol=1e-6,
        precision=FP32_REFINE64, bc=CHANNEL,
        soup=lambda: soups.dirty_sphere(seed=2), seed=2, a_ref=np.pi * 32.0 ** 2 / 4.0,
        note="dirty icosphere D=32 (holes, overlaps, jitter, nested shell, disk), Re=1e4"),
    "cube_plate_512x256x256": Config(
        "cube_plate_512x256x256", 512, 256, 256, nu=32.0 / 4e4, dt=0.2, steps=1000, tol=1e-6,
        precision=FP32_REFINE64, bc=GROUND,
        soup=soups.cube_and_plate, seed=3, a_ref=32.0 * 32.0,
        note="cube on a no-slip floor + 10 deg zero-thickness plate, Re=4e4 on the cube edge"),
    "vehicle_1024x512x384": Config(
        "vehicle_1024x512x384", 1024, 512, 384, nu=640.0 / 1e6, dt=0.2, steps=200, tol=1e-6,
        precision=FP32_REFINE64, bc=GROUND, deadend_on=1,
        soup=lambda: soups.vehicle_assembly(seed=4), seed=4, a_ref=240.0 * 160.0,
        note="union of 300 boxes/cylinders/plates, ~2M triangles, ground effect, Re=1e6"),
}


def get_config(name):
    return CONFIGS[name]


def initial_fields(cfg, dtype=np.float64, seed=None):
    """Uniform stream (1,0,0) plus a 1e-3 N(0,1) perturbation; returns u[3, nz, ny, nx]."""
    rng = np.random.default_rng(cfg.seed if seed is None else seed)
    u = 1e-3 * rng.standard_normal((3, cfg.nz, cfg.ny, cfg.nx))
    u[0] += cfg.u_in[0]
    u[1] += cfg.u_in[1]
    u[2] += cfg.u_in[2]
    return u.astype(dtype)


def taylor_green_velocity(x, y, t, re):
    """Analytic Taylor-Green velocity of Sec. 2.5 at physical points (x, y); returns [..., 3]."""
    f = np.exp(-2.0 * np.pi ** 2 * t / re)
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    return np.stack([-np.cos(np.pi * x) * np.sin(np.pi * y) * f, np.sin(np.pi * x) * np.cos(np.pi * y) * f,
                     np.zeros_like(x)], -1)


def taylor_green(n, t, re, nz=1, lo=-2.0, hi=2.0):
    """Analytic 2-D Taylor-Green vortex of Sec. 2.5 sampled at cell centres of an n x n x nz grid on
    [lo, hi]^2 (periodic); returns (u[3,nz,n,n], p[nz,n,n], dx)."""
    dx = (hi - lo) / n
    x = lo + (np.arange(n) + 0.5) * dx
    X, Y = np.meshgrid(x, x, indexing="xy")          # X varies along the last (x) axis
    f = np.exp(-2.0 * np.pi ** 2 * t / re)
    u1 = -np.cos(np.pi * X) * np.sin(np.pi * Y) * f
    u2 = np.sin(np.pi * X) * np.cos(np.pi * Y) * f
    p = -0.25 * (np.cos(2 * np.pi * X) + np.cos(2 * np.pi * Y)) * f * f
    u = np.zeros((3, nz, n, n))
    u[0] = u1[None]
    u[1] = u2[None]
    return u, np.broadcast_to(p[None], (nz, n, n)).copy(), dx
