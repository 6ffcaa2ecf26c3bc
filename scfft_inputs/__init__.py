"""Seeded, synthetic inputs shared by the tests, the benchmark and the smoke check.

This module holds no arithmetic of the method itself: it builds voxel masks of
the solids (the superconductor Omega of §2), applied-field knot lists (§3),
grid/box choices and seeded random arrays.  Both the CUDA path and the CPU
oracle receive the arrays it makes; neither imports the other.

Node placement (cell centres x_i = -L + (i + 1/2) dx) is the same convention
both sides use; a node belongs to Omega iff its coordinates satisfy the solid's
closed inequalities, evaluated in float64 with no tolerance.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

__all__ = ["node_axes", "cube", "sphere", "cylinder", "shield", "lens", "biconical_lens", "disk_region",
           "Config", "config", "CONFIGS", "random_field", "jc_noise", "batch_configs", "shield_case_path"]


def node_axes(n, L):
    """Cell-centre coordinates along x, y, z for grid n=(nx,ny,nz), half extents L."""
    return tuple(-Lh + (np.arange(k) + 0.5) * (2.0 * Lh / k) for Lh, k in zip(L, n))


def _zyx(n, L):
    x, y, z = node_axes(n, L)
    return z[:, None, None], y[None, :, None], x[None, None, :]


def cube(n, L, side: float) -> np.ndarray:
    """|x|, |y|, |z| <= side/2."""
    Z, Y, X = _zyx(n, L)
    h = 0.5 * side
    return (np.abs(X) <= h) & (np.abs(Y) <= h) & (np.abs(Z) <= h)


def sphere(n, L, R: float) -> np.ndarray:
    Z, Y, X = _zyx(n, L)
    return X * X + Y * Y + Z * Z <= R * R


def cylinder(n, L, R: float, height: float) -> np.ndarray:
    """Solid cylinder r <= R, |z| <= height/2 (axis z)."""
    Z, Y, X = _zyx(n, L)
    return (X * X + Y * Y <= R * R) & (np.abs(Z) <= 0.5 * height)


def shield(n, L, R_out: float, R_in: float, height: float, cap: float) -> np.ndarray:
    """Hollow cylinder R_in <= r <= R_out, |z| <= height/2, sealed at the -z end by
    a solid disc r <= R_out of thickness cap."""
    Z, Y, X = _zyx(n, L)
    r2 = X * X + Y * Y
    zlo = -0.5 * height
    wall = (r2 >= R_in * R_in) & (r2 <= R_out * R_out) & (np.abs(Z) <= 0.5 * height)
    lid = (r2 <= R_out * R_out) & (Z >= zlo) & (Z <= zlo + cap)
    return wall | lid


def lens(n, L, R: float, height: float, bore: float, slit: float) -> np.ndarray:
    """Cylinder r <= R, |z| <= height/2 with a coaxial bore r < bore and a radial
    slit |y| < slit/2, x > 0 from the bore to the outer surface."""
    Z, Y, X = _zyx(n, L)
    r2 = X * X + Y * Y
    body = (r2 <= R * R) & (np.abs(Z) <= 0.5 * height)
    hole = r2 < bore * bore
    cut = (np.abs(Y) < 0.5 * slit) & (X > 0)
    return body & ~hole & ~cut


def biconical_lens(n, L, R: float, height: float, r_mid: float, r_face: float, slit: float) -> np.ndarray:
    """Cylinder r <= R, |z| <= height/2 with a coaxial biconical hole whose radius grows
    linearly from r_mid at z = 0 to r_face at |z| = height/2, and a radial slit |y| < slit/2,
    x > 0 from the hole to the outer surface (the lens shape of §3; its dimensions are
    readings, the paper gives them only in a figure)."""
    Z, Y, X = _zyx(n, L)
    r = np.sqrt(X * X + Y * Y)
    body = (r <= R) & (np.abs(Z) <= 0.5 * height)
    hole = r < r_mid + (r_face - r_mid) * np.abs(Z) / (0.5 * height)
    cut = (np.abs(Y) < 0.5 * slit) & (X > 0)
    return body & ~hole & ~cut


def disk_region(n, L, z_center: float, thickness: float, radius: float) -> np.ndarray:
    """Nodes of the coaxial disk r <= radius, |z - z_center| <= thickness/2 (an averaging zone)."""
    Z, Y, X = _zyx(n, L)
    return (X * X + Y * Y <= radius * radius) & (np.abs(Z - z_center) <= 0.5 * thickness) & (X * 0 == 0)


def shield_case_path(case: str, tau: float = 0.09):
    """Applied-field knots of the shield experiment of §3: case A ramps along the axis to tau,
    then perpendicular (h_e = (t - tau, 0, tau)); case B the same ramps in the inverse order."""
    if case == "A":
        return [0.0, tau, 2 * tau], [[0, 0, 0], [0, 0, tau], [tau, 0, tau]]
    if case == "B":
        return [0.0, tau, 2 * tau], [[0, 0, 0], [tau, 0, 0], [tau, 0, tau]]
    raise KeyError(case)


@dataclass
class Config:
    """One workload: grid, box, solid, material and applied-field path."""
    name: str
    n: tuple
    L: tuple
    mask: np.ndarray
    n_power: float
    rho_out: float
    knots_t: list
    knots_he: list
    sin_amp: float = 0.0
    sin_period: float = 1.0
    sin_t0: float = 0.0
    sin_t1: float = 0.0
    sin_dir: tuple = (0.0, 0.0, 1.0)
    rtol: float = 2e-4
    atol: float = 1e-6
    t_end: float = 1.0
    snapshots: list = field(default_factory=list)
    jc: object = 1.0
    note: str = ""


def config(name: str, scale: Optional[tuple] = None) -> Config:
    """The five workloads of the benchmark suite (shapes of the paper's shield and
    lens, §3).  `scale` overrides the grid (same box) for small parity copies."""
    if name == "cube16":
        n = scale or (16, 16, 16)
        L = (1.0, 1.0, 1.0)
        return Config(name, n, L, cube(n, L, 1.0), 20.0, 20.0,
                      [0.0, 1.0, 2.0], [[0, 0, 0], [0, 0, 0.5], [0, 0, 0]],
                      rtol=1e-6, atol=1e-6 * 0.5, t_end=2.0,
                      snapshots=[0.1 * (i + 1) for i in range(20)],
                      note="cube side 1, 16^3 grid, box side 2, z ramp 0->0.5->0 over [0,2]")
    if name == "shield64x64x96":
        n = scale or (64, 64, 96)
        L = (1.6, 1.6, 2.4)
        amp = 1.2 * (1.0 - 0.8)
        s = math.sqrt(0.5)
        d = (s, 0.0, s)
        tr = amp  # ramp at rate 1
        per = tr / 3.0
        return Config(name, n, L, shield(n, L, 1.0, 0.8, 3.0, 0.2), 25.0, 20.0,
                      [0.0, tr], [[0, 0, 0], [amp * d[0], amp * d[1], amp * d[2]]],
                      sin_amp=0.1 * amp, sin_period=per, sin_t0=tr, sin_t1=tr + 3 * per, sin_dir=d,
                      rtol=2e-4, atol=1e-6 * amp, t_end=tr + 3 * per,
                      note="shield R 1/0.8, height 3, cap 0.2, 45 deg field, ramp to 0.24 + 3 sine periods")
    if name == "lens128":
        n = scale or (128, 128, 128)
        L = (1.6, 1.6, 1.6)
        return Config(name, n, L, lens(n, L, 1.0, 1.0, 0.15, 0.05), 30.0, 100.0,
                      [0.0, 0.8], [[0, 0, 0], [0, 0, 0.8]],
                      rtol=2e-4, atol=1e-6 * 0.8, t_end=1.0,
                      note="lens R 1, height 1, bore 0.15, slit 0.05, axial ramp to 0.8 then hold")
    if name == "lens96":
        n = scale or (96, 96, 96)
        L = (1.6, 1.6, 1.6)
        return Config(name, n, L, lens(n, L, 1.0, 1.0, 0.15, 0.05), 30.0, 100.0,
                      [0.0, 0.8], [[0, 0, 0], [0, 0, 0.8]],
                      rtol=2e-4, atol=1e-6 * 0.8, t_end=1.0,
                      jc=jc_noise((n[2], n[1], n[0]), 1346),
                      note="lens at 96^3 with a seeded +-5% jc map")
    raise KeyError(name)


CONFIGS = ("cube16", "shield64x64x96", "lens128", "lens96")


def random_field(shape, seed: int, scale: float = 1.0) -> np.ndarray:
    """Seeded Gaussian float64 array."""
    return scale * np.random.default_rng(seed).standard_normal(shape)


def jc_noise(shape, seed: int, amp: float = 0.05) -> np.ndarray:
    """jc = 1 + U[-amp, amp] per node (seeded)."""
    return 1.0 + np.random.default_rng(seed).uniform(-amp, amp, size=shape)


def batch_configs(count: int = 64, seed: int = 1803) -> list:
    """Independent shield instances for batched runs: grids drawn from
    {32, 48, 64, 96}^3 in a cubic box of side 3.2, a hollow cylinder R 1 / 0.8,
    height 2, cap 0.2 (the shield shortened so that it keeps a margin in the
    cubic box), applied-field direction uniform on the sphere, ramp amplitude
    U[0.3, 1.5] x 0.2 (jc times the wall thickness) reached at rate 1, n drawn
    from {15, 25, 50}, rho_out = 20."""
    rng = np.random.default_rng(seed)
    out = []
    L = (1.6, 1.6, 1.6)
    for i in range(count):
        N = int(rng.choice([32, 48, 64, 96]))
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        amp = float(rng.uniform(0.3, 1.5) * 0.2)
        npow = float(rng.choice([15.0, 25.0, 50.0]))
        n = (N, N, N)
        out.append(Config(f"shield{N}_{i}", n, L, shield(n, L, 1.0, 0.8, 2.0, 0.2), npow, 20.0,
                          [0.0, amp, amp + 1.0], [[0, 0, 0], list(amp * d), list(amp * d)],
                          rtol=2e-4, atol=1e-6 * amp, t_end=amp + 1.0,
                          note=f"shield instance {i}: {N}^3, n={npow}, |h_e|={amp:.3f}"))
    return out
