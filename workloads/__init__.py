"""Seeded synthetic workloads for the thermocapillary phase-field LBM.

Coordinates are cell-centred: cell (i, j, k) sits at (i + 1/2, j + 1/2,
k + 1/2), so an n-cell axis spans [0, n] and its centre is n/2.  Walls are
the faces z = 0 and z = nz.  Heater patches are given by integer cell index.

This module is shared by the FP64 oracle and the CUDA path.  It holds only
*inputs*: lattice sizes, physical parameters, droplet and heater placements
drawn from a seeded ``numpy.random.Generator(PCG64(seed))``.  It contains
none of the method's arithmetic (no equilibria, no interface profile, no
forces); each side builds its initial state from these numbers on its own.

The five workloads stand in for the paper's own droplet set-ups (Sec. 3.3,
Sec. 3.4: droplets of radius R ~ 10-32 lu, interface width 4-5 lu, Gaussian
laser heat sources of width w_s = 6, Eq. HeatSource) and for its single-GPU
throughput study (Sec. 4.2).  There is no public dataset involved.
"""
from __future__ import annotations

import dataclasses
import math
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

# Thermal-scheme names, in the order the C ABI enumerates them.
THERMAL_SCHEMES = ("D3Q7", "D3Q15", "D3Q19", "D3Q27", "RK2", "RK4")
PRECISIONS = ("fp64", "fp32", "fp16")


@dataclass
class Params:
    """Physical/numerical parameters of one run (lattice units, dx = dt = 1)."""
    nu_L: float = 0.1            # kinematic viscosity, light phase (phi = 0)
    nu_H: float = 0.1            # kinematic viscosity, heavy phase (phi = 1)
    rho_L: float = 1.0           # density, light phase
    rho_H: float = 1.0           # density, heavy phase
    mobility: float = 0.02       # Allen-Cahn mobility M
    xi: float = 5.0              # interface width
    sigma_ref: float = 5e-3      # surface tension at T_ref
    sigma_T: float = -5e-4       # d sigma / d T
    T_ref: float = 0.0
    alpha_L: float = 0.05        # thermal conductivity kappa, light phase (the diffusivity when rho c_p = 1)
    alpha_H: float = 0.05        # thermal conductivity kappa, heavy phase
    gravity: tuple = (0.0, 0.0, 0.0)
    walls_z: bool = False        # no-slip walls at both z faces (x, y periodic)
    T_bottom: float = 0.0        # wall temperature at z = 0
    T_top: float = 0.0           # wall temperature at z = nz
    grad_T: tuple = (0.0, 0.0, 0.0)     # imposed background temperature gradient
    grad_T_origin: tuple = (0.0, 0.0, 0.0)  # point where the background part is 0
    eps_n: float = 1e-12         # regulariser of the interface normal
    omega_high: float = 1.0      # relaxation rate of central moments of order >= 3
    rk_isotropic_fd: bool = False  # RK path: isotropic D3Q27 operators instead of 7-point
    T_bottom_amp: float = 0.0    # bottom wall T_bottom + T_bottom_amp cos(2 pi k x / nx)
    T_bottom_waves: int = 0      # k (0: uniform bottom wall)
    wall_u_bottom: tuple = (0.0, 0.0)   # tangential (x, y) velocity of the bottom wall
    wall_u_top: tuple = (0.0, 0.0)      # tangential (x, y) velocity of the top wall
    theta_bottom: float = 90.0   # contact angle at the bottom wall, degrees, through phi = 1
    theta_top: float = 90.0      # contact angle at the top wall
    cp_L: float = 1.0            # specific heat capacity c_p, light phase
    cp_H: float = 1.0            # specific heat capacity c_p, heavy phase


@dataclass
class HeatSource:
    """Gaussian laser heat source, Eq. HeatSource: Q exp(-2 r^2 / w^2) for r <= d."""
    x: float
    y: float
    z: float
    Q: float
    w: float
    d: float = math.inf          # cut-off radius (inf = no cut-off)


@dataclass
class Droplet:
    cx: float
    cy: float
    cz: float
    R: float
    ux: float = 0.0
    uy: float = 0.0
    uz: float = 0.0


@dataclass
class HeaterPatches:
    """Rectangular heater patches on one z layer (the adjoint workload).

    Patch k covers x in [x0_k, x0_k + sx), y in [y0_k, y0_k + sy) on layer z;
    its heat source density is the intensity I_k.
    """
    z: int
    sx: int
    sy: int
    x0: List[int]
    y0: List[int]
    intensity: List[float]


@dataclass
class Workload:
    name: str
    nx: int
    ny: int
    nz: int
    steps: int
    params: Params
    droplets: List[Droplet]
    sources: List[HeatSource] = field(default_factory=list)
    patches: Optional[HeaterPatches] = None
    q_phase: int = 15            # phase-field stencil: 15 (D3Q15) or 27
    thermal: str = "D3Q7"
    precision: str = "fp64"
    target: Optional[tuple] = None  # adjoint objective target point

    @property
    def cells(self) -> int:
        return self.nx * self.ny * self.nz

    def replace(self, **kw) -> "Workload":
        return dataclasses.replace(self, **kw)


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _place_droplets(rng, n, box, r_lo, r_hi, gap, walls_z, wall_clear=3.0,
                    speed=0.0, max_tries=200000):
    """Rejection-sample n non-overlapping spheres (minimum-image distances)."""
    nx, ny, nz = box
    out: List[Droplet] = []
    tries = 0
    while len(out) < n:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("droplet placement failed; box too crowded")
        R = float(rng.uniform(r_lo, r_hi))
        cx = float(rng.uniform(0, nx))
        cy = float(rng.uniform(0, ny))
        if walls_z:
            lo = R + wall_clear
            hi = nz - R - wall_clear
            if hi <= lo:
                continue
            cz = float(rng.uniform(lo, hi))
        else:
            cz = float(rng.uniform(0, nz))
        ok = True
        for d in out:
            dx = cx - d.cx
            dx -= nx * round(dx / nx)
            dy = cy - d.cy
            dy -= ny * round(dy / ny)
            dz = cz - d.cz
            if not walls_z:
                dz -= nz * round(dz / nz)
            if math.sqrt(dx * dx + dy * dy + dz * dz) < R + d.R + gap:
                ok = False
                break
        if not ok:
            continue
        ux = uy = 0.0
        if speed:
            ang = float(rng.uniform(0, 2 * math.pi))
            ux, uy = speed * math.cos(ang), speed * math.sin(ang)
        out.append(Droplet(cx, cy, cz, R, ux, uy, 0.0))
    return out


def config1() -> Workload:
    """32^3 periodic, one droplet R = 8 at the centre, D3Q15 phase field,
    D3Q7 thermal LB, background gradient dT/dx = 1e-3, 200 steps, FP64."""
    p = Params(nu_L=0.1, nu_H=0.1, mobility=0.02, xi=5.0, sigma_ref=5e-3,
               sigma_T=-5e-4, T_ref=0.0, alpha_L=0.05, alpha_H=0.05,
               grad_T=(1e-3, 0.0, 0.0), grad_T_origin=(16.0, 16.0, 16.0))
    return Workload("cfg1_32cube_periodic", 32, 32, 32, 200, p,
                    [Droplet(16.0, 16.0, 16.0, 8.0)], q_phase=15,
                    thermal="D3Q7", precision="fp64")


def config2(thermal: str = "D3Q7", precision: str = "fp64") -> Workload:
    """64x64x128 channel, walls at z with T = -0.5 (bottom) / +0.5 (top),
    droplet R = 12, nu = 0.05, 5000 steps (thermocapillary migration)."""
    p = Params(nu_L=0.05, nu_H=0.05, mobility=0.02, xi=5.0, sigma_ref=5e-3,
               sigma_T=-5e-4, T_ref=0.0, alpha_L=0.05, alpha_H=0.05,
               walls_z=True, T_bottom=-0.5, T_top=0.5)
    return Workload("cfg2_64x64x128_walls", 64, 64, 128, 5000, p,
                    [Droplet(32.0, 32.0, 64.0, 12.0)], q_phase=15,
                    thermal=thermal, precision=precision)


def config3(precision: str = "fp32") -> Workload:
    """256x128x128 channel, walls at z (T = 0), four Gaussian heaters on the
    bottom wall (Q = 0.2, w = 6), three seeded droplets R ~ U[10, 16] moving
    at 1e-3 lu/step, sigma(T) = 1e-3 - 2e-4 T, D3Q7, 20000 steps."""
    rng = _rng(3)
    nx, ny, nz = 256, 128, 128
    p = Params(nu_L=0.05, nu_H=0.05, mobility=0.02, xi=5.0, sigma_ref=1e-3,
               sigma_T=-2e-4, T_ref=0.0, alpha_L=0.05, alpha_H=0.05,
               walls_z=True, T_bottom=0.0, T_top=0.0)
    sources = [HeatSource(float(rng.uniform(0, nx)), float(rng.uniform(0, ny)),
                          0.0, 0.2, 6.0) for _ in range(4)]
    drops = _place_droplets(rng, 3, (nx, ny, nz), 10.0, 16.0, 2 * p.xi, True,
                            speed=1e-3)
    return Workload("cfg3_256x128x128_capture", nx, ny, nz, 20000, p, drops,
                    sources, q_phase=15, thermal="D3Q7", precision=precision)


def config4(thermal: str = "D3Q7", precision: str = "fp32", n: int = 512,
            n_droplets: Optional[int] = None) -> Workload:
    """n^3 periodic throughput lattice (n = 512 by default), a seeded array of
    droplets (R ~ U[8, 20], gap >= 2 xi; 64 droplets at 512^3, the same
    density at other sizes), weak gradient dT/dx = 1e-4."""
    if n_droplets is None:
        n_droplets = max(1, int(round(64 * (n / 512.0) ** 3)))
    rng = _rng(4)
    p = Params(nu_L=0.05, nu_H=0.05, mobility=0.02, xi=5.0, sigma_ref=5e-3,
               sigma_T=-5e-4, T_ref=0.0, alpha_L=0.05, alpha_H=0.05,
               grad_T=(1e-4, 0.0, 0.0), grad_T_origin=(n / 2, n / 2, n / 2))
    drops = _place_droplets(rng, n_droplets, (n, n, n), 8.0, 20.0, 2 * p.xi,
                            False)
    return Workload(f"cfg4_{n}cube_periodic_{n_droplets}drops", n, n, n, 50, p,
                    drops, q_phase=15, thermal=thermal, precision=precision)


def config5(n: int = 64) -> Workload:
    """Adjoint workload: n^3 with walls at z (T = 0), 16 heater patches
    (4 x 4 grid of (n/4)^2 cells) on the first fluid layer, intensity 0.1,
    one droplet of radius 10 (n = 64) at a seeded offset, D3Q7."""
    rng = _rng(5)
    p = Params(nu_L=0.05, nu_H=0.05, mobility=0.02,
               xi=5.0 if n >= 32 else 3.0, sigma_ref=1e-3, sigma_T=-2e-4,
               T_ref=0.0, alpha_L=0.05, alpha_H=0.05, walls_z=True,
               T_bottom=0.0, T_top=0.0)
    s = n // 4
    x0 = [s * (k % 4) for k in range(16)]
    y0 = [s * (k // 4) for k in range(16)]
    patches = HeaterPatches(z=0, sx=s, sy=s, x0=x0, y0=y0,
                            intensity=[0.1] * 16)
    R = 10.0 * n / 64.0
    off = n / 8.0
    cx = n / 2 + float(rng.uniform(-off, off))
    cy = n / 2 + float(rng.uniform(-off, off))
    cz = 20.0 * n / 64.0
    steps = 2000 if n >= 64 else 200
    return Workload(f"cfg5_{n}cube_adjoint", n, n, n, steps, p,
                    [Droplet(cx, cy, cz, R)], patches=patches, q_phase=15,
                    thermal="D3Q7", precision="fp64",
                    target=(cx + 8.0 * n / 64.0, cy, cz))


def crop(w: Workload, nx: int, ny: int, nz: int) -> Workload:
    """Same parameters and droplet density on a smaller box (droplets whose
    centre falls inside the box are kept; used for bounded CPU samples)."""
    keep = [d for d in w.droplets if d.cx < nx and d.cy < ny and d.cz < nz]
    return w.replace(name=w.name + f"_crop{nx}x{ny}x{nz}", nx=nx, ny=ny, nz=nz,
                     droplets=keep)


def random_state(seed: int, shape, scale: float = 1.0) -> np.ndarray:
    """Seeded FP64 noise (used to perturb PDFs in parity tests)."""
    return _rng(seed).standard_normal(shape) * scale


def heater_field(seed: int, shape, peak: float = 2e-3) -> np.ndarray:
    """Seeded per-cell heat-source density, dense [z][y][x] FP64: a few
    randomly placed Gaussian spots of random width (the shape of laser
    heating) plus uniform background noise of 1 % of the peak."""
    rng = _rng(seed)
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz) + 0.5, np.arange(ny) + 0.5, np.arange(nx) + 0.5,
                          indexing="ij")
    q = 0.01 * peak * rng.uniform(0.0, 1.0, shape)
    for _ in range(3):
        c = rng.uniform(0.0, 1.0, 3) * np.array([nx, ny, nz])
        w = float(rng.uniform(2.0, 6.0))
        q += peak * float(rng.uniform(0.3, 1.0)) * np.exp(
            -2.0 * ((x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2) / (w * w))
    return q
