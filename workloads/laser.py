"""Seeded synthetic inputs for the laser-envelope advance.

Describes problems only; no part of the envelope arithmetic lives here, so the
FP64 CPU oracle and the CUDA library are fed the same arrays.  Units are the
paper's normalised ones (k_p = 1).  The demonstration follows the paper's
laser-driven blowout (Sec. 7.3, Table 1): omega_0 / omega_p = 20, base slice
0.08, a box of 25 k_p^-1 (here 24.0 so that 256 cells give h = 0.094).
Arrays are [slice, iy, ix] on the cell-centred grid of the slice advance.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Tuple

import numpy as np

__all__ = ["LaserWorkload", "LASER_WORKLOADS", "laser_workload", "gaussian_pulse",
           "bubble_susceptibility", "cell_centres"]


@dataclasses.dataclass(frozen=True)
class LaserWorkload:
    name: str
    n: int              # cells per side
    width: float        # box side (k_p^-1)
    n_xi: int           # slices
    dxi: float          # slice spacing
    k0: float           # omega_0 / omega_p
    dt: float           # time step (1/omega_p)
    a0: float = 2.0     # peak normalised vector potential
    w0: float = 3.0     # spot size (1/e of the field)
    sigma_xi: float = 2.0
    xi_c: float = 4.0   # pulse centre behind the window head
    bubble_radius: float = 4.0
    tol: float = 1e-10


def cell_centres(n: int, width: float) -> np.ndarray:
    h = width / n
    return -0.5 * width + (np.arange(n) + 0.5) * h


def gaussian_pulse(wl: LaserWorkload) -> np.ndarray:
    """A = a0 exp(-r^2 / w0^2 - (xi - xi_c)^2 / sigma_xi^2), complex128."""
    x = cell_centres(wl.n, wl.width)
    X, Y = np.meshgrid(x, x)
    xi = (np.arange(wl.n_xi) + 0.5) * wl.dxi
    env = np.exp(-((xi - wl.xi_c) / wl.sigma_xi) ** 2)
    a = wl.a0 * env[:, None, None] * np.exp(-(X * X + Y * Y) / wl.w0 ** 2)[None]
    return a.astype(np.complex128)


def bubble_susceptibility(wl: LaserWorkload) -> np.ndarray:
    """chi = n_* / (1 + psi) of a synthetic blowout: 1 ahead of the pulse
    centre, then a cavity of the given radius whose radius follows a circle in
    xi, a compressed sheath around it; float64 [n_xi, n, n]."""
    x = cell_centres(wl.n, wl.width)
    X, Y = np.meshgrid(x, x)
    r = np.sqrt(X * X + Y * Y)[None]
    xi = (np.arange(wl.n_xi) + 0.5) * wl.dxi
    d = xi - wl.xi_c
    rb = np.sqrt(np.clip(wl.bubble_radius ** 2 - (d - wl.bubble_radius) ** 2, 0.0, None))
    rb = rb[:, None, None]
    cavity = 1.0 / (1.0 + np.exp(-(r - rb) / 0.1))
    sheath = 2.0 * np.exp(-((r - rb - 0.3) / 0.3) ** 2) * (rb > 0)
    return np.ascontiguousarray(cavity * (1.0 + sheath), dtype=np.float64)


LASER_WORKLOADS = {
    # 256^2 cells, 256 slices of 0.08 (a 20.5 k_p^-1 window), k0 = 20, dt = 5
    "laser256": LaserWorkload(name="laser256", n=256, width=24.0, n_xi=256, dxi=0.08,
                              k0=20.0, dt=5.0),
}


def laser_workload(name: str) -> LaserWorkload:
    return LASER_WORKLOADS[name]
