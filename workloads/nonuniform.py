"""Seeded synthetic inputs for the nonuniform transverse grid.

This module describes grids and source fields only; it holds no part of the
field-solver arithmetic, so the FP64 CPU oracle and the CUDA library are fed
the same arrays without sharing any of the method's code.

Layout: an axis is given by its n + 2 node coordinates, strictly increasing;
the first and the last are the walls (where the fields are zero) and the n
nodes between them are the unknowns.  2D arrays are indexed [iy, ix] with ix
fastest.  The multigrid hierarchy takes every other node, so n = 2^k - 1.

The three-region profile follows the demonstration of Sec. "Multigrid Solver
with Nonuniform Grids" (Fig. 5(c)): the densest spacing on the axis where the
bunches are (region III), an intermediate one across the bubble and its sheath
(region II), and the coarsest in the quiet plasma (region I), with spacing
ratios 3 : ~1.4-2 : 1 against the densest.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, Tuple

import numpy as np

__all__ = [
    "uniform_axis",
    "alternating_axis",
    "three_region_axis",
    "NonuniformWorkload",
    "NONUNIFORM_WORKLOADS",
    "nonuniform_workload",
    "bubble_sources",
]


def uniform_axis(n: int, half_width: float) -> np.ndarray:
    """n interior nodes, equal spacing 2 half_width / (n + 1), walls included."""
    return np.linspace(-half_width, half_width, n + 2)


def alternating_axis(n: int, half_width: float, ratio: float = 2.0,
                     first_long: bool = False) -> np.ndarray:
    """Spacings alternating h, ratio*h (or ratio*h, h) across [-hw, hw].

    Every interior node then has a left and a right spacing that differ by a
    fixed factor, the largest local non-uniformity a grid refinement keeps.
    n + 1 (the number of intervals) must be even."""
    if (n + 1) % 2:
        raise ValueError("alternating_axis needs an even number of intervals")
    pattern = np.array([ratio, 1.0] if first_long else [1.0, ratio])
    steps = np.tile(pattern, (n + 1) // 2)
    steps *= 2.0 * half_width / steps.sum()
    x = np.concatenate([[0.0], np.cumsum(steps)]) - half_width
    x[-1] = half_width
    return x


def _three_region_spacing(r: np.ndarray) -> np.ndarray:
    """Target spacing versus |x| before scaling: 0.05 on the beam axis
    (|x| < 0.8), 0.1 inside the bubble, 0.07 across the sheath (2.8 < |x| <
    4.3), 0.15 in the quiet plasma; linear ramps of 0.5 between regions."""
    knots_r = np.array([0.0, 0.8, 1.3, 2.3, 2.8, 4.3, 4.8, 1e9])
    knots_h = np.array([0.05, 0.05, 0.10, 0.10, 0.07, 0.07, 0.15, 0.15])
    return np.interp(np.abs(r), knots_r, knots_h)


def three_region_axis(n: int, half_width: float) -> np.ndarray:
    """Symmetric node coordinates whose local spacing follows the three-region
    profile, scaled so that exactly n + 1 intervals span [-hw, hw].

    The map is the inverse of s(x) = int_0^x dx' / spacing(x'), sampled at
    equal steps of s; n + 1 must be even so that x = 0 is a node."""
    if (n + 1) % 2:
        raise ValueError("three_region_axis needs an even number of intervals")
    xf = np.linspace(0.0, half_width, 200_001)
    inv = 1.0 / _three_region_spacing(xf)
    s = np.concatenate([[0.0], np.cumsum(0.5 * (inv[1:] + inv[:-1]) * np.diff(xf))])
    half = (n + 1) // 2
    targets = np.linspace(0.0, s[-1], half + 1)
    pos = np.interp(targets, s, xf)
    pos[0], pos[-1] = 0.0, half_width
    return np.concatenate([-pos[::-1], pos[1:]])


@dataclasses.dataclass(frozen=True)
class NonuniformWorkload:
    """A field-solve problem on a nonuniform transverse grid."""

    name: str
    n: int                 # interior nodes per side, 2^k - 1
    half_width: float      # box [-hw, hw]^2
    profile: str           # "three_region" | "uniform" | "alternating"
    bubble_radius: float = 3.0
    mg_tol: float = 1e-10

    def axis(self) -> np.ndarray:
        if self.profile == "three_region":
            return three_region_axis(self.n, self.half_width)
        if self.profile == "alternating":
            return alternating_axis(self.n, self.half_width)
        return uniform_axis(self.n, self.half_width)


def bubble_sources(xn: np.ndarray, yn: np.ndarray, radius: float = 3.0) -> Dict[str, np.ndarray]:
    """Synthetic right-hand sides and screening of one blowout slice.

    Electron density n_e(r): zero inside a bubble of the given radius, a
    compressed sheath just outside it, 1 far away.  From it:
      psi : n_e - 1                       (Poisson source)
      ez  : radial ring dipole             (Poisson source)
      bz  : weak quadrupole                (Poisson source)
      bx, by : azimuthal ring current      (screened sources)
      m   : -n_e / (1 + psi_0(r)),  psi_0 the bubble's potential well
    Every source decays to round-off level well before the walls.  Arrays are
    float64 [ny, nx] on the interior nodes."""
    x = xn[1:-1][None, :]
    y = yn[1:-1][:, None]
    r = np.sqrt(x * x + y * y)
    step = 1.0 / (1.0 + np.exp(-(r - radius) / 0.08))
    sheath = (radius / 0.5) * np.exp(-((r - radius - 0.15) / 0.25) ** 2) / math.sqrt(math.pi)
    n_e = step * (1.0 + 0.5 * sheath)
    well = 0.25 * radius * radius * np.exp(-(r / radius) ** 4)
    ring = np.exp(-((r - radius) / 0.35) ** 2)
    out = {
        "psi": (n_e - 1.0) * np.exp(-(r / (2.5 * radius)) ** 8),
        "ez": (r - radius) * ring,
        "bz": 0.1 * x * y * np.exp(-r * r / 4.0),
        "bx": y * ring,
        "by": -x * ring,
        "m": -n_e / (1.0 + well),
    }
    return {k: np.ascontiguousarray(np.broadcast_to(v, r.shape), dtype=np.float64)
            for k, v in out.items()}


# The demonstration grid of the nonuniform-grid section: 255 x 255 nodes on a
# three-region profile (the paper seeds 250 x 250 cells), the width that a
# uniform 0.05 grid would cover with 500 cells.
NONUNIFORM_WORKLOADS = {
    "nonuni255": NonuniformWorkload(name="nonuni255", n=255, half_width=12.5,
                                    profile="three_region"),
    "nonuni63": NonuniformWorkload(name="nonuni63", n=63, half_width=12.5,
                                   profile="three_region"),
}


def nonuniform_workload(name: str) -> NonuniformWorkload:
    return NONUNIFORM_WORKLOADS[name]


def driver_current_nodes(xn: np.ndarray, yn: np.ndarray, n_xi: int, xi_len: float,
                         amplitude: float, sigma_r: float, sigma_z: float,
                         xi_c: float) -> np.ndarray:
    """j_z of a bi-Gaussian electron driver, amplitude exp(-r^2/sigma_r^2 -
    (xi - xi_c)^2/sigma_z^2) (Sec. 5.1's convention, v_z = 1), at the interior
    nodes of the base slices xi_j = j xi_len / n_xi: float64 [n_xi, ny, nx]."""
    X, Y = np.meshgrid(np.asarray(xn)[1:-1], np.asarray(yn)[1:-1])
    xi = np.arange(n_xi) * xi_len / n_xi
    prof = np.exp(-((xi - xi_c) / sigma_z) ** 2)
    return np.ascontiguousarray(amplitude * prof[:, None, None] *
                                np.exp(-(X * X + Y * Y) / sigma_r ** 2)[None])
