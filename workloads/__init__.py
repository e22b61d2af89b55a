"""Seeded synthetic workloads for the quasi-static slice advance.

This module only *describes* problems and draws the random numbers that a
problem needs (driver-beam macroparticles).  It holds no part of the
slice-advance arithmetic, so both the FP64 CPU oracle and the CUDA library can
be fed the same arrays without sharing any code of the method.

Units are the paper's normalised units (Sec. 3 opening paragraph): lengths in
k_p^-1, momenta in mc, densities in n0.  Driver beams use the bi-Gaussian
density n_b * exp(-r^2/sigma_r^2 - (xi-xi_c)^2/sigma_z^2) of Sec. 5.1 (no factor
of 2 in the exponent), so a macroparticle coordinate is distributed as a normal
with standard deviation sigma/sqrt(2).  The total number of beam electrons in
units of n0 k_p^-3 is n_b pi^(3/2) sigma_x sigma_y sigma_z and the paper's
normalised charge is Q = that number / (4 pi) (Sec. 5.1).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Tuple

import numpy as np

__all__ = [
    "BeamSpec",
    "Workload",
    "beam_from_normals",
    "beam_normals",
    "sample_beam",
    "beam_total_number",
    "normalised_charge",
    "radial_profile_table",
    "WORKLOADS",
    "workload",
]


@dataclasses.dataclass(frozen=True)
class BeamSpec:
    """One bi-Gaussian bunch.

    amplitude      peak density n_b / n0
    sigma_x/y/z    e-folding lengths of the density (k_p^-1), paper convention
    x_c, y_c, xi_c centroid; xi is measured backwards from the window head
    tilt           centroid slope dx_c/dxi (0 = straight bunch)
    gamma          Lorentz factor of every macroparticle (cold beam)
    n_particles    number of macroparticles
    seed           numpy Generator seed for the normals
    charge         charge in units of e (electron = -1)
    q_over_m       charge-to-mass ratio in units of e/m (electron = -1)
    """

    amplitude: float
    sigma_x: float
    sigma_y: float
    sigma_z: float
    xi_c: float
    n_particles: int
    seed: int
    x_c: float = 0.0
    y_c: float = 0.0
    tilt: float = 0.0
    gamma: float = 2000.0
    charge: float = -1.0
    q_over_m: float = -1.0

    def with_(self, **kw) -> "BeamSpec":
        return dataclasses.replace(self, **kw)


@dataclasses.dataclass(frozen=True)
class Workload:
    """A complete problem: transverse grid, xi window, plasma and drivers."""

    name: str
    n: int                      # transverse cells per side (square grid)
    half_width: float           # box is [-half_width, half_width]^2
    n_xi: int                   # base xi slices
    xi_len: float               # window length; xi in [0, xi_len)
    ppc: int                    # plasma macroparticles per cell (a square)
    beams: Tuple[BeamSpec, ...]
    profile: Optional[Tuple[Tuple[float, ...], float]] = None  # (n at radii, r_max)
    precision: str = "fp64"     # "fp64" | "fp32r"
    steps: int = 1
    dt: float = 10.0
    refine_k: int = 8
    mg_tol: float = 1e-10
    psi_floor: float = 1e-3

    @property
    def h(self) -> float:
        return 2.0 * self.half_width / self.n

    @property
    def dxi0(self) -> float:
        return self.xi_len / self.n_xi

    @property
    def n_plasma(self) -> int:
        return self.n * self.n * self.ppc

    def with_(self, **kw) -> "Workload":
        return dataclasses.replace(self, **kw)


def beam_normals(n: int, seed: int) -> np.ndarray:
    """Standard normals (3, n) for x, y, xi from numpy's PCG64 generator."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((3, n))


def beam_total_number(spec: BeamSpec) -> float:
    """Integral of the bi-Gaussian density: n_b pi^(3/2) sx sy sz (n0 k_p^-3)."""
    return spec.amplitude * math.pi ** 1.5 * spec.sigma_x * spec.sigma_y * spec.sigma_z


def normalised_charge(spec: BeamSpec) -> float:
    """Q = k_p^3 q / (4 pi e n0) of Sec. 5.1."""
    return beam_total_number(spec) / (4.0 * math.pi)


def beam_from_normals(spec: BeamSpec, z: np.ndarray) -> dict:
    """Map standard normals to macroparticles of `spec` (float64 SoA dict).

    x  = x_c + tilt*(xi - xi_c) + sigma_x/sqrt2 * z0
    y  = y_c + sigma_y/sqrt2 * z1
    xi = xi_c + sigma_z/sqrt2 * z2
    Every macroparticle carries the same weight (number of electrons in units
    of n0 k_p^-3) and the momentum (0, 0, sqrt(gamma^2-1)).
    """
    n = z.shape[1]
    s2 = math.sqrt(2.0)
    xi = spec.xi_c + spec.sigma_z / s2 * z[2]
    x = spec.x_c + spec.tilt * (xi - spec.xi_c) + spec.sigma_x / s2 * z[0]
    y = spec.y_c + spec.sigma_y / s2 * z[1]
    pz = math.sqrt(spec.gamma * spec.gamma - 1.0)
    w = beam_total_number(spec) / n
    return {
        "x": np.ascontiguousarray(x, dtype=np.float64),
        "y": np.ascontiguousarray(y, dtype=np.float64),
        "xi": np.ascontiguousarray(xi, dtype=np.float64),
        "px": np.zeros(n),
        "py": np.zeros(n),
        "pz": np.full(n, pz),
        "w": np.full(n, w),
        "charge": float(spec.charge),
        "q_over_m": float(spec.q_over_m),
    }


def sample_beam(spec: BeamSpec) -> dict:
    """Draw the macroparticles of one bunch (deterministic for a given seed)."""
    return beam_from_normals(spec, beam_normals(spec.n_particles, spec.seed))


def radial_profile_table(fn, r_max: float, n_coef: int) -> Tuple[Tuple[float, ...], float]:
    """Tabulate a transverse density profile n(r) at n_coef equispaced radii on
    [0, r_max]; the library interpolates the table piecewise-linearly and holds
    the last value beyond r_max."""
    r = np.linspace(0.0, r_max, n_coef)
    return tuple(float(v) for v in fn(r)), float(r_max)


def _driver(amplitude, sr, sz, n, seed, xi_c=None, **kw) -> BeamSpec:
    return BeamSpec(amplitude=amplitude, sigma_x=sr, sigma_y=sr, sigma_z=sz,
                    xi_c=3.0 * sz if xi_c is None else xi_c, n_particles=n,
                    seed=seed, **kw)


def _c4_instances() -> List[Workload]:
    out = []
    sizes = (128, 192, 256)
    for i in range(48):
        nb = 0.5 + 7.5 * i / 47.0
        sr = 0.3 + 0.5 * i / 47.0
        out.append(Workload(
            name=f"scan{i:02d}", n=sizes[i % 3], half_width=8.0, n_xi=512,
            xi_len=12.0, ppc=4,
            beams=(_driver(nb, sr, 0.7, 100_000, seed=i),),
            precision="fp32r"))
    return out


# The five problem families (transverse grid, window, plasma, drivers).
# Choices the problem statement leaves open: driver centre xi_c = 3 sigma_z,
# witness 4.5 behind the driver, window 12 (16 for the 512^2 case), dt = 10.
WORKLOADS = {
    "linear64": Workload(
        name="linear64", n=64, half_width=6.0, n_xi=128, xi_len=12.0, ppc=4,
        beams=(_driver(0.3, 0.5, 1.0, 20_000, seed=0),), precision="fp64",
        steps=1),
    "blowout256": Workload(
        name="blowout256", n=256, half_width=8.0, n_xi=1024, xi_len=12.0, ppc=4,
        beams=(_driver(5.0, 0.3, 0.7, 500_000, seed=0),
               _driver(2.0, 0.3, 0.3, 200_000, seed=1, xi_c=2.1 + 4.5)),
        precision="fp64", steps=50),
    "blowout512": Workload(
        name="blowout512", n=512, half_width=10.0, n_xi=2048, xi_len=16.0, ppc=9,
        beams=(_driver(10.0, 1.0, 1.21, 2_000_000, seed=0),),
        profile=radial_profile_table(lambda r: 1.0 + 0.05 * r * r, 10.0 * math.sqrt(2.0), 257),
        precision="fp32r", steps=20),
    "grad256": Workload(
        name="grad256", n=256, half_width=8.0, n_xi=512, xi_len=12.0, ppc=4,
        beams=(_driver(5.0, 0.3, 0.7, 500_000, seed=0),
               _driver(2.0, 0.3, 0.3, 200_000, seed=1, xi_c=2.1 + 4.5)),
        profile=(tuple([1.0] * 16), 8.0 * math.sqrt(2.0)),
        precision="fp64", steps=1),
}


def workload(name: str) -> Workload:
    return WORKLOADS[name]


def scan_instances() -> List[Workload]:
    """The 48-instance parameter scan (sizes 128^2/192^2/256^2, 16 each)."""
    return _c4_instances()
