"""FP64 CPU oracle of the laser-envelope advance (Eq. laser_Enve).

TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the CPU
baseline leg of the benchmark may import this module; the CUDA library never
does, and this module imports nothing from the CUDA path.

Sec. "Description of different plasma wake drivers": the complex envelope
A(x, y, xi, t) of a laser with vector potential A exp(-i k0 xi) obeys the
paraxial equation
    (2 i k0 d_t - 2 d_t d_xi + lap_perp) A = chi A,    chi = n_* / (1 + psi),
which the paper rearranges into a Poisson-like equation per slice and solves
with its multigrid solver, warm-started from the previous time step (Sec. 7.1,
last paragraphs).  Units are the paper's normalised ones (k_p = 1).

Readings taken where the paper is silent (mirrored by the CUDA library, which
was written separately):

L1. Time discretisation.  Time-centred (Crank-Nicolson) for lap_perp and chi;
    the mixed derivative d_t d_xi as the time difference of a backward
    difference in xi (towards the head, j - 1), so slices advance from the
    head (j = 0) to the tail with A^{n+1}_{j-1} already known.  Multiplying
    the discrete equation by 2 gives, per slice,
        (lap - chi_j + c) A^{n+1}_j = (c - lap + chi_j) A^n_j
                                      - q (A^{n+1}_{j-1} - A^n_{j-1}),
        c = 4 (i k0 - 1/dxi) / dt,   q = 4 / (dt dxi).
L2. chi is held at t_n (the wake of step n) for both time levels.
L3. A = 0 ahead of the window (slice j = -1) and on the transverse walls
    (odd ghosts, the slice advance's 5-point Laplacian of Eq. 2D_Laplac_Uni
    on its cell-centred grid).
L4. dxi is the base slice spacing.  dxi = inf drops the xi coupling (q = 0,
    c = 4 i k0 / dt): each slice then obeys the Schroedinger-like equation
    2 i k0 d_t A = (chi - lap) A, whose Crank-Nicolson step is unitary.

One library routine is used as a step: scipy's sparse LU (SuperLU) solves each
slice's complex system exactly to rounding.  Everything is complex128 /
float64.  Arrays are [slice, iy, ix].  Pinned by tests/test_laser_pins.py
(unitarity without the xi coupling, the paraxial Gaussian beam's closed form,
the group-velocity slip (chi + k_perp^2) / (2 k0^2) of a pulse in plasma, and
the coupled step handing chi ~ 1 of a weakly perturbed plasma to the
envelope).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .qs_oracle import Config, Grid, _second_difference_1d, step3d

__all__ = ["laplacian_matrix", "step_coefficients", "envelope_advance", "envelope_step",
           "laser_step3d"]


def laplacian_matrix(n: int, h: float) -> sp.csr_matrix:
    """The 5-point Laplacian with odd ghosts (Dirichlet walls), N^2 x N^2."""
    t = _second_difference_1d(n)
    eye = sp.identity(n, format="csr")
    return ((sp.kron(eye, t) + sp.kron(t, eye)) / (h * h)).tocsr()


def step_coefficients(k0: float, dt: float, dxi: float):
    """(c, q) of reading L1; dxi = inf gives (4 i k0 / dt, 0)."""
    q = 0.0 if math.isinf(dxi) else 4.0 / (dt * dxi)
    return 4.0j * k0 / dt - q, q


def envelope_advance(g: Grid, a, chi, k0: float, dt: float, dxi: float, steps: int = 1):
    """`steps` time steps of Eq. laser_Enve from a (complex [n_xi, N, N]) with
    chi (real [n_xi, N, N]) held fixed; returns the envelope at the end.

    Each slice's matrix lap - chi_j + c does not change between steps, so it
    is factorised once."""
    a = np.array(a, dtype=np.complex128)
    chi = np.asarray(chi, dtype=np.float64)
    n_xi, n = a.shape[0], g.n
    lap = laplacian_matrix(n, g.h)
    c, q = step_coefficients(k0, dt, dxi)
    lus = [spla.splu((lap + sp.diags(c - chi[j].ravel())).tocsc()) for j in range(n_xi)]
    for _ in range(steps):
        new = np.zeros_like(a)
        for j in range(n_xi):
            aj = a[j].ravel()
            rhs = (c + chi[j].ravel()) * aj - lap @ aj
            if j > 0:
                rhs -= q * (new[j - 1].ravel() - a[j - 1].ravel())
            new[j] = lus[j].solve(rhs).reshape(n, n)
        a = new
    return a


def envelope_step(g: Grid, a, chi, k0: float, dt: float, dxi: float):
    """One time step (see envelope_advance)."""
    return envelope_advance(g, a, chi, k0, dt, dxi, 1)


def laser_step3d(cfg: Config, plasma0, n_ion, envelope, k0: float, dt: float, beams=(),
                 jzb=None, m_schedule=None):
    """One 3D step with a laser driver (Algorithm 1 with the laser): the xi
    loop with |A|^2 of the envelope (the slice advance's laser terms), which
    also yields chi = n_*/(1+psi) at the base slices, then one time step of
    Eq. laser_Enve with that chi over the same slices.  Returns (the step's
    result, the envelope at t + dt)."""
    a2 = np.abs(np.asarray(envelope)) ** 2
    if jzb is None and not beams:
        jzb = np.zeros(a2.shape)
    r = step3d(cfg, plasma0, n_ion, beams, jzb=jzb, laser_a2=a2, m_schedule=m_schedule)
    return r, envelope_advance(cfg.grid, envelope, r.chi, k0, dt, cfg.dxi0, 1)
