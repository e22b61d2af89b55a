"""FP64 CPU oracle of the driver push in the laser's high-frequency fields.

TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the CPU
baseline leg of the benchmark may import this module; the CUDA library never
does, and this module imports nothing from the CUDA path.

Sec. "Description of different plasma wake drivers": driver (or witness)
particles are not ponderomotive: they feel the laser's own fields, rebuilt
from the envelope A (vector potential A exp(-i k0 xi), polarised along x) by
Eq. E_B_Fields,
    E_x = -((d_t A + d_xi A) - i k0 A) e^{-i k0 xi},   B_y = (-d_xi A + i k0 A) e^{-i k0 xi},
    E_z = -d_x A e^{-i k0 xi},                          B_z = -d_y A e^{-i k0 xi},
added to the wake in Eqs. EoM_beam_1/2, and are advanced by a Boris-like
pusher sub-cycled N_sub times per laser time step (the DLA comparison of Sec.
"Comparison with full 3D PIC simulations" uses N_sub = 50).

Readings taken where the paper is silent (the CUDA path must take the same):

D1. The physical fields are the real parts of the printed complex
    expressions (the vector potential is Re(A e^{-i k0 xi}), whose square
    averages to |A|^2/2, the |A|^2/2 of the plasma's gamma).
D2. The envelope and its derivatives are gathered at the particle like the
    wake (CIC in x, y on the base slices, linear in xi, zero outside the box
    and the window); the carrier phase e^{-i k0 xi} is applied at the
    particle's own xi, so it is not interpolated.
D3. d_xi A and d_x A, d_y A are central differences on the base slices (A is
    zero ahead of and behind the window and odd at the walls); d_t A is the
    difference of the envelopes at t_n and t_{n+1} over dt, and A itself is
    interpolated linearly in t between them at each sub-step.
D4. Each of the N_sub sub-steps is the driver push's Boris step (fields at
    the particle's position at the start of the sub-step, then the drift),
    of length dt / N_sub, with the wake frozen over the whole step.

One library routine is used as a step: numpy's complex exponential.
Everything is float64 / complex128.  Pinned by tests/test_dla_pins.py (the
exact orbit of an electron in a plane wave, zero divergence of the rebuilt
E and B, and the laser-free limit equal to sub-stepped wake pushes).
"""
from __future__ import annotations

from typing import Sequence, Tuple

import numpy as np

from .qs_oracle import Config, boris_step, ddx, ddy, gather, wake_at

__all__ = ["envelope_derivatives", "laser_fields_at", "push_beam_dla"]


def _ddx_c(u: np.ndarray, h: float) -> np.ndarray:
    return ddx(u.real, h, "odd") + 1j * ddx(u.imag, h, "odd")


def _ddy_c(u: np.ndarray, h: float) -> np.ndarray:
    return ddy(u.real, h, "odd") + 1j * ddy(u.imag, h, "odd")


def envelope_derivatives(cfg: Config, env: np.ndarray):
    """(d_xi A, d_x A, d_y A) of an envelope [n_xi, N, N] (reading D3)."""
    h = cfg.grid.h
    pad = np.zeros((env.shape[0] + 2,) + env.shape[1:], dtype=np.complex128)
    pad[1:-1] = env
    dxi = (pad[2:] - pad[:-2]) / (2.0 * cfg.dxi0)
    dx = np.stack([_ddx_c(env[j], h) for j in range(env.shape[0])])
    dy = np.stack([_ddy_c(env[j], h) for j in range(env.shape[0])])
    return dxi, dx, dy


def _gather_slices(cfg: Config, grids: Sequence[np.ndarray], x, y, xi) -> np.ndarray:
    """CIC in x, y and linear in xi of complex [n_xi, N, N] grids (reading D2)."""
    g = cfg.grid
    nb = grids[0].shape[0]
    inside = (x >= g.x_min) & (x <= g.x_max) & (y >= g.y_min) & (y <= g.y_max)
    s = (xi - cfg.xi_min) / cfg.dxi0
    j0 = np.floor(s)
    f = s - j0
    j0 = j0.astype(np.int64)
    out = np.zeros((len(grids), len(x)), dtype=np.complex128)
    for jj, wj in ((j0, 1.0 - f), (j0 + 1, f)):
        ok = inside & (jj >= 0) & (jj < nb)
        for sl in np.unique(jj[ok]):
            sel = ok & (jj == sl)
            for c, u in enumerate(grids):
                val = gather(u[sl].real, x[sel], y[sel], g) + 1j * gather(u[sl].imag, x[sel], y[sel], g)
                out[c, sel] += wj[sel] * val
    return out


def laser_fields_at(cfg: Config, env_n: np.ndarray, env_np1: np.ndarray, frac: float,
                    dt: float, k0: float, x, y, xi) -> Tuple[np.ndarray, ...]:
    """(E_x, B_y, E_z, B_z) of Eq. E_B_Fields at the particles, for the
    envelope at t_n + frac dt (readings D1-D3)."""
    env = (1.0 - frac) * env_n + frac * env_np1
    dadt = (env_np1 - env_n) / dt
    dxi, dx, dy = envelope_derivatives(cfg, env)
    a, adt, axi, ax, ay = _gather_slices(cfg, (env, dadt, dxi, dx, dy), x, y, xi)
    ph = np.exp(-1j * k0 * np.asarray(xi))
    ex = (-((adt + axi) - 1j * k0 * a) * ph).real
    by = ((-axi + 1j * k0 * a) * ph).real
    ez = (-ax * ph).real
    bz = (-ay * ph).real
    return ex, by, ez, bz


def push_beam_dla(cfg: Config, hist: np.ndarray, env_n: np.ndarray, env_np1: np.ndarray,
                  k0: float, beam: dict, dt: float, n_sub: int) -> dict:
    """Push_Driver with the laser's fields: n_sub Boris sub-steps of dt/n_sub
    in the frozen wake (E_perp = -grad(psi) - e_z x B_perp) plus the fields of
    Eq. E_B_Fields (Eqs. EoM_beam_1/2; reading D4)."""
    b = dict(beam)
    h = dt / n_sub
    for s in range(n_sub):
        x, y, xi = b["x"], b["y"], b["xi"]
        ez, bz, bx, by, gx, gy = wake_at(cfg, hist, x, y, xi)
        exl, byl, ezl, bzl = laser_fields_at(cfg, env_n, env_np1, s / n_sub, dt, k0, x, y, xi)
        b = boris_step(b, -gx + by + exl, -gy - bx, ez + ezl, bx, by + byl, bz + bzl, h)
    return b
