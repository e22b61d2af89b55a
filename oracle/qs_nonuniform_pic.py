"""FP64 CPU oracle of the slice advance on a nonuniform transverse grid.

TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the CPU
baseline leg of the benchmark may import this module; the CUDA library never
does, and this module imports nothing from the CUDA path.

Sec. "Multigrid Solver with Nonuniform Grids" deploys nonuniform grids for the
whole quasi-static PIC loop, not only for its solver.  This module is the
uniform-grid slice advance of qs_oracle (Algorithm 1: deposit, psi, moments,
sources, E_z and B_z, B_perp, push) with every grid operation taken on the
node grid of qs_nonuniform:

* deposits and gathers: CIC on the nodes (reading N5 of qs_nonuniform);
* gradients: the three-point first difference printed after Eq.
  2D_Laplac_3rd, with the wall value zero (fields vanish there; moments are
  differenced with zero outside, as on the uniform grid);
* the five field equations: the 9-point operator with the third-order
  correction (Eqs. 2D_Laplac, 2D_Laplac_3rd), M = 0 for psi, E_z, B_z and
  M = -kappa for B_perp, solved exactly by qs_nonuniform.solve;
* the push: the uniform oracle's Boris-like step (reading 10 of qs_oracle)
  with the node gathers, specular walls at the box edges.

The quiet start puts sqrt(ppc)^2 particles in every interval rectangle
between neighbouring nodes (walls included) at offsets (k + 1/2)/sqrt(ppc) of
it, with weight = its area / ppc (density 1), and n_ion = their deposit.
Pinned by tests/test_nonuniform_pins.py (the linear beam wake of the
uniform oracle's closed form, with the node grid's own (1 - lap)^-1).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional, Sequence

import numpy as np
import scipy.sparse as sp

from . import qs_nonuniform as nu
from .qs_oracle import Plasma, SliceFields, gamma_qs, refine_m

__all__ = ["NodeGrid", "init_plasma_nodes", "slice_fields_nodes", "push_plasma_nodes",
           "step3d_nodes"]


@dataclasses.dataclass(frozen=True)
class NodeGrid:
    xn: np.ndarray   # n_x + 2 node coordinates, walls included
    yn: np.ndarray

    @property
    def shape(self):
        return (len(self.yn) - 2, len(self.xn) - 2)

    @property
    def h_min(self) -> float:
        return float(min(np.diff(self.xn).min(), np.diff(self.yn).min()))

    def ddx(self, u: np.ndarray) -> np.ndarray:
        return (nu.first_difference(self.xn) @ u.T).T

    def ddy(self, u: np.ndarray) -> np.ndarray:
        return nu.first_difference(self.yn) @ u

    def deposit(self, x, y, q) -> np.ndarray:
        return nu.deposit(self.xn, self.yn, x, y, q)

    def gather(self, u, x, y) -> np.ndarray:
        return nu.gather(u, self.xn, self.yn, x, y)

    def poisson(self, f: np.ndarray) -> np.ndarray:
        return nu.solve(self.xn, self.yn, f)

    def screened(self, f: np.ndarray, kappa: np.ndarray) -> np.ndarray:
        return nu.solve(self.xn, self.yn, f, -kappa)


def init_plasma_nodes(G: NodeGrid, ppc: int):
    """Quiet-start lattice on the node grid; returns (plasma, n_ion)."""
    s = int(round(math.sqrt(ppc)))
    if s * s != ppc:
        raise ValueError("ppc must be a perfect square")
    off = (np.arange(s) + 0.5) / s

    def sub(xn):
        lo, d = xn[:-1], np.diff(xn)
        return (lo[:, None] + d[:, None] * off[None, :]).ravel(), np.repeat(d, s) / s

    xs, dx = sub(np.asarray(G.xn, dtype=np.float64))
    ys, dy = sub(np.asarray(G.yn, dtype=np.float64))
    X, Y = np.meshgrid(xs, ys)
    W = np.outer(dy, dx)
    x, y, w = X.ravel(), Y.ravel(), W.ravel()
    z = np.zeros_like(x)
    pl = Plasma(x, y, z.copy(), z.copy(), w, np.arange(x.size, dtype=np.int64))
    return pl, G.deposit(x, y, w)


def _guard(a, floor):
    low = a < floor
    return np.where(low, floor, a), int(np.sum(low))


def slice_fields_nodes(G: NodeGrid, pl: Plasma, n_ion: np.ndarray, jzb: np.ndarray,
                       psi_floor: float) -> SliceFields:
    """Collect_Source + Solve_Wakefield of Algorithm 1 on the node grid (the
    formulas of qs_oracle.slice_fields, term by term)."""
    n_star = G.deposit(pl.x, pl.y, pl.w)
    psi = G.poisson(n_star - n_ion)
    a_p, hits = _guard(1.0 + G.gather(psi, pl.x, pl.y), psi_floor)
    gam = gamma_qs(pl.px, pl.py, a_p)
    vx, vy = pl.px / a_p, pl.py / a_p
    jx = G.deposit(pl.x, pl.y, pl.w * vx)
    jy = G.deposit(pl.x, pl.y, pl.w * vy)
    txx = G.deposit(pl.x, pl.y, pl.w * vx * vx)
    txy = G.deposit(pl.x, pl.y, pl.w * vx * vy)
    tyy = G.deposit(pl.x, pl.y, pl.w * vy * vy)
    gsum = G.deposit(pl.x, pl.y, pl.w * gam)
    ez = G.poisson(-(G.ddx(jx) + G.ddy(jy)))
    bz = G.poisson(G.ddx(jy) - G.ddy(jx))
    a_g, hits_g = _guard(1.0 + psi, psi_floor)
    jz = gsum / a_g - n_star + jzb
    kappa = n_star / a_g
    dpx, dpy = G.ddx(psi), G.ddy(psi)
    sx = (G.ddx(jz) - G.ddx(txx) - G.ddy(txy) - jy * bz / a_g + gsum * dpx / (a_g * a_g)
          - jx * ez / a_g - (txx * dpx + txy * dpy) / a_g)
    sy = (G.ddy(jz) - G.ddx(txy) - G.ddy(tyy) + jx * bz / a_g + gsum * dpy / (a_g * a_g)
          - jy * ez / a_g - (txy * dpx + tyy * dpy) / a_g)
    bx = G.screened(sy, kappa)
    by = G.screened(-sx, kappa)
    vmax_in = float(np.sqrt(vx * vx + vy * vy).max()) if len(vx) else 0.0
    mom = dict(n_star=n_star, jx=jx, jy=jy, txx=txx, txy=txy, tyy=tyy, G=gsum, jz=jz,
               kappa=kappa, Sx=sx, Sy=sy)
    return SliceFields(psi, ez, bz, bx, by, dpx, dpy, mom, vmax_in, hits + hits_g)


def push_plasma_nodes(G: NodeGrid, pl: Plasma, F: SliceFields, dxi: float, psi_floor: float):
    """The Boris-like push of qs_oracle.push_plasma with node gathers."""
    x, y = pl.x, pl.y
    a, hits = _guard(1.0 + G.gather(F.psi, x, y), psi_floor)
    gx, gy = G.gather(F.dpsi_dx, x, y), G.gather(F.dpsi_dy, x, y)
    bx, by, bz = G.gather(F.Bx, x, y), G.gather(F.By, x, y), G.gather(F.Bz, x, y)
    half = 0.5 * dxi
    gam = gamma_qs(pl.px, pl.py, a)
    pxm = pl.px + half * (gam * gx / a - by)
    pym = pl.py + half * (gam * gy / a + bx)
    tau = half * bz / a
    pxp_, pyp_ = pxm - tau * pym, pym + tau * pxm
    s = 2.0 * tau / (1.0 + tau * tau)
    pxr, pyr = pxm - s * pyp_, pym + s * pxp_
    gam2 = gamma_qs(pxr, pyr, a)
    px = pxr + half * (gam2 * gx / a - by)
    py = pyr + half * (gam2 * gy / a + bx)
    nx, ny = x + dxi * px / a, y + dxi * py / a
    for lo, hi, pos, mom in ((G.xn[0], G.xn[-1], nx, px), (G.yn[0], G.yn[-1], ny, py)):
        over = pos > hi
        pos[over] = 2.0 * hi - pos[over]
        mom[over] = -mom[over]
        under = pos < lo
        pos[under] = 2.0 * lo - pos[under]
        mom[under] = -mom[under]
    vmax = float(np.max(np.sqrt(px * px + py * py) / a)) if len(a) else 0.0
    return Plasma(nx, ny, px, py, pl.w, pl.pid), vmax, hits


def step3d_nodes(G: NodeGrid, n_xi: int, dxi0: float, plasma0: Plasma, n_ion: np.ndarray,
                 jzb: np.ndarray, refine_k: int = 8, psi_floor: float = 1e-3,
                 m_schedule: Optional[Sequence[int]] = None):
    """The xi loop of Algorithm 1 on the node grid with a given driver current
    jzb [n_xi, ny, nx]; returns (history [5, n_xi, ny, nx], sub-steps used).
    V0 of Step_Size_Refinement uses the smallest spacing."""
    v0 = G.h_min / dxi0
    hist = np.zeros((5, n_xi) + G.shape)
    ms = np.ones(n_xi, dtype=np.int64)
    pl = plasma0.copy()
    m = 1 if m_schedule is None else int(m_schedule[0])
    zero = np.zeros(G.shape)
    vmax = 0.0
    for j in range(n_xi):
        ms[j] = m
        nxt = jzb[j + 1] if j + 1 < n_xi else zero
        for q in range(m):
            frac = q / m
            jz_here = jzb[j] if q == 0 else (1.0 - frac) * jzb[j] + frac * nxt
            F = slice_fields_nodes(G, pl, n_ion, jz_here, psi_floor)
            if q == 0:
                hist[:, j] = F.stack()
            if j == n_xi - 1:
                break
            pl, vmax, _ = push_plasma_nodes(G, pl, F, dxi0 / m, psi_floor)
        if j == n_xi - 1:
            break
        m = refine_m(vmax, v0, refine_k) if m_schedule is None else int(m_schedule[j + 1])
    return hist, ms
