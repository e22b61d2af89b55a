"""Gradient oracle of the differentiable slice advance (float64, CPU).

TEST INFRASTRUCTURE ONLY.  Only tests/ use this module; the CUDA library never
imports it, and it imports nothing from the CUDA path.

What it computes.  The loss of the differentiable form is the mean energy
gain of the witness bunch over one 3D step,

    L = mean_p [ gamma_p after the driver-beam push of length dt - gamma_p before ],

with the wake of one 3D step of the quasi-static advance (Algorithm 1 and
Sec. 7.1; every bunch deposits j_z) and the frozen-field relativistic Boris
push of Eqs. EoM_beam_1/2 (qs_oracle.push_beam).  Its parameters are

* the driver bunch, theta = (A, sigma_x, sigma_y, sigma_z, x_c, y_c, xi_c,
  tilt), acting on fixed standard normals z (the bi-Gaussian of Sec. 5.1,
  n_b = A exp(-r^2/sigma_r^2 - xi^2/sigma_z^2)):
      xi = xi_c + sigma_z/sqrt2 z2,  x = x_c + tilt (xi - xi_c) + sigma_x/sqrt2 z0,
      y = y_c + sigma_y/sqrt2 z1,    w = A pi^(3/2) sigma_x sigma_y sigma_z / N;
* the transverse plasma density n(r), a table of values at equispaced radii
  on [0, r_max] interpolated piecewise-linearly: the lattice weights are
  n(r0) h^2 / ppc and the ion background is the deposit of that lattice.

The sub-step schedule m_j is held fixed (it is piecewise constant in the
parameters) and the 1 + psi guard must not trigger.

How.  The forward steps of qs_oracle are restated with float64 torch ops, in
the same order and with the same formulas, and torch.autograd differentiates
them.  The elliptic solves are autograd functions whose backward is the same
exact solve, the 5-point operators being symmetric: for (lap - kappa) u = f,
    dL/df = (lap - kappa)^-1 dL/du,   dL/dkappa = u * dL/df.

Pins (tests/test_grad_oracle.py): the restated forward equals qs_oracle's to
rounding, and the gradient equals central finite differences of the loss
computed with qs_oracle alone.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional, Sequence, Tuple

import numpy as np
import torch

from . import qs_oracle as O

F64 = torch.float64
N_DRIVER_PARAMS = 8
DRIVER_PARAM_NAMES = ("amplitude", "sigma_x", "sigma_y", "sigma_z", "x_c", "y_c", "xi_c", "tilt")


# --------------------------------------------------------------------------
# problem description
# --------------------------------------------------------------------------
@dataclasses.dataclass
class GradProblem:
    cfg: O.Config
    ppc: int
    r_max: float                 # radius of the last profile sample
    driver_z: np.ndarray         # (3, N) standard normals of the driver
    driver_gamma: float
    driver_charge: float
    witness: dict                # witness bunch (numpy SoA, fixed)
    dt: float
    m_schedule: Optional[np.ndarray] = None   # fixed sub-steps per base interval


def driver_beam_numpy(theta: Sequence[float], z: np.ndarray, gamma: float, charge: float,
                      q_over_m: float = -1.0) -> dict:
    """Driver macroparticles for parameters theta (see the module text)."""
    a, sx, sy, sz, xc, yc, xic, tilt = [float(v) for v in theta]
    n = z.shape[1]
    s2 = math.sqrt(2.0)
    xi = xic + sz / s2 * z[2]
    x = xc + tilt * (xi - xic) + sx / s2 * z[0]
    y = yc + sy / s2 * z[1]
    w = a * math.pi ** 1.5 * sx * sy * sz / n
    return {"x": x, "y": y, "xi": xi, "px": np.zeros(n), "py": np.zeros(n),
            "pz": np.full(n, math.sqrt(gamma * gamma - 1.0)), "w": np.full(n, w),
            "charge": charge, "q_over_m": q_over_m}


# --------------------------------------------------------------------------
# the loss with qs_oracle alone (used for finite differences)
# --------------------------------------------------------------------------
def loss_numpy(P: GradProblem, theta: Sequence[float], table: Sequence[float]) -> float:
    cfg = P.cfg
    pl, n_ion = O.init_plasma(cfg.grid, P.ppc, list(table), P.r_max)
    drv = driver_beam_numpy(theta, P.driver_z, P.driver_gamma, P.driver_charge)
    res = O.step3d(cfg, pl, n_ion, [drv, P.witness], m_schedule=P.m_schedule)
    if res.guard_hits:
        raise ValueError("the 1 + psi guard triggered")
    after = O.push_beam(cfg, res.history, P.witness, P.dt)
    return float(np.mean(O.beam_gamma(after) - O.beam_gamma(P.witness)))


def schedule(P: GradProblem, theta, table) -> np.ndarray:
    """The adaptive sub-step schedule of the forward run at (theta, table)."""
    cfg = P.cfg
    pl, n_ion = O.init_plasma(cfg.grid, P.ppc, list(table), P.r_max)
    drv = driver_beam_numpy(theta, P.driver_z, P.driver_gamma, P.driver_charge)
    return O.step3d(cfg, pl, n_ion, [drv, P.witness]).m.copy()


# --------------------------------------------------------------------------
# the same forward in torch
# --------------------------------------------------------------------------
def _cic_1d(s: torch.Tensor, n: int):
    t = s - 0.5
    fl = torch.floor(t)
    f = t - fl
    i0 = fl.long()
    i1 = i0 + 1
    i0 = torch.where(i0 < 0, -1 - i0, i0)
    i1 = torch.where(i1 > n - 1, 2 * n - 1 - i1, i1)
    return i0, i1, 1.0 - f, f


def _stencil(x, y, g: O.Grid):
    ix0, ix1, wx0, wx1 = _cic_1d((x - g.x_min) / g.h, g.n)
    iy0, iy1, wy0, wy1 = _cic_1d((y - g.y_min) / g.h, g.n)
    n = g.n
    return ((iy0 * n + ix0, iy0 * n + ix1, iy1 * n + ix0, iy1 * n + ix1),
            (wy0 * wx0, wy0 * wx1, wy1 * wx0, wy1 * wx1))


def deposit(x, y, q, g: O.Grid) -> torch.Tensor:
    idx, wts = _stencil(x, y, g)
    out = torch.zeros(g.n * g.n, dtype=F64)
    for i, wgt in zip(idx, wts):
        out = out.index_add(0, i, q * wgt)
    return (out / (g.h * g.h)).reshape(g.n, g.n)


def gather(u, x, y, g: O.Grid) -> torch.Tensor:
    idx, wts = _stencil(x, y, g)
    uf = u.reshape(-1)
    val = torch.zeros_like(x)
    for i, wgt in zip(idx, wts):
        val = val + uf[i] * wgt
    return val


def ddx(u, h: float, ghost: str):
    s = -1.0 if ghost == "odd" else 0.0
    left = torch.cat([s * u[:, :1], u[:, :-1]], 1)
    right = torch.cat([u[:, 1:], s * u[:, -1:]], 1)
    return (right - left) / (2.0 * h)


def ddy(u, h: float, ghost: str):
    s = -1.0 if ghost == "odd" else 0.0
    below = torch.cat([s * u[:1, :], u[:-1, :]], 0)
    above = torch.cat([u[1:, :], s * u[-1:, :]], 0)
    return (above - below) / (2.0 * h)


class _Poisson(torch.autograd.Function):
    """u = lap^-1 f with an exact sparse LU; backward: the same solve."""

    @staticmethod
    def forward(ctx, f, h):
        n = f.shape[0]
        ctx.n, ctx.h = n, float(h)
        u = O.solve_poisson(f.detach().numpy(), float(h))
        return torch.from_numpy(u)

    @staticmethod
    def backward(ctx, gu):
        return torch.from_numpy(O.solve_poisson(gu.detach().numpy(), ctx.h)), None


class _Screened(torch.autograd.Function):
    """(u1, u2) = (lap - kappa)^-1 (f1, f2); backward: the same solve for the
    right-hand sides and u1 mu1 + u2 mu2 for kappa."""

    @staticmethod
    def forward(ctx, f1, f2, kappa, h):
        k = kappa.detach().numpy()
        u1, lu = O.solve_screened(f1.detach().numpy(), k, float(h))
        u2, _ = O.solve_screened(f2.detach().numpy(), k, float(h), lu)
        ctx.lu = lu
        u1t, u2t = torch.from_numpy(u1), torch.from_numpy(u2)
        ctx.save_for_backward(u1t, u2t)
        return u1t, u2t

    @staticmethod
    def backward(ctx, g1, g2):
        u1, u2 = ctx.saved_tensors
        n = u1.shape[0]

        def solve(gv):
            if gv is None:
                return torch.zeros_like(u1)
            return torch.from_numpy(ctx.lu.solve(gv.detach().numpy().ravel()).reshape(n, n))

        m1, m2 = solve(g1), solve(g2)
        return m1, m2, m1 * u1 + m2 * u2, None


def _guard(a, floor: float):
    hits = int((a < floor).sum())
    return torch.clamp(a, min=floor), hits


def gamma_qs(px, py, a):
    return (1.0 + px * px + py * py + a * a) / (2.0 * a)


def slice_fields(g: O.Grid, x, y, px, py, w, n_ion, jzb, psi_floor: float):
    """qs_oracle.slice_fields in torch: returns (psi, Ez, Bz, Bx, By, dpsi_dx,
    dpsi_dy, guard hits)."""
    h = g.h
    n_star = deposit(x, y, w, g)
    psi = _Poisson.apply(n_star - n_ion, h)
    a_p, hits = _guard(1.0 + gather(psi, x, y, g), psi_floor)
    gam = gamma_qs(px, py, a_p)
    vx = px / a_p
    vy = py / a_p
    jx = deposit(x, y, w * vx, g)
    jy = deposit(x, y, w * vy, g)
    txx = deposit(x, y, w * vx * vx, g)
    txy = deposit(x, y, w * vx * vy, g)
    tyy = deposit(x, y, w * vy * vy, g)
    gsum = deposit(x, y, w * gam, g)
    ez = _Poisson.apply(-(ddx(jx, h, "zero") + ddy(jy, h, "zero")), h)
    bz = _Poisson.apply(ddx(jy, h, "zero") - ddy(jx, h, "zero"), h)
    a_g, hits_g = _guard(1.0 + psi, psi_floor)
    jz = gsum / a_g - n_star + jzb
    kappa = n_star / a_g
    dpx = ddx(psi, h, "odd")
    dpy = ddy(psi, h, "odd")
    sx = (ddx(jz, h, "zero") - ddx(txx, h, "zero") - ddy(txy, h, "zero")
          - jy * bz / a_g + gsum * dpx / (a_g * a_g) - jx * ez / a_g
          - (txx * dpx + txy * dpy) / a_g)
    sy = (ddy(jz, h, "zero") - ddx(txy, h, "zero") - ddy(tyy, h, "zero")
          + jx * bz / a_g + gsum * dpy / (a_g * a_g) - jy * ez / a_g
          - (txy * dpx + tyy * dpy) / a_g)
    bx, by = _Screened.apply(sy, -sx, kappa, h)
    return psi, ez, bz, bx, by, dpx, dpy, hits + hits_g


def push_plasma(g: O.Grid, x, y, px, py, fields, dxi: float, psi_floor: float):
    """qs_oracle.push_plasma in torch; returns (x, y, px, py, guard hits)."""
    psi, ez, bz_g, bx_g, by_g, dpx, dpy = fields
    a, hits = _guard(1.0 + gather(psi, x, y, g), psi_floor)
    gx = gather(dpx, x, y, g)
    gy = gather(dpy, x, y, g)
    bx = gather(bx_g, x, y, g)
    by = gather(by_g, x, y, g)
    bz = gather(bz_g, x, y, g)
    half = 0.5 * dxi
    gam = gamma_qs(px, py, a)
    pxm = px + half * (gam * gx / a - by)
    pym = py + half * (gam * gy / a + bx)
    tau = half * bz / a
    pxp_ = pxm - tau * pym
    pyp_ = pym + tau * pxm
    s = 2.0 * tau / (1.0 + tau * tau)
    pxr = pxm - s * pyp_
    pyr = pym + s * pxp_
    gam2 = gamma_qs(pxr, pyr, a)
    px2 = pxr + half * (gam2 * gx / a - by)
    py2 = pyr + half * (gam2 * gy / a + bx)
    nx = x + dxi * px2 / a
    ny = y + dxi * py2 / a
    out = []
    for lo, hi, pos, mom in ((g.x_min, g.x_max, nx, px2), (g.y_min, g.y_max, ny, py2)):
        over = pos > hi
        pos = torch.where(over, 2.0 * hi - pos, pos)
        mom = torch.where(over, -mom, mom)
        under = pos < lo
        pos = torch.where(under, 2.0 * lo - pos, pos)
        mom = torch.where(under, -mom, mom)
        out.append((pos, mom))
    (nx, px2), (ny, py2) = out
    return nx, ny, px2, py2, hits


def deposit_beam(cfg: O.Config, beams, ns: int) -> torch.Tensor:
    """qs_oracle.deposit_beam in torch over the first ns base slices."""
    g = cfg.grid
    n = g.n
    out = torch.zeros(ns * n * n, dtype=F64)
    for b in beams:
        x, y, xi = b["x"], b["y"], b["xi"]
        gam = torch.sqrt(1.0 + b["px"] ** 2 + b["py"] ** 2 + b["pz"] ** 2)
        q = -b["charge"] * b["w"] * b["pz"] / gam
        inside = (x >= g.x_min) & (x <= g.x_max) & (y >= g.y_min) & (y <= g.y_max)
        s = (xi - cfg.xi_min) / cfg.dxi0
        j0f = torch.floor(s)
        f = s - j0f
        j0 = j0f.long()
        idx, wts = _stencil(x, y, g)
        for jj, wj in ((j0, 1.0 - f), (j0 + 1, f)):
            ok = inside & (jj >= 0) & (jj < ns)
            for i, wgt in zip(idx, wts):
                out = out.index_add(0, (jj * n * n + i)[ok], (q * wj * wgt)[ok])
    return (out / (g.h * g.h * cfg.dxi0)).reshape(ns, n, n)


def step3d(cfg: O.Config, x, y, w, n_ion, jzb, m_schedule) -> torch.Tensor:
    """Base-slice history (5, n_xi, N, N) of one 3D step (qs_oracle.step3d
    with a fixed schedule); the plasma starts cold at (x, y)."""
    g = cfg.grid
    nb = cfg.n_xi
    px = torch.zeros_like(x)
    py = torch.zeros_like(x)
    zero = torch.zeros((g.n, g.n), dtype=F64)
    hist = []
    hits = 0
    for j in range(nb):
        m = int(m_schedule[j])
        nxt = jzb[j + 1] if j + 1 < nb else zero
        for q in range(m):
            frac = q / m
            jz_here = jzb[j] if q == 0 else (1.0 - frac) * jzb[j] + frac * nxt
            F = slice_fields(g, x, y, px, py, w, n_ion, jz_here, cfg.psi_floor)
            hits += F[7]
            if q == 0:
                hist.append(torch.stack(F[:5]))
            if j == nb - 1:
                break
            x, y, px, py, hp = push_plasma(g, x, y, px, py, F[:7], cfg.dxi0 / m, cfg.psi_floor)
            hits += hp
    if hits:
        raise ValueError("the 1 + psi guard triggered")
    return torch.stack(hist, 1)


def wake_at(cfg: O.Config, hist, x, y, xi):
    """qs_oracle.wake_at in torch: (Ez, Bz, Bx, By, dpsi/dx, dpsi/dy) at the
    particles, trilinear from the base slices."""
    g = cfg.grid
    nb = hist.shape[1]
    inside = (x >= g.x_min) & (x <= g.x_max) & (y >= g.y_min) & (y <= g.y_max)
    s = (xi - cfg.xi_min) / cfg.dxi0
    j0f = torch.floor(s)
    f = s - j0f
    j0 = j0f.long()
    out = [torch.zeros_like(x) for _ in range(6)]
    for jj, wj in ((j0, 1.0 - f), (j0 + 1, f)):
        ok = inside & (jj >= 0) & (jj < nb)
        for sl in torch.unique(jj[ok]).tolist():
            sel = torch.nonzero(ok & (jj == sl)).reshape(-1)
            comps = (hist[1, sl], hist[2, sl], hist[3, sl], hist[4, sl],
                     ddx(hist[0, sl], g.h, "odd"), ddy(hist[0, sl], g.h, "odd"))
            for c, u in enumerate(comps):
                val = wj[sel] * gather(u, x[sel], y[sel], g)
                out[c] = out[c].index_add(0, sel, val)
    return out


def push_beam_gamma(cfg: O.Config, hist, beam: dict, dt: float):
    """Lorentz factor after qs_oracle.push_beam (relativistic Boris, frozen
    wake, E_perp = -grad psi - e_z x B_perp), in torch."""
    x, y, xi = beam["x"], beam["y"], beam["xi"]
    ez, bz, bx, by, gx, gy = wake_at(cfg, hist, x, y, xi)
    ex = -gx + by
    ey = -gy - bx
    hq = 0.5 * dt * beam["q_over_m"]
    ux = beam["px"] + hq * ex
    uy = beam["py"] + hq * ey
    uz = beam["pz"] + hq * ez
    gam = torch.sqrt(1.0 + ux * ux + uy * uy + uz * uz)
    tx, ty, tz = hq * bx / gam, hq * by / gam, hq * bz / gam
    ss = 2.0 / (1.0 + tx * tx + ty * ty + tz * tz)
    upx = ux + (uy * tz - uz * ty)
    upy = uy + (uz * tx - ux * tz)
    upz = uz + (ux * ty - uy * tx)
    ux2 = ux + ss * (upy * tz - upz * ty)
    uy2 = uy + ss * (upz * tx - upx * tz)
    uz2 = uz + ss * (upx * ty - upy * tx)
    ux2 = ux2 + hq * ex
    uy2 = uy2 + hq * ey
    uz2 = uz2 + hq * ez
    return torch.sqrt(1.0 + ux2 * ux2 + uy2 * uy2 + uz2 * uz2)


def _profile(r, table, r_max: float):
    m = table.shape[0]
    if m == 1:
        return table[0] * torch.ones_like(r)
    s = torch.clamp(r / r_max * (m - 1), max=float(m - 1))
    i = torch.clamp(torch.floor(s).long(), max=m - 2)
    f = s - i.to(F64)
    return table[i] * (1.0 - f) + table[i + 1] * f


def loss_torch(P: GradProblem, theta: torch.Tensor, table: torch.Tensor,
               return_history: bool = False):
    """The loss as a torch scalar of (theta, table)."""
    cfg = P.cfg
    g = cfg.grid
    pl, _ = O.init_plasma(g, P.ppc, None, 1.0)      # lattice positions only
    x0 = torch.from_numpy(pl.x)
    y0 = torch.from_numpy(pl.y)
    w = _profile(torch.sqrt(x0 * x0 + y0 * y0), table, P.r_max) * (g.h * g.h / P.ppc)
    n_ion = deposit(x0, y0, w, g)
    z = torch.from_numpy(P.driver_z)
    a, sx, sy, sz, xc, yc, xic, tilt = theta
    s2 = math.sqrt(2.0)
    nd = z.shape[1]
    xi = xic + sz / s2 * z[2]
    drv = {"x": xc + tilt * (xi - xic) + sx / s2 * z[0], "y": yc + sy / s2 * z[1], "xi": xi,
           "px": torch.zeros(nd, dtype=F64), "py": torch.zeros(nd, dtype=F64),
           "pz": torch.full((nd,), math.sqrt(P.driver_gamma ** 2 - 1.0), dtype=F64),
           "w": (a * math.pi ** 1.5 * sx * sy * sz / nd) * torch.ones(nd, dtype=F64),
           "charge": P.driver_charge}
    wit = {k: (torch.from_numpy(np.asarray(v, dtype=np.float64)) if isinstance(v, np.ndarray)
               else v) for k, v in P.witness.items()}
    jzb = deposit_beam(cfg, [drv, wit], cfg.n_xi)
    hist = step3d(cfg, x0, y0, w, n_ion, jzb, P.m_schedule)
    gam = push_beam_gamma(cfg, hist, wit, P.dt)
    gam0 = torch.sqrt(1.0 + wit["px"] ** 2 + wit["py"] ** 2 + wit["pz"] ** 2)
    loss = torch.mean(gam - gam0)
    return (loss, hist) if return_history else loss


def gradient(P: GradProblem, theta: Sequence[float], table: Sequence[float]
             ) -> Tuple[float, np.ndarray, np.ndarray]:
    """(L, dL/dtheta, dL/dtable) at (theta, table) by reverse-mode
    differentiation of the restated forward."""
    th = torch.tensor(list(theta), dtype=F64, requires_grad=True)
    tb = torch.tensor(list(table), dtype=F64, requires_grad=True)
    loss = loss_torch(P, th, tb)
    dth, dtb = torch.autograd.grad(loss, (th, tb))
    return float(loss.detach()), dth.numpy(), dtb.numpy()


def problem_from_workload(wl, dt: Optional[float] = None) -> Tuple[GradProblem, np.ndarray, np.ndarray]:
    """GradProblem for a workloads.Workload whose first bunch is the driver
    and second the witness; returns (problem, theta, table) at the workload's
    values (the schedule is taken from the forward run there)."""
    import workloads as W
    drv, wit = wl.beams[0], wl.beams[1]
    theta = np.array([drv.amplitude, drv.sigma_x, drv.sigma_y, drv.sigma_z, drv.x_c, drv.y_c,
                      drv.xi_c, drv.tilt])
    if wl.profile is None:
        table, r_max = (1.0,), 1.0
    else:
        table, r_max = wl.profile
    P = GradProblem(cfg=O.config_from_workload(wl), ppc=wl.ppc, r_max=float(r_max),
                    driver_z=W.beam_normals(drv.n_particles, drv.seed),
                    driver_gamma=drv.gamma, driver_charge=float(drv.charge),
                    witness=W.sample_beam(wit), dt=wl.dt if dt is None else dt)
    table = np.asarray(table, dtype=np.float64)
    P.m_schedule = schedule(P, theta, table)
    return P, theta, table
