"""Plain FP64 CPU oracle of the quasi-static slice advance and driver push.

TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the CPU
baseline leg of the benchmark may import this module; the CUDA library never
does, and this module imports nothing from the CUDA path.

What it computes follows Wang, Khudik, Kim, Shvets, "WAND-PIC: an accelerated
three-dimensional quasi-static particle-in-cell code" (arXiv 2012.00881):

* plasma macroparticle motion in the transverse plane, Eqs. EoM_112_A and
  EoM_111 (laser terms zero), with the constant of motion gamma - p_z = 1 + psi
  (Eq. substitute_A and the line after Eq. Jr);
* the fluid moments of Eq. Jr and the pressure tensor T of Eq. FluxPres;
* the field equations EqM_N8_AA (psi), EqM_N8_A (E_z), Mag_z_A (B_z) and the
  explicit screened-Poisson equation Main_Eq_A with the source FluxCurr1_A for
  B_perp, solved in the order psi; E_z, B_z; B_perp (text after Eq. matrix);
* the adaptive xi-step of Algorithm 1 (Step_Size_Refinement) with the
  refinement cap of Sec. 5.1;
* the driver equations of motion EoM_beam_1/2 with the wake E^W, B^W.

The arithmetic is written out plainly in the order of those equations.  One
library routine is used as a step: scipy's sparse LU (SuperLU) solves the
assembled 5-point systems exactly to rounding.  Everything is float64.

Readings taken where the paper is silent or garbled (all mirrored by the CUDA
library, which was written separately):

1.  Grid: N x N cell-centred cells on [x_min, x_max]^2, h = (x_max-x_min)/N,
    arrays indexed [iy, ix].  5-point Laplacian of Eq. 2D_Laplac_Uni.
2.  Fields are zero on the walls: odd ghosts (ghost = -first interior cell)
    for the Laplacian and for central differences of psi.  Moment grids use
    zero ghosts for their central differences.
3.  CIC (area weighting) on cell centres; a weight that falls into a ghost
    cell is folded back into its mirror interior cell, so deposits conserve
    sum(w) exactly.  The gather uses the same weights (it is the transpose of
    the deposit).
4.  Particles reflect specularly at the walls.
5.  Ion background n_ion = deposit of the initial lattice (quiet start), so
    the psi source is n_* - n_ion (Eq. EqM_N8_AA with a background profile).
6.  Sign of E_perp in the driver push: E_perp = -grad psi - e_z x B_perp
    (the line after Eq. EoM_beam_2 prints "+"; psi = phi - A_z, d_t = d_xi,
    d_z = -d_xi give "-", and that sign is the one consistent with Eq. EoM_111
    for an electron).
7.  Rows 4-5 of M_1 in Eq. matrix are read with B_x on the diagonal of row 4
    (the printed matrix repeats column 5); this is Eq. Main_Eq_A.
8.  n_* <T_ab> in Eq. matrix is the deposited sum w V_a V_b / h^2.
9.  The products of Eq. FluxCurr1_A are evaluated on the grid from the seven
    deposited moments {n_*, j_x, j_y, T_xx, T_xy, T_yy, G = n_* <gamma>}, with
    central differences for the gradients.
10. "Boris-like" push (Sec. 7.1): fields of the current slice frozen at the
    particle; half kick, rotation by B_z, half kick, then the drift with the
    new momentum.
11. Adaptive step: each base interval is split into m equal sub-steps,
    m = min(k, max(1, ceil(V_max / V0))), V0 = h / dxi0, V_max from the last
    push.  Sub-step fields are computed but only base slices are stored.
12. Guard: 1 + psi is replaced by max(1 + psi, psi_floor) wherever it divides,
    at particles and on the grid; every replacement is counted.
13. The driver beam enters only through j_z (electron flux units): a beam of
    charge q adds -q * w * v_z deposited by CIC in x, y and linearly in xi.
14. The driver push is the relativistic Boris scheme (a volume-preserving
    integrator) with the wake gathered trilinearly from the stored base
    slices; xi = t - z advances by dt (1 - v_z).
15. Laser driver (optional; Eq. EoM_111, the line after it, Eq.
    FluxCurr1_A): |A|^2 of the envelope is given at the base slices and
    taken linearly in xi at sub-steps, like the driver current.  It adds
    |A|^2/2 to the numerator of gamma, -grad(|A|^2/4)/(1+psi) to the kicks
    of the push, and -n_* grad(|A|^2/4)/(1+psi)^2 to S.  grad(|A|^2) is a
    central difference with even ghosts (A is odd at the walls, so |A|^2 is
    mirrored) gathered by CIC like grad(psi).  The step returns
    chi = n_*/(1+psi) at the base slices for the envelope advance of Eq.
    laser_Enve.

Parity status: every function here is pinned by tests under tests/ marked
"not gpu" (eigenmodes, manufactured solutions, the linear-wake closed form,
conservation laws, the xi-derivative identity behind Eq. FluxCurr1_A, and
exact orbits of the driver push; the laser terms by the mass shell with
|A|^2/2, ponderomotive expulsion with energy conservation, and the linear
laser wake (d_xi^2 + 1) psi = |A|^2/4 in tests/test_laser_wake_pins.py).
"""
from __future__ import annotations

import dataclasses
import math
from functools import lru_cache
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

FIELD_NAMES = ("psi", "Ez", "Bz", "Bx", "By")


# --------------------------------------------------------------------------
# grid, CIC deposit / gather
# --------------------------------------------------------------------------
@dataclasses.dataclass(frozen=True)
class Grid:
    """Square cell-centred grid: cell (iy, ix) has centre
    (x_min + (ix + 1/2) h, y_min + (iy + 1/2) h)."""

    n: int
    x_min: float
    x_max: float
    y_min: float
    y_max: float

    @property
    def h(self) -> float:
        return (self.x_max - self.x_min) / self.n

    @staticmethod
    def square(n: int, half_width: float) -> "Grid":
        return Grid(n, -half_width, half_width, -half_width, half_width)


def _cic_1d(s: np.ndarray, n: int):
    """Two-cell linear weights for coordinate s in cell units, s = (x-x_min)/h.

    Cell centres sit at s = i + 1/2.  Returns folded indices (i0, i1) and
    weights (w0, w1); index -1 folds to 0 and index n folds to n-1 (reading 3).
    """
    t = s - 0.5
    i0 = np.floor(t)
    f = t - i0
    i0 = i0.astype(np.int64)
    i1 = i0 + 1
    i0 = np.where(i0 < 0, -1 - i0, i0)
    i1 = np.where(i1 > n - 1, 2 * n - 1 - i1, i1)
    return i0, i1, 1.0 - f, f


def cic_stencil(x: np.ndarray, y: np.ndarray, g: Grid):
    """Four (flat index, weight) pairs per particle."""
    ix0, ix1, wx0, wx1 = _cic_1d((x - g.x_min) / g.h, g.n)
    iy0, iy1, wy0, wy1 = _cic_1d((y - g.y_min) / g.h, g.n)
    n = g.n
    idx = (iy0 * n + ix0, iy0 * n + ix1, iy1 * n + ix0, iy1 * n + ix1)
    wts = (wy0 * wx0, wy0 * wx1, wy1 * wx0, wy1 * wx1)
    return idx, wts


def deposit(x, y, q, g: Grid) -> np.ndarray:
    """Surface density sum_p q_p S(r - r_p) / h^2 on the grid (Eq. continuity's
    n_* for q = w; the moments of Eq. Jr for other q)."""
    idx, wts = cic_stencil(x, y, g)
    out = np.zeros(g.n * g.n)
    for i, wgt in zip(idx, wts):
        out += np.bincount(i, weights=q * wgt, minlength=g.n * g.n)
    return (out / (g.h * g.h)).reshape(g.n, g.n)


def gather(u: np.ndarray, x, y, g: Grid) -> np.ndarray:
    """Field value at particles: sum over the same four cells and weights."""
    idx, wts = cic_stencil(x, y, g)
    uf = u.ravel()
    val = np.zeros(len(x))
    for i, wgt in zip(idx, wts):
        val += uf[i] * wgt
    return val


# --------------------------------------------------------------------------
# cell sort (stable by particle id)
# --------------------------------------------------------------------------
def cell_index(x, y, g: Grid) -> np.ndarray:
    """c = iy * N + ix with ix = floor((x - x_min) / h) clamped to [0, N-1]."""
    ix = np.clip(np.floor((x - g.x_min) / g.h), 0, g.n - 1).astype(np.int64)
    iy = np.clip(np.floor((y - g.y_min) / g.h), 0, g.n - 1).astype(np.int64)
    return iy * g.n + ix


def cell_sort(x, y, pid, g: Grid):
    """Counting sort by cell; ties ordered by ascending particle id.

    Returns (cell, count[N^2], offset[N^2+1], perm) where perm lists the input
    positions in sorted order.
    """
    c = cell_index(x, y, g)
    count = np.bincount(c, minlength=g.n * g.n).astype(np.int64)
    offset = np.zeros(g.n * g.n + 1, dtype=np.int64)
    np.cumsum(count, out=offset[1:])
    perm = np.lexsort((pid, c))
    return c, count, offset, perm


# --------------------------------------------------------------------------
# finite differences (Eq. 2D_Laplac_Uni) and the elliptic solves
# --------------------------------------------------------------------------
def _pad(u: np.ndarray, ghost: str) -> np.ndarray:
    p = np.zeros((u.shape[0] + 2, u.shape[1] + 2))
    p[1:-1, 1:-1] = u
    if ghost == "odd":
        p[0, 1:-1] = -u[0, :]
        p[-1, 1:-1] = -u[-1, :]
        p[1:-1, 0] = -u[:, 0]
        p[1:-1, -1] = -u[:, -1]
    elif ghost == "even":
        p[0, 1:-1] = u[0, :]
        p[-1, 1:-1] = u[-1, :]
        p[1:-1, 0] = u[:, 0]
        p[1:-1, -1] = u[:, -1]
    elif ghost != "zero":
        raise ValueError(ghost)
    return p


def laplacian(u: np.ndarray, h: float) -> np.ndarray:
    """5-point Laplacian with zero-Dirichlet (odd) ghosts."""
    p = _pad(u, "odd")
    return (p[:-2, 1:-1] + p[2:, 1:-1] + p[1:-1, :-2] + p[1:-1, 2:] - 4.0 * u) / (h * h)


def ddx(u: np.ndarray, h: float, ghost: str) -> np.ndarray:
    """Central difference along x (axis 1)."""
    p = _pad(u, ghost)
    return (p[1:-1, 2:] - p[1:-1, :-2]) / (2.0 * h)


def ddy(u: np.ndarray, h: float, ghost: str) -> np.ndarray:
    """Central difference along y (axis 0)."""
    p = _pad(u, ghost)
    return (p[2:, 1:-1] - p[:-2, 1:-1]) / (2.0 * h)


def _second_difference_1d(n: int) -> sp.csr_matrix:
    """Tridiagonal [1, -2, 1] with the odd-ghost wall rows [-3, 1] / [1, -3]."""
    main = np.full(n, -2.0)
    main[0] = main[-1] = -3.0
    off = np.ones(n - 1)
    return sp.diags([off, main, off], [-1, 0, 1], format="csr")


@lru_cache(maxsize=8)
def _poisson_lu(n: int, h: float):
    t = _second_difference_1d(n)
    eye = sp.identity(n, format="csr")
    a = (sp.kron(eye, t) + sp.kron(t, eye)) / (h * h)
    return spla.splu(a.tocsc())


def solve_poisson(f: np.ndarray, h: float) -> np.ndarray:
    """u with laplacian(u) = f (zero walls), exact sparse LU solve."""
    n = f.shape[0]
    return _poisson_lu(n, float(h)).solve(f.ravel()).reshape(n, n)


def solve_screened(f: np.ndarray, kappa: np.ndarray, h: float, lu=None):
    """u with laplacian(u) - kappa u = f (zero walls).  Returns (u, lu) so a
    second right-hand side with the same kappa reuses the factorisation."""
    n = f.shape[0]
    if lu is None:
        t = _second_difference_1d(n)
        eye = sp.identity(n, format="csr")
        a = (sp.kron(eye, t) + sp.kron(t, eye)) / (h * h) - sp.diags(kappa.ravel())
        lu = spla.splu(a.tocsc())
    return lu.solve(f.ravel()).reshape(n, n), lu


# --------------------------------------------------------------------------
# plasma initialisation
# --------------------------------------------------------------------------
def profile_density(r: np.ndarray, table: Optional[Sequence[float]], r_max: float) -> np.ndarray:
    """n(r) from equispaced samples on [0, r_max], piecewise linear, held
    constant beyond r_max; None means uniform n = 1."""
    if table is None:
        return np.ones_like(r)
    tab = np.asarray(table, dtype=np.float64)
    m = len(tab)
    if m == 1:
        return np.full_like(r, tab[0])
    s = np.minimum(r / r_max * (m - 1), m - 1)
    i = np.minimum(np.floor(s).astype(np.int64), m - 2)
    f = s - i
    return tab[i] * (1.0 - f) + tab[i + 1] * f


@dataclasses.dataclass
class Plasma:
    x: np.ndarray
    y: np.ndarray
    px: np.ndarray
    py: np.ndarray
    w: np.ndarray
    pid: np.ndarray

    def copy(self) -> "Plasma":
        return Plasma(self.x.copy(), self.y.copy(), self.px.copy(), self.py.copy(),
                      self.w.copy(), self.pid.copy())


def init_plasma(g: Grid, ppc: int, table=None, r_max: float = 1.0):
    """Cold quiet-start lattice: sqrt(ppc)^2 particles per cell at offsets
    (k + 1/2)/sqrt(ppc) of a cell, p_perp = 0 (cold plasma before the driver,
    Sec. 3.1), weight n(r0) h^2 / ppc, id = cell * ppc + ky * s + kx.
    Returns (plasma, n_ion) with n_ion the deposit of the lattice."""
    s = int(round(math.sqrt(ppc)))
    if s * s != ppc:
        raise ValueError("ppc must be a perfect square")
    n, h = g.n, g.h
    iy, ix, ky, kx = np.meshgrid(np.arange(n), np.arange(n), np.arange(s), np.arange(s),
                                 indexing="ij")
    x = g.x_min + (ix + (kx + 0.5) / s) * h
    y = g.y_min + (iy + (ky + 0.5) / s) * h
    x, y = x.ravel(), y.ravel()
    pid = ((iy * n + ix) * ppc + ky * s + kx).ravel().astype(np.int64)
    w = profile_density(np.sqrt(x * x + y * y), table, r_max) * (h * h / ppc)
    pl = Plasma(x, y, np.zeros_like(x), np.zeros_like(x), w, pid)
    return pl, deposit(x, y, w, g)


# --------------------------------------------------------------------------
# one slice: sources and fields
# --------------------------------------------------------------------------
@dataclasses.dataclass
class SliceFields:
    psi: np.ndarray
    Ez: np.ndarray
    Bz: np.ndarray
    Bx: np.ndarray
    By: np.ndarray
    dpsi_dx: np.ndarray
    dpsi_dy: np.ndarray
    moments: Dict[str, np.ndarray]
    vmax_in: float
    guard_hits: int
    # laser driver (Eq. EoM_111): |A|^2 on the grid and grad(|A|^2 / 4)
    a2: Optional[np.ndarray] = None
    pond_x: Optional[np.ndarray] = None
    pond_y: Optional[np.ndarray] = None

    def stack(self) -> np.ndarray:
        return np.stack([self.psi, self.Ez, self.Bz, self.Bx, self.By])


def gamma_qs(px, py, a, a2=0.0):
    """Lorentz factor of a plasma electron from the constant of motion
    gamma - p_z = 1 + psi: gamma = (1 + p_perp^2 + (1+psi)^2 + |A|^2/2) /
    (2 (1+psi)) (line after Eq. EoM_111); a = 1 + psi, a2 = |A|^2 of the laser
    envelope at the particle (0 without a laser)."""
    return (1.0 + px * px + py * py + a * a + 0.5 * a2) / (2.0 * a)


def _guard(a: np.ndarray, floor: float):
    low = a < floor
    return np.where(low, floor, a), int(low.sum())


def slice_fields(g: Grid, pl: Plasma, n_ion: np.ndarray, jzb: np.ndarray,
                 psi_floor: float, a2: Optional[np.ndarray] = None) -> SliceFields:
    """Collect_Source + Solve_Wakefield of Algorithm 1 for one slice.

    `a2` is |A|^2 of a laser envelope on the grid (None: no laser).  It enters
    gamma (line after Eq. EoM_111), hence <gamma> and j_z, and the source S
    through -n_* grad(|A|^2/4) / (1+psi)^2 (Eq. FluxCurr1_A).  |A|^2 takes
    even ghosts at the walls (A is odd there)."""
    h = g.h
    # surface density n_* (Eq. continuity) and psi (Eq. EqM_N8_AA)
    n_star = deposit(pl.x, pl.y, pl.w, g)
    psi = solve_poisson(n_star - n_ion, h)
    # per-particle 1 + psi, gamma (line after Eq. EoM_111), V (Eq. EoM_112_A)
    a_p, hits = _guard(1.0 + gather(psi, pl.x, pl.y, g), psi_floor)
    a2_p = 0.0 if a2 is None else gather(a2, pl.x, pl.y, g)
    gam = gamma_qs(pl.px, pl.py, a_p, a2_p)
    vx = pl.px / a_p
    vy = pl.py / a_p
    # moments: j_perp = n_* <V> (Eq. Jr), T = n_* <V V> (Eq. FluxPres), G = n_* <gamma>
    jx = deposit(pl.x, pl.y, pl.w * vx, g)
    jy = deposit(pl.x, pl.y, pl.w * vy, g)
    txx = deposit(pl.x, pl.y, pl.w * vx * vx, g)
    txy = deposit(pl.x, pl.y, pl.w * vx * vy, g)
    tyy = deposit(pl.x, pl.y, pl.w * vy * vy, g)
    gsum = deposit(pl.x, pl.y, pl.w * gam, g)
    # E_z (Eq. EqM_N8_A) and B_z (Eq. Mag_z_A)
    ez = solve_poisson(-(ddx(jx, h, "zero") + ddy(jy, h, "zero")), h)
    bz = solve_poisson(ddx(jy, h, "zero") - ddy(jx, h, "zero"), h)
    # j_z = n_* <p_z> / (1 + psi) with <p_z> = <gamma> - psi - 1 (Eq. Jr), plus the driver
    a_g, hits_g = _guard(1.0 + psi, psi_floor)
    jz = gsum / a_g - n_star + jzb
    kappa = n_star / a_g
    dpx = ddx(psi, h, "odd")
    dpy = ddy(psi, h, "odd")
    # source S of Eq. FluxCurr1_A, term by term
    sx = (ddx(jz, h, "zero") - ddx(txx, h, "zero") - ddy(txy, h, "zero")
          - jy * bz / a_g
          + gsum * dpx / (a_g * a_g)
          - jx * ez / a_g
          - (txx * dpx + txy * dpy) / a_g)
    sy = (ddy(jz, h, "zero") - ddx(txy, h, "zero") - ddy(tyy, h, "zero")
          + jx * bz / a_g
          + gsum * dpy / (a_g * a_g)
          - jy * ez / a_g
          - (txy * dpx + tyy * dpy) / a_g)
    pond_x = pond_y = None
    if a2 is not None:
        # ponderomotive term of Eq. FluxCurr1_A: -n_* grad(|A|^2/4) / (1+psi)^2
        pond_x = ddx(0.25 * a2, h, "even")
        pond_y = ddy(0.25 * a2, h, "even")
        sx = sx - n_star * pond_x / (a_g * a_g)
        sy = sy - n_star * pond_y / (a_g * a_g)
    # B_perp: laplacian(B) - kappa B = -e_z x S = (S_y, -S_x)  (Eq. Main_Eq_A)
    bx, lu = solve_screened(sy, kappa, h)
    by, _ = solve_screened(-sx, kappa, h, lu)
    vmax_in = float(np.sqrt(vx * vx + vy * vy).max()) if len(vx) else 0.0
    mom = dict(n_star=n_star, jx=jx, jy=jy, txx=txx, txy=txy, tyy=tyy, G=gsum, jz=jz,
               kappa=kappa, Sx=sx, Sy=sy)
    return SliceFields(psi, ez, bz, bx, by, dpx, dpy, mom, vmax_in, hits + hits_g,
                       a2, pond_x, pond_y)


# --------------------------------------------------------------------------
# plasma push (Eqs. EoM_112_A, EoM_111) and step refinement (Algorithm 1)
# --------------------------------------------------------------------------
def push_plasma(g: Grid, pl: Plasma, F: SliceFields, dxi: float, psi_floor: float):
    """Advance every trajectory from xi to xi + dxi with the fields of this
    slice frozen at its position.  Returns (new plasma, V_max, guard hits)."""
    x, y = pl.x, pl.y
    a, hits = _guard(1.0 + gather(F.psi, x, y, g), psi_floor)
    gx = gather(F.dpsi_dx, x, y, g)
    gy = gather(F.dpsi_dy, x, y, g)
    bx = gather(F.Bx, x, y, g)
    by = gather(F.By, x, y, g)
    bz = gather(F.Bz, x, y, g)
    half = 0.5 * dxi
    # laser (Eq. EoM_111): |A|^2 in gamma and the force -grad(|A|^2/4)/(1+psi)
    if F.a2 is not None:
        a2 = gather(F.a2, x, y, g)
        px_pond = gather(F.pond_x, x, y, g)
        py_pond = gather(F.pond_y, x, y, g)
    else:
        a2 = 0.0
        px_pond = py_pond = 0.0
    # electric-like part of Eq. EoM_111:
    # gamma grad(psi)/(1+psi) - grad(|A|^2/4)/(1+psi) + e_z x B_perp
    gam = gamma_qs(pl.px, pl.py, a, a2)
    pxm = pl.px + half * ((gam * gx - px_pond) / a - by)
    pym = pl.py + half * ((gam * gy - py_pond) / a + bx)
    # rotation by the B_z term: dp/dxi = (e_z x p) B_z / (1+psi)
    tau = half * bz / a
    pxp_ = pxm - tau * pym
    pyp_ = pym + tau * pxm
    s = 2.0 * tau / (1.0 + tau * tau)
    pxr = pxm - s * pyp_
    pyr = pym + s * pxp_
    gam2 = gamma_qs(pxr, pyr, a, a2)
    px = pxr + half * ((gam2 * gx - px_pond) / a - by)
    py = pyr + half * ((gam2 * gy - py_pond) / a + bx)
    # drift with V = p / (1 + psi)
    nx = x + dxi * px / a
    ny = y + dxi * py / a
    # specular walls
    for lo, hi, pos, mom in ((g.x_min, g.x_max, nx, px), (g.y_min, g.y_max, ny, py)):
        over = pos > hi
        pos[over] = 2.0 * hi - pos[over]
        mom[over] = -mom[over]
        under = pos < lo
        pos[under] = 2.0 * lo - pos[under]
        mom[under] = -mom[under]
    vmax = float(np.max(np.sqrt(px * px + py * py) / a)) if len(a) else 0.0
    return Plasma(nx, ny, px, py, pl.w, pl.pid), vmax, hits


def refine_m(vmax: float, v0: float, k: int) -> int:
    """Sub-steps for the next base interval: Step_Size_Refinement of
    Algorithm 1 (dxi = dxi0 V0 / V_max when V_max > V0) rounded up to an
    integer division of dxi0 and capped by dxi >= dxi0 / k (Sec. 5.1)."""
    if vmax <= v0:
        return 1
    return int(min(k, max(1, math.ceil(vmax / v0))))


# --------------------------------------------------------------------------
# driver beam: deposit (Sec. 7.1, last paragraph) and push (Eqs. EoM_beam_1/2)
# --------------------------------------------------------------------------
@dataclasses.dataclass(frozen=True)
class Config:
    n: int
    x_min: float
    x_max: float
    y_min: float
    y_max: float
    n_xi: int
    xi_min: float
    xi_max: float
    refine_k: int = 8
    psi_floor: float = 1e-3

    @property
    def grid(self) -> Grid:
        return Grid(self.n, self.x_min, self.x_max, self.y_min, self.y_max)

    @property
    def dxi0(self) -> float:
        return (self.xi_max - self.xi_min) / self.n_xi


def deposit_beam(cfg: Config, beams: Sequence[dict], n_slices: Optional[int] = None) -> np.ndarray:
    """j_z of the drivers on the base slices, shape (n_xi, N, N), or on the
    first `n_slices` base slices only (the rest of the window is not stored).

    CIC in x, y (folded at the walls like the plasma deposit) and linear in xi
    between base slices; particles outside the transverse box, and weight that
    falls outside the slice range, are dropped.  A beam of charge q in units of
    e contributes -q w v_z (j is normalised to -e n0 c).
    """
    g = cfg.grid
    n = g.n
    ns = cfg.n_xi if n_slices is None else min(cfg.n_xi, n_slices)
    out = np.zeros(ns * n * n)
    for b in beams:
        x, y, xi = b["x"], b["y"], b["xi"]
        gam = np.sqrt(1.0 + b["px"] ** 2 + b["py"] ** 2 + b["pz"] ** 2)
        q = -b["charge"] * b["w"] * b["pz"] / gam
        inside = (x >= g.x_min) & (x <= g.x_max) & (y >= g.y_min) & (y <= g.y_max)
        s = (xi - cfg.xi_min) / cfg.dxi0
        j0 = np.floor(s)
        f = s - j0
        j0 = j0.astype(np.int64)
        idx, wts = cic_stencil(x, y, g)
        for jj, wj in ((j0, 1.0 - f), (j0 + 1, f)):
            ok = inside & (jj >= 0) & (jj < ns)
            for i, wgt in zip(idx, wts):
                out += np.bincount((jj[ok] * n * n + i[ok]), weights=(q * wj * wgt)[ok],
                                   minlength=ns * n * n)
    return (out / (g.h * g.h * cfg.dxi0)).reshape(ns, n, n)


@dataclasses.dataclass
class StepResult:
    history: np.ndarray          # (5, n_xi, N, N): psi, Ez, Bz, Bx, By at base slices
    m: np.ndarray                # sub-steps used for each base interval
    vmax: np.ndarray             # V_max after the last push of each interval
    charge: np.ndarray           # sum n_* h^2 at each base slice
    slices: int                  # computed slices including sub-steps
    pushes: int                  # plasma particle pushes
    guard_hits: int
    final_plasma: Plasma
    chi: Optional[np.ndarray] = None   # (n_xi, N, N) n_* / (1+psi) with a laser driver


def step3d(cfg: Config, plasma0: Plasma, n_ion: np.ndarray, beams: Sequence[dict],
           jzb: Optional[np.ndarray] = None, n_slices: Optional[int] = None,
           m_schedule: Optional[Sequence[int]] = None,
           laser_a2: Optional[np.ndarray] = None) -> StepResult:
    """One 3D step with frozen drivers: the xi loop of Algorithm 1.

    `jzb` may be given directly (shape (n_xi, N, N)) instead of beam particles.
    `n_slices` truncates the loop after that many base slices.
    `m_schedule` fixes the sub-steps of every base interval instead of the
    adaptive rule (used to freeze the schedule of a previous run).
    `laser_a2` is |A|^2 of a laser envelope at the base slices (shape
    (n_xi, N, N)), interpolated linearly in xi at sub-steps like the driver
    current; the result then also holds the laser susceptibility
    chi = n_* / (1+psi) of Eq. laser_Enve at the base slices.
    """
    g = cfg.grid
    nb = cfg.n_xi if n_slices is None else n_slices
    if jzb is None:
        jzb = deposit_beam(cfg, beams, n_slices=min(cfg.n_xi, nb + 1))
    v0 = g.h / cfg.dxi0
    hist = np.zeros((5, nb, g.n, g.n))
    ms = np.ones(nb, dtype=np.int64)
    vmaxs = np.zeros(nb)
    charge = np.zeros(nb)
    pl = plasma0.copy()
    m = 1 if m_schedule is None else int(m_schedule[0])
    slices = pushes = hits = 0
    zero = np.zeros((g.n, g.n))
    chi = None if laser_a2 is None else np.zeros((nb, g.n, g.n))
    for j in range(nb):
        ms[j] = m
        nxt = jzb[j + 1] if j + 1 < min(cfg.n_xi, jzb.shape[0]) else zero
        if laser_a2 is not None:
            a2_nxt = laser_a2[j + 1] if j + 1 < laser_a2.shape[0] else zero
        for q in range(m):
            frac = q / m
            jz_here = jzb[j] if q == 0 else (1.0 - frac) * jzb[j] + frac * nxt
            a2_here = None
            if laser_a2 is not None:
                a2_here = laser_a2[j] if q == 0 else (1.0 - frac) * laser_a2[j] + frac * a2_nxt
            F = slice_fields(g, pl, n_ion, jz_here, cfg.psi_floor, a2_here)
            slices += 1
            hits += F.guard_hits
            if q == 0:
                hist[:, j] = F.stack()
                charge[j] = float(F.moments["n_star"].sum() * g.h * g.h)
                if chi is not None:
                    chi[j] = F.moments["kappa"]
            if j == nb - 1:
                break
            pl, vmax, hp = push_plasma(g, pl, F, cfg.dxi0 / m, cfg.psi_floor)
            pushes += len(pl.x)
            hits += hp
        if j == nb - 1:
            break
        vmaxs[j] = vmax
        m = refine_m(vmax, v0, cfg.refine_k) if m_schedule is None else int(m_schedule[j + 1])
    return StepResult(hist, ms, vmaxs, charge, slices, pushes, hits, pl, chi)


def wake_at(cfg: Config, hist: np.ndarray, x, y, xi):
    """Trilinear gather of (E_z, B_z, B_x, B_y, dpsi/dx, dpsi/dy) from the base
    slices: CIC in x, y; linear in xi; zero outside the box or the window."""
    g = cfg.grid
    nb = hist.shape[1]
    inside = (x >= g.x_min) & (x <= g.x_max) & (y >= g.y_min) & (y <= g.y_max)
    s = (xi - cfg.xi_min) / cfg.dxi0
    j0 = np.floor(s)
    f = s - j0
    j0 = j0.astype(np.int64)
    out = np.zeros((6, len(x)))
    grads = {}
    for jj, wj in ((j0, 1.0 - f), (j0 + 1, f)):
        ok = inside & (jj >= 0) & (jj < nb)
        if not ok.any():
            continue
        for sl in np.unique(jj[ok]):
            sel = ok & (jj == sl)
            if sl not in grads:
                grads[sl] = (ddx(hist[0, sl], g.h, "odd"), ddy(hist[0, sl], g.h, "odd"))
            comps = (hist[1, sl], hist[2, sl], hist[3, sl], hist[4, sl]) + grads[sl]
            for c, u in enumerate(comps):
                out[c, sel] += wj[sel] * gather(u, x[sel], y[sel], g)
    return out


def boris_step(beam: dict, ex, ey, ez, bx, by, bz, dt: float) -> dict:
    """One relativistic Boris step of length dt (half kick, rotation, half
    kick, then the drift with the new velocity; xi = t - z advances by
    dt (1 - v_z)) of Eqs. EoM_beam_1/2 in the given fields at the particles."""
    x, y, xi = beam["x"], beam["y"], beam["xi"]
    qm = beam["q_over_m"]
    hq = 0.5 * dt * qm
    ux = beam["px"] + hq * ex
    uy = beam["py"] + hq * ey
    uz = beam["pz"] + hq * ez
    gam = np.sqrt(1.0 + ux * ux + uy * uy + uz * uz)
    tx, ty, tz = hq * bx / gam, hq * by / gam, hq * bz / gam
    ss = 2.0 / (1.0 + tx * tx + ty * ty + tz * tz)
    # u' = u- + u- x t
    upx = ux + (uy * tz - uz * ty)
    upy = uy + (uz * tx - ux * tz)
    upz = uz + (ux * ty - uy * tx)
    # u+ = u- + u' x s
    ux = ux + ss * (upy * tz - upz * ty)
    uy = uy + ss * (upz * tx - upx * tz)
    uz = uz + ss * (upx * ty - upy * tx)
    ux = ux + hq * ex
    uy = uy + hq * ey
    uz = uz + hq * ez
    gam = np.sqrt(1.0 + ux * ux + uy * uy + uz * uz)
    out = dict(beam)
    out.update(x=x + dt * ux / gam, y=y + dt * uy / gam, xi=xi + dt * (1.0 - uz / gam),
               px=ux, py=uy, pz=uz)
    return out


def push_beam(cfg: Config, hist: np.ndarray, beam: dict, dt: float) -> dict:
    """Push_Driver of Algorithm 1: one relativistic Boris step of length dt in
    the frozen wake, E^W = e_z E_z + E_perp, B^W = e_z B_z + B_perp, with
    E_perp = -grad(psi) - e_z x B_perp (Eqs. EoM_beam_1/2; reading 6)."""
    ez, bz, bx, by, gx, gy = wake_at(cfg, hist, beam["x"], beam["y"], beam["xi"])
    return boris_step(beam, -gx + by, -gy - bx, ez, bx, by, bz, dt)


def beam_gamma(beam: dict) -> np.ndarray:
    return np.sqrt(1.0 + beam["px"] ** 2 + beam["py"] ** 2 + beam["pz"] ** 2)


def config_from_workload(wl) -> Config:
    """Build an oracle Config from a workloads.Workload description."""
    return Config(n=wl.n, x_min=-wl.half_width, x_max=wl.half_width,
                  y_min=-wl.half_width, y_max=wl.half_width, n_xi=wl.n_xi,
                  xi_min=0.0, xi_max=wl.xi_len, refine_k=wl.refine_k,
                  psi_floor=wl.psi_floor)


def plasma_from_workload(wl):
    g = Grid.square(wl.n, wl.half_width)
    if wl.profile is None:
        return init_plasma(g, wl.ppc)
    table, r_max = wl.profile
    return init_plasma(g, wl.ppc, table, r_max)
