"""FP64 CPU oracle of the field equations on a nonuniform transverse grid.

TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the CPU
baseline leg of the benchmark may import this module; the CUDA library never
does, and this module imports nothing from the CUDA path.

It follows Sec. "Multigrid Solver with Nonuniform Grids" of Wang, Khudik, Kim,
Shvets, arXiv 2012.00881.  The equations have the general form
    (d^2/dx^2 + d^2/dy^2) Psi + M Psi = J                (the section's opening)
and are discretised on a tensor-product grid of nodes x_i, y_j with local
spacings h^- = x_i - x_{i-1}, h^+ = x_{i+1} - x_i, h^a = h^+ + h^-,
h^b = h^+ - h^-:

* D2 is the three-point second difference of Eq. 2D_Laplac,
      2 / (h^- h^+ h^a) (h^+ Psi_{i-1} - h^a Psi_i + h^- Psi_{i+1});
* D1 is the three-point first difference printed after Eq. 2D_Laplac_3rd;
* the third-order terms of Eq. 2D_Laplac are replaced as in Eq.
  2D_Laplac_3rd: d_x^3 = d_x(lap) - d_x d_y^2 with lap -> J - M Psi, the mixed
  third derivatives approximated by D1 applied to the other axis' D2.

Collecting terms, the discrete system is A Psi = J' with
    A  = D2x + D2y + M + Cx (D1x D2y + D1x M) + Cy (D1y D2x + D1y M),
    J' = J + (Cx D1x + Cy D1y) J,            Cx = diag(h_x^b / 3), Cy likewise,
where M stands for the diagonal matrix of the screening field.  With
`correction=False` the third-order terms are dropped (A = D2x + D2y + M,
J' = J), the plain second-order scheme the section warns about.

Readings taken where the section is silent or garbled (mirrored by the CUDA
library, which was written separately):

N1. Sign of the third-order term.  Taylor expansion of the three-point
    difference gives D2 = d^2 + (h^b / 3) d^3 + O(h^2), so the Laplacian is
    D2 - (h^b / 3) d^3; Eq. 2D_Laplac prints "+", which with h^b = h^+ - h^-
    would double the error instead of removing it.
N2. In Eq. 2D_Laplac_3rd the second bracket (d_y of the x second difference)
    carries h_y^b, as the first line of the same equation shows; the printed
    h_x^b is read as a typo.
N3. Layout: vertex-centred.  Each axis has n interior nodes plus the two walls
    as nodes where Psi = 0 (Dirichlet, as on the uniform grid).  J is zero on
    the walls (every source decays before the wall) and so is M Psi; the
    difference operators below therefore drop the wall columns.
N4. The J part of d_x(lap) moves to the right-hand side (J'); the M Psi part
    stays in the operator, so A is a 9-point, non-symmetric matrix.
N5. Particles (the section's grids carry the whole PIC, not only the solver):
    a particle's weight goes to the four nodes around it with linear weights
    in physical coordinates (CIC on the node grid); weight that falls on a
    wall node is folded into the adjacent interior node, so deposits conserve
    charge, and the density is the deposit over the node's dual area, the
    first and last nodes owning the whole interval to the wall.  The gather
    uses the same weights (it is the transpose of the deposit).

One library routine is used as a step: scipy's sparse LU (SuperLU) solves the
assembled system exactly to rounding.  Everything is float64.  Arrays are
indexed [iy, ix], flattened with ix fastest.  Pinned by
tests/test_nonuniform_pins.py (uniform-grid reduction to the 5-point scheme of
Eq. 2D_Laplac_Uni, exactness on quadratics, second-order truncation with the
correction and first-order without it, second-order convergence of the
solution; for particles, charge conservation, the gather as the deposit's
transpose, exact bilinear gathers, and unit density from a uniform lattice).
"""
from __future__ import annotations

from typing import Optional, Tuple

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

__all__ = [
    "node_areas",
    "cic_node_weights",
    "deposit",
    "gather",
    "spacings",
    "second_difference",
    "first_difference",
    "operator",
    "corrected_source",
    "apply",
    "solve",
]


def spacings(xn: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    """(h^-, h^+) at the interior nodes of an axis given with its walls."""
    xn = np.asarray(xn, dtype=np.float64)
    if xn.ndim != 1 or xn.size < 3 or np.any(np.diff(xn) <= 0.0):
        raise ValueError("node coordinates must be strictly increasing, walls included")
    return xn[1:-1] - xn[:-2], xn[2:] - xn[1:-1]


def second_difference(xn: np.ndarray) -> sp.csr_matrix:
    """The n x n three-point d^2/dx^2 of Eq. 2D_Laplac (wall values zero)."""
    hm, hp = spacings(xn)
    ha = hm + hp
    scale = 2.0 / (hm * hp * ha)
    lower = scale * hp          # coefficient of Psi_{i-1}
    diag = -scale * ha          # coefficient of Psi_i
    upper = scale * hm          # coefficient of Psi_{i+1}
    n = hm.size
    return sp.diags([lower[1:], diag, upper[:-1]], [-1, 0, 1], shape=(n, n), format="csr")


def first_difference(xn: np.ndarray) -> sp.csr_matrix:
    """The n x n three-point d/dx printed after Eq. 2D_Laplac_3rd:
    h^-/(h^a h^+) (Psi_{i+1} - Psi_i) + h^+/(h^a h^-) (Psi_i - Psi_{i-1})."""
    hm, hp = spacings(xn)
    ha = hm + hp
    a = hm / (ha * hp)          # weight of the forward difference
    b = hp / (ha * hm)          # weight of the backward difference
    n = hm.size
    return sp.diags([-b[1:], b - a, a[:-1]], [-1, 0, 1], shape=(n, n), format="csr")


def _along_x(op_1d: sp.spmatrix, ny: int) -> sp.csr_matrix:
    return sp.kron(sp.identity(ny, format="csr"), op_1d, format="csr")


def _along_y(op_1d: sp.spmatrix, nx: int) -> sp.csr_matrix:
    return sp.kron(op_1d, sp.identity(nx, format="csr"), format="csr")


def _third_order_weights(xn, yn):
    """Cx, Cy = diag(h^b / 3) as 2D diagonal matrices."""
    hmx, hpx = spacings(xn)
    hmy, hpy = spacings(yn)
    cx = np.tile((hpx - hmx) / 3.0, hmy.size)
    cy = np.repeat((hpy - hmy) / 3.0, hmx.size)
    return sp.diags(cx, format="csr"), sp.diags(cy, format="csr")


def operator(xn: np.ndarray, yn: np.ndarray, m: Optional[np.ndarray] = None,
             correction: bool = True) -> sp.csr_matrix:
    """The assembled discrete operator A (N = nx*ny rows, ix fastest)."""
    nx, ny = len(xn) - 2, len(yn) - 2
    d2x = _along_x(second_difference(xn), ny)
    d2y = _along_y(second_difference(yn), nx)
    mm = sp.diags(np.zeros(nx * ny) if m is None else np.asarray(m, np.float64).reshape(-1),
                  format="csr")
    a = d2x + d2y + mm
    if correction:
        d1x = _along_x(first_difference(xn), ny)
        d1y = _along_y(first_difference(yn), nx)
        cx, cy = _third_order_weights(xn, yn)
        a = a + cx @ (d1x @ d2y + d1x @ mm) + cy @ (d1y @ d2x + d1y @ mm)
    return a.tocsr()


def corrected_source(xn: np.ndarray, yn: np.ndarray, j: np.ndarray,
                     correction: bool = True) -> np.ndarray:
    """J' = J + (Cx D1x + Cy D1y) J (J itself without the correction)."""
    nx, ny = len(xn) - 2, len(yn) - 2
    jv = np.asarray(j, np.float64).reshape(-1)
    if not correction:
        return jv.reshape(ny, nx).copy()
    d1x = _along_x(first_difference(xn), ny)
    d1y = _along_y(first_difference(yn), nx)
    cx, cy = _third_order_weights(xn, yn)
    return (jv + cx @ (d1x @ jv) + cy @ (d1y @ jv)).reshape(ny, nx)


def apply(xn, yn, u, m=None, correction: bool = True) -> np.ndarray:
    """A u on the interior nodes, [ny, nx]."""
    nx, ny = len(xn) - 2, len(yn) - 2
    return (operator(xn, yn, m, correction) @ np.asarray(u, np.float64).reshape(-1)).reshape(ny, nx)


def solve(xn, yn, j, m=None, correction: bool = True) -> np.ndarray:
    """The discrete solution of A Psi = J' (exact to rounding), [ny, nx]."""
    nx, ny = len(xn) - 2, len(yn) - 2
    a = operator(xn, yn, m, correction).tocsc()
    rhs = corrected_source(xn, yn, j, correction).reshape(-1)
    return spla.spsolve(a, rhs).reshape(ny, nx)


# --------------------------------------------------------------------------
# particles on the node grid (reading N5)
# --------------------------------------------------------------------------
def _dual_lengths(xn: np.ndarray) -> np.ndarray:
    """Length each interior node owns: half of each adjacent interval, and the
    whole interval to the wall for the first and last node."""
    xn = np.asarray(xn, dtype=np.float64)
    hm, hp = spacings(xn)
    v = 0.5 * (hm + hp)
    v[0] += 0.5 * hm[0]
    v[-1] += 0.5 * hp[-1]
    return v


def node_areas(xn: np.ndarray, yn: np.ndarray) -> np.ndarray:
    """Dual areas [ny, nx] of the interior nodes; they sum to the box area."""
    return np.outer(_dual_lengths(yn), _dual_lengths(xn))


def cic_node_weights(xn: np.ndarray, x: np.ndarray):
    """(left node, weight of the right node) of each coordinate: the interval
    [xn[k], xn[k+1]] holding it (walls included, clamped to the box) and the
    linear weight; interior node indices, -1 / n for the walls."""
    xn = np.asarray(xn, dtype=np.float64)
    n = xn.size - 2
    x = np.clip(np.asarray(x, dtype=np.float64), xn[0], xn[-1])
    k = np.clip(np.searchsorted(xn, x, side="right") - 1, 0, n)
    f = (x - xn[k]) / (xn[k + 1] - xn[k])
    return k - 1, f


def _fold(i: np.ndarray, n: int) -> np.ndarray:
    return np.clip(i, 0, n - 1)


def _stencil(xn, yn, x, y):
    ix, fx = cic_node_weights(xn, x)
    iy, fy = cic_node_weights(yn, y)
    nx, ny = len(xn) - 2, len(yn) - 2
    out = []
    for dy, wy in ((0, 1.0 - fy), (1, fy)):
        for dx, wx in ((0, 1.0 - fx), (1, fx)):
            out.append((_fold(iy + dy, ny), _fold(ix + dx, nx), wy * wx))
    return out


def deposit(xn, yn, x, y, q) -> np.ndarray:
    """Density [ny, nx] of particle weights q at (x, y) (reading N5)."""
    nx, ny = len(xn) - 2, len(yn) - 2
    out = np.zeros(ny * nx)
    q = np.asarray(q, dtype=np.float64)
    for jy, jx, w in _stencil(xn, yn, x, y):
        out += np.bincount(jy * nx + jx, weights=q * w, minlength=ny * nx)
    return out.reshape(ny, nx) / node_areas(xn, yn)


def gather(u, xn, yn, x, y) -> np.ndarray:
    """Node field u [ny, nx] at the particles, with the deposit's weights."""
    u = np.asarray(u, dtype=np.float64)
    out = np.zeros(len(np.atleast_1d(x)))
    for jy, jx, w in _stencil(xn, yn, x, y):
        out += w * u[jy, jx]
    return out
