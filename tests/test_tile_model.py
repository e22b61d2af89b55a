"""A numpy model of the staged (temporally blocked) grid levels (CPU).

The GPU stages a tile plus a halo in shared memory and runs all the
red-black half sweeps of a leg there: half sweep s updates only the cells at
least s + 1 from a cut side of the region (the domain walls are not cut).
This model checks the invariant the kernels rely on, with plain numpy
arithmetic in the same order as a grid-wide sweep: after ns half sweeps the
tile and the ring of cells around it hold exactly the grid-wide values when
the halo is ns + 1 wide (the down leg's 2 nu1 + 1, the level-0 up leg's
2 nu2 + 1, which also needs the ring for the residual), and the tile alone
when it is ns wide (the other up legs, 2 nu2).
"""
import numpy as np
import pytest


def _gs_point(u, f, h2, x, y, n, omega):
    nb = 0.0
    walls = 0
    if x > 0:
        nb += u[y, x - 1]
    else:
        walls += 1
    if x < n - 1:
        nb += u[y, x + 1]
    else:
        walls += 1
    if y > 0:
        nb += u[y - 1, x]
    else:
        walls += 1
    if y < n - 1:
        nb += u[y + 1, x]
    else:
        walls += 1
    g = (nb - h2 * f[y, x]) / (4 + walls)
    u[y, x] = u[y, x] + omega * (g - u[y, x])


def grid_sweeps(u, f, h2, ns, omega):
    """ns red-black half sweeps over the whole grid (colour s & 1)."""
    n = u.shape[0]
    u = u.copy()
    for s in range(ns):
        for y in range(n):
            for x in range(n):
                if (x + y) % 2 == s % 2:
                    _gs_point(u, f, h2, x, y, n, omega)
    return u


def staged_sweeps(u, f, h2, ns, omega, tx0, ty0, TX, TY, H):
    """The same half sweeps on the region of one tile (halo H), updating in
    half sweep s only the cells at least s + 1 from every cut side; returns
    the region's values (NaN outside it)."""
    n = u.shape[0]
    ax, bx = max(tx0 - H, 0), min(tx0 + TX + H - 1, n - 1)
    ay, by = max(ty0 - H, 0), min(ty0 + TY + H - 1, n - 1)
    cl, cr, cb, ct = ax > 0, bx < n - 1, ay > 0, by < n - 1
    r = np.full_like(u, np.nan)
    r[ay:by + 1, ax:bx + 1] = u[ay:by + 1, ax:bx + 1]
    for s in range(ns):
        X0 = ax + s + 1 if cl else ax
        X1 = bx - s - 1 if cr else bx
        Y0 = ay + s + 1 if cb else ay
        Y1 = by - s - 1 if ct else by
        for y in range(Y0, Y1 + 1):
            for x in range(X0, X1 + 1):
                if (x + y) % 2 == s % 2:
                    _gs_point(r, f, h2, x, y, n, omega)
    return r


@pytest.mark.parametrize("ns", [2, 4, 6])
@pytest.mark.parametrize("warm", [False, True])
def test_staged_tiles_reproduce_the_grid_sweeps(ns, warm):
    rng = np.random.default_rng(ns + 10 * warm)
    n, TX, TY = 24, 8, 4
    f = rng.standard_normal((n, n))
    u0 = rng.standard_normal((n, n)) if warm else np.zeros((n, n))
    h2, omega = 0.1, 1.2
    ref = grid_sweeps(u0, f, h2, ns, omega)
    for ty0 in range(0, n, TY):
        for tx0 in range(0, n, TX):
            # halo ns + 1: the tile and its ring are exact
            r = staged_sweeps(u0, f, h2, ns, omega, tx0, ty0, TX, TY, ns + 1)
            y0, y1 = max(ty0 - 1, 0), min(ty0 + TY, n - 1)
            x0, x1 = max(tx0 - 1, 0), min(tx0 + TX, n - 1)
            assert np.array_equal(r[y0:y1 + 1, x0:x1 + 1], ref[y0:y1 + 1, x0:x1 + 1])
            # halo ns: the tile alone is exact
            r = staged_sweeps(u0, f, h2, ns, omega, tx0, ty0, TX, TY, ns)
            assert np.array_equal(r[ty0:ty0 + TY, tx0:tx0 + TX], ref[ty0:ty0 + TY, tx0:tx0 + TX])


def test_a_narrower_halo_is_not_exact():
    """With a halo of ns - 1 a tile away from the walls differs: the halo
    widths above are the smallest that work."""
    rng = np.random.default_rng(7)
    n, ns, TX, TY = 24, 4, 8, 4
    f = rng.standard_normal((n, n))
    u0 = rng.standard_normal((n, n))
    ref = grid_sweeps(u0, f, 0.1, ns, 1.2)
    r = staged_sweeps(u0, f, 0.1, ns, 1.2, 8, 8, TX, TY, ns - 1)
    assert not np.array_equal(r[8:12, 8:16], ref[8:12, 8:16])
