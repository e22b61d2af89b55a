"""Pins of the nonuniform-grid oracle against facts the mathematics fixes.

Sec. "Multigrid Solver with Nonuniform Grids": on a uniform grid the operator
must be the 5-point scheme of Eq. 2D_Laplac_Uni; the three-point differences
are exact on quadratics; the third-order term of Eq. 2D_Laplac is what Taylor
expansion says it is; with the correction of Eq. 2D_Laplac_3rd the truncation
error is second order even where neighbouring spacings differ by a fixed
factor, and first order without it.  Manufactured solutions are products of
sines that vanish on the walls, so J = lap u + M u vanishes there too.
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import qs_nonuniform as nu
from workloads.nonuniform import alternating_axis, three_region_axis, uniform_axis


def _textbook_laplacian(nx, hx, ny, hy):
    tx = sp.diags([1.0, -2.0, 1.0], [-1, 0, 1], shape=(nx, nx)) / (hx * hx)
    ty = sp.diags([1.0, -2.0, 1.0], [-1, 0, 1], shape=(ny, ny)) / (hy * hy)
    return sp.kron(sp.identity(ny), tx) + sp.kron(ty, sp.identity(nx))


def test_uniform_grid_is_five_point():
    xn, yn = uniform_axis(15, 3.0), uniform_axis(11, 2.0)
    rng = np.random.default_rng(5)
    m = -rng.uniform(0.0, 2.0, (11, 15))
    j = rng.standard_normal((11, 15))
    a = nu.operator(xn, yn, m, correction=True)
    ref = _textbook_laplacian(15, xn[1] - xn[0], 11, yn[1] - yn[0]) + sp.diags(m.reshape(-1))
    scale = abs(ref).max()
    assert abs(a - ref).max() <= 1e-13 * scale
    np.testing.assert_allclose(nu.corrected_source(xn, yn, j), j, rtol=0, atol=1e-13)


def _random_axis(n, rng, lo=-2.0, hi=3.0):
    steps = rng.uniform(0.3, 2.0, n + 1)
    x = lo + (hi - lo) * np.concatenate([[0.0], np.cumsum(steps)]) / steps.sum()
    x[-1] = hi
    return x


def test_differences_exact_on_quadratics():
    rng = np.random.default_rng(11)
    xn = _random_axis(40, rng)
    xl, xr = xn[0], xn[-1]
    x = xn[1:-1]
    u = (x - xl) * (xr - x)                  # vanishes on both walls
    np.testing.assert_allclose(nu.second_difference(xn) @ u, -2.0, rtol=0, atol=1e-11)
    np.testing.assert_allclose(nu.first_difference(xn) @ u, xl + xr - 2.0 * x, rtol=0, atol=1e-11)


def test_third_order_term_of_the_second_difference():
    """D2 u = u'' + (h^+ - h^-)/3 u''' exactly for a cubic (Taylor, reading N1)."""
    rng = np.random.default_rng(12)
    xn = _random_axis(30, rng)
    xl, xr, c = xn[0], xn[-1], 0.37
    x = xn[1:-1]
    u = (x - xl) * (xr - x) * (x - c)
    # u = -x^3 + (xl + xr + c) x^2 - ... : u'' = -6x + 2 (xl + xr + c), u''' = -6
    u2 = -6.0 * x + 2.0 * (xl + xr + c)
    hm, hp = nu.spacings(xn)
    np.testing.assert_allclose(nu.second_difference(xn) @ u, u2 + (hp - hm) / 3.0 * -6.0,
                               rtol=0, atol=1e-10)


def _manufactured(xn, yn):
    """u, J = lap u + M u (continuous), M on the interior nodes."""
    wx, wy = xn[-1], yn[-1]
    x = xn[1:-1][None, :]
    y = yn[1:-1][:, None]
    ax1, by1 = math.pi / (2 * wx), 2 * math.pi / (2 * wy)
    ax2, by2 = 2 * math.pi / (2 * wx), math.pi / (2 * wy)
    s1 = np.sin(ax1 * (x + wx)) * np.sin(by1 * (y + wy))
    s2 = np.sin(ax2 * (x + wx)) * np.sin(by2 * (y + wy))
    u = s1 + 0.5 * s2
    lap = -(ax1 ** 2 + by1 ** 2) * s1 - 0.5 * (ax2 ** 2 + by2 ** 2) * s2
    m = -(1.0 + 0.3 * np.sin(x) * np.cos(0.7 * y))
    return u, lap + m * u, m


def _truncation(n, correction):
    xn = alternating_axis(n, 2.0, ratio=2.0)
    yn = alternating_axis(n, 1.5, ratio=3.0, first_long=True)
    u, j, m = _manufactured(xn, yn)
    tau = nu.apply(xn, yn, u, m, correction) - nu.corrected_source(xn, yn, j, correction)
    return np.abs(tau).max()


def test_truncation_second_order_with_correction_first_without():
    sizes = (31, 63, 127, 255)
    corr = [_truncation(n, True) for n in sizes]
    plain = [_truncation(n, False) for n in sizes]
    p_corr = [math.log2(corr[k] / corr[k + 1]) for k in range(len(sizes) - 1)]
    p_plain = [math.log2(plain[k] / plain[k + 1]) for k in range(len(sizes) - 1)]
    assert min(p_corr[-2:]) > 1.8, p_corr
    assert all(0.8 < p < 1.2 for p in p_plain[-2:]), p_plain
    assert corr[-1] < 0.05 * plain[-1]


@pytest.mark.parametrize("axis", ["alternating", "three_region"])
def test_solution_converges_second_order(axis):
    errs = []
    for n in (31, 63, 127):
        if axis == "alternating":
            xn = alternating_axis(n, 2.0, ratio=2.0)
            yn = alternating_axis(n, 1.5, ratio=3.0, first_long=True)
        else:
            xn, yn = three_region_axis(n, 2.0), three_region_axis(n, 1.5)
        u, j, m = _manufactured(xn, yn)
        errs.append(np.abs(nu.solve(xn, yn, j, m) - u).max())
    orders = [math.log2(errs[k] / errs[k + 1]) for k in range(2)]
    assert min(orders) > 1.8, orders


def test_mirror_symmetry():
    """A grid and data symmetric under x -> -x give a symmetric solution."""
    xn = three_region_axis(63, 6.0)
    yn = alternating_axis(31, 3.0, ratio=2.5)
    np.testing.assert_allclose(xn, -xn[::-1], rtol=0, atol=1e-14)
    x = xn[1:-1][None, :]
    y = yn[1:-1][:, None]
    j = np.exp(-(x * x) - (y - 0.3) ** 2) * (1.0 + 0.2 * y)
    m = -(1.0 + 0.5 * np.cos(x) * np.exp(-y * y))
    u = nu.solve(xn, yn, j, m)
    np.testing.assert_allclose(u, u[:, ::-1], rtol=0, atol=1e-12 * np.abs(u).max())


def test_rejects_bad_axes():
    with pytest.raises(ValueError):
        nu.spacings(np.array([0.0, 1.0, 0.5, 2.0]))
    with pytest.raises(ValueError):
        nu.spacings(np.array([0.0, 1.0]))


# ---------------------------------------------------------------- particles (reading N5)
def _particles(xn, yn, count, seed):
    rng = np.random.default_rng(seed)
    x = rng.uniform(xn[0], xn[-1], count)
    y = rng.uniform(yn[0], yn[-1], count)
    return x, y, rng.uniform(0.5, 1.5, count)


def test_node_deposit_conserves_charge_and_areas_tile_the_box():
    xn, yn = three_region_axis(31, 5.0), alternating_axis(15, 3.0, 2.5)
    np.testing.assert_allclose(nu.node_areas(xn, yn).sum(), 10.0 * 6.0, rtol=1e-14)
    x, y, q = _particles(xn, yn, 5000, 1)
    n = nu.deposit(xn, yn, x, y, q)
    np.testing.assert_allclose((n * nu.node_areas(xn, yn)).sum(), q.sum(), rtol=1e-13)


def test_node_gather_is_the_deposit_transpose():
    xn, yn = three_region_axis(31, 5.0), alternating_axis(15, 3.0, 2.5)
    x, y, q = _particles(xn, yn, 3000, 2)
    u = np.random.default_rng(3).standard_normal((15, 31))
    lhs = (nu.gather(u, xn, yn, x, y) * q).sum()
    rhs = (u * nu.deposit(xn, yn, x, y, q) * nu.node_areas(xn, yn)).sum()
    np.testing.assert_allclose(lhs, rhs, rtol=1e-13)


def test_node_gather_reproduces_bilinear_fields_inside():
    xn, yn = three_region_axis(31, 5.0), alternating_axis(15, 3.0, 2.5)
    X, Y = np.meshgrid(xn[1:-1], yn[1:-1])
    u = 0.7 * X - 1.3 * Y + 0.2 * X * Y + 0.5
    rng = np.random.default_rng(4)
    x = rng.uniform(xn[1], xn[-2], 500)          # between interior nodes only
    y = rng.uniform(yn[1], yn[-2], 500)
    np.testing.assert_allclose(nu.gather(u, xn, yn, x, y), 0.7 * x - 1.3 * y + 0.2 * x * y + 0.5,
                               rtol=0, atol=1e-12)


def test_node_deposit_of_a_uniform_density_is_one():
    """A fine uniform lattice of equal weights (density 1) deposits n = 1 at
    every node, walls included, up to the lattice's own discreteness."""
    xn, yn = three_region_axis(31, 5.0), alternating_axis(15, 3.0, 2.5)
    m = 1200
    xs = xn[0] + (np.arange(m) + 0.5) * (xn[-1] - xn[0]) / m
    ys = yn[0] + (np.arange(m) + 0.5) * (yn[-1] - yn[0]) / m
    X, Y = np.meshgrid(xs, ys)
    q = np.full(X.size, (xn[-1] - xn[0]) * (yn[-1] - yn[0]) / X.size)
    n = nu.deposit(xn, yn, X.ravel(), Y.ravel(), q)
    assert np.abs(n - 1.0).max() < 5e-3


def _node_linear_wake_error(n):
    """psi of the node-grid slice advance under a weak bi-Gaussian driver
    against the linear theory of the uniform oracle's closed-form pin:
    psi = n_b int sin(xi - xi') f(xi') dxi' (1 - lap)^-1 g, with the node
    grid's own (1 - lap)^-1 (9-point operator, M = -1)."""
    from oracle import qs_nonuniform_pic as P
    hw, n_xi, nb, sr, sz, xic, length = 6.0, 192, 1e-3, 1.0, 1.0, 3.0, 9.0
    ax = three_region_axis(n, hw)
    G = P.NodeGrid(ax, ax)
    X, Y = np.meshgrid(ax[1:-1], ax[1:-1])
    gr = np.exp(-(X ** 2 + Y ** 2) / sr ** 2)
    dxi = length / n_xi
    xi = np.arange(n_xi) * dxi
    jzb = nb * np.exp(-(xi - xic) ** 2 / sz ** 2)[:, None, None] * gr[None]
    pl, n_ion = P.init_plasma_nodes(G, 4)
    hist, _ = P.step3d_nodes(G, n_xi, dxi, pl, n_ion, jzb)
    ghat = nu.solve(ax, ax, -gr, -np.ones_like(gr))
    xf = np.linspace(0.0, length, 90001)
    ff = np.exp(-(xf - xic) ** 2 / sz ** 2)
    conv = []
    for x0 in xi:
        sel = xf <= x0
        conv.append(np.trapezoid(np.sin(x0 - xf[sel]) * ff[sel], dx=xf[1] - xf[0])
                    if sel.sum() > 1 else 0.0)
    psi_l = nb * np.array(conv)[:, None, None] * ghat[None]
    m = n // 6
    return (np.linalg.norm((hist[0] - psi_l)[:, m:-m, m:-m])
            / np.linalg.norm(psi_l[:, m:-m, m:-m]))


@pytest.mark.slow
def test_node_grid_slice_advance_linear_wake():
    """The whole slice loop on the three-region node grid (deposits, the
    9-point solves of the five fields, the push) reaches the linear beam wake
    at second order in the spacing."""
    e31, e63 = _node_linear_wake_error(31), _node_linear_wake_error(63)
    assert e63 < 0.06, e63
    assert e31 / e63 > 2.5, (e31, e63)


def test_node_quiet_start_is_unit_density():
    from oracle import qs_nonuniform_pic as P
    ax = three_region_axis(31, 5.0)
    G = P.NodeGrid(ax, alternating_axis(15, 3.0, 2.0))
    pl, n_ion = P.init_plasma_nodes(G, 4)
    np.testing.assert_allclose(pl.w.sum(), 10.0 * 6.0, rtol=1e-13)
    assert np.abs(n_ion - 1.0).max() < 0.02
