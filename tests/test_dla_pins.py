"""Pins of the driver push in the laser's fields (Eqs. E_B_Fields,
EoM_beam_1/2, sub-cycling).

An electron starting at rest in a plane wave A_x = a0 cos(k0 xi) keeps
gamma - p_z = 1 and p_x = A_x(xi) - A_x(xi_0) (conserved canonical momentum
for charge -1, luminal phase velocity); the rebuilt fields of a transversely
shaped envelope satisfy Gauss's law d_x E_x + d_z E_z = 0 and div B =
d_y B_y + d_z B_z = 0 (d_z = -d_xi at fixed t); without a laser the push is
the wake push sub-stepped.
"""
import math

import numpy as np

from oracle import qs_dla as D
from oracle import qs_oracle as Q


def _cfg(n=16, hw=4.0, n_xi=40, length=4.0):
    return Q.Config(n, -hw, hw, -hw, hw, n_xi, 0.0, length)


def _electron(xi0, x=0.0, y=0.0, pz=0.0):
    return dict(x=np.array([x]), y=np.array([y]), xi=np.array([xi0]), px=np.zeros(1),
                py=np.zeros(1), pz=np.array([pz]), w=np.ones(1), charge=-1.0, q_over_m=-1.0)


def _plane_wave_errors(n_sub, a0=0.5, k0=5.0, dt=1.0):
    cfg = _cfg()
    env = np.full((cfg.n_xi, cfg.n, cfg.n), a0, dtype=np.complex128)
    hist = np.zeros((5, cfg.n_xi, cfg.n, cfg.n))
    b0 = _electron(2.0)
    b = D.push_beam_dla(cfg, hist, env, env, k0, b0, dt, n_sub)
    gam = math.sqrt(1.0 + b["px"][0] ** 2 + b["py"][0] ** 2 + b["pz"][0] ** 2)
    ax = lambda xi: a0 * math.cos(k0 * xi)
    canon = b["px"][0] - (ax(b["xi"][0]) - ax(b0["xi"][0]))
    return abs(gam - b["pz"][0] - 1.0), abs(canon), b


def test_electron_in_a_plane_wave():
    g200, c200, _ = _plane_wave_errors(200)
    g400, c400, b = _plane_wave_errors(400)
    assert g400 < 1e-6 and g200 / g400 > 3.5          # gamma - p_z = 1, second order
    assert c400 < 5e-3 and 1.7 < c200 / c400 < 2.3    # canonical momentum, first order
    assert b["pz"][0] > 0.0 and abs(b["py"][0]) < 1e-14
    assert abs(b["pz"][0] - 0.5 * b["px"][0] ** 2) < 1e-5


def test_rebuilt_fields_are_divergence_free():
    cfg = _cfg(n=32, hw=4.0)
    g = cfg.grid
    xc = g.x_min + (np.arange(g.n) + 0.5) * g.h
    X, Y = np.meshgrid(xc, xc)
    a = (0.8 * np.exp(-(X ** 2 + Y ** 2) / 2.0)).astype(np.complex128)
    env = np.repeat(a[None], cfg.n_xi, axis=0)
    k0, xi0 = 6.0, 2.05
    pts_x = xc[8:24]
    y0 = xc[13]
    xs = np.concatenate([pts_x - g.h, pts_x + g.h, pts_x, pts_x])
    eps = 1e-4
    xis = np.concatenate([np.full(32, xi0), np.full(16, xi0 + eps), np.full(16, xi0 - eps)])
    ex, by, ez, bz = D.laser_fields_at(cfg, env, env, 0.0, 1.0, k0, xs, np.full(64, y0), xis)
    dex_dx = (ex[16:32] - ex[:16]) / (2 * g.h)
    dez_dz = -(ez[32:48] - ez[48:64]) / (2 * eps)      # d_z = -d_xi at fixed t
    scale = k0 * np.abs(ez[32:48]).max()
    assert np.abs(dex_dx + dez_dz).max() < 1e-6 * scale
    assert np.abs(dex_dx).max() > 0.1 * scale          # the two terms are not zero alone
    np.testing.assert_allclose(ex, by, rtol=0, atol=1e-12)   # E_x = B_y without d_xi, d_t
    # div B = d_y B_y + d_z B_z = 0 along a column
    pts_y = xc[8:24]
    x0 = xc[13]
    ys = np.concatenate([pts_y - g.h, pts_y + g.h, pts_y, pts_y])
    ex, by, ez, bz = D.laser_fields_at(cfg, env, env, 0.0, 1.0, k0, np.full(64, x0), ys, xis)
    dby_dy = (by[16:32] - by[:16]) / (2 * g.h)
    dbz_dz = -(bz[32:48] - bz[48:64]) / (2 * eps)
    scale = k0 * np.abs(bz[32:48]).max()
    assert np.abs(dby_dy + dbz_dz).max() < 1e-6 * scale
    assert np.abs(dby_dy).max() > 0.1 * scale


def test_without_laser_it_is_the_sub_stepped_wake_push():
    cfg = _cfg()
    rng = np.random.default_rng(9)
    hist = rng.normal(0.0, 0.3, (5, cfg.n_xi, cfg.n, cfg.n))
    zero = np.zeros((cfg.n_xi, cfg.n, cfg.n), dtype=np.complex128)
    b0 = dict(x=rng.uniform(-2, 2, 50), y=rng.uniform(-2, 2, 50), xi=rng.uniform(0.5, 3.5, 50),
              px=rng.normal(0, 1, 50), py=rng.normal(0, 1, 50), pz=np.full(50, 100.0),
              w=np.ones(50), charge=-1.0, q_over_m=-1.0)
    got = D.push_beam_dla(cfg, hist, zero, zero, 5.0, b0, 2.0, 7)
    ref = dict(b0)
    for _ in range(7):
        ref = Q.push_beam(cfg, hist, ref, 2.0 / 7)
    for k in ("x", "y", "xi", "px", "py", "pz"):
        np.testing.assert_array_equal(got[k], ref[k])
