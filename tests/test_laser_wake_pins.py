"""Pins of the oracle's laser-driver terms in the slice advance.

Eq. EoM_111 and the line after it: gamma = (1 + p_perp^2 + (1+psi)^2 +
|A|^2/2) / (2 (1+psi)) and the ponderomotive force -grad(|A|^2/4) / (1+psi);
Eq. FluxCurr1_A: the matching term of S.  Checked against the mass shell
gamma^2 = 1 + p^2 + |A|^2/2 (the envelope-averaged a^2 is |A|^2/2), energy
conservation of an electron expelled from a static envelope (H = p^2/2 +
|A|^2/4 with psi = 0), and the linear laser wake: for a weak envelope the
push, deposit and psi solve give grad_perp^2 [(d_xi^2 + 1) psi - |A|^2/4] = 0,
so psi = int sin(xi - xi') |A|^2(xi')/4 dxi' at every transverse point.
"""
import math

import numpy as np

from oracle import qs_oracle as Q


def test_mass_shell_with_laser():
    rng = np.random.default_rng(4)
    px, py = rng.normal(0, 2, 1000), rng.normal(0, 2, 1000)
    a = rng.uniform(0.05, 3.0, 1000)
    a2 = rng.uniform(0.0, 9.0, 1000)
    gam = Q.gamma_qs(px, py, a, a2)
    pz = gam - a
    np.testing.assert_allclose(gam * gam - px * px - py * py - pz * pz, 1.0 + 0.5 * a2,
                               rtol=1e-10)


def _expel(n, dxi, steps):
    g = Q.Grid.square(n, 6.0)
    x = g.x_min + (np.arange(n) + 0.5) * g.h
    X, Y = np.meshgrid(x, x)
    a2 = 0.25 * np.exp(-2.0 * (X ** 2 + Y ** 2) / 4.0)
    z = np.zeros((n, n))
    F = Q.SliceFields(z, z, z, z, z, z, z, {}, 0.0, 0, a2, Q.ddx(0.25 * a2, g.h, "even"),
                      Q.ddy(0.25 * a2, g.h, "even"))
    pl = Q.Plasma(np.array([0.8]), np.array([0.3]), np.zeros(1), np.zeros(1), np.ones(1),
                  np.zeros(1, dtype=np.int32))
    h0 = 0.25 * Q.gather(a2, pl.x, pl.y, g)[0]
    worst = 0.0
    for _ in range(steps):
        pl, _, _ = Q.push_plasma(g, pl, F, dxi, 1e-3)
        hk = 0.5 * (pl.px[0] ** 2 + pl.py[0] ** 2) + 0.25 * Q.gather(a2, pl.x, pl.y, g)[0]
        worst = max(worst, abs(hk - h0) / h0)
    return pl, worst


def test_ponderomotive_expulsion_conserves_energy():
    pl, worst = _expel(128, 0.01, 600)
    r = math.hypot(pl.x[0], pl.y[0])
    assert r > 1.4                                   # pushed out of the intensity
    assert abs(pl.px[0] / pl.py[0] - 0.8 / 0.3) < 0.05   # radially
    assert worst < 5e-3
    _, worst64 = _expel(64, 0.01, 600)
    assert worst64 / worst > 3.0                     # the error is the grid's, O(h^2)


def _linear_wake_error(n):
    hw, w0, a0, n_xi, length, xic, sig = 8.0, 3.0, 0.1, 160, 8.0, 2.0, 0.7
    cfg = Q.Config(n, -hw, hw, -hw, hw, n_xi, 0.0, length, refine_k=1)
    g = cfg.grid
    pl, n_ion = Q.init_plasma(g, 4)
    x = g.x_min + (np.arange(n) + 0.5) * g.h
    X, Y = np.meshgrid(x, x)
    xi = np.arange(n_xi) * cfg.dxi0
    a2 = (a0 * a0 * np.exp(-2.0 * ((xi - xic) / sig) ** 2)[:, None, None]
          * np.exp(-2.0 * (X ** 2 + Y ** 2) / w0 ** 2)[None])
    r = Q.step3d(cfg, pl, n_ion, [], jzb=np.zeros((n_xi, n, n)), laser_a2=a2,
                 m_schedule=[1] * n_xi)
    psi = r.history[0]
    assert r.chi is not None and r.chi.shape == psi.shape
    ref = np.zeros_like(psi)
    for j in range(n_xi):
        w = np.sin(xi[j] - xi[:j + 1]) * cfg.dxi0
        w[0] *= 0.5
        w[-1] *= 0.5
        ref[j] = np.tensordot(w, a2[:j + 1] / 4.0, axes=(0, 0))
    behind = xi > xic + 3 * sig
    return np.abs(psi[behind] - ref[behind]).max() / np.abs(ref[behind]).max()


def test_linear_laser_wake():
    e32, e64 = _linear_wake_error(32), _linear_wake_error(64)
    assert e64 < 0.05, e64
    assert e32 / e64 > 3.0, (e32, e64)
