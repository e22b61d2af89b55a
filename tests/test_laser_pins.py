"""Pins of the laser-envelope oracle (Eq. laser_Enve) against closed forms.

Without the xi coupling the time-centred step of 2 i k0 d_t A = (chi - lap) A
is unitary; in vacuum a Gaussian envelope diffracts as the paraxial beam
A = exp(-r^2 / (w0^2 Q)) / Q, Q = 1 + i t / z_R, z_R = k0 w0^2 / 2; in plasma a
pulse on the transverse mode of wavenumber k_perp slips back in xi at
(chi + k_perp^2) / (2 k0^2) (the dispersion relation Omega = (chi + k_perp^2) /
(2 (k0 - kappa)) of the equation, at kappa = 0); and the xi coupling only
carries information from the head backwards.
"""
import math

import numpy as np

from oracle import qs_laser as QL
from oracle.qs_oracle import Grid


def _centres(g):
    x = g.x_min + (np.arange(g.n) + 0.5) * g.h
    return np.meshgrid(x, x)


def test_unitary_without_xi_coupling():
    g = Grid.square(16, 3.0)
    rng = np.random.default_rng(3)
    a0 = rng.standard_normal((3, 16, 16)) + 1j * rng.standard_normal((3, 16, 16))
    chi = rng.uniform(0.0, 2.0, (3, 16, 16))
    a = QL.envelope_advance(g, a0, chi, k0=5.0, dt=0.7, dxi=math.inf, steps=10)
    for j in range(3):
        np.testing.assert_allclose(np.linalg.norm(a[j]), np.linalg.norm(a0[j]), rtol=1e-12)
    assert np.abs(a - a0).max() > 0.1          # it did evolve


def test_paraxial_gaussian_beam():
    g = Grid.square(128, 10.0)
    X, Y = _centres(g)
    w0, k0 = 2.5, 10.0
    zr = k0 * w0 * w0 / 2.0
    a0 = np.exp(-(X ** 2 + Y ** 2) / w0 ** 2)[None]
    a = QL.envelope_advance(g, a0, np.zeros((1, 128, 128)), k0, zr / 40, math.inf, 40)
    q = 1.0 + 1j                               # t = z_R
    ref = np.exp(-(X ** 2 + Y ** 2) / (w0 ** 2 * q)) / q
    err = np.linalg.norm(a[0] - ref) / np.linalg.norm(ref)
    assert err < 5e-3, err
    # on-axis intensity halves at one Rayleigh length
    c = g.n // 2
    on_axis = np.abs(a[0][c - 1:c + 1, c - 1:c + 1]).mean() ** 2
    assert abs(on_axis - 0.5) < 0.01


def test_group_velocity_slip_in_plasma():
    hw, n = 4.0, 8
    g = Grid.square(n, hw)
    X, Y = _centres(g)
    mode = np.sin(math.pi * (X + hw) / (2 * hw)) * np.sin(math.pi * (Y + hw) / (2 * hw))
    # the mode's eigenvalue under the discrete Laplacian (k_perp^2 = -lam)
    lam = -(8.0 / g.h ** 2) * math.sin(math.pi * g.h / (4 * hw)) ** 2
    k0, dxi, dt, steps = 6.0, 0.05, 1.0, 400
    xi = (np.arange(800) + 0.5) * dxi
    env = np.exp(-((xi - 10.0) / 3.0) ** 2)
    a0 = env[:, None, None] * mode[None]
    a = QL.envelope_advance(g, a0, np.ones((800, n, n)), k0, dt, dxi, steps)
    i0 = (np.abs(a0) ** 2).sum(axis=(1, 2))
    i1 = (np.abs(a) ** 2).sum(axis=(1, 2))
    shift = (xi * i1).sum() / i1.sum() - (xi * i0).sum() / i0.sum()
    expected = (1.0 - lam) / (2 * k0 * k0) * dt * steps
    assert abs(shift / expected - 1.0) < 0.02, (shift, expected)


def test_xi_coupling_runs_from_head_to_tail():
    """Slices ahead of the pulse stay exactly zero."""
    g = Grid.square(8, 2.0)
    X, Y = _centres(g)
    xi = (np.arange(60) + 0.5) * 0.1
    env = np.where(xi > 3.0, np.exp(-((xi - 4.5) / 0.8) ** 2), 0.0)
    a0 = env[:, None, None] * np.exp(-(X ** 2 + Y ** 2))[None]
    a = QL.envelope_advance(g, a0, np.full((60, 8, 8), 0.5), 4.0, 0.5, 0.1, 5)
    assert not a[xi < 3.0].any()
    assert np.abs(a[xi > 3.0]).max() > 0.1


def test_laser_step_hands_the_plasma_susceptibility_to_the_envelope():
    """A weak pulse in uniform plasma: the wake's chi = n_*/(1+psi) is 1 up to
    O(a0^2), and the envelope then advances as it does with chi = 1, not as in
    vacuum."""
    from oracle import qs_oracle as Q
    n, hw, n_xi = 16, 4.0, 48
    cfg = Q.Config(n, -hw, hw, -hw, hw, n_xi, 0.0, 4.8, refine_k=1)
    g = cfg.grid
    X, Y = _centres(g)
    xi = (np.arange(n_xi) + 0.5) * cfg.dxi0
    env = (0.05 * np.exp(-((xi - 2.0) / 0.8) ** 2)[:, None, None]
           * np.exp(-(X ** 2 + Y ** 2) / 2.0)[None]).astype(np.complex128)
    pl, n_ion = Q.init_plasma(g, 4)
    r, new = QL.laser_step3d(cfg, pl, n_ion, env, k0=3.0, dt=2.0, m_schedule=[1] * n_xi)
    assert np.abs(r.chi - 1.0).max() < 5e-3
    with_one = QL.envelope_advance(g, env, np.ones_like(r.chi), 3.0, 2.0, cfg.dxi0, 1)
    vacuum = QL.envelope_advance(g, env, np.zeros_like(r.chi), 3.0, 2.0, cfg.dxi0, 1)
    d1 = np.linalg.norm(new - with_one)
    d0 = np.linalg.norm(new - vacuum)
    assert d1 < 0.02 * d0, (d1, d0)
