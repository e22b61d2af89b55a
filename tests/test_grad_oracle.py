"""Pins of the gradient oracle (CPU).

The gradient oracle restates the forward of qs_oracle in torch and lets
autograd differentiate it.  It is pinned to two things outside itself:
the forward of qs_oracle (same history and loss to rounding), and central
finite differences of the loss computed by qs_oracle alone, for every
driver parameter and every profile coefficient.
"""
import math

import numpy as np
import pytest
import torch

import oracle as O
from oracle import qs_grad as QG
import workloads as W


def small_problem(strong=False):
    """16^2 cells, 14 slices; the strong driver (n_b = 20 on a finer box)
    refines the xi step (sub-steps) and drives orbits across cells."""
    if strong:
        hw, xl, amp, sx, sy, ws = 2.0, 7.0, 20.0, 0.35, 0.3, 0.25
    else:
        hw, xl, amp, sx, sy, ws = 4.0, 3.5, 1.5, 0.6, 0.5, 0.4
    wl = W.Workload(
        name="g16", n=16, half_width=hw, n_xi=14, xi_len=xl, ppc=4,
        beams=(W.BeamSpec(amplitude=amp, sigma_x=sx, sigma_y=sy, sigma_z=0.45, xi_c=1.0,
                          n_particles=1500, seed=3, x_c=0.1 * hw / 4, y_c=-0.05 * hw / 4,
                          tilt=0.05),
               W.BeamSpec(amplitude=1.0, sigma_x=ws, sigma_y=ws, sigma_z=0.25, xi_c=2.6,
                          n_particles=400, seed=4)),
        profile=((1.0, 1.03, 1.07, 1.12, 1.18, 1.25), hw * math.sqrt(2.0)),
        precision="fp64", dt=2.0)
    return QG.problem_from_workload(wl)


def test_driver_mapping_matches_the_input_generator():
    spec = W.BeamSpec(amplitude=2.0, sigma_x=0.6, sigma_y=0.5, sigma_z=0.45, xi_c=1.0,
                      n_particles=300, seed=3, x_c=0.1, y_c=-0.05, tilt=0.05)
    a = W.sample_beam(spec)
    b = QG.driver_beam_numpy([2.0, 0.6, 0.5, 0.45, 0.1, -0.05, 1.0, 0.05],
                             W.beam_normals(300, 3), spec.gamma, spec.charge)
    for k in ("x", "y", "xi", "px", "py", "pz", "w"):
        np.testing.assert_allclose(a[k], b[k], rtol=1e-15, atol=0)


def test_torch_forward_equals_oracle_forward():
    P, theta, table = small_problem()
    loss, hist = QG.loss_torch(P, torch.tensor(theta), torch.tensor(table), return_history=True)
    pl, n_ion = O.init_plasma(P.cfg.grid, P.ppc, list(table), P.r_max)
    drv = QG.driver_beam_numpy(theta, P.driver_z, P.driver_gamma, P.driver_charge)
    ref = O.step3d(P.cfg, pl, n_ion, [drv, P.witness], m_schedule=P.m_schedule)
    h = hist.detach().numpy()
    assert np.linalg.norm(h - ref.history) <= 1e-12 * np.linalg.norm(ref.history)
    ln = QG.loss_numpy(P, theta, table)
    assert abs(float(loss) - ln) <= 1e-12 * abs(ln)
    assert ln != 0.0


@pytest.mark.parametrize("strong", [False, True])
def test_gradient_equals_central_differences(strong):
    """Every driver parameter and profile coefficient; the strong driver
    makes the schedule refine (sub-steps) and the plasma orbits cross cells."""
    P, theta, table = small_problem(strong=strong)
    if strong:
        assert P.m_schedule.max() > 1
    L, dth, dtb = QG.gradient(P, theta, table)
    scale = max(np.abs(dth).max(), np.abs(dtb).max())

    def fd(vec, k, other, is_theta):
        eps = 1e-6 * max(abs(vec[k]), 1.0)
        out = []
        for s in (1.0, -1.0):
            v = vec.copy()
            v[k] += s * eps
            out.append(QG.loss_numpy(P, v, other) if is_theta else QG.loss_numpy(P, other, v))
        return (out[0] - out[1]) / (2 * eps)

    for k in range(len(theta)):
        d = fd(theta, k, table, True)
        assert abs(d - dth[k]) <= 1e-5 * scale + 1e-4 * abs(d), (QG.DRIVER_PARAM_NAMES[k], d, dth[k])
    for k in range(len(table)):
        d = fd(table, k, theta, False)
        assert abs(d - dtb[k]) <= 1e-5 * scale + 1e-4 * abs(d), ("table", k, d, dtb[k])
