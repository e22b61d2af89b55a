"""Differentiable form on the GPU: gradients of the witness energy gain (GPU).

The loss L(theta, table) = mean energy gain of the witness over one bunch
push after one 3D step; theta are the driver's eight bi-Gaussian parameters
and table the radial plasma-density profile.  The CUDA adjoint (reverse
slice loop with checkpoints, behind a torch.autograd.Function) is checked
against the gradient oracle (autograd of the float64 restatement, itself
pinned by finite differences of the oracle), against central finite
differences of the CUDA forward, and for invariance under the checkpoint
interval.
"""
import math

import numpy as np
import pytest
import torch

from oracle import qs_grad as QG
import workloads as W

pytestmark = pytest.mark.gpu


def _workload(strong: bool):
    if strong:
        hw, xl, amp, sx, sy, ws = 2.0, 7.0, 20.0, 0.35, 0.3, 0.25
    else:
        hw, xl, amp, sx, sy, ws = 4.0, 3.5, 1.5, 0.6, 0.5, 0.4
    return W.Workload(
        name="g16", n=16, half_width=hw, n_xi=14, xi_len=xl, ppc=4,
        beams=(W.BeamSpec(amplitude=amp, sigma_x=sx, sigma_y=sy, sigma_z=0.45, xi_c=1.0,
                          n_particles=1500, seed=3, x_c=0.1 * hw / 4, y_c=-0.05 * hw / 4,
                          tilt=0.05),
               W.BeamSpec(amplitude=1.0, sigma_x=ws, sigma_y=ws, sigma_z=0.25, xi_c=2.6,
                          n_particles=400, seed=4)),
        profile=((1.0, 1.03, 1.07, 1.12, 1.18, 1.25), hw * math.sqrt(2.0)),
        precision="fp64", dt=2.0)


def _gpu_gradient(qs, wl, P, theta, table, form="fp64", checkpoint_every=0, stored=0,
                  schedule=None):
    ctx = qs.Context(qs.config_from_workload(wl, precision=form, mg_tol=1e-12,
                                             checkpoint_every=stored))
    z = torch.tensor(P.driver_z, dtype=torch.float64, device="cuda")
    witness = qs.Beam(P.witness)
    th = torch.tensor(theta, dtype=torch.float64, requires_grad=True)
    tb = torch.tensor(table, dtype=torch.float64, requires_grad=True)
    L = qs.witness_gain(ctx, th, tb, z, P.driver_gamma, witness, P.dt, wl.ppc, P.r_max,
                        checkpoint_every, schedule)
    m = ctx.slice_diagnostics()[0]
    L.backward()
    return float(L.detach()), th.grad.numpy().copy(), tb.grad.numpy().copy(), m


def _rel(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


@pytest.mark.parametrize("strong", [False, True])
def test_fp64_gradient_matches_the_gradient_oracle(qs, strong):
    wl = _workload(strong)
    P, theta, table = QG.problem_from_workload(wl)
    L, dth, dtb, m = _gpu_gradient(qs, wl, P, theta, table)
    np.testing.assert_array_equal(m, P.m_schedule)
    Lo, dtho, dtbo = QG.gradient(P, theta, table)
    assert abs(L - Lo) <= 1e-9 * abs(Lo)
    scale = max(np.abs(dtho).max(), np.abs(dtbo).max())
    assert np.max(np.abs(dth - dtho)) <= 1e-7 * scale, (dth, dtho)
    assert np.max(np.abs(dtb - dtbo)) <= 1e-7 * scale, (dtb, dtbo)


def test_fp64_gradient_matches_central_differences_of_the_gpu_loss(qs):
    wl = _workload(True)
    P, theta, table = QG.problem_from_workload(wl)
    _, dth, dtb, _ = _gpu_gradient(qs, wl, P, theta, table)
    scale = max(np.abs(dth).max(), np.abs(dtb).max())
    ctx = qs.Context(qs.config_from_workload(wl, mg_tol=1e-13))
    z = torch.tensor(P.driver_z, dtype=torch.float64, device="cuda")
    witness = qs.Beam(P.witness)

    def loss(th, tb):
        ctx.init_plasma(wl.ppc, list(tb), P.r_max)
        drv = qs.bigaussian_beam(th, z, P.driver_gamma)
        ctx.step3d([drv, witness], schedule=P.m_schedule)
        return ctx.beam_gain(witness, P.dt)

    for k in range(8):
        eps = 1e-5 * max(abs(theta[k]), 1.0)
        tp, tm = theta.copy(), theta.copy()
        tp[k] += eps
        tm[k] -= eps
        d = (loss(tp, table) - loss(tm, table)) / (2 * eps)
        assert abs(d - dth[k]) <= 1e-4 * max(abs(d), 1e-3 * scale), (k, d, dth[k])
    for k in range(len(table)):
        eps = 1e-5
        tp, tm = table.copy(), table.copy()
        tp[k] += eps
        tm[k] -= eps
        d = (loss(theta, tp) - loss(theta, tm)) / (2 * eps)
        assert abs(d - dtb[k]) <= 1e-4 * max(abs(d), 1e-3 * scale), ("table", k, d, dtb[k])


def test_refined_gradient_matches_central_differences(qs):
    """The refined form's adjoint (float32 particles and inner cycles in the
    forward, float64 adjoint), schedule frozen, against central differences
    of the float64 CUDA loss with the same schedule: 1e-4 relative.  (The
    refined loss itself carries float32 rounding noise of ~1e-7, too much
    for a difference quotient at 1e-4.)"""
    wl = _workload(True)
    P, theta, table = QG.problem_from_workload(wl)
    _, dth, dtb, m = _gpu_gradient(qs, wl, P, theta, table, form="fp32r",
                                   schedule=P.m_schedule)
    np.testing.assert_array_equal(m, P.m_schedule)
    scale = max(np.abs(dth).max(), np.abs(dtb).max())
    ctx = qs.Context(qs.config_from_workload(wl, mg_tol=1e-13))
    z = torch.tensor(P.driver_z, dtype=torch.float64, device="cuda")
    witness = qs.Beam(P.witness)

    def loss(th, tb):
        ctx.init_plasma(wl.ppc, list(tb), P.r_max)
        drv = qs.bigaussian_beam(th, z, P.driver_gamma)
        ctx.step3d([drv, witness], schedule=P.m_schedule)
        return ctx.beam_gain(witness, P.dt)

    for k in range(8):
        eps = 1e-5 * max(abs(theta[k]), 1.0)
        tp, tm = theta.copy(), theta.copy()
        tp[k] += eps
        tm[k] -= eps
        d = (loss(tp, table) - loss(tm, table)) / (2 * eps)
        assert abs(d - dth[k]) <= 1e-4 * max(abs(d), 1e-2 * scale), (k, d, dth[k])
    for k in range(len(table)):
        eps = 1e-5
        tp, tm = table.copy(), table.copy()
        tp[k] += eps
        tm[k] -= eps
        d = (loss(theta, tp) - loss(theta, tm)) / (2 * eps)
        assert abs(d - dtb[k]) <= 1e-4 * max(abs(d), 1e-2 * scale), ("table", k, d, dtb[k])


def test_checkpoint_interval_does_not_change_the_gradient(qs):
    wl = _workload(True)
    P, theta, table = QG.problem_from_workload(wl)
    ref = _gpu_gradient(qs, wl, P, theta, table, checkpoint_every=0)
    for K in (1, 3, 14):
        got = _gpu_gradient(qs, wl, P, theta, table, checkpoint_every=K)
        assert _rel(got[1], ref[1]) <= 1e-9 and _rel(got[2], ref[2]) <= 1e-9, K
    # checkpoints stored by the forward step itself (no replay in the adjoint);
    # K >= n_xi keeps every slice, so the adjoint recomputes nothing
    for K in (4, 14, 32):
        got = _gpu_gradient(qs, wl, P, theta, table, checkpoint_every=0, stored=K)
        assert _rel(got[1], ref[1]) <= 1e-9 and _rel(got[2], ref[2]) <= 1e-9, ("stored", K)


@pytest.mark.parametrize("strong", [False, True])
def test_refined_form_gradient_against_the_gradient_oracle(qs, strong):
    """Float32 particles and inner cycles in the forward replay, float64
    adjoint arithmetic, the oracle's sub-step schedule held fixed: the
    gradient follows the float64 one to 1e-3."""
    wl = _workload(strong)
    P, theta, table = QG.problem_from_workload(wl)
    L, dth, dtb, m = _gpu_gradient(qs, wl, P, theta, table, form="fp32r",
                                   schedule=P.m_schedule)
    np.testing.assert_array_equal(m, P.m_schedule)
    Lo, dtho, dtbo = QG.gradient(P, theta, table)
    assert abs(L - Lo) <= 1e-4 * abs(Lo)
    scale = max(np.abs(dtho).max(), np.abs(dtbo).max())
    assert np.max(np.abs(dth - dtho)) <= 1e-3 * scale, (dth, dtho)
    assert np.max(np.abs(dtb - dtbo)) <= 1e-3 * scale, (dtb, dtbo)


def test_adjoint_needs_a_forward_step(qs):
    wl = _workload(False)
    ctx = qs.Context(qs.config_from_workload(wl))
    ctx.init_plasma(wl.ppc)
    with pytest.raises(qs.QsError) as e:
        ctx.step3d_adjoint(None)
    assert e.value.status == qs.QS_ERR_STATE


def test_fullsize_directional_derivative(qs):
    """The 256^2 differentiable case (512 slices, 262,144 plasma particles,
    500k + 200k bunch particles, 16-value table): the adjoint's directional
    derivative along a random direction equals the central difference of
    the CUDA loss (same schedule), float64."""
    wl = W.workload("grad256")
    drv, wit = wl.beams
    theta = np.array([drv.amplitude, drv.sigma_x, drv.sigma_y, drv.sigma_z, drv.x_c, drv.y_c,
                      drv.xi_c, drv.tilt])
    table, r_max = np.array(wl.profile[0]), wl.profile[1]
    z = torch.tensor(W.beam_normals(drv.n_particles, drv.seed), dtype=torch.float64,
                     device="cuda")
    witness = qs.Beam(W.sample_beam(wit))
    ctx = qs.Context(qs.config_from_workload(wl, mg_tol=1e-12))
    th = torch.tensor(theta, requires_grad=True)
    tb = torch.tensor(table, requires_grad=True)
    L = qs.witness_gain(ctx, th, tb, z, drv.gamma, witness, wl.dt, wl.ppc, r_max)
    m = ctx.slice_diagnostics()[0]
    L.backward()
    rng = np.random.default_rng(7)
    vth = rng.standard_normal(8) * np.maximum(np.abs(theta), 0.1)
    vtb = rng.standard_normal(len(table)) * 0.05
    dd = float(th.grad.numpy() @ vth + tb.grad.numpy() @ vtb)

    def loss(t):
        ctx.init_plasma(wl.ppc, list(table + t * vtb), r_max)
        b = qs.bigaussian_beam(theta + t * vth, z, drv.gamma)
        st = ctx.step3d([b, witness], schedule=m)
        assert st["psi_guard_hits"] == 0
        return ctx.beam_gain(witness, wl.dt)

    eps = 1e-5
    fd = (loss(eps) - loss(-eps)) / (2 * eps)
    assert abs(fd - dd) <= 1e-4 * abs(fd), (fd, dd)


@pytest.mark.parametrize("n_xi", [1, 2, 5])
def test_short_windows_and_zero_cotangent(qs, n_xi):
    """Edge cases: windows of 1, 2 and 5 slices (the last slice has no push;
    checkpoint interval 1 and 2), against the gradient oracle; a zero
    cotangent gives zero outputs.  With one slice the loss is ~1e-11 (the
    wake of slice 0 alone): the gradient is then at the solver's absolute
    tolerance and only its magnitude is compared."""
    base = _workload(True)
    drv, wit = base.beams
    wl = base.with_(n_xi=n_xi, xi_len=0.5 * n_xi,
                    beams=(drv.with_(xi_c=0.15), wit.with_(xi_c=0.3 * n_xi, sigma_z=0.1)))
    P, theta, table = QG.problem_from_workload(wl)
    for K in (1, 2):
        L, dth, dtb, _ = _gpu_gradient(qs, wl, P, theta, table, checkpoint_every=K)
        Lo, dtho, dtbo = QG.gradient(P, theta, table)
        scale = max(np.abs(dtho).max(), np.abs(dtbo).max(), 1e-300)
        tol = 1e-6 if n_xi > 1 else 1e-2
        assert np.max(np.abs(dth - dtho)) <= tol * scale, (K, dth, dtho)
        assert np.max(np.abs(dtb - dtbo)) <= tol * scale, (K, dtb, dtbo)
    ctx = qs.Context(qs.config_from_workload(wl, mg_tol=1e-12))
    ctx.init_plasma(wl.ppc, list(table), P.r_max)
    ctx.step3d([qs.Beam(W.sample_beam(b)) for b in wl.beams])
    d_jzb, d_w, d_nion, st = ctx.step3d_adjoint(None, 1)
    assert float(d_jzb.abs().max()) == 0.0 and float(d_w.abs().max()) == 0.0
    assert float(d_nion.abs().max()) == 0.0
    assert st["slices"] >= n_xi


def test_fullsize_refined_gradient_follows_the_fp64_gradient(qs):
    """grad256 at full size: the refined form's gradient (float32 particles
    and inner cycles in the forward, float64 adjoint arithmetic) against the
    float64 form's, which the directional-derivative test pins to central
    differences; checkpoints stored by the forward step."""
    wl = W.workload("grad256")
    drv, wit = wl.beams
    theta = [drv.amplitude, drv.sigma_x, drv.sigma_y, drv.sigma_z, drv.x_c, drv.y_c, drv.xi_c,
             drv.tilt]
    table, r_max = list(wl.profile[0]), wl.profile[1]
    z = torch.tensor(W.beam_normals(drv.n_particles, drv.seed), dtype=torch.float64,
                     device="cuda")
    witness = qs.Beam(W.sample_beam(wit))
    out = {}
    for form in ("fp64", "fp32r"):
        ctx = qs.Context(qs.config_from_workload(wl, precision=form, checkpoint_every=32))
        th = torch.tensor(theta, dtype=torch.float64, requires_grad=True)
        tb = torch.tensor(table, dtype=torch.float64, requires_grad=True)
        L = qs.witness_gain(ctx, th, tb, z, drv.gamma, witness, wl.dt, wl.ppc, r_max)
        L.backward()
        out[form] = (float(L.detach()), th.grad.numpy().copy(), tb.grad.numpy().copy())
        ctx.close()
    (L64, g64, t64), (L32, g32, t32) = out["fp64"], out["fp32r"]
    assert abs(L32 - L64) <= 1e-6 * abs(L64)
    scale = max(np.abs(g64).max(), np.abs(t64).max())
    assert np.max(np.abs(g32 - g64)) <= 1e-4 * scale, (g32, g64)
    assert np.max(np.abs(t32 - t64)) <= 1e-4 * scale, (t32, t64)


def test_slice_store_overflow_falls_back_to_recompute(qs):
    """With every slice kept by the forward step (checkpoint_every >= n_xi),
    a schedule with more sub-steps than the store holds (two per base slice)
    is recomputed from the checkpoint instead: same cotangents as without a
    store."""
    wl = _workload(True)
    beams = [qs.Beam(W.sample_beam(b)) for b in wl.beams]
    sched = [3] * wl.n_xi
    outs = []
    for K in (0, 14):
        ctx = qs.Context(qs.config_from_workload(wl, mg_tol=1e-12, checkpoint_every=K))
        ctx.init_plasma(wl.ppc, list(wl.profile[0]), wl.profile[1])
        st = ctx.step3d(beams, schedule=sched)
        assert st["slices"] == 3 * (wl.n_xi - 1) + 1
        d_hist = torch.zeros((5, wl.n_xi, wl.n, wl.n), dtype=torch.float64, device="cuda")
        ctx.beam_gain(beams[1], wl.dt, d_hist)
        outs.append([t.cpu().numpy() for t in ctx.step3d_adjoint(d_hist)[:3]])
    for a, b in zip(*outs):
        assert np.max(np.abs(a - b)) <= 1e-9 * max(np.max(np.abs(b)), 1e-300)
