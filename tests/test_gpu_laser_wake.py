"""The laser driver inside the slice loop on the GPU against the oracle (GPU).

qs_step3d_laser adds the laser terms of the slice advance (|A|^2 / 2 in
gamma, the ponderomotive force -grad(|A|^2/4)/(1+psi) in the push, Eq.
EoM_111 and the line after it; -n_* grad(|A|^2/4)/(1+psi)^2 in the source S
of Eq. FluxCurr1_A) and returns chi = n_*/(1+psi) at the base slices for Eq.
laser_Enve.  qs_laser_step3d chains it with one envelope time step.  Both are
compared element by element with the oracle's step3d(laser_a2=...) and
laser_step3d: 1e-9 relative L2 per field in float64, 2e-5 in the refined form.
"""
import math

import numpy as np
import pytest
import torch

import oracle as O
from oracle import qs_laser as QL
import workloads as W

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-9, "fp32r": 2e-5}


def _a2(wl, a0, w0, sigma, xi_c):
    """|A|^2 of a Gaussian envelope A = a0 exp(-r^2/w0^2 - (xi - xi_c)^2 /
    sigma^2) at the cell centres of the base slices."""
    h = 2 * wl.half_width / wl.n
    x = -wl.half_width + (np.arange(wl.n) + 0.5) * h
    X, Y = np.meshgrid(x, x)
    xi = np.arange(wl.n_xi) * wl.xi_len / wl.n_xi
    env = np.exp(-2.0 * ((xi - xi_c) / sigma) ** 2)
    return a0 * a0 * env[:, None, None] * np.exp(-2.0 * (X * X + Y * Y) / w0 ** 2)[None]


def _gpu(qs, wl, form, a2, beams_np=(), n_prefix=None):
    ctx = qs.Context(qs.config_from_workload(wl, precision=form, mg_tol=1e-12))
    ctx.init_plasma(wl.ppc)
    a2_d = torch.tensor(a2, device="cuda")
    chi = torch.zeros_like(a2_d)
    st = ctx.step3d_laser([qs.Beam(b) for b in beams_np], a2_d, chi)
    n = n_prefix or wl.n_xi
    got = ctx.fields(qs.FIELD_ALL, 0, n, device=False).numpy()
    out = got, chi[:n].cpu().numpy(), st
    ctx.close()
    return out


def _compare(got, chi, ref_hist, ref_chi, tol):
    scale = np.linalg.norm(ref_hist[0])
    errs = {nm: np.linalg.norm(got[i] - ref_hist[i]) / max(np.linalg.norm(ref_hist[i]), scale)
            for i, nm in enumerate(O.FIELD_NAMES)}
    errs["chi"] = np.linalg.norm(chi - ref_chi) / np.linalg.norm(ref_chi)
    assert max(errs.values()) < tol, errs
    return errs


@pytest.mark.parametrize("form", ["fp64", "fp32r"])
def test_laser_only_wake(qs, form):
    wl = W.Workload(name="l32", n=32, half_width=4.0, n_xi=32, xi_len=6.4, ppc=4, beams=())
    a2 = _a2(wl, a0=1.5, w0=1.5, sigma=1.0, xi_c=2.0)
    got, chi, st = _gpu(qs, wl, form, a2)
    assert st["psi_guard_hits"] == 0
    cfg = O.config_from_workload(wl)
    pl, n_ion = O.plasma_from_workload(wl)
    ref = O.step3d(cfg, pl, n_ion, [], jzb=np.zeros_like(a2), laser_a2=a2)
    _compare(got, chi, ref.history, ref.chi, TOL[form])
    np.testing.assert_array_equal(qs_m(qs, wl, form, a2), ref.m)


def qs_m(qs, wl, form, a2):
    ctx = qs.Context(qs.config_from_workload(wl, precision=form, mg_tol=1e-12))
    ctx.init_plasma(wl.ppc)
    ctx.step3d_laser([], torch.tensor(a2, device="cuda"))
    m = ctx.slice_diagnostics()[0]
    ctx.close()
    return m


@pytest.mark.parametrize("form", ["fp64", "fp32r"])
def test_laser_and_beam_driver_on_a_ragged_grid(qs, form):
    """48^2 (coarsest level 3), a laser with a weaker beam behind it and
    sub-steps from the refinement rule."""
    wl = W.Workload(name="lb48", n=48, half_width=4.0, n_xi=30, xi_len=9.0, ppc=4,
                    beams=(W.BeamSpec(amplitude=6.0, sigma_x=0.4, sigma_y=0.4, sigma_z=0.6,
                                      xi_c=5.7, n_particles=6000, seed=9),))
    a2 = _a2(wl, a0=2.5, w0=1.2, sigma=1.2, xi_c=2.4)
    beams_np = [W.sample_beam(b) for b in wl.beams]
    got, chi, st = _gpu(qs, wl, form, a2, beams_np)
    assert st["psi_guard_hits"] == 0
    cfg = O.config_from_workload(wl)
    pl, n_ion = O.plasma_from_workload(wl)
    ref = O.step3d(cfg, pl, n_ion, beams_np, laser_a2=a2)
    assert ref.m.max() > 1  # the sub-step path with interpolated |A|^2
    _compare(got, chi, ref.history, ref.chi, TOL[form])


def test_zero_envelope_is_the_plain_step(qs):
    wl = W.workload("linear64").with_(n_xi=24, xi_len=3.0)
    beams_np = [W.sample_beam(b.with_(xi_c=1.5)) for b in wl.beams]
    ctx = qs.Context(qs.config_from_workload(wl, mg_tol=1e-12))
    ctx.init_plasma(wl.ppc)
    ctx.step3d([qs.Beam(b) for b in beams_np])
    plain = ctx.fields(qs.FIELD_ALL, device=False).numpy()
    z = torch.zeros((wl.n_xi, wl.n, wl.n), dtype=torch.float64, device="cuda")
    chi = torch.zeros_like(z)
    ctx.step3d_laser([qs.Beam(b) for b in beams_np], z, chi)
    las = ctx.fields(qs.FIELD_ALL, device=False).numpy()
    assert np.linalg.norm(las - plain) <= 1e-12 * np.linalg.norm(plain)
    # chi = n_*/(1+psi) at the base slices, n_* = 1 at the head
    assert abs(float(chi[0].mean()) - 1.0) < 1e-12
    # the adjoint does not cover the laser terms
    with pytest.raises(qs.QsError) as e:
        ctx.step3d_adjoint(None)
    assert e.value.status == qs.QS_ERR_STATE
    with pytest.raises(qs.QsError):
        ctx.step3d_laser([], z[:-1].contiguous())
    ctx.close()


@pytest.mark.parametrize("form", ["fp64", "fp32r"])
def test_laser_driven_step_with_the_envelope_advance(qs, form):
    """qs_laser_step3d = the wake with |A|^2 of the envelope, then one time
    step of Eq. laser_Enve with the wake's chi, against QL.laser_step3d."""
    wl = W.Workload(name="ld32", n=32, half_width=4.0, n_xi=24, xi_len=4.8, ppc=4, beams=())
    k0, dt = 6.0, 1.0
    h = 2 * wl.half_width / wl.n
    x = -wl.half_width + (np.arange(wl.n) + 0.5) * h
    X, Y = np.meshgrid(x, x)
    xi = np.arange(wl.n_xi) * wl.xi_len / wl.n_xi
    env = (1.2 * np.exp(-((xi - 1.6) / 0.7) ** 2)[:, None, None] *
           np.exp(-(X * X + Y * Y) / 1.5 ** 2)[None]).astype(np.complex128)
    env = env * np.exp(0.3j * X)[None]  # a tilted phase front
    ctx = qs.Context(qs.config_from_workload(wl, precision=form, mg_tol=1e-12))
    ctx.init_plasma(wl.ppc)
    lz = qs.LaserEnvelope(wl.n, 2 * wl.half_width, wl.n_xi, k0, dt, wl.xi_len / wl.n_xi)
    a = torch.tensor(env, device="cuda")
    st = ctx.laser_step3d(lz, a, tol=1e-12)
    got = ctx.fields(qs.FIELD_ALL, device=False).numpy()
    new = a.cpu().numpy()
    lz.close()
    ctx.close()
    cfg = O.config_from_workload(wl)
    pl, n_ion = O.plasma_from_workload(wl)
    ref, ref_env = QL.laser_step3d(cfg, pl, n_ion, env, k0=k0, dt=dt)
    assert st["env_cycles"] > 0
    scale = np.linalg.norm(ref.history[0])
    for i in range(5):
        assert np.linalg.norm(got[i] - ref.history[i]) <= TOL[form] * max(
            np.linalg.norm(ref.history[i]), scale), i
    assert np.linalg.norm(new - ref_env) <= TOL[form] * np.linalg.norm(ref_env)


def test_laser_step_rejects_a_mismatched_envelope(qs):
    wl = W.Workload(name="m", n=32, half_width=4.0, n_xi=8, xi_len=1.6, ppc=4, beams=())
    ctx = qs.Context(qs.config_from_workload(wl))
    ctx.init_plasma(wl.ppc)
    lz = qs.LaserEnvelope(wl.n, 2 * wl.half_width, wl.n_xi, 6.0, 1.0, 0.3)  # other spacing
    a = torch.zeros((wl.n_xi, wl.n, wl.n), dtype=torch.complex128, device="cuda")
    with pytest.raises(qs.QsError) as e:
        ctx.laser_step3d(lz, a)
    assert e.value.status == qs.QS_ERR_ARG
    lz.close()
    ctx.close()


@pytest.mark.slow
@pytest.mark.parametrize("form", ["fp64", "fp32r"])
def test_fullsize_laser_wake_prefix(qs, form):
    """The 256^2 laser case (box 24, slices of 0.08, a0 = 2, w0 = 3,
    sigma_xi = 2 centred 4 behind the head, as the paper's laser blowout of
    Table 1 scaled to this grid): the first 80 base slices, through the
    pulse's peak, element by element."""
    from workloads.laser import gaussian_pulse, laser_workload
    lw = laser_workload("laser256")
    wl = W.Workload(name="lw256", n=lw.n, half_width=lw.width / 2, n_xi=lw.n_xi,
                    xi_len=lw.n_xi * lw.dxi, ppc=4, beams=())
    a2 = np.abs(gaussian_pulse(lw)) ** 2
    n = 80
    got, chi, st = _gpu(qs, wl, form, a2, n_prefix=n)
    assert st["psi_guard_hits"] == 0
    cfg = O.config_from_workload(wl)
    pl, n_ion = O.plasma_from_workload(wl)
    ref = O.step3d(cfg, pl, n_ion, [], jzb=np.zeros((n + 1, wl.n, wl.n)), n_slices=n,
                   laser_a2=a2)
    errs = _compare(got, chi, ref.history, ref.chi, TOL[form])
    print(form, {k: f"{v:.2e}" for k, v in errs.items()})
