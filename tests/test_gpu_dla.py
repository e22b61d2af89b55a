"""Driver push in the laser's high-frequency fields on the GPU (GPU).

qs_push_beam_dla against oracle/qs_dla.push_beam_dla (Eqs. E_B_Fields,
EoM_beam_1/2, sub-cycled): both start from their own 3D step of the same
problem (the stored wakes agree to the solver tolerance) and push the same
witness bunch in the same envelopes; and, without a laser, the sub-cycled push
equals the plain driver push repeated, bit for bit.
"""
import math

import numpy as np
import pytest
import torch

import oracle as O
from oracle import qs_dla as D
import workloads as W

pytestmark = pytest.mark.gpu


def _problem():
    wl = W.Workload(name="dla32", n=32, half_width=4.0, n_xi=40, xi_len=8.0, ppc=4,
                    beams=(W.BeamSpec(amplitude=1.0, sigma_x=0.5, sigma_y=0.5, sigma_z=0.6,
                                      xi_c=1.8, n_particles=6000, seed=1),))
    h = 2 * wl.half_width / wl.n
    x = -wl.half_width + (np.arange(wl.n) + 0.5) * h
    X, Y = np.meshgrid(x, x)
    xi = np.arange(wl.n_xi) * wl.xi_len / wl.n_xi

    def env(shift):
        e = (0.8 * np.exp(-((xi - 4.0 - shift) / 1.2) ** 2)[:, None, None]
             * np.exp(-(X * X + Y * Y) / 2.0 ** 2)[None]).astype(np.complex128)
        return e * np.exp(0.2j * Y + 0.1j * shift)[None]
    wit = W.sample_beam(W.BeamSpec(amplitude=0.05, sigma_x=0.7, sigma_y=0.7, sigma_z=0.5,
                                   xi_c=4.5, n_particles=3000, seed=2))
    wit["pz"] = np.full_like(wit["pz"], 20.0)  # a slow witness that dephases
    return wl, env(0.0), env(0.05), wit


def test_dla_push_matches_the_oracle(qs):
    wl, env_n, env_np1, wit = _problem()
    k0, dt, n_sub = 5.0, 1.5, 12
    beams_np = [W.sample_beam(b) for b in wl.beams]
    ctx = qs.Context(qs.config_from_workload(wl, mg_tol=1e-12))
    ctx.init_plasma(wl.ppc)
    ctx.step3d([qs.Beam(b) for b in beams_np])
    b = qs.Beam(wit)
    en = torch.tensor(env_n, device="cuda")
    ep = torch.tensor(env_np1, device="cuda")
    ctx.push_beam_dla([b], dt, en, ep, k0, n_sub)
    got = b.numpy()
    cfg = O.config_from_workload(wl)
    pl, n_ion = O.plasma_from_workload(wl)
    hist = O.step3d(cfg, pl, n_ion, beams_np).history
    ref = D.push_beam_dla(cfg, hist, env_n, env_np1, k0, dict(wit), dt, n_sub)
    for k in ("px", "py", "pz"):
        d_ref = ref[k] - wit[k]
        assert np.max(np.abs((got[k] - wit[k]) - d_ref)) <= 1e-8 * np.max(np.abs(d_ref)), k
    for k in ("x", "y", "xi"):
        assert np.max(np.abs(got[k] - ref[k])) <= 1e-10 * max(1.0, np.max(np.abs(ref[k]))), k
    # the laser did something: the momentum change differs from the wake push's
    b2 = qs.Beam(wit)
    ctx.push_beam([b2], dt)
    assert np.max(np.abs(b2.numpy()["px"] - got["px"])) > 1e-3
    ctx.close()


def test_no_laser_is_the_plain_push_repeated(qs):
    wl, env_n, _, wit = _problem()
    beams_np = [W.sample_beam(b) for b in wl.beams]
    ctx = qs.Context(qs.config_from_workload(wl))
    ctx.init_plasma(wl.ppc)
    ctx.step3d([qs.Beam(b) for b in beams_np])
    zero = torch.zeros(env_n.shape, dtype=torch.complex128, device="cuda")
    a, b = qs.Beam(wit), qs.Beam(wit)
    ctx.push_beam_dla([a], 2.0, zero, zero, 5.0, 4)
    for _ in range(4):
        ctx.push_beam([b], 0.5)
    torch.cuda.synchronize()
    for k in qs.Beam.KEYS:
        assert torch.equal(a.t[k], b.t[k]), k
    with pytest.raises(qs.QsError):
        ctx.push_beam_dla([a], 2.0, zero, zero, 5.0, 0)
    ctx.close()


def test_electron_in_a_plane_wave(qs):
    """A constant envelope a0 is the plane wave A_x = a0 cos(k0 xi): an
    electron starting at rest keeps gamma - p_z = 1 and p_x = A_x(xi) -
    A_x(xi_0), to second and first order in the sub-step (the oracle's pin),
    and the GPU follows the oracle."""
    wl = W.Workload(name="pw", n=16, half_width=4.0, n_xi=40, xi_len=4.0, ppc=1, beams=())
    ctx = qs.Context(qs.config_from_workload(wl))
    ctx.init_plasma(1)
    ctx.step3d([])
    a0, k0, dt = 0.5, 5.0, 1.0
    env = torch.full((wl.n_xi, wl.n, wl.n), a0, dtype=torch.complex128, device="cuda")
    e = dict(x=np.array([0.0]), y=np.array([0.0]), xi=np.array([2.0]), px=np.zeros(1),
             py=np.zeros(1), pz=np.zeros(1), w=np.ones(1), charge=-1.0, q_over_m=-1.0)
    errs = []
    for n_sub in (200, 400):
        b = qs.Beam(e)
        ctx.push_beam_dla([b], dt, env, env, k0, n_sub)
        r = b.numpy()
        gam = math.sqrt(1 + r["px"][0] ** 2 + r["py"][0] ** 2 + r["pz"][0] ** 2)
        errs.append(abs(gam - r["pz"][0] - 1.0))
        canon = r["px"][0] - a0 * (math.cos(k0 * r["xi"][0]) - math.cos(k0 * 2.0))
        assert abs(canon) < 0.02, canon
    assert errs[1] < errs[0] / 3.0, errs
    ctx.close()
