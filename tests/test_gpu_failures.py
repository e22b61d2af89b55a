"""Failure statuses of the slice loop, made without faulting the GPU (GPU).

QS_ERR_TIMEOUT: every grid-barrier wait of the persistent slice engine is
bounded.  With the limit set to one clock cycle the first block that has to
wait gives up, records the status and returns, and every other block returns
at its next barrier; the call reports QS_ERR_TIMEOUT and the CUDA context
stays usable: another context on the same device then computes a step that
matches the oracle.

QS_ERR_PSI_FLOOR: 1 + psi is clamped to psi_floor wherever it divides, and a
step that clamps more often than max_psi_guard_hits reports the status.  A
floor just below 1 makes every point where psi < 0 clamp.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu


def _small(n_xi=16):
    return W.Workload(name="f", n=32, half_width=4.0, n_xi=n_xi, xi_len=4.0, ppc=4,
                      beams=(W.BeamSpec(amplitude=1.0, sigma_x=0.5, sigma_y=0.5, sigma_z=0.6,
                                        xi_c=1.5, n_particles=4000, seed=3),), mg_tol=1e-12)


@pytest.mark.parametrize("form", ["fp64", "fp32r"])
def test_barrier_wait_runs_out_and_the_device_stays_usable(qs, form):
    import torch
    wl = _small()
    beams_np = [W.sample_beam(b) for b in wl.beams]
    beams = [qs.Beam(b) for b in beams_np]
    ctx = qs.Context(qs.config_from_workload(wl, precision=form, barrier_wait_cycles=1))
    ctx.init_plasma(wl.ppc)
    st = ctx.step3d(beams, raise_on_error=False)
    assert st["status"] == qs.QS_ERR_TIMEOUT, st
    # the same context reports the same status again (no CUDA error)
    st = ctx.step3d(beams, raise_on_error=False)
    assert st["status"] == qs.QS_ERR_TIMEOUT, st
    ctx.close()
    # the device still works: torch, and a context with the default limit
    assert float(torch.ones(4, device="cuda").sum()) == 4.0
    ctx = qs.Context(qs.config_from_workload(wl, precision=form))
    ctx.init_plasma(wl.ppc)
    ctx.step3d(beams)
    got = ctx.fields(qs.FIELD_ALL, device=False).numpy()
    ctx.close()
    cfg = O.config_from_workload(wl)
    pl, n_ion = O.plasma_from_workload(wl)
    ref = O.step3d(cfg, pl, n_ion, beams_np).history
    tol = 1e-9 if form == "fp64" else 2e-5
    scale = np.linalg.norm(ref[0])
    for i in range(5):
        assert np.linalg.norm(got[i] - ref[i]) <= tol * max(np.linalg.norm(ref[i]), scale)


def test_psi_floor_status_and_count(qs):
    wl = _small()
    beams = [qs.Beam(W.sample_beam(b)) for b in wl.beams]
    # unlimited hits: the step completes and counts the clamps
    ctx = qs.Context(qs.config_from_workload(wl, psi_floor=0.999999))
    ctx.init_plasma(wl.ppc)
    st = ctx.step3d(beams)
    hits = st["psi_guard_hits"]
    assert hits > 0
    ctx.close()
    # a limit well below the count gives QS_ERR_PSI_FLOOR (the count itself
    # may move by a few between runs: float atomics deposit in any order)
    ctx = qs.Context(qs.config_from_workload(wl, psi_floor=0.999999,
                                             max_psi_guard_hits=hits // 2))
    ctx.init_plasma(wl.ppc)
    st = ctx.step3d(beams, raise_on_error=False)
    assert st["status"] == qs.QS_ERR_PSI_FLOOR and st["psi_guard_hits"] > hits // 2
    ctx.close()
    # a limit well above it passes; the default floor clamps nothing here
    ctx = qs.Context(qs.config_from_workload(wl, psi_floor=0.999999,
                                             max_psi_guard_hits=2 * hits))
    ctx.init_plasma(wl.ppc)
    assert ctx.step3d(beams)["status"] == qs.QS_OK
    ctx.close()
    ctx = qs.Context(qs.config_from_workload(wl, max_psi_guard_hits=0))
    ctx.init_plasma(wl.ppc)
    assert ctx.step3d(beams)["psi_guard_hits"] == 0
    ctx.close()
