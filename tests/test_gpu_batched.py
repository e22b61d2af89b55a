"""Batched form: several independent instances in one persistent launch (GPU).

Each instance of the batch must give the result of its own single-instance
step (same arithmetic, other blocks), for uneven sizes, several team sizes
and both forms; one instance is also checked against the FP64 oracle.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu


def _instances(form):
    out = []
    for i, n in enumerate((32, 48, 64, 32, 48)):
        out.append(W.Workload(
            name=f"b{i}", n=n, half_width=4.0, n_xi=20, xi_len=4.0, ppc=4,
            beams=(W.BeamSpec(amplitude=0.5 + 1.5 * i, sigma_x=0.4 + 0.05 * i, sigma_y=0.5,
                              sigma_z=0.6, xi_c=1.5, n_particles=6000, seed=i),),
            precision=form))
    return out


def _contexts(qs, wls, **over):
    ctxs, beams = [], []
    for wl in wls:
        c = qs.Context(qs.config_from_workload(wl, mg_tol=1e-12, **over))
        c.init_plasma(wl.ppc)
        ctxs.append(c)
        beams.append([qs.Beam(W.sample_beam(b)) for b in wl.beams])
    return ctxs, beams


@pytest.mark.parametrize("form", ["fp64", "fp32r"])
def test_batched_equals_single_instance_steps(qs, form):
    wls = _instances(form)
    ctxs, beams = _contexts(qs, wls)
    tol = 1e-12 if form == "fp64" else 1e-6
    for team in (0, 3, 16):
        st = qs.step3d_batched(ctxs, beams, team_blocks=team)
        batched = [c.fields(qs.FIELD_ALL, device=False).numpy() for c in ctxs]
        for c, b, f, s in zip(ctxs, beams, batched, st):
            single = c.step3d(b)
            g = c.fields(qs.FIELD_ALL, device=False).numpy()
            assert np.linalg.norm(g - f) <= tol * np.linalg.norm(g), (team, c.n)
            assert s["slices"] == single["slices"]


def test_batched_instance_matches_oracle(qs):
    wls = _instances("fp64")
    ctxs, beams = _contexts(qs, wls)
    qs.step3d_batched(ctxs, beams)
    k = 2  # the 64^2 instance
    got = ctxs[k].fields(qs.FIELD_ALL, device=False).numpy()
    wl = wls[k]
    cfg = O.config_from_workload(wl)
    pl, n_ion = O.plasma_from_workload(wl)
    ref = O.step3d(cfg, pl, n_ion, [W.sample_beam(b) for b in wl.beams]).history
    assert np.linalg.norm(got - ref) <= 1e-9 * np.linalg.norm(ref)


def test_batched_rejects_repeated_and_mixed_contexts(qs):
    wls = _instances("fp64")[:2]
    ctxs, beams = _contexts(qs, wls)
    with pytest.raises(qs.QsError) as e:
        qs.step3d_batched([ctxs[0], ctxs[0]], [beams[0], beams[0]])
    assert e.value.status == qs.QS_ERR_ARG
    other, ob = _contexts(qs, [wls[1].with_(precision="fp32r")])
    with pytest.raises(qs.QsError) as e:
        qs.step3d_batched([ctxs[0], other[0]], [beams[0], ob[0]])
    assert e.value.status == qs.QS_ERR_ARG


def test_batched_scan_sizes_match_oracle(qs):
    """The parameter scan's sizes in the refined form: the three strongest
    drivers of the scan (128^2, 192^2, 256^2; n_b near 8) in one batched
    launch, each with other autotuner-style settings (tiles, sweeps,
    single-block threshold), over a 40-slice prefix through the driver's
    peak, against the FP64 oracle at the refined form's bar."""
    insts = W.scan_instances()[45:48]
    settings = (dict(tile_x=64, tile_y=32, pre_sweeps=2, post_sweeps=1, coarse_block_n=16),
                dict(),
                dict(tile_x=32, tile_y=16, pre_sweeps=3, post_sweeps=2, coarse_block_n=32))
    wls = [wl.with_(n_xi=40, xi_len=wl.xi_len * 40 / wl.n_xi,
                    beams=tuple(b.with_(xi_c=0.75, n_particles=20000) for b in wl.beams))
           for wl in insts]
    ctxs, beams = [], []
    for wl, over in zip(wls, settings):
        c = qs.Context(qs.config_from_workload(wl, precision="fp32r", mg_tol=1e-12, **over))
        c.init_plasma(wl.ppc)
        ctxs.append(c)
        beams.append([qs.Beam(W.sample_beam(b)) for b in wl.beams])
    st = qs.step3d_batched(ctxs, beams)
    for c, wl, s in zip(ctxs, wls, st):
        got = c.fields(qs.FIELD_ALL, device=False).numpy()
        cfg = O.config_from_workload(wl)
        pl, n_ion = O.plasma_from_workload(wl)
        ref = O.step3d(cfg, pl, n_ion, [W.sample_beam(b) for b in wl.beams])
        assert s["slices"] == ref.slices
        scale = np.linalg.norm(ref.history[0])
        for i in range(5):
            err = np.linalg.norm(got[i] - ref.history[i]) / max(np.linalg.norm(ref.history[i]), scale)
            assert err < 2e-5, (wl.n, i, err)
    assert max(abs(h).max() for h in [ctxs[2].fields(qs.FIELD_PSI, device=False).numpy()]) > 0.3
