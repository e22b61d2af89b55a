"""CUDA path vs the FP64 oracle, element by element, through the C ABI (GPU)."""
import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu


def _rel(a, b, scale=None):
    d = np.linalg.norm(a - b)
    s = max(np.linalg.norm(b), scale or 0.0, 1e-300)
    return d / s


def _run_both(qs, wl, tol=1e-12, schedule=None, **cfg_over):
    beams_np = [W.sample_beam(b) for b in wl.beams]
    ctx = qs.Context(qs.config_from_workload(wl, mg_tol=tol, **cfg_over))
    if wl.profile is None:
        ctx.init_plasma(wl.ppc)
    else:
        ctx.init_plasma(wl.ppc, wl.profile[0], wl.profile[1])
    beams = [qs.Beam(b) for b in beams_np]
    stats = ctx.step3d(beams, schedule=schedule)
    got = ctx.fields(qs.FIELD_ALL | qs.FIELD_JZB, device=False).numpy()
    m, vmax, charge = ctx.slice_diagnostics()
    cfg = O.config_from_workload(wl)
    pl, n_ion = O.plasma_from_workload(wl)
    ref = O.step3d(cfg, pl, n_ion, beams_np, m_schedule=schedule)
    jzb = O.deposit_beam(cfg, beams_np)
    return dict(ctx=ctx, stats=stats, got=got, m=m, vmax=vmax, charge=charge, ref=ref, jzb=jzb,
                beams=beams, beams_np=beams_np, cfg=cfg, pl=pl)


TOL = {"fp64": 1e-9, "fp32r": 2e-5}


def _check_fields(r, tol):
    ref = r["ref"].history
    scale = np.linalg.norm(ref[0])
    errs = {}
    for i, name in enumerate(O.FIELD_NAMES):
        errs[name] = _rel(r["got"][i], ref[i], scale)
    assert max(errs.values()) < tol, errs
    return errs


def test_init_plasma_matches_oracle_lattice(qs):
    wl = W.workload("linear64")
    ctx = qs.Context(qs.config_from_workload(wl))
    ctx.init_plasma(4)
    p = ctx.plasma()
    pl, _ = O.plasma_from_workload(wl)
    assert np.array_equal(p["id"], pl.pid)
    assert np.max(np.abs(p["x"] - pl.x)) < 1e-14 and np.max(np.abs(p["y"] - pl.y)) < 1e-14
    assert np.max(np.abs(p["w"] - pl.w)) < 1e-16
    # parabolic channel weights
    prof = W.workload("blowout512").profile
    ctx2 = qs.Context(qs.config_from_workload(wl))
    ctx2.init_plasma(9, prof[0], prof[1])
    p2 = ctx2.plasma()
    g = O.Grid.square(wl.n, wl.half_width)
    pl2, _ = O.init_plasma(g, 9, prof[0], prof[1])
    assert np.max(np.abs(p2["w"] - pl2.w)) < 1e-15 * pl2.w.max()


@pytest.mark.parametrize("n,np_", [(8, 1000), (64, 50000), (256, 262144)])
def test_cell_sort_bit_exact(qs, n, np_):
    import torch
    rng = np.random.default_rng(n)
    L = 8.0
    x = rng.uniform(-L, L, np_)
    y = rng.uniform(-L, L, np_)
    h = 2 * L / n
    x[: min(50, np_)] = -L + h * rng.integers(0, n + 1, min(50, np_))  # on cell faces and walls
    pid = rng.permutation(np_).astype(np.int32)
    wl = W.Workload(name="s", n=n, half_width=L, n_xi=4, xi_len=1.0, ppc=4, beams=())
    ctx = qs.Context(qs.config_from_workload(wl))
    t = lambda a: torch.as_tensor(a, device="cuda")
    cell, count, offset, perm = (v.cpu().numpy() for v in ctx.cell_sort(t(x), t(y), t(pid)))
    c_o, count_o, off_o, perm_o = O.cell_sort(x, y, pid, O.Grid.square(n, L))
    assert np.array_equal(cell, c_o)
    assert np.array_equal(count, count_o)
    assert np.array_equal(offset, off_o)
    assert np.array_equal(perm, perm_o)


@pytest.mark.parametrize("form", ["fp64", "fp32r"])
def test_linear_driver_step_parity(qs, form):
    """The 64^2, 128-slice linear workload: every field of every base slice.
    The refined form reaches the float64 solution by iterative refinement."""
    wl = W.workload("linear64").with_(precision=form)
    r = _run_both(qs, wl)
    _check_fields(r, TOL[form])
    assert r["stats"]["slices"] == r["ref"].slices == 128
    assert np.array_equal(r["m"], r["ref"].m)
    ctol = 1e-11 if form == "fp64" else 1e-6  # float32 deposits round at 1e-7
    assert np.max(np.abs(r["charge"] - r["pl"].w.sum())) < ctol * r["pl"].w.sum()
    assert _rel(r["got"][5], r["jzb"]) < 1e-13


@pytest.mark.parametrize("form,cb", [("fp64", 0), ("fp32r", 0), ("fp64", 4), ("fp32r", 32)])
def test_nonlinear_refined_step_parity(qs, form, cb):
    """A strong driver on a small grid: adaptive sub-steps, nonlinear sources;
    both forms, with the single-block coarse part starting at several levels."""
    wl = W.Workload(name="t", n=32, half_width=3.0, n_xi=32, xi_len=8.0, ppc=4,
                    beams=(W.BeamSpec(amplitude=20.0, sigma_x=0.5, sigma_y=0.5, sigma_z=0.6,
                                      xi_c=1.8, n_particles=20000, seed=3),), precision=form)
    if form == "fp32r":
        # float32 particles may round a V_max across a refinement threshold:
        # replay the oracle's sub-step schedule and compare the arithmetic
        cfg = O.config_from_workload(wl)
        pl, n_ion = O.plasma_from_workload(wl)
        sched = O.step3d(cfg, pl, n_ion, [W.sample_beam(b) for b in wl.beams]).m
        r = _run_both(qs, wl, schedule=list(sched), coarse_block_n=cb)
    else:
        r = _run_both(qs, wl, coarse_block_n=cb)
    assert np.array_equal(r["m"], r["ref"].m), (r["m"], r["ref"].m)
    assert r["ref"].m.max() > 2
    assert r["stats"]["slices"] == r["ref"].slices
    _check_fields(r, TOL[form])


def test_beam_push_parity(qs):
    wl = W.workload("linear64")
    r = _run_both(qs, wl)
    ctx = r["ctx"]
    ctx.push_beam(r["beams"], 10.0)
    got = r["beams"][0].numpy()
    b0 = r["beams_np"][0]
    ref = O.push_beam(r["cfg"], r["ref"].history, b0, 10.0)
    for k in ("px", "py", "pz"):
        dg, dr = got[k] - b0[k], ref[k] - b0[k]
        assert _rel(dg, dr) < 1e-8, k
    for k in ("x", "y", "xi"):
        assert np.max(np.abs(got[k] - ref[k])) < 1e-10, k


def test_schedule_replay(qs):
    wl = W.workload("linear64").with_(n_xi=32, xi_len=3.0)
    sched = [1, 2, 1, 3] * 8
    r = _run_both(qs, wl, schedule=sched)
    assert list(r["m"]) == sched
    assert r["stats"]["slices"] == r["ref"].slices
    _check_fields(r, 1e-9)


def test_errors_are_statuses(qs):
    wl = W.workload("linear64")
    ctx = qs.Context(qs.config_from_workload(wl))
    with pytest.raises(qs.QsError) as e:
        ctx.step3d([])
    assert e.value.status == qs.QS_ERR_STATE
    with pytest.raises(qs.QsError) as e:
        ctx.fields()
    assert e.value.status == qs.QS_ERR_STATE
    # a V-cycle cap of one with a tight tolerance cannot converge
    ctx2 = qs.Context(qs.config_from_workload(wl.with_(n_xi=8, xi_len=2.0), mg_tol=1e-14,
                                              mg_max_vcycles=1))
    ctx2.init_plasma(4)
    st = ctx2.step3d([qs.Beam(W.sample_beam(wl.beams[0]))], raise_on_error=False)
    assert st["status"] == qs.QS_ERR_NOT_CONVERGED
    # the context stays usable afterwards
    ctx3 = qs.Context(qs.config_from_workload(wl.with_(n_xi=8, xi_len=2.0)))
    ctx3.init_plasma(4)
    assert ctx3.step3d([])["status"] == 0


@pytest.mark.parametrize("form,n", [("fp64", 32), ("fp64", 64), ("fp64", 128),
                                    ("fp32r", 64), ("fp32r", 128), ("fp32r", 256)])
def test_cluster_solves_match_the_oracle_and_the_grid_solves(qs, form, n):
    """Solves whose V-cycles run in thread-block clusters (cluster_size 8 and
    16: the grid's rows split over the cluster's shared memory; in the refined
    form the float32 cycles of the correction, with the float64 update
    grid-wide) against the oracle and against the grid-wide solves
    (cluster_size 1), on the linear wake."""
    bar, agree = (1e-9, 1e-10) if form == "fp64" else (2e-5, 1e-6)
    wl = W.workload("linear64").with_(n=n, n_xi=32, xi_len=3.0)
    beams_np = [W.sample_beam(b.with_(xi_c=1.5)) for b in wl.beams]
    cfg = O.config_from_workload(wl)
    pl, n_ion = O.plasma_from_workload(wl)
    ref = O.step3d(cfg, pl, n_ion, beams_np).history
    scale = np.linalg.norm(ref[0])
    out = {}
    for cs in (1, 8, 16):
        if cs > 1 and n % (2 * cs):
            continue
        ctx = qs.Context(qs.config_from_workload(wl, precision=form, mg_tol=1e-12,
                                                 cluster_size=cs))
        ctx.init_plasma(wl.ppc)
        st = ctx.step3d([qs.Beam(b) for b in beams_np])
        out[cs] = ctx.fields(qs.FIELD_ALL, device=False).numpy(), st
        ctx.close()
        got = out[cs][0]
        for i in range(5):
            err = np.linalg.norm(got[i] - ref[i]) / max(np.linalg.norm(ref[i]), scale)
            assert err < bar, (cs, i, err)
    for cs in out:
        assert np.linalg.norm(out[cs][0] - out[1][0]) <= agree * np.linalg.norm(out[1][0]), cs


@pytest.mark.parametrize("form", ["fp64", "fp32r"])
def test_plasma_sorted_by_cell_inside_the_loop(qs, form):
    """sort_every = 1 reorders the plasma by (cell, id) before every base
    slice (the last slice has no push, so the final order is that of the
    final positions): bit-exact against the oracle's counting sort; the wake
    and the particles (matched by id) equal those of the unsorted loop."""
    wl = W.workload("linear64").with_(n_xi=24, xi_len=3.0)
    beams_np = [W.sample_beam(b.with_(xi_c=1.5, amplitude=2.0)) for b in wl.beams]
    out = {}
    for K in (0, 1, 5):
        ctx = qs.Context(qs.config_from_workload(wl, precision=form, mg_tol=1e-12,
                                                 sort_every=K))
        ctx.init_plasma(wl.ppc)
        st = ctx.step3d([qs.Beam(b) for b in beams_np])
        out[K] = (ctx.fields(qs.FIELD_ALL, device=False).numpy(), ctx.plasma(), st)
        ctx.close()
    assert out[0][2]["sorts"] == 0
    assert out[1][2]["sorts"] == wl.n_xi - 1 and out[5][2]["sorts"] == (wl.n_xi - 1) // 5
    p = out[1][1]
    cell, count, offset, perm = O.cell_sort(p["x"], p["y"], p["id"], O.Grid.square(wl.n, wl.half_width))
    assert np.array_equal(perm, np.arange(len(perm)))  # already in (cell, id) order
    tol = 1e-11 if form == "fp64" else 2e-6
    base = out[0][0]
    for K in (1, 5):
        assert np.linalg.norm(out[K][0] - base) <= tol * np.linalg.norm(base)
        a, b = out[0][1], out[K][1]
        ia, ib = np.argsort(a["id"]), np.argsort(b["id"])
        assert np.array_equal(a["id"][ia], b["id"][ib])
        for k in ("x", "y", "px", "py", "w"):
            assert np.max(np.abs(a[k][ia] - b[k][ib])) <= (1e-9 if form == "fp64" else 1e-4), k


@pytest.mark.parametrize("form", ["fp64", "fp32r"])
def test_privatised_deposits_match_the_oracle_and_the_grid_atomics(qs, form):
    """The moments and n_* deposited through shared-memory bands of grid rows
    (as many rows as fit, -1; 3 rows, so that many stencils of the expelled
    particles go to the grid directly; no in-loop sort, so that the chunks
    are the lattice's) against plain grid atomics (deposit_band_rows = 0)
    and against the oracle, on a driver strong enough to refine the step."""
    wl = W.Workload(name="t", n=64, half_width=4.0, n_xi=32, xi_len=8.0, ppc=4,
                    beams=(W.BeamSpec(amplitude=20.0, sigma_x=0.5, sigma_y=0.5, sigma_z=0.6,
                                      xi_c=1.8, n_particles=20000, seed=3),), precision=form)
    cfg = O.config_from_workload(wl)
    pl, n_ion = O.plasma_from_workload(wl)
    beams_np = [W.sample_beam(b) for b in wl.beams]
    ref = O.step3d(cfg, pl, n_ion, beams_np)
    sched = list(ref.m) if form == "fp32r" else None
    scale = np.linalg.norm(ref.history[0])
    out = {}
    for rows, sort in ((0, 16), (-1, 16), (3, 16), (-1, 0)):
        ctx = qs.Context(qs.config_from_workload(wl, mg_tol=1e-12, deposit_band_rows=rows,
                                                 sort_every=sort))
        ctx.init_plasma(wl.ppc)
        st = ctx.step3d([qs.Beam(b) for b in beams_np], schedule=sched)
        got = ctx.fields(qs.FIELD_ALL, device=False).numpy()
        m, _, _ = ctx.slice_diagnostics()
        ctx.close()
        assert np.array_equal(m, ref.m), (rows, sort)
        assert ref.m.max() > 2
        errs = [_rel(got[i], ref.history[i], scale) for i in range(5)]
        assert max(errs) < TOL[form], (rows, sort, errs)
        out[(rows, sort)] = got
    base = out[(0, 16)]
    # only the order of the floating-point additions differs
    agree = 1e-9 if form == "fp64" else 1e-5
    for key, got in out.items():
        assert np.linalg.norm(got - base) <= agree * np.linalg.norm(base), key
