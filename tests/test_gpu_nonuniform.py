"""Nonuniform-grid field solver vs the FP64 oracle, through the C ABI (GPU).

Sec. "Multigrid Solver with Nonuniform Grids": the operator (Eq. 2D_Laplac
with the correction of Eq. 2D_Laplac_3rd) and the corrected source are
compared element by element; the multigrid solution against the oracle's
sparse-LU solution of the same discrete system.  Solves here run to a
relative residual of 1e-13 (1e-12 from 127^2 up, where the float64 residual
of these grids levels off at 1e-13 .. 6e-13), so two exact solvers of the
system agree to about cond(A) times that (cond ~ (L / h_min)^2 ~ 1e5 here);
the agreement observed is 1e-13 .. 1e-15, and the bound is the float64 bar
of the slice advance, 1e-9 relative in L2.
"""
import numpy as np
import pytest

from oracle import qs_nonuniform as nu
from workloads.nonuniform import (alternating_axis, bubble_sources, nonuniform_workload,
                                  three_region_axis, uniform_axis)

pytestmark = pytest.mark.gpu

PARITY = 1e-9


def _solve_tol(n):
    return 1e-13 if n <= 63 else 1e-12


def _axes(kind, n):
    if kind == "three_region":
        return three_region_axis(n, 12.5), three_region_axis(n, 12.5)
    if kind == "alternating":
        return alternating_axis(n, 4.0, 2.0), alternating_axis(n, 3.0, 3.0, first_long=True)
    if kind == "uniform":
        return uniform_axis(n, 5.0), uniform_axis(n, 5.0)
    # strongly irregular, seeded
    rng = np.random.default_rng(n)
    out = []
    for hw in (4.0, 3.0):
        steps = rng.uniform(0.4, 1.6, n + 1)
        x = np.concatenate([[0.0], np.cumsum(steps)]) * (2 * hw / steps.sum()) - hw
        x[-1] = hw
        out.append(x)
    return tuple(out)


def _t(a):
    import torch
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("kind", ["three_region", "alternating", "random", "uniform"])
@pytest.mark.parametrize("correction", [True, False])
@pytest.mark.parametrize("n", [31, 127])
def test_operator_and_source_match_oracle(qs, kind, correction, n):
    xn, yn = _axes(kind, n)
    src = bubble_sources(xn, yn, radius=1.5)
    rng = np.random.default_rng(7)
    u = rng.standard_normal((n, n))
    s = qs.NonuniformSolver(xn, yn, correction=correction,
                            precision="fp64" if n == 31 else "fp32r")
    for m in (None, src["m"]):
        got = s.apply(_t(u), None if m is None else _t(m)).cpu().numpy()
        ref = nu.apply(xn, yn, u, m, correction)
        scale = np.abs(ref).max()
        np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12 * scale)
    got = s.source(_t(src["ez"])).cpu().numpy()
    ref = nu.corrected_source(xn, yn, src["ez"], correction)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-13 * np.abs(ref).max())


@pytest.mark.parametrize("precision", ["fp64", "fp32r"])
@pytest.mark.parametrize("kind", ["three_region", "alternating", "random"])
@pytest.mark.parametrize("n", [7, 63, 255])
def test_solve_matches_oracle(qs, kind, n, precision):
    """Both forms stop on the float64 residual, so both meet the same bound."""
    xn, yn = _axes(kind, n)
    src = bubble_sources(xn, yn, radius=3.0 if kind == "three_region" else 1.5)
    s = qs.NonuniformSolver(xn, yn, correction=True, precision=precision)
    j = np.stack([src["psi"], src["bx"]])
    # Poisson (M = 0) and screened (M = -kappa) solves, two fields each
    for m in (None, src["m"]):
        u, cycles, relres = s.solve(_t(j), m=None if m is None else _t(m), tol=_solve_tol(n),
                                    max_cycles=60)
        got = u.cpu().numpy()
        assert max(relres) <= _solve_tol(n)
        for c in range(2):
            ref = nu.solve(xn, yn, j[c], m)
            assert _rel(got[c], ref) < PARITY, (c, _rel(got[c], ref))


@pytest.mark.parametrize("precision", ["fp64", "fp32r"])
def test_plain_scheme_solve_matches_oracle(qs, precision):
    xn, yn = _axes("alternating", 127)
    src = bubble_sources(xn, yn, radius=1.5)
    s = qs.NonuniformSolver(xn, yn, correction=False, precision=precision)
    u, _, _ = s.solve(_t(src["by"]), m=_t(src["m"]), tol=_solve_tol(127), max_cycles=60)
    ref = nu.solve(xn, yn, src["by"], src["m"], correction=False)
    assert _rel(u.cpu().numpy(), ref) < PARITY


@pytest.mark.parametrize("precision", ["fp64", "fp32r"])
def test_coarsest_only_grid(qs, precision):
    """n = 3: the exact coarse solve is the whole method (one float32 solve
    plus float64 refinement in the refined form)."""
    xn = np.array([-1.0, -0.7, 0.1, 0.4, 1.0])
    yn = np.array([-2.0, -0.5, 0.0, 1.5, 2.0])
    j = np.arange(9.0).reshape(3, 3) - 3.0
    m = -np.linspace(0.5, 1.5, 9).reshape(3, 3)
    s = qs.NonuniformSolver(xn, yn, correction=True, precision=precision)
    u, cycles, relres = s.solve(_t(j), m=_t(m), tol=1e-14, max_cycles=4)
    assert cycles == 1 if precision == "fp64" else cycles <= 3
    np.testing.assert_allclose(u.cpu().numpy(), nu.solve(xn, yn, j, m), rtol=1e-13, atol=1e-14)


@pytest.mark.parametrize("precision", ["fp64", "fp32r"])
def test_convergence_rate_and_warm_start(qs, precision):
    """Per V-cycle residual reduction on the three-region demonstration grid
    (cells up to 3:1 in aspect, which slows point smoothing), and a converged
    initial guess costs no cycle."""
    wl = nonuniform_workload("nonuni255")
    xn = wl.axis()
    src = bubble_sources(xn, xn, wl.bubble_radius)
    s = qs.NonuniformSolver(xn, xn, correction=True, precision=precision)
    for key, m in (("psi", None), ("bx", src["m"])):
        mt = None if m is None else _t(m)
        u, cycles, relres = s.solve(_t(src[key]), m=mt, tol=1e-10, max_cycles=40)
        # from zero: 1e-10 in at most 16 cycles means an average factor < 0.24
        assert cycles <= 16, (key, cycles)
        u2, cycles2, _ = s.solve(_t(src[key]), u=u.clone(), m=mt, tol=1e-10, max_cycles=40)
        assert cycles2 == 0
        np.testing.assert_array_equal(u2.cpu().numpy(), u.cpu().numpy())


@pytest.mark.parametrize("precision", ["fp64", "fp32r"])
def test_fields_are_independent(qs, precision):
    """A batch of fields gives what each gives alone; a zero source gives zero."""
    xn, yn = _axes("random", 63)
    src = bubble_sources(xn, yn, radius=1.5)
    s = qs.NonuniformSolver(xn, yn, correction=True, precision=precision)
    j = np.stack([src["ez"], np.zeros_like(src["ez"]), src["bz"], src["by"]])
    u4, _, relres = s.solve(_t(j), u=_t(np.ones_like(j)), m=_t(src["m"]), tol=1e-12,
                            max_cycles=60)
    assert relres[1] == 0.0
    got = u4.cpu().numpy()
    assert not got[1].any()
    for c in (0, 2, 3):
        u1, _, _ = s.solve(_t(j[c]), m=_t(src["m"]), tol=1e-12, max_cycles=60)
        ref = nu.solve(xn, yn, j[c], src["m"])
        assert _rel(got[c], ref) < 1e-7 and _rel(u1.cpu().numpy(), ref) < 1e-7


def test_cycle_cap_reports_not_converged(qs):
    xn, yn = _axes("three_region", 127)
    src = bubble_sources(xn, yn)
    s = qs.NonuniformSolver(xn, yn)
    u, cycles, relres = s.solve(_t(src["psi"]), tol=1e-14, max_cycles=2, raise_on_error=False)
    assert s.status == qs.QS_ERR_NOT_CONVERGED and cycles == 2
    assert 0.0 < relres[0] < 1.0
    # the last iterate is kept: it continues to convergence from there
    u2, cycles2, _ = s.solve(_t(src["psi"]), u=u.clone(), tol=1e-10, max_cycles=40)
    assert s.status == qs.QS_OK


def test_solver_rejects_bad_calls(qs):
    xn, yn = _axes("uniform", 15)
    s = qs.NonuniformSolver(xn, yn)
    j = _t(np.zeros((15, 15)))
    lib = qs.load_library()
    assert lib.qs_nu_solve(s.h, None, 0, j.data_ptr(), j.data_ptr(), 1e-10, 10, None, None) == qs.QS_ERR_ARG
    assert lib.qs_nu_solve(s.h, None, 5, j.data_ptr(), j.data_ptr(), 1e-10, 10, None, None) == qs.QS_ERR_ARG
    assert lib.qs_nu_solve(s.h, None, 1, j.data_ptr(), j.data_ptr(), 0.0, 10, None, None) == qs.QS_ERR_ARG
    assert lib.qs_nu_solve(s.h, None, 1, j.data_ptr(), j.data_ptr(), 1e-10, 0, None, None) == qs.QS_ERR_ARG


@pytest.mark.parametrize("precision", ["fp64", "fp32r"])
def test_cycle_settings(qs, precision):
    """Other sweep counts and relaxation reach the same solution; bad settings
    are rejected."""
    xn, yn = _axes("three_region", 127)
    src = bubble_sources(xn, yn)
    s = qs.NonuniformSolver(xn, yn, precision=precision)
    ref = nu.solve(xn, yn, src["bx"], src["m"])
    for pre, post, omega, blk in ((1, 1, 1.0, 0), (3, 2, 1.2, 3), (0, 2, 1.1, 63),
                                  (2, 0, 1.0, 127), (2, 2, 1.3, 4095)):
        s.set_cycle(pre, post, omega, blk)
        u, cycles, _ = s.solve(_t(src["bx"]), m=_t(src["m"]), tol=1e-12, max_cycles=200)
        assert _rel(u.cpu().numpy(), ref) < PARITY, (pre, post, omega)
    lib = qs.load_library()
    for bad in ((0, 0, 1.0, 0, 1), (-1, 2, 1.0, 0, 1), (9, 2, 1.0, 0, 1), (2, 2, 0.0, 0, 1),
                (2, 2, 2.0, 0, 1), (2, 2, float("nan"), 0, 1), (2, 2, 1.3, -1, 1),
                (2, 2, 1.3, 0, 2)):
        assert lib.qs_nu_set_cycle(s.h, *bad) == qs.QS_ERR_ARG, bad


@pytest.mark.parametrize("precision", ["fp64", "fp32r"])
@pytest.mark.parametrize("sweeps", [(2, 2), (1, 2), (3, 1)])
def test_staged_smoothing_is_exact(qs, precision, sweeps):
    """Shared-memory staged smoothing (halo 4 max(nu) + 2, recomputed) gives
    the iterates of grid-wide colour sweeps, including on levels whose tiles
    are clipped by the domain's end and the one-block levels staged whole
    (level 63 with one-block level 63 does not fit and mixes both ways of
    smoothing).  The arithmetic is the same; the
    compiler contracts multiply-adds differently in the two code paths, so
    they agree to rounding: 1e-11 of the largest value in float64 (about
    1e-15 absolute here), 1e-5 in the refined form's float32 cycles."""
    xn, yn = _axes("random", 255)
    src = bubble_sources(xn, yn, radius=1.5)
    s = qs.NonuniformSolver(xn, yn, precision=precision)
    j = _t(np.stack([src["bx"], src["by"]]))
    m = _t(src["m"])
    got = {}
    for staged in (True, False):
        for blk in (63, 31, 7):
            s.set_cycle(sweeps[0], sweeps[1], 1.3, blk, staged)
            u, cycles, relres = s.solve(j, u=_t(np.full((2, 255, 255), 0.1)), m=m, tol=1e-11,
                                        max_cycles=4, raise_on_error=False)
            got[(staged, blk)] = (u.cpu().numpy(), cycles, relres)
    tol = 1e-11 if precision == "fp64" else 1e-5
    for blk in (63, 31, 7):
        a, b = got[(True, blk)], got[(False, blk)]
        np.testing.assert_allclose(a[0], b[0], rtol=0, atol=tol * np.abs(b[0]).max())
        assert a[1] == b[1]
        np.testing.assert_allclose(a[2], b[2], rtol=1e-3 if precision == "fp32r" else 1e-8)
