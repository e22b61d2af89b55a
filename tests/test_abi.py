"""The C-ABI library builds, loads and exports what include/qs.h declares (CPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"\b(qs_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2012_00881_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(lib):
    names = _declared_functions()
    assert "qs_step3d" in names and "qs_init_plasma" in names and "qs_fields" in names
    for n in names:
        assert hasattr(lib, n), n


def test_binding_prototypes_cover_the_header():
    import paper_2012_00881_gb300 as qs
    assert set(_declared_functions()) == set(qs.PROTOTYPES)


def test_default_config_through_the_abi(lib):
    """qs_config_default fills the ctypes mirror field by field."""
    import paper_2012_00881_gb300 as qs
    cfg = qs.default_config()
    assert cfg.nx == 64 and cfg.ny == 64 and cfg.refine_k == 8 and cfg.mg_tol == 1e-10
    assert cfg.x_min == -6.0 and cfg.xi_max == 12.0 and cfg.n_xi == 128
    assert cfg.max_psi_guard_hits == -1 and cfg.sort_every == 16
    assert cfg.pre_sweeps == -1 and cfg.post_sweeps == 2 and cfg.coarse_block_n == 0
    assert cfg.trace_capacity == 0 and cfg.warm_start_order == 2
    assert cfg.tile_x == 0 and cfg.tile_y == 0 and cfg.checkpoint_every == 0
    assert cfg.omega_pct == 0 and cfg.coarse_pre_sweeps == 1


def test_status_strings(lib):
    import paper_2012_00881_gb300 as qs
    l = qs.load_library()
    assert l.qs_strerror(0) == b"ok"
    assert l.qs_strerror(qs.QS_ERR_NOT_CONVERGED) == b"multigrid did not converge"
    assert l.qs_strerror(12345) == b"unknown status"


def test_invalid_config_rejected_without_gpu(lib):
    """Argument validation runs before any device call."""
    import paper_2012_00881_gb300 as qs
    l = qs.load_library()
    h = ctypes.c_void_p()
    for bad in (dict(nx=64, ny=32), dict(nx=100, ny=100), dict(refine_k=0),
                dict(precision=7), dict(mg_tol=0.0), dict(x_max=7.0), dict(tile_x=7, tile_y=8),
                dict(warm_start_order=3), dict(omega_pct=40), dict(omega_pct=200), dict(coarse_pre_sweeps=9), dict(checkpoint_every=-1),
                dict(pre_sweeps=-2), dict(pre_sweeps=0, post_sweeps=0), dict(post_sweeps=9),
                dict(deposit_band_rows=2), dict(deposit_band_rows=-2), dict(cluster_size=4)):
        cfg = qs.default_config(**bad)
        assert l.qs_create(ctypes.byref(cfg), None, ctypes.byref(h)) == qs.QS_ERR_ARG, bad
    assert l.qs_create(None, None, ctypes.byref(h)) == qs.QS_ERR_ARG


def test_nonuniform_solver_arguments_rejected_without_gpu(lib):
    """qs_nu_create validates n and the axes before any device call."""
    import numpy as np
    import paper_2012_00881_gb300 as qs
    l = qs.load_library()
    h = ctypes.c_void_p()

    def create(n, xn, yn, corr=1, prec=0):
        xa = np.ascontiguousarray(xn, dtype=np.float64)
        ya = np.ascontiguousarray(yn, dtype=np.float64)
        return l.qs_nu_create(n, xa.ctypes.data, ya.ctypes.data, corr, prec, None,
                              ctypes.byref(h))

    good = np.linspace(-1.0, 1.0, 17)
    for n in (0, 1, 2, 4, 5, 6, 14, 16, 4096, 8191):
        axis = np.linspace(-1.0, 1.0, max(n, 1) + 2)
        assert create(n, axis, axis) == qs.QS_ERR_ARG, n
    bad = good.copy()
    bad[5] = bad[4]                       # repeated node
    assert create(15, bad, good) == qs.QS_ERR_ARG
    assert create(15, good, bad[::-1].copy()) == qs.QS_ERR_ARG
    nan = good.copy()
    nan[3] = float("nan")
    assert create(15, nan, good) == qs.QS_ERR_ARG
    assert create(15, good, good, corr=2) == qs.QS_ERR_ARG
    assert create(15, good, good, prec=2) == qs.QS_ERR_ARG
    assert l.qs_nu_create(15, None, None, 1, 0, None, ctypes.byref(h)) == qs.QS_ERR_ARG
    assert l.qs_nu_create(15, good.ctypes.data, good.ctypes.data, 1, 0, None, None) == qs.QS_ERR_ARG
    for args in ((None, None, 1, None, None, 1e-10, 10, None, None),):
        assert l.qs_nu_solve(*args) == qs.QS_ERR_ARG
    l.qs_nu_destroy(None)


def test_laser_arguments_rejected_without_gpu(lib):
    """qs_laser_create validates its arguments before any device call."""
    import math
    import paper_2012_00881_gb300 as qs
    l = qs.load_library()
    h = ctypes.c_void_p()
    good = dict(n=16, width=4.0, n_xi=4, k0=3.0, dt=0.5, dxi=0.1)
    for bad in (dict(n=1), dict(n=9000), dict(width=0.0), dict(width=math.inf), dict(n_xi=0),
                dict(k0=0.0), dict(k0=math.nan), dict(dt=-1.0), dict(dt=math.inf),
                dict(dxi=0.0), dict(dxi=-0.1), dict(dxi=math.nan)):
        a = dict(good, **bad)
        assert l.qs_laser_create(a["n"], a["width"], a["n_xi"], a["k0"], a["dt"], a["dxi"],
                                 None, ctypes.byref(h)) == qs.QS_ERR_ARG, bad
    assert l.qs_laser_create(16, 4.0, 4, 3.0, 0.5, 0.1, None, None) == qs.QS_ERR_ARG
    assert l.qs_laser_advance(None, None, None, 1, 1e-10, 10, None, None) == qs.QS_ERR_ARG
    l.qs_laser_destroy(None)


def test_sort_bindings_reject_host_tensors_and_oversized_grids():
    """The sort bindings check their tensors before any library call, so a
    wrong tensor never reaches a kernel (CPU: no CUDA is needed to fail)."""
    import torch

    import paper_2012_00881_gb300 as qs
    x = torch.zeros(10, dtype=torch.float64)
    pid = torch.arange(10, dtype=torch.int32)
    with pytest.raises(ValueError):  # host tensors
        qs.cell_sort_noalloc(4, -1.0, -1.0, 0.5, x, x, pid)
    with pytest.raises(ValueError):  # more cells than the fixed scratch holds
        qs.cell_sort_noalloc(513, -1.0, -1.0, 0.5, x, x, pid)
    with pytest.raises(ValueError):
        qs.cell_sort_noalloc(4, -1.0, -1.0, 0.5, [0.0] * 10, x, pid)
