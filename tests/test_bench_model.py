"""The bench's algorithmic byte model (CPU): the multigrid term follows the
sweeps per level, so a change of smoother settings changes the bytes a
V-cycle must move, not only the V-cycle count."""
import importlib.util
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    old = sys.argv
    sys.argv = ["bench.py"]
    try:
        spec = importlib.util.spec_from_file_location("bench_model", os.path.join(ROOT, "bench.py"))
        mod = importlib.util.module_from_spec(spec)
        spec.loader.exec_module(mod)
    finally:
        sys.argv = old
    return mod


class _Wl:
    n = 64
    n_plasma = 0


def _mg_bytes(bench, form, sweeps, v):
    st = {"slices": 1, "vcycles": v}
    base = bench.algorithmic_bytes({"slices": 1, "vcycles": [0, 0, 0]}, _Wl, form, 0, sweeps)
    return bench.algorithmic_bytes(st, _Wl, form, 0, sweeps) - base


def test_cycle_sweeps_defaults(bench):
    assert bench.cycle_sweeps("fp32r") == 5
    assert bench.cycle_sweeps("fp64") == 4
    assert bench.cycle_sweeps("fp32r", {"pre_sweeps": 2, "post_sweeps": 1}) == 3
    assert bench.cycle_sweeps("fp64", {"pre_sweeps": -1, "post_sweeps": 3}) == 5


def test_multigrid_bytes_per_cycle(bench):
    nn = _Wl.n * _Wl.n
    # one psi cycle (one component) in the float64 form with V(2,2): 24 words of 8 bytes
    assert _mg_bytes(bench, "fp64", 4, [1, 0, 0]) == pytest.approx(24 * 8 * nn)
    # V(3,2): 3 nu b + 4.5b = 19.5b on the fine level, a third of it on the
    # coarse ones, 2b for the norm: 28b
    assert _mg_bytes(bench, "fp64", 5, [1, 0, 0]) == pytest.approx(28 * 8 * nn)
    # a screened cycle: two components and kappa
    assert _mg_bytes(bench, "fp64", 4, [0, 0, 1]) == pytest.approx((2 * 24 + 8) * 8 * nn)
    # the refined form adds its float64 outer update per component and cycle
    assert _mg_bytes(bench, "fp32r", 4, [1, 0, 0]) == pytest.approx((24 * 4 + 40) * nn)
