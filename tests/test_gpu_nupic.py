"""The slice advance on a nonuniform node grid on the GPU against the oracle (GPU).

qs_nu_pic_* runs Algorithm 1 with node deposits and gathers, three-point first
differences and the 9-point corrected solves (Sec. "Multigrid Solver with
Nonuniform Grids"); oracle/qs_nonuniform_pic.step3d_nodes is the same loop in
float64 numpy with exact sparse solves.  Both get the same node axes and the
same driver current on the nodes; the wake of every base slice is compared
element by element (1e-9 relative per field, solves to 1e-12 on the GPU).
"""
import numpy as np
import pytest
import torch

from oracle import qs_nonuniform_pic as P
from workloads.nonuniform import alternating_axis, three_region_axis, uniform_axis

pytestmark = pytest.mark.gpu


def _driver(xn, yn, n_xi, length, nb, sr, sz, xic):
    x, y = xn[1:-1], yn[1:-1]
    X, Y = np.meshgrid(x, y)
    xi = np.arange(n_xi) * length / n_xi
    return (nb * np.exp(-((xi - xic) / sz) ** 2)[:, None, None]
            * np.exp(-(X * X + Y * Y) / sr ** 2)[None]).astype(np.float64)


def _compare(qs, xn, yn, n_xi, length, jzb, precision="fp64", ppc=4):
    pic = qs.NonuniformPIC(xn, yn, n_xi, length, precision=precision)
    pic.init_plasma(ppc)
    hist, st = pic.step3d(torch.tensor(jzb, device="cuda"), tol=1e-12, max_cycles=100)
    got = hist.cpu().numpy()
    G = P.NodeGrid(xn, yn)
    pl, n_ion = P.init_plasma_nodes(G, ppc)
    ref, ms = P.step3d_nodes(G, n_xi, length / n_xi, pl, n_ion, jzb)
    scale = np.linalg.norm(ref[0])
    errs = [np.linalg.norm(got[i] - ref[i]) / max(np.linalg.norm(ref[i]), scale) for i in range(5)]
    pic.close()
    return errs, st, ms


@pytest.mark.parametrize("precision", ["fp64", "fp32r"])
def test_three_region_grid_driver_wake(qs, precision):
    ax = three_region_axis(31, 5.0)
    jzb = _driver(ax, ax, 30, 6.0, nb=2.0, sr=0.6, sz=0.6, xic=1.5)
    errs, st, ms = _compare(qs, ax, ax, 30, 6.0, jzb, precision)
    assert max(errs) < 1e-9, errs
    assert st["max_m"] == int(ms.max())


def test_refined_steps_on_an_alternating_grid(qs):
    """A strong driver on a grid whose neighbouring spacings differ 2:1 in x
    and 3:1 in y (different axes): the refinement rule subdivides."""
    xn = alternating_axis(31, 4.0, 2.0)
    yn = alternating_axis(31, 4.0, 3.0, first_long=True)
    jzb = _driver(xn, yn, 24, 7.2, nb=8.0, sr=0.4, sz=0.75, xic=1.8)
    errs, st, ms = _compare(qs, xn, yn, 24, 7.2, jzb)
    assert ms.max() > 1 and st["max_m"] == int(ms.max())
    assert max(errs) < 1e-9, errs


def test_uniform_nodes_and_one_particle_per_cell(qs):
    ax = uniform_axis(63, 6.0)
    jzb = _driver(ax, ax, 16, 3.2, nb=0.5, sr=0.8, sz=0.6, xic=1.0)
    errs, _, _ = _compare(qs, ax, ax, 16, 3.2, jzb, ppc=1)
    assert max(errs) < 1e-9, errs


def test_arguments_and_state(qs):
    ax = uniform_axis(15, 3.0)
    pic = qs.NonuniformPIC(ax, ax, 4, 1.0)
    z = torch.zeros((4, 15, 15), dtype=torch.float64, device="cuda")
    _, st = pic.step3d(z, raise_on_error=False)
    assert st["status"] == qs.QS_ERR_STATE
    pic.init_plasma(9)
    pic.init_plasma(4)  # a second lattice replaces the first
    assert len(pic.plasma()["x"]) == 16 * 16 * 4
    hist, st = pic.step3d(z)
    assert float(hist.abs().max()) < 1e-12 and st["slices"] == 4
    with pytest.raises(qs.QsError):
        pic.step3d(z[:3].contiguous())
    pic.close()
    with pytest.raises(qs.QsError):
        qs.NonuniformPIC(np.array([0.0, 1.0, 0.5, 2.0]), uniform_axis(2, 1.0), 4, 1.0)
