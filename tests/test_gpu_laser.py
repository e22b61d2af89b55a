"""Laser-envelope advance (Eq. laser_Enve) vs the FP64 oracle, through the C ABI (GPU).

Both sides take the same time-centred, head-to-tail discretisation; the GPU
solves each slice by complex multigrid to a relative residual of 1e-13 and the
oracle by sparse LU, so they agree to about cond * 1e-13 per slice: the bound
is 1e-9 relative in L2 after a few steps.
"""
import math

import numpy as np
import pytest

from oracle import qs_laser as QL
from oracle.qs_oracle import Grid
from workloads.laser import bubble_susceptibility, gaussian_pulse, laser_workload

pytestmark = pytest.mark.gpu


def _c(a):
    import torch
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.complex128, device="cuda")


def _r(a):
    import torch
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("n,n_xi,dxi", [(32, 8, 0.2), (48, 5, 0.1), (64, 3, math.inf),
                                        (16, 12, 0.05), (34, 4, 0.2), (40, 4, 0.1)])
def test_advance_matches_oracle(qs, n, n_xi, dxi):
    """Sizes cover each form of the coarse part: staged levels above 8 with
    the levels of side <= 8 in every block's shared memory and an exact
    coarsest inverse (32, 48, 64, 16), a 5^2 coarsest level too large for
    the inverse (40: sweeps), a 17^2 coarsest level too large for shared
    memory (34: block 0 in global memory)."""
    width = 8.0
    g = Grid.square(n, width / 2)
    rng = np.random.default_rng(n)
    x = -width / 2 + (np.arange(n) + 0.5) * g.h
    X, Y = np.meshgrid(x, x)
    xi = np.arange(n_xi)
    a0 = (np.exp(-(X ** 2 + Y ** 2) / 4.0)[None] * np.exp(-((xi - n_xi / 3) / 2.0) ** 2)[:, None, None]
          * (1.0 + 0.3j * rng.standard_normal((n_xi, n, n))))
    chi = rng.uniform(0.0, 2.0, (n_xi, n, n))
    ref = QL.envelope_advance(g, a0, chi, 5.0, 1.0, dxi, 3)
    lz = qs.LaserEnvelope(n, width, n_xi, 5.0, 1.0, dxi)
    a = _c(a0)
    _, cycles, relres = lz.advance(_r(chi), a, steps=3, tol=1e-13, max_cycles=60)
    assert relres <= 1e-13 and cycles > 0
    assert _rel(a.cpu().numpy(), ref) < 1e-9


def test_paraxial_gaussian_on_gpu(qs):
    """No xi coupling, vacuum: the GPU reproduces the oracle and the closed form."""
    n, width, w0, k0 = 128, 20.0, 2.5, 10.0
    g = Grid.square(n, width / 2)
    x = -width / 2 + (np.arange(n) + 0.5) * g.h
    X, Y = np.meshgrid(x, x)
    zr = k0 * w0 * w0 / 2
    a0 = np.exp(-(X ** 2 + Y ** 2) / w0 ** 2)[None]
    lz = qs.LaserEnvelope(n, width, 1, k0, zr / 40, math.inf)
    a = _c(a0)
    lz.advance(_r(np.zeros((1, n, n))), a, steps=40, tol=1e-13, max_cycles=80)
    got = a.cpu().numpy()
    ref = QL.envelope_advance(g, a0, np.zeros((1, n, n)), k0, zr / 40, math.inf, 40)
    assert _rel(got, ref) < 1e-9
    q = 1.0 + 1j
    closed = np.exp(-(X ** 2 + Y ** 2) / (w0 ** 2 * q)) / q
    assert _rel(got[0], closed) < 5e-3


def test_full_grid_slices(qs):
    """The 256^2 grid of the benchmark, first 12 slices of its pulse and
    blowout susceptibility, one step, against the oracle."""
    wl = laser_workload("laser256")
    a0 = gaussian_pulse(wl)[:12]
    chi = bubble_susceptibility(wl)[:12]
    g = Grid.square(wl.n, wl.width / 2)
    ref = QL.envelope_advance(g, a0, chi, wl.k0, wl.dt, wl.dxi, 1)
    lz = qs.LaserEnvelope(wl.n, wl.width, 12, wl.k0, wl.dt, wl.dxi)
    a = _c(a0)
    lz.advance(_r(chi), a, steps=1, tol=1e-13, max_cycles=60)
    assert _rel(a.cpu().numpy(), ref) < 1e-9


def test_edge_cases(qs):
    n = 16
    lz = qs.LaserEnvelope(n, 4.0, 4, 3.0, 0.5, 0.1)
    chi = _r(np.ones((4, n, n)))
    a = _c(np.zeros((4, n, n)))
    _, cycles, relres = lz.advance(chi, a, steps=3)
    assert not a.abs().max().item() and cycles == 0
    b = _c(np.ones((4, n, n)))
    b0 = b.clone()
    _, cycles, _ = lz.advance(chi, b, steps=0)
    assert cycles == 0 and bool((b == b0).all())
    _, cycles, relres = lz.advance(chi, b, steps=1, tol=1e-15, max_cycles=1,
                                   raise_on_error=False)
    assert lz.status == qs.QS_ERR_NOT_CONVERGED and cycles == 4 and relres > 1e-15
    lib = qs.load_library()
    assert lib.qs_laser_advance(lz.h, None, b.data_ptr(), 1, 1e-10, 10, None, None) == qs.QS_ERR_ARG
    assert lib.qs_laser_advance(lz.h, chi.data_ptr(), b.data_ptr(), -1, 1e-10, 10, None, None) == qs.QS_ERR_ARG
    assert lib.qs_laser_advance(lz.h, chi.data_ptr(), b.data_ptr(), 1, 0.0, 10, None, None) == qs.QS_ERR_ARG
