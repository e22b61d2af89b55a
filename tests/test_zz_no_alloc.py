"""The allocation-free cell sort agrees with the context-based one (GPU).

qs_cell_sort_noalloc is for callers that cannot let a library allocate
device memory (their own memory pool owns the GPU, a host passes only raw
buffers, or cudaMalloc's possible device synchronisation is not acceptable).
Its only scratch is a fixed device array shared by all calls, so the check
runs two different sorts back to back: the second must not see anything left
over from the first.  Bit-exact agreement is required (integer outputs).
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _inputs(seed, n, L, npart):
    rng = np.random.default_rng(seed)
    h = 2 * L / n
    x = rng.uniform(-L, L, npart)
    y = rng.uniform(-L, L, npart)
    k = min(64, npart)
    x[:k] = -L + h * rng.integers(0, n + 1, k)  # cell faces and both walls
    pid = rng.permutation(npart).astype(np.int32)
    return x, y, pid, h


def _noalloc(qs, n, L, h, x, y, pid):
    import torch
    lib = qs.load_library()
    npart = int(x.numel())
    cell = torch.full((npart,), -1, dtype=torch.int32, device="cuda")
    count = torch.full((n * n,), -1, dtype=torch.int32, device="cuda")
    offset = torch.full((n * n + 1,), -1, dtype=torch.int32, device="cuda")
    perm = torch.full((npart,), -1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    rc = lib.qs_cell_sort_noalloc(n, -L, -L, h, x.data_ptr(), y.data_ptr(), pid.data_ptr(),
                                  npart, cell.data_ptr(), count.data_ptr(), offset.data_ptr(),
                                  perm.data_ptr(), ctypes.c_void_p(stream.cuda_stream))
    assert rc == qs.QS_OK, lib.qs_strerror(rc)
    stream.synchronize()
    return [t.cpu().numpy() for t in (cell, count, offset, perm)]


def test_noalloc_cell_sort_matches_context_sort_twice(qs):
    import torch
    import workloads as W

    # two different problems in a row: a large one, then a smaller one whose
    # cursors occupy only part of the shared scratch array
    for seed, n, L, npart in ((1, 256, 8.0, 262144), (2, 96, 5.0, 40000)):
        xh, yh, ph, h = _inputs(seed, n, L, npart)
        t = lambda a: torch.as_tensor(a, device="cuda")
        x, y, pid = t(xh), t(yh), t(ph)
        got = _noalloc(qs, n, L, h, x, y, pid)
        wl = W.Workload(name="s", n=n, half_width=L, n_xi=2, xi_len=1.0, ppc=4, beams=())
        ctx = qs.Context(qs.config_from_workload(wl))
        ref = [v.cpu().numpy() for v in ctx.cell_sort(x, y, pid)]
        ctx.close()
        for a, b, name in zip(got, ref, ("cell", "count", "offset", "perm")):
            assert np.array_equal(a, b), (seed, name)
        assert got[2][-1] == npart
        # and directly against the oracle's counting sort (ties by id)
        import oracle as O
        want = O.cell_sort(xh, yh, ph, O.Grid.square(n, L))
        for a, b, name in zip(got, want, ("cell", "count", "offset", "perm")):
            assert np.array_equal(a.astype(np.int64), np.asarray(b, dtype=np.int64)), (seed, name)


def test_noalloc_binding_rejects_bad_tensors_before_launch(qs):
    import torch
    x = torch.zeros(100, dtype=torch.float64, device="cuda")
    pid = torch.arange(100, dtype=torch.int32, device="cuda")
    with pytest.raises(ValueError):  # float32 positions
        qs.cell_sort_noalloc(8, -1.0, -1.0, 0.25, x.float(), x, pid)
    with pytest.raises(ValueError):  # ids of another length
        qs.cell_sort_noalloc(8, -1.0, -1.0, 0.25, x, x, pid[:50])
    short = (torch.empty(100, dtype=torch.int32, device="cuda"),
             torch.empty(10, dtype=torch.int32, device="cuda"),
             torch.empty(65, dtype=torch.int32, device="cuda"),
             torch.empty(100, dtype=torch.int32, device="cuda"))
    with pytest.raises(ValueError):  # count shorter than n * n
        qs.cell_sort_noalloc(8, -1.0, -1.0, 0.25, x, x, pid, out=short)
    with pytest.raises(ValueError):  # non-contiguous
        qs.cell_sort_noalloc(8, -1.0, -1.0, 0.25, torch.zeros(200, dtype=torch.float64,
                                                              device="cuda")[::2], x, pid)


def test_noalloc_rejects_grids_beyond_its_scratch(qs):
    lib = qs.load_library()
    side = 513  # 513^2 cells exceed the 512^2 the fixed scratch holds
    rc = lib.qs_cell_sort_noalloc(side, -1.0, -1.0, 2.0 / side, None, None, None, 0, None,
                                  None, None, None, None)
    assert rc == qs.QS_ERR_ARG
