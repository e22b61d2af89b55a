"""ctypes binding of libqs (include/qs.h): argument marshalling only.

Every step of the slice advance runs in the CUDA library; this module only
converts torch tensors to device pointers and structs to ctypes.  If the
library is missing, loading fails loudly: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Dict, List, Optional, Sequence

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "lib", "libqs.so")

QS_OK = 0
QS_ERR_ARG = -1
QS_ERR_CUDA = -2
QS_ERR_OOM = -3
QS_ERR_NOT_CONVERGED = -4
QS_ERR_PSI_FLOOR = -5
QS_ERR_STATE = -6
QS_ERR_TIMEOUT = -7
QS_FP64 = 0
QS_FP32_REFINED = 1
FIELD_PSI, FIELD_EZ, FIELD_BZ, FIELD_BX, FIELD_BY, FIELD_JZB = 1, 2, 4, 8, 16, 32
FIELD_ALL = 31
FIELD_NAMES = ("psi", "Ez", "Bz", "Bx", "By", "jzb")


class QsConfig(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("x_min", ctypes.c_double), ("x_max", ctypes.c_double),
        ("y_min", ctypes.c_double), ("y_max", ctypes.c_double),
        ("n_xi", ctypes.c_int),
        ("xi_min", ctypes.c_double), ("xi_max", ctypes.c_double),
        ("refine_k", ctypes.c_int),
        ("precision", ctypes.c_int),
        ("mg_tol", ctypes.c_double),
        ("mg_max_vcycles", ctypes.c_int),
        ("psi_floor", ctypes.c_double),
        ("max_psi_guard_hits", ctypes.c_int64),
        ("sort_every", ctypes.c_int),
        ("pre_sweeps", ctypes.c_int), ("post_sweeps", ctypes.c_int),
        ("coarse_block_n", ctypes.c_int),
        ("trace_capacity", ctypes.c_int),
        ("warm_start_order", ctypes.c_int),
        ("tile_x", ctypes.c_int), ("tile_y", ctypes.c_int),
        ("omega_pct", ctypes.c_int),
        ("coarse_pre_sweeps", ctypes.c_int),
        ("checkpoint_every", ctypes.c_int),
        ("barrier_wait_cycles", ctypes.c_int64),
        ("cluster_size", ctypes.c_int),
        ("deposit_band_rows", ctypes.c_int),
    ]


class QsBeam(ctypes.Structure):
    _fields_ = [
        ("x", ctypes.c_void_p), ("y", ctypes.c_void_p), ("xi", ctypes.c_void_p),
        ("px", ctypes.c_void_p), ("py", ctypes.c_void_p), ("pz", ctypes.c_void_p),
        ("w", ctypes.c_void_p),
        ("n", ctypes.c_int64),
        ("charge", ctypes.c_double), ("q_over_m", ctypes.c_double),
    ]


class QsStepStats(ctypes.Structure):
    _fields_ = [
        ("slices", ctypes.c_int64), ("substeps", ctypes.c_int64), ("pushes", ctypes.c_int64),
        ("vcycles", ctypes.c_int64 * 3), ("psi_guard_hits", ctypes.c_int64),
        ("sorts", ctypes.c_int64), ("max_relres", ctypes.c_double), ("vmax", ctypes.c_double),
        ("max_m", ctypes.c_int32), ("status", ctypes.c_int32), ("gpu_ms", ctypes.c_double),
    ]


_P = ctypes.c_void_p
_I = ctypes.c_int
_I64 = ctypes.c_int64
_D = ctypes.c_double

# name -> (restype, argtypes), mirroring include/qs.h
PROTOTYPES = {
    "qs_config_default": (None, [ctypes.POINTER(QsConfig)]),
    "qs_create": (_I, [ctypes.POINTER(QsConfig), _P, ctypes.POINTER(_P)]),
    "qs_destroy": (None, [_P]),
    "qs_init_plasma": (_I, [_P, _I, _P, _I, _D]),
    "qs_step3d": (_I, [_P, _P, _I, ctypes.POINTER(QsStepStats)]),
    "qs_step3d_schedule": (_I, [_P, _P, _I, _P, ctypes.POINTER(QsStepStats)]),
    "qs_push_beam": (_I, [_P, _P, _I, _D]),
    "qs_push_beam_dla": (_I, [_P, _P, _I, _D, _P, _P, _D, _I]),
    "qs_step3d_laser": (_I, [_P, _P, _I, _P, _P, ctypes.POINTER(QsStepStats)]),
    "qs_laser_step3d": (_I, [_P, _P, _P, _I, _P, _D, _I, ctypes.POINTER(QsStepStats), _P, _P]),
    "qs_step3d_batched": (_I, [_P, _I, _P, _P, _I, _P]),
    "qs_fields": (_I, [_P, _I, _I, _I, _P, _I]),
    "qs_slice_diagnostics": (_I, [_P, _P, _P, _P]),
    "qs_get_plasma": (_I, [_P, _P, _P, _P, _P, _P, _P]),
    "qs_plasma_count": (_I64, [_P]),
    "qs_cell_sort": (_I, [_P, _P, _P, _P, _I64, _P, _P, _P, _P]),
    "qs_phase_trace": (_I, [_P, _P, _P, _I]),
    "qs_cell_sort_noalloc": (_I, [_I, _D, _D, _D, _P, _P, _P, _I64, _P, _P, _P, _P, _P]),
    "qs_step3d_adjoint": (_I, [_P, _P, _I, _P, _P, _P, ctypes.POINTER(QsStepStats)]),
    "qs_beam_gain": (_I, [_P, _P, _D, ctypes.POINTER(_D), _P]),
    "qs_beam_deposit_adjoint": (_I, [_P, _P, _P, _P, _P, _P, _P]),
    "qs_profile_adjoint": (_I, [_P, _P, _P, _I, _D, _P]),
    "qs_bigaussian_beam": (_I, [_P, _P, _I64, _D, _P, _P]),
    "qs_bigaussian_adjoint": (_I, [_P, _P, _I64, _P, _P, _P, _P, _P, _P]),
    "qs_nu_create": (_I, [_I, _P, _P, _I, _I, _P, ctypes.POINTER(_P)]),
    "qs_nu_solve": (_I, [_P, _P, _I, _P, _P, _D, _I, _P, _P]),
    "qs_nu_set_cycle": (_I, [_P, _I, _I, _D, _I, _I]),
    "qs_nu_apply": (_I, [_P, _P, _P, _P]),
    "qs_nu_source": (_I, [_P, _P, _P]),
    "qs_nu_destroy": (None, [_P]),
    "qs_nu_pic_create": (_I, [_I, _P, _P, _I, _D, _I, _D, _I, _P, ctypes.POINTER(_P)]),
    "qs_nu_pic_init_plasma": (_I, [_P, _I]),
    "qs_nu_pic_step3d": (_I, [_P, _P, _P, _D, _I, ctypes.POINTER(QsStepStats)]),
    "qs_nu_pic_get_plasma": (_I, [_P, _P, _P, _P, _P, _P]),
    "qs_nu_pic_count": (_I64, [_P]),
    "qs_nu_pic_destroy": (None, [_P]),
    "qs_laser_create": (_I, [_I, _D, _I, _D, _D, _D, _P, ctypes.POINTER(_P)]),
    "qs_laser_advance": (_I, [_P, _P, _P, _I, _D, _I, _P, _P]),
    "qs_laser_destroy": (None, [_P]),
    "qs_strerror": (ctypes.c_char_p, [_I]),
    "qs_last_error": (ctypes.c_char_p, [_P]),
}

_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libqs.so (built in-tree by build()).  Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libqs.so not found at {path}; run paper_2012_00881_gb300.build.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in PROTOTYPES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class QsError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{message} (status {status})")
        self.status = status


def default_config(**overrides) -> QsConfig:
    lib = load_library()
    cfg = QsConfig()
    lib.qs_config_default(ctypes.byref(cfg))
    for k, v in overrides.items():
        setattr(cfg, k, v)
    return cfg


def config_from_workload(wl, precision: Optional[str] = None, **overrides) -> QsConfig:
    prec = precision or wl.precision
    cfg = default_config(
        nx=wl.n, ny=wl.n, x_min=-wl.half_width, x_max=wl.half_width, y_min=-wl.half_width,
        y_max=wl.half_width, n_xi=wl.n_xi, xi_min=0.0, xi_max=wl.xi_len,
        refine_k=wl.refine_k, precision=QS_FP64 if prec == "fp64" else QS_FP32_REFINED,
        mg_tol=wl.mg_tol, psi_floor=wl.psi_floor)
    for k, v in overrides.items():
        setattr(cfg, k, v)
    return cfg


def _ptr(t) -> int:
    return 0 if t is None else int(t.data_ptr())


def _check_sort_tensors(x, y, pid, out, n_cells: int, device=None):
    """Checks the tensors of a cell sort before any launch: x, y contiguous
    CUDA float64 of one length, pid int32 of that length, the outputs int32
    of sizes (npart, n_cells, n_cells + 1, npart), all on one device (and on
    `device` when given).  Raises ValueError on a mismatch."""
    import torch
    npart = int(x.numel()) if hasattr(x, "numel") else -1
    dev = x.device if hasattr(x, "device") else None
    for name, t, dt, size in (("x", x, torch.float64, npart), ("y", y, torch.float64, npart),
                              ("pid", pid, torch.int32, npart)):
        if not isinstance(t, torch.Tensor):
            raise ValueError(f"cell sort: {name} must be a torch tensor")
        if not t.is_cuda or t.dtype != dt or not t.is_contiguous() or t.numel() != size:
            raise ValueError(f"cell sort: {name} must be a contiguous CUDA {dt} tensor of "
                             f"{size} entries (got {t.dtype}, {t.numel()}, cuda={t.is_cuda})")
        if t.device != dev:
            raise ValueError(f"cell sort: {name} is on {t.device}, x on {dev}")
    if device is not None and dev != torch.device(device):
        raise ValueError(f"cell sort: tensors on {dev}, the context's device is {device}")
    if out is not None:
        if len(out) != 4:
            raise ValueError("cell sort: out must be (cell, count, offset, perm)")
        for name, t, size in zip(("cell", "count", "offset", "perm"), out,
                                 (npart, n_cells, n_cells + 1, npart)):
            if (not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.int32
                    or not t.is_contiguous() or t.numel() != size or t.device != dev):
                raise ValueError(f"cell sort: out {name} must be a contiguous int32 tensor of "
                                 f"{size} entries on {dev}")
    return npart


class Beam:
    """Driver macroparticles as float64 CUDA tensors (caller-owned memory)."""

    KEYS = ("x", "y", "xi", "px", "py", "pz", "w")

    def __init__(self, arrays: Dict, charge: float = -1.0, q_over_m: float = -1.0, device="cuda"):
        import torch
        self.t = {k: torch.as_tensor(arrays[k], dtype=torch.float64, device=device).contiguous()
                  for k in self.KEYS}
        self.charge = float(arrays.get("charge", charge)) if isinstance(arrays, dict) else charge
        self.q_over_m = float(arrays.get("q_over_m", q_over_m)) if isinstance(arrays, dict) else q_over_m

    @property
    def n(self) -> int:
        return int(self.t["x"].numel())

    def struct(self) -> QsBeam:
        b = QsBeam()
        for k in self.KEYS:
            setattr(b, k, _ptr(self.t[k]))
        b.n = self.n
        b.charge = self.charge
        b.q_over_m = self.q_over_m
        return b

    def numpy(self) -> Dict:
        out = {k: v.detach().cpu().numpy() for k, v in self.t.items()}
        out["charge"] = self.charge
        out["q_over_m"] = self.q_over_m
        return out


def _beam_array(beams: Sequence[Beam]):
    arr = (QsBeam * max(1, len(beams)))()
    for i, b in enumerate(beams):
        arr[i] = b.struct()
    return arr


class Context:
    """One slice-advance problem on the current CUDA device (qs_ctx)."""

    def __init__(self, cfg: QsConfig, stream=None):
        import torch
        self.lib = load_library()
        self.cfg = cfg
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        self.device = torch.device("cuda", torch.cuda.current_device())
        h = _P()
        st = self.lib.qs_create(ctypes.byref(cfg), _P(stream.cuda_stream), ctypes.byref(h))
        if st != QS_OK:
            raise QsError(st, "qs_create: " + self.lib.qs_strerror(st).decode())
        self.h = h

    # ---- helpers
    def _check(self, st: int, what: str):
        if st != QS_OK:
            msg = self.lib.qs_last_error(self.h).decode()
            raise QsError(st, f"{what}: {self.lib.qs_strerror(st).decode()}: {msg}")

    def close(self):
        if getattr(self, "h", None):
            self.lib.qs_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def n(self) -> int:
        return self.cfg.nx

    @property
    def n_xi(self) -> int:
        return self.cfg.n_xi

    # ---- API
    def init_plasma(self, ppc: int, profile: Optional[Sequence[float]] = None, r_max: float = 1.0):
        if profile is None:
            st = self.lib.qs_init_plasma(self.h, ppc, None, 0, 0.0)
        else:
            arr = (ctypes.c_double * len(profile))(*[float(v) for v in profile])
            st = self.lib.qs_init_plasma(self.h, ppc, ctypes.cast(arr, _P), len(profile), float(r_max))
        self._check(st, "qs_init_plasma")

    def step3d(self, beams: Sequence[Beam] = (), schedule: Optional[Sequence[int]] = None,
               raise_on_error: bool = True) -> Dict:
        arr = _beam_array(beams)
        stats = QsStepStats()
        if schedule is None:
            st = self.lib.qs_step3d(self.h, ctypes.cast(arr, _P), len(beams), ctypes.byref(stats))
        else:
            sch = (ctypes.c_int32 * len(schedule))(*[int(v) for v in schedule])
            st = self.lib.qs_step3d_schedule(self.h, ctypes.cast(arr, _P), len(beams),
                                             ctypes.cast(sch, _P), ctypes.byref(stats))
        if raise_on_error:
            self._check(st, "qs_step3d")
        return dict(status=st, slices=stats.slices, substeps=stats.substeps, pushes=stats.pushes,
                    vcycles=list(stats.vcycles), psi_guard_hits=stats.psi_guard_hits,
                    sorts=stats.sorts, max_relres=stats.max_relres, vmax=stats.vmax,
                    max_m=stats.max_m, gpu_ms=stats.gpu_ms)

    @staticmethod
    def _stats_dict(st: int, stats) -> Dict:
        return dict(status=st, slices=stats.slices, substeps=stats.substeps, pushes=stats.pushes,
                    vcycles=list(stats.vcycles), psi_guard_hits=stats.psi_guard_hits,
                    sorts=stats.sorts, max_relres=stats.max_relres, vmax=stats.vmax,
                    max_m=stats.max_m, gpu_ms=stats.gpu_ms)

    def _field_tensor(self, t, name: str, dtype=None):
        """Checks a CUDA tensor of shape [n_xi, N, N] for a laser step."""
        import torch
        shape = (self.n_xi, self.n, self.n)
        dtype = dtype or torch.float64
        if (not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != dtype
                or not t.is_contiguous() or tuple(t.shape) != shape or t.device != self.device):
            raise QsError(QS_ERR_ARG, f"{name} must be a contiguous {dtype} CUDA tensor "
                                      f"{list(shape)} on {self.device}")
        return t

    def step3d_laser(self, beams: Sequence[Beam], a2, chi=None,
                     raise_on_error: bool = True) -> Dict:
        """qs_step3d_laser: the slice loop with |A|^2 of a laser envelope
        (float64 [n_xi, N, N] CUDA tensor) at the base slices; `chi` (same
        shape, optional) receives n_* / (1+psi) at the base slices."""
        self._field_tensor(a2, "a2")
        if chi is not None:
            self._field_tensor(chi, "chi")
        arr = _beam_array(beams)
        stats = QsStepStats()
        st = self.lib.qs_step3d_laser(self.h, ctypes.cast(arr, _P), len(beams), _ptr(a2),
                                      _ptr(chi), ctypes.byref(stats))
        if raise_on_error:
            self._check(st, "qs_step3d_laser")
        return self._stats_dict(st, stats)

    def laser_step3d(self, laser: "LaserEnvelope", envelope, beams: Sequence[Beam] = (),
                     tol: float = 1e-10, max_cycles: int = 50,
                     raise_on_error: bool = True) -> Dict:
        """qs_laser_step3d: one laser-driven 3D step (the wake with |A|^2 of
        `envelope`, then one envelope time step with the wake's chi); the
        complex128 [n_xi, N, N] envelope is advanced in place."""
        import torch
        self._field_tensor(envelope, "envelope", torch.complex128)
        arr = _beam_array(beams)
        stats = QsStepStats()
        cyc = ctypes.c_int64(0)
        rel = ctypes.c_double(0.0)
        st = self.lib.qs_laser_step3d(self.h, _P(laser.h), ctypes.cast(arr, _P), len(beams),
                                      _ptr(envelope), float(tol), int(max_cycles),
                                      ctypes.byref(stats), ctypes.byref(cyc), ctypes.byref(rel))
        if raise_on_error:
            self._check(st, "qs_laser_step3d")
        out = self._stats_dict(st, stats)
        out.update(env_cycles=cyc.value, env_relres=rel.value)
        return out

    def push_beam_dla(self, beams: Sequence[Beam], dt: float, env_n, env_np1, k0: float,
                      n_sub: int):
        """qs_push_beam_dla: n_sub Boris sub-steps of dt/n_sub in the stored wake
        plus the laser fields rebuilt from the envelopes at t and t + dt
        (complex128 [n_xi, N, N] CUDA tensors)."""
        import torch
        self._field_tensor(env_n, "env_n", torch.complex128)
        self._field_tensor(env_np1, "env_np1", torch.complex128)
        arr = _beam_array(beams)
        self._check(self.lib.qs_push_beam_dla(self.h, ctypes.cast(arr, _P), len(beams), float(dt),
                                              _ptr(env_n), _ptr(env_np1), float(k0), int(n_sub)),
                    "qs_push_beam_dla")
        self.stream.synchronize()

    def push_beam(self, beams: Sequence[Beam], dt: float):
        arr = _beam_array(beams)
        self._check(self.lib.qs_push_beam(self.h, ctypes.cast(arr, _P), len(beams), float(dt)),
                    "qs_push_beam")

    def fields(self, mask: int = FIELD_ALL, begin: int = 0, end: Optional[int] = None,
               device: bool = True):
        """Base-slice fields as a float64 tensor [field][slice][iy][ix]."""
        import torch
        end = self.n_xi if end is None else end
        nf = bin(mask).count("1")
        shape = (nf, end - begin, self.n, self.n)
        if device:
            out = torch.empty(shape, dtype=torch.float64, device="cuda")
        else:
            out = torch.empty(shape, dtype=torch.float64).pin_memory()
        self._check(self.lib.qs_fields(self.h, mask, begin, end, _ptr(out), 1 if device else 0),
                    "qs_fields")
        return out

    def slice_diagnostics(self):
        import numpy as np
        m = np.zeros(self.n_xi, dtype=np.int32)
        vm = np.zeros(self.n_xi)
        ch = np.zeros(self.n_xi)
        self._check(self.lib.qs_slice_diagnostics(self.h, m.ctypes.data, vm.ctypes.data,
                                                  ch.ctypes.data), "qs_slice_diagnostics")
        return m, vm, ch

    def plasma(self):
        import numpy as np
        n = int(self.lib.qs_plasma_count(self.h))
        arrs = [np.zeros(n) for _ in range(5)]
        pid = np.zeros(n, dtype=np.int32)
        self._check(self.lib.qs_get_plasma(self.h, *[a.ctypes.data for a in arrs], pid.ctypes.data),
                    "qs_get_plasma")
        return dict(zip(("x", "y", "px", "py", "w"), arrs), id=pid)

    def phase_trace(self):
        """(where, t_ns) arrays of the last step's phase trace."""
        import numpy as np
        cap = max(1, int(self.cfg.trace_capacity))
        wh = np.zeros(cap, dtype=np.int32)
        tn = np.zeros(cap, dtype=np.int64)
        k = self.lib.qs_phase_trace(self.h, wh.ctypes.data, tn.ctypes.data, cap)
        if k < 0:
            self._check(k, "qs_phase_trace")
        return wh[:k], tn[:k]

    # ---- differentiable form
    def step3d_adjoint(self, d_hist=None, checkpoint_every: int = 0):
        """qs_step3d_adjoint: returns (d_jzb [n_xi,N,N], d_w [np], d_nion [N,N],
        stats) as float64 CUDA tensors for the cotangent d_hist [5,n_xi,N,N]."""
        import torch
        n = self.n
        np_ = int(self.lib.qs_plasma_count(self.h))
        d_jzb = torch.empty((self.n_xi, n, n), dtype=torch.float64, device="cuda")
        d_w = torch.empty(np_, dtype=torch.float64, device="cuda")
        d_nion = torch.empty((n, n), dtype=torch.float64, device="cuda")
        if d_hist is not None:
            d_hist = d_hist.to(dtype=torch.float64, device="cuda").contiguous()
        stats = QsStepStats()
        self._check(self.lib.qs_step3d_adjoint(self.h, _ptr(d_hist), int(checkpoint_every),
                                               _ptr(d_jzb), _ptr(d_w), _ptr(d_nion),
                                               ctypes.byref(stats)), "qs_step3d_adjoint")
        return d_jzb, d_w, d_nion, dict(slices=stats.slices, vcycles=list(stats.vcycles),
                                        gpu_ms=stats.gpu_ms)

    def beam_gain(self, beam: Beam, dt: float, d_hist=None) -> float:
        """qs_beam_gain: mean energy gain of `beam` over a push of dt (the beam
        is not moved); adds dL/d(history) into d_hist when given."""
        g = _D()
        b = beam.struct()
        self._check(self.lib.qs_beam_gain(self.h, ctypes.byref(b), float(dt), ctypes.byref(g),
                                          _ptr(d_hist)), "qs_beam_gain")
        return g.value

    def beam_deposit_adjoint(self, beam: Beam, d_jzb):
        """qs_beam_deposit_adjoint: (d_x, d_y, d_xi, d_w) of a bunch."""
        import torch
        out = [torch.empty(beam.n, dtype=torch.float64, device="cuda") for _ in range(4)]
        b = beam.struct()
        self._check(self.lib.qs_beam_deposit_adjoint(self.h, ctypes.byref(b), _ptr(d_jzb),
                                                     *[_ptr(t) for t in out]),
                    "qs_beam_deposit_adjoint")
        return tuple(out)

    def profile_adjoint(self, d_w, d_nion, n_coef: int, r_max: float):
        """qs_profile_adjoint: dL/d(profile table) as a numpy array."""
        import numpy as np
        out = np.zeros(int(n_coef))
        self._check(self.lib.qs_profile_adjoint(self.h, _ptr(d_w), _ptr(d_nion), int(n_coef),
                                                float(r_max), out.ctypes.data),
                    "qs_profile_adjoint")
        return out

    def cell_sort(self, x, y, pid):
        """Run the library's cell sort on CUDA tensors; returns (cell, count, offset, perm)."""
        import torch
        m = self.n * self.n
        n = _check_sort_tensors(x, y, pid, None, m, device=self.device)
        cell = torch.empty(n, dtype=torch.int32, device=x.device)
        count = torch.empty(m, dtype=torch.int32, device=x.device)
        offset = torch.empty(m + 1, dtype=torch.int32, device=x.device)
        perm = torch.empty(n, dtype=torch.int32, device=x.device)
        self._check(self.lib.qs_cell_sort(self.h, _ptr(x), _ptr(y), _ptr(pid), n, _ptr(cell),
                                          _ptr(count), _ptr(offset), _ptr(perm)), "qs_cell_sort")
        return cell, count, offset, perm


NOALLOC_MAX_CELLS = 512 * 512


def cell_sort_noalloc(n: int, x_min: float, y_min: float, h: float, x, y, pid, out=None,
                      stream=None):
    """qs_cell_sort_noalloc on CUDA tensors.  `out` may supply the output
    tensors (cell, count, offset, perm); the library allocates nothing.
    Waits for the stream before returning."""
    import torch
    if not (1 <= int(n) and int(n) * int(n) <= NOALLOC_MAX_CELLS):
        raise ValueError(f"cell_sort_noalloc: n * n must be in [1, {NOALLOC_MAX_CELLS}]")
    npart = _check_sort_tensors(x, y, pid, out, int(n) * int(n))
    lib = load_library()
    # the C call uses the current device's stream and scratch array
    with torch.cuda.device(x.device):
        if out is None:
            out = (torch.empty(npart, dtype=torch.int32, device=x.device),
                   torch.empty(n * n, dtype=torch.int32, device=x.device),
                   torch.empty(n * n + 1, dtype=torch.int32, device=x.device),
                   torch.empty(npart, dtype=torch.int32, device=x.device))
        cell, count, offset, perm = out
        st = torch.cuda.current_stream(x.device) if stream is None else stream
        rc = lib.qs_cell_sort_noalloc(n, float(x_min), float(y_min), float(h), _ptr(x), _ptr(y),
                                      _ptr(pid), npart, _ptr(cell), _ptr(count), _ptr(offset),
                                      _ptr(perm), _P(st.cuda_stream))
        if rc != QS_OK:
            raise QsError(rc, "qs_cell_sort_noalloc: " + lib.qs_strerror(rc).decode())
        st.synchronize()
    return cell, count, offset, perm


def step3d_batched(contexts: Sequence["Context"], beams: Sequence[Sequence[Beam]] = None,
                   team_blocks: int = 0, raise_on_error: bool = True) -> List[Dict]:
    """qs_step3d_batched over several contexts; returns one stats dict each."""
    lib = load_library()
    n = len(contexts)
    handles = (_P * n)(*[c.h for c in contexts])
    arrays = []
    ptrs = (_P * n)()
    counts = (ctypes.c_int * n)()
    for i in range(n):
        bl = list(beams[i]) if beams is not None else []
        arr = _beam_array(bl)
        arrays.append(arr)
        ptrs[i] = ctypes.cast(arr, _P)
        counts[i] = len(bl)
    stats = (QsStepStats * n)()
    st = lib.qs_step3d_batched(ctypes.cast(handles, _P), n, ctypes.cast(ptrs, _P),
                               ctypes.cast(counts, _P), int(team_blocks), ctypes.cast(stats, _P))
    if raise_on_error and st != QS_OK:
        msg = lib.qs_last_error(contexts[0].h).decode()
        raise QsError(st, f"qs_step3d_batched: {lib.qs_strerror(st).decode()}: {msg}")
    out = []
    for s_ in stats:
        out.append(dict(status=s_.status, slices=s_.slices, substeps=s_.substeps,
                        pushes=s_.pushes, vcycles=list(s_.vcycles),
                        psi_guard_hits=s_.psi_guard_hits, max_relres=s_.max_relres,
                        vmax=s_.vmax, max_m=s_.max_m, gpu_ms=s_.gpu_ms))
    return out


def bigaussian_beam(theta: Sequence[float], z, gamma: float, charge: float = -1.0,
                    q_over_m: float = -1.0) -> Beam:
    """qs_bigaussian_beam: the bunch of parameters theta on normals z [3, n]
    (float64 CUDA tensor)."""
    import torch
    lib = load_library()
    n = int(z.shape[1])
    arrays = {k: torch.empty(n, dtype=torch.float64, device="cuda") for k in Beam.KEYS}
    beam = Beam(arrays, charge=charge, q_over_m=q_over_m)
    th = (ctypes.c_double * 8)(*[float(v) for v in theta])
    b = beam.struct()
    st = torch.cuda.current_stream()
    rc = lib.qs_bigaussian_beam(ctypes.cast(th, _P), _ptr(z), n, float(gamma), ctypes.byref(b),
                                _P(st.cuda_stream))
    if rc != QS_OK:
        raise QsError(rc, "qs_bigaussian_beam: " + lib.qs_strerror(rc).decode())
    return beam


def bigaussian_adjoint(theta: Sequence[float], z, d_x, d_y, d_xi, d_w):
    """qs_bigaussian_adjoint: dL/dtheta (numpy, 8)."""
    import numpy as np
    import torch
    lib = load_library()
    th = (ctypes.c_double * 8)(*[float(v) for v in theta])
    out = np.zeros(8)
    st = torch.cuda.current_stream()
    rc = lib.qs_bigaussian_adjoint(ctypes.cast(th, _P), _ptr(z), int(z.shape[1]), _ptr(d_x),
                                   _ptr(d_y), _ptr(d_xi), _ptr(d_w), out.ctypes.data,
                                   _P(st.cuda_stream))
    if rc != QS_OK:
        raise QsError(rc, "qs_bigaussian_adjoint: " + lib.qs_strerror(rc).decode())
    return out


class NonuniformSolver:
    """qs_nu_* on a nonuniform tensor-product grid (float64 CUDA tensors).

    x_nodes, y_nodes: n + 2 increasing coordinates, walls first and last
    (array-likes, copied by the library).  correction=True selects the 9-point
    operator with the third-order correction; precision "fp64" or "fp32r"
    (float32 cycles refining a float64 solution)."""

    def __init__(self, x_nodes, y_nodes, correction: bool = True, precision: str = "fp64",
                 stream=None):
        import numpy as np
        import torch
        self._lib = load_library()
        self.h = None
        xn = np.ascontiguousarray(x_nodes, dtype=np.float64)
        yn = np.ascontiguousarray(y_nodes, dtype=np.float64)
        if xn.size != yn.size:
            raise QsError(QS_ERR_ARG, "x_nodes and y_nodes differ in length")
        self.n = int(xn.size) - 2
        self._stream = torch.cuda.current_stream() if stream is None else stream
        h = _P()
        if precision not in ("fp64", "fp32r"):
            raise QsError(QS_ERR_ARG, f"precision {precision!r}")
        prec = QS_FP64 if precision == "fp64" else QS_FP32_REFINED
        rc = self._lib.qs_nu_create(self.n, xn.ctypes.data, yn.ctypes.data, int(bool(correction)),
                                    prec, _P(self._stream.cuda_stream), ctypes.byref(h))
        if rc != QS_OK:
            raise QsError(rc, "qs_nu_create: " + self._lib.qs_strerror(rc).decode())
        self.h = h.value

    def _check(self, rc: int, what: str):
        if rc != QS_OK:
            raise QsError(rc, f"{what}: " + self._lib.qs_strerror(rc).decode())

    def solve(self, j, u=None, m=None, tol: float = 1e-10, max_cycles: int = 50,
              raise_on_error: bool = True):
        """Solve for j of shape [n, n] or [nrhs, n, n]; u (same shape) is the
        initial guess and receives the solution.  Returns (u, cycles, relres)."""
        import torch
        squeeze = j.dim() == 2
        jj = j.reshape(-1, self.n, self.n).contiguous()
        if u is None:
            u = torch.zeros_like(jj)
        # the library writes u in place: it must be the caller's own storage
        if not u.is_contiguous() or u.numel() != jj.numel():
            raise QsError(QS_ERR_ARG, "u must be a contiguous tensor shaped like j")
        uu = u.view(-1, self.n, self.n)
        mm = None if m is None else m.contiguous()
        for t in (jj, uu) + (() if mm is None else (mm,)):
            if t.dtype != torch.float64 or not t.is_cuda:
                raise QsError(QS_ERR_ARG, "j, u and m must be float64 CUDA tensors")
        if mm is not None and mm.numel() != self.n * self.n:
            raise QsError(QS_ERR_ARG, "m must hold n * n values")
        nrhs = int(jj.shape[0])
        cycles = ctypes.c_int(0)
        relres = (ctypes.c_double * 4)()
        rc = self._lib.qs_nu_solve(self.h, _ptr(mm), nrhs, _ptr(jj), _ptr(uu), float(tol),
                                   int(max_cycles), ctypes.byref(cycles),
                                   ctypes.cast(relres, _P))
        self.status = rc
        if raise_on_error:
            self._check(rc, "qs_nu_solve")
        out = uu[0] if squeeze else uu
        return out, cycles.value, [relres[c] for c in range(nrhs)]

    def set_cycle(self, pre_sweeps: int = 2, post_sweeps: int = 2, omega: float = 1.3,
                  coarse_block_n: int = 0, staged: bool = True):
        """Sweeps per level, Gauss-Seidel relaxation, the one-block level size
        (0 = default) and shared-memory staged smoothing of later solves."""
        self._check(self._lib.qs_nu_set_cycle(self.h, int(pre_sweeps), int(post_sweeps),
                                              float(omega), int(coarse_block_n),
                                              int(bool(staged))), "qs_nu_set_cycle")

    def apply(self, u, m=None):
        import torch
        uc = u.contiguous()
        mm = None if m is None else m.contiguous()
        out = torch.empty_like(uc)
        self._check(self._lib.qs_nu_apply(self.h, _ptr(mm), _ptr(uc), _ptr(out)), "qs_nu_apply")
        self._stream.synchronize()
        return out

    def source(self, j):
        import torch
        jc = j.contiguous()
        out = torch.empty_like(jc)
        self._check(self._lib.qs_nu_source(self.h, _ptr(jc), _ptr(out)), "qs_nu_source")
        self._stream.synchronize()
        return out

    def close(self):
        if self.h:
            self._lib.qs_nu_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class NonuniformPIC:
    """qs_nu_pic_*: the slice loop on a nonuniform node grid (n x n interior
    nodes, node coordinates with the walls), float64 particles and grids,
    solves in `precision` ("fp64" or "fp32r")."""

    def __init__(self, x_nodes, y_nodes, n_xi: int, xi_len: float, refine_k: int = 8,
                 psi_floor: float = 1e-3, precision: str = "fp64", stream=None):
        import numpy as np
        import torch
        self._lib = load_library()
        self.h = None
        xn = np.ascontiguousarray(x_nodes, dtype=np.float64)
        yn = np.ascontiguousarray(y_nodes, dtype=np.float64)
        self.n, self.n_xi = int(xn.size) - 2, int(n_xi)
        self.stream = torch.cuda.current_stream() if stream is None else stream
        h = _P()
        rc = self._lib.qs_nu_pic_create(self.n, xn.ctypes.data, yn.ctypes.data, self.n_xi,
                                        float(xi_len), int(refine_k), float(psi_floor),
                                        QS_FP64 if precision == "fp64" else QS_FP32_REFINED,
                                        _P(self.stream.cuda_stream), ctypes.byref(h))
        if rc != QS_OK:
            raise QsError(rc, "qs_nu_pic_create: " + self._lib.qs_strerror(rc).decode())
        self.h = h.value

    def init_plasma(self, ppc: int):
        rc = self._lib.qs_nu_pic_init_plasma(self.h, int(ppc))
        if rc != QS_OK:
            raise QsError(rc, "qs_nu_pic_init_plasma: " + self._lib.qs_strerror(rc).decode())

    def step3d(self, jzb, tol: float = 1e-10, max_cycles: int = 60,
               raise_on_error: bool = True):
        """One 3D step with the driver current jzb (float64 CUDA [n_xi, n, n]);
        returns (history [5, n_xi, n, n] CUDA tensor, stats dict)."""
        import torch
        shape = (self.n_xi, self.n, self.n)
        if (not isinstance(jzb, torch.Tensor) or not jzb.is_cuda or jzb.dtype != torch.float64
                or not jzb.is_contiguous() or tuple(jzb.shape) != shape):
            raise QsError(QS_ERR_ARG, f"jzb must be a contiguous float64 CUDA tensor {shape}")
        hist = torch.empty((5,) + shape, dtype=torch.float64, device=jzb.device)
        stats = QsStepStats()
        rc = self._lib.qs_nu_pic_step3d(self.h, _ptr(jzb), _ptr(hist), float(tol),
                                        int(max_cycles), ctypes.byref(stats))
        if raise_on_error and rc != QS_OK:
            raise QsError(rc, "qs_nu_pic_step3d: " + self._lib.qs_strerror(rc).decode())
        return hist, Context._stats_dict(rc, stats)

    def plasma(self):
        import numpy as np
        n = int(self._lib.qs_nu_pic_count(self.h))
        arrs = [np.zeros(n) for _ in range(5)]
        rc = self._lib.qs_nu_pic_get_plasma(self.h, *[a.ctypes.data for a in arrs])
        if rc != QS_OK:
            raise QsError(rc, "qs_nu_pic_get_plasma")
        return dict(zip(("x", "y", "px", "py", "w"), arrs))

    def close(self):
        if self.h is not None:
            self._lib.qs_nu_pic_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class LaserEnvelope:
    """qs_laser_* : the envelope advance of Eq. laser_Enve on an n x n
    cell-centred grid of side `width` with n_xi slices (float64 / complex128
    CUDA tensors).  dxi = math.inf drops the xi coupling."""

    def __init__(self, n: int, width: float, n_xi: int, k0: float, dt: float, dxi: float,
                 stream=None):
        import torch
        self._lib = load_library()
        self.h = None
        self.n, self.n_xi = int(n), int(n_xi)
        self._stream = torch.cuda.current_stream() if stream is None else stream
        h = _P()
        rc = self._lib.qs_laser_create(self.n, float(width), self.n_xi, float(k0), float(dt),
                                       float(dxi), _P(self._stream.cuda_stream),
                                       ctypes.byref(h))
        if rc != QS_OK:
            raise QsError(rc, "qs_laser_create: " + self._lib.qs_strerror(rc).decode())
        self.h = h.value

    def advance(self, chi, a, steps: int = 1, tol: float = 1e-10, max_cycles: int = 50,
                raise_on_error: bool = True):
        """Advance `a` (complex128 [n_xi, n, n], in place) by `steps` steps with
        `chi` (float64, same shape) fixed.  Returns (a, cycles, max_relres)."""
        import torch
        shape = (self.n_xi, self.n, self.n)
        if a.dtype != torch.complex128 or not a.is_contiguous() or tuple(a.shape) != shape:
            raise QsError(QS_ERR_ARG, "a must be a contiguous complex128 tensor [n_xi, n, n]")
        # keep the contiguous copy alive until the call has returned
        chi_c = chi.contiguous()
        if chi_c.dtype != torch.float64 or tuple(chi_c.shape) != shape:
            raise QsError(QS_ERR_ARG, "chi must be a float64 tensor [n_xi, n, n]")
        cycles = ctypes.c_int64(0)
        relres = ctypes.c_double(0.0)
        rc = self._lib.qs_laser_advance(self.h, _ptr(chi_c), _ptr(a), int(steps),
                                        float(tol), int(max_cycles), ctypes.byref(cycles),
                                        ctypes.byref(relres))
        self.status = rc
        if raise_on_error and rc != QS_OK:
            raise QsError(rc, "qs_laser_advance: " + self._lib.qs_strerror(rc).decode())
        return a, cycles.value, relres.value

    def close(self):
        if self.h:
            self._lib.qs_laser_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
