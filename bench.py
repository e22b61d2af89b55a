#!/usr/bin/env python
"""Throughput of the quasi-static slice advance on one GB300 (or N replicas).

A "step" is one 3D step of the method: the driver current deposit, the full
xi-slice loop (deposit, psi / E_z, B_z / B_perp multigrid solves, moments,
explicit sources, push, adaptive sub-steps) and the frozen-field driver push.
The workload is the 256^2 blowout case: [-8,8]^2, 1024 base slices over a
12 k_p^-1 window, 4 plasma particles per cell (262,144), a driver (n_b = 5,
sigma_r = 0.3, sigma_z = 0.7, 500k macroparticles) and a witness (n_b = 2,
sigma_z = 0.3, 200k).  Inputs are synthetic (seeded bi-Gaussian beams, lattice
plasma).

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle on
a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import atexit
import json
import os
import signal
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "blowout256"
METRIC = "xi_slices_per_s"
UNIT = "slices/s"


def _args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="native", choices=["native", "reference"])
    p.add_argument("--form", default="both", choices=["fp64", "fp32r", "both"])
    p.add_argument("--cpu-seconds", type=float, default=15.0,
                   help="target CPU time of the oracle baseline sample")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--workload", default=WORKLOAD)
    p.add_argument("--slices", type=int, default=0,
                   help="profiling only: truncate the window to this many base slices")
    p.add_argument("--parity-slices", type=int, default=-1,
                   help="base slices of the live parity check against the oracle "
                        "(-1: the workload's default, 0: off)")
    return p.parse_args()


# live parity: base slices of the oracle prefix that the bench compares the
# GPU forms with (a few minutes of one host core at most, run concurrently
# with the GPU legs): through the driver and the first bubble at 256^2
PARITY_SLICES = {"linear64": 128, "blowout256": 256, "blowout512": 24}
PARITY_TOL = 1e-12  # solver tolerance of the parity steps (both sides solve exactly)


def _oracle_prefix_job(name: str, n_prefix: int, path: str):
    """Spawned process: the oracle's history of the first n_prefix base slices
    of workload `name`, saved to `path` (.npy) with its run time."""
    import numpy as np

    import oracle as O
    import workloads as W
    wl = W.workload(name)
    beams = [W.sample_beam(b) for b in wl.beams]
    cfg = O.config_from_workload(wl)
    pl, n_ion = O.plasma_from_workload(wl)
    t0 = time.perf_counter()
    r = O.step3d(cfg, pl, n_ion, beams, n_slices=n_prefix)
    np.save(path, r.history)
    with open(path + ".s", "w") as f:
        f.write(f"{time.perf_counter() - t0:.3f}")


def _start_parity(args, rank, world):
    """Starts the oracle prefix in a spawned process before any CUDA work."""
    n = args.parity_slices
    if n < 0:
        n = PARITY_SLICES.get(args.workload, 0)
    if n <= 0 or rank != 0 or world != 1 or args.slices > 0:
        return None
    import multiprocessing as mp
    d = tempfile.mkdtemp(prefix="qs_parity_")
    path = os.path.join(d, "oracle.npy")
    proc = mp.get_context("spawn").Process(target=_oracle_prefix_job,
                                          args=(args.workload, n, path), daemon=True)
    proc.start()
    return {"proc": proc, "path": path, "n": n, "dir": d}


def _finish_parity(job, qs, wl, forms):
    """Per-field relative L2 error of each form against the oracle prefix:
    ||F_gpu - F_oracle|| / max(||F_oracle||, ||psi_oracle||) over the first
    n base slices, from one untimed step per form solved to PARITY_TOL."""
    import numpy as np
    import workloads as W
    if job is None:
        return None
    n = job["n"]
    got = {}
    beams_np = [W.sample_beam(b) for b in wl.beams]
    for form in forms:
        ctx = qs.Context(qs.config_from_workload(wl, precision=form, mg_tol=PARITY_TOL))
        if wl.profile is None:
            ctx.init_plasma(wl.ppc)
        else:
            ctx.init_plasma(wl.ppc, wl.profile[0], wl.profile[1])
        st = ctx.step3d([qs.Beam(b) for b in beams_np])
        got[form] = (ctx.fields(qs.FIELD_ALL, 0, n, device=False).numpy(), st["psi_guard_hits"])
        ctx.close()
    job["proc"].join(timeout=900)
    if job["proc"].is_alive() or not os.path.exists(job["path"]):
        job["proc"].terminate()
        return {"slices": n, "error": "oracle prefix did not finish"}
    ref = np.load(job["path"])
    oracle_s = float(open(job["path"] + ".s").read())
    import shutil
    shutil.rmtree(job["dir"], ignore_errors=True)
    names = ("psi", "Ez", "Bz", "Bx", "By")
    out = {"slices": n, "xi_end": n * wl.xi_len / wl.n_xi, "mg_tol": PARITY_TOL,
           "oracle_s": oracle_s, "bar": {"fp64": 1e-9, "fp32r": 2e-5},
           "norm": "||F - F_oracle|| / max(||F_oracle||, ||psi_oracle||) over the prefix"}
    scale = np.linalg.norm(ref[0])
    for form, (g, hits) in got.items():
        out[form] = {nm: float(np.linalg.norm(g[i] - ref[i]) /
                               max(np.linalg.norm(ref[i]), scale, 1e-300))
                     for i, nm in enumerate(names)}
        out[form]["psi_guard_hits"] = int(hits)
    return out


SCAN = "scan48"


def _load_workload(args):
    import workloads as W
    if args.workload == SCAN:
        return None
    wl = W.workload(args.workload)
    if args.slices > 0:
        wl = wl.with_(n_xi=args.slices, xi_len=wl.xi_len * args.slices / wl.n_xi)
    return wl


def _dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(value: float, device="cpu") -> float:
    """The largest `value` over the ranks of the default process group (the
    job's time is the slowest rank's); the value itself with no group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, world: int, max_seconds: float) -> float:
    """Whole-job throughput of replicas (weak scaling): every rank processed
    `units_per_rank` units; the job took the slowest rank's time."""
    return units_per_rank * world / max_seconds


def _workload_desc(wl):
    beams = ", ".join(f"n_b={b.amplitude:g} sigma_r={b.sigma_x:g} sigma_z={b.sigma_z:g} "
                      f"xi_c={b.xi_c:g} N={b.n_particles}" for b in wl.beams)
    return (f"{wl.name}: {wl.n}x{wl.n} cells over [-{wl.half_width:g},{wl.half_width:g}]^2, "
            f"{wl.n_xi} base xi-slices over {wl.xi_len:g}, {wl.ppc} ppc "
            f"({wl.n_plasma} plasma macroparticles), beams [{beams}], refine_k={wl.refine_k}, "
            f"mg_tol={wl.mg_tol:g}, dt={wl.dt:g}")


# the float64 ALU roofline of the solver kernels: no measured float64 peak is
# available, so the nominal one, derived from the unit counts and clocks
FP64_PEAK_SOURCE = ("nominal: 152 SMs x 2.07 GHz x 2 FP64 FMA/clk/SM x 2 flop/FMA "
                    "= 1258 GFLOP/s, rounded to the 1250 of the data sheet")

# ---------------------------------------------------------------- ncu traffic
ENGINE_SOURCES = ("qs_engine.cuh", "qs_engine_fp64.cu", "qs_engine_fp32r.cu", "qs_solve.cuh",
                  "qs_mg.cuh", "qs_tile.cuh", "qs_internal.cuh")


def engine_source_hash(sources=ENGINE_SOURCES) -> str:
    import hashlib
    h = hashlib.sha256()
    for f in sources:
        with open(os.path.join(ROOT, "paper_2012_00881_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic(kernel: str, workload: str, form: str, profiles_dir: str = None,
                     source_hash: str = None):
    """DRAM bytes per launch from the committed ncu summary of this kernel and
    workload, if it was captured on the current engine source; else None."""
    d = profiles_dir or os.path.join(ROOT, "profiles")
    want = source_hash or engine_source_hash()
    if not os.path.isdir(d):
        return None
    for fn in sorted(os.listdir(d)):
        if not fn.endswith(".md"):
            continue
        with open(os.path.join(d, fn)) as f:
            for line in f:
                if not line.startswith("<!-- traffic "):
                    continue
                meta = {}
                for kv in line[len("<!-- traffic "):].replace("-->", "").split():
                    k, _, v = kv.partition("=")
                    meta[k] = v
                if (meta.get("kernel") == kernel and meta.get("workload") == workload
                        and meta.get("form") == form and meta.get("source_sha256") == want):
                    try:
                        return float(meta["bytes_per_launch"])
                    except (KeyError, ValueError):
                        return None
    return None


# ---------------------------------------------------------------- roofline model
def cycle_sweeps(form: str, over=None) -> int:
    """Red-black sweeps per level and V-cycle (pre + post) of a context made
    with these overrides: pre_sweeps -1 is the library's default for the form
    (3 refined, 2 float64), post_sweeps defaults to 2."""
    over = over or {}
    pre = over.get("pre_sweeps", -1)
    if pre < 0:
        pre = 3 if form == "fp32r" else 2
    return pre + over.get("post_sweeps", 2)


def algorithmic_bytes(stats, wl, form: str, n_xi: int, sweeps: int = None) -> float:
    """Bytes one slice-engine launch must move at minimum (the byte model).

    b = 8 (float64 form) or 4 (refined form: float32 momenta, weights, moment
    grids and inner multigrid cycles); positions, n_*, the fields and the
    history are float64 in both forms.
      particles, per pushed slice: positions read twice and written once
        (48 B), momenta read twice and written once (6b), weights read by the
        moment and density deposits (b + 8); the last slice reads positions,
        momenta and weights once (16 + 3b);
      grid phases, per slice: 50 words per point, of which 21 are moment
        grids (clears, deposits, reads in the assembly: b) and 29 float64
        (sources, fields, gradients, kappa, guesses); per base slice the
        history store 10 float64 words per point;
      multigrid, per V-cycle and component, with nu sweeps per level (pre +
        post): the fine level 3 nu b (read u, f, write u) + 4.5b (residual and
        restriction 2.25b, prolongation and correction 2.25b) + 2b (residual
        norm), the coarse levels a third of the fine level's 3 nu b + 4.5b
        (24b for nu = 4, 28b for nu = 5), plus 8b per point
        for kappa in a screened cycle; the refined form adds its float64
        outer residual and correction, 40 B per point and component (read u,
        r, write u, r, float32 r), and 32 B per point and component for the
        float64 residual that starts each solve."""
    b = 8 if form == "fp64" else 4
    nn = wl.n * wl.n
    np_ = wl.n_plasma
    slices = stats["slices"]
    part = ((48 + 6 * b + b + 8) * (slices - 1) + (16 + 3 * b)) * np_
    grid = ((21 * b + 29 * 8) * slices + 10 * 8 * n_xi) * nn
    v = stats["vcycles"]
    comp_cycles = v[0] + 2 * v[1] + 2 * v[2]
    nu = sweeps if sweeps is not None else cycle_sweeps(form)
    fine = 3 * nu * b + 4.5 * b
    mg = (comp_cycles * (fine + 2 * b + fine / 3) + v[2] * 8 * b) * nn
    if form != "fp64":
        mg += (comp_cycles * 40 + 5 * slices * 32) * nn
    return float(part + grid + mg)


# ---------------------------------------------------------------- clocks
def _die_with_parent():
    """Child side of Popen: receive SIGTERM when the parent process dies, so
    that a sampler never outlives a bench run that ended by an exception or a
    signal (a profiler waits for every process of the tree)."""
    try:
        import ctypes
        ctypes.CDLL(None, use_errno=True).prctl(1, int(signal.SIGTERM))  # PR_SET_PDEATHSIG
    except (OSError, AttributeError):
        pass


class ClockSampler:
    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None
        atexit.register(self._kill)

    def _kill(self):
        if self.proc and self.proc.poll() is None:
            self.proc.kill()

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL,
                preexec_fn=_die_with_parent)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for nm, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        loaded = [s for s in sm if mx and s > 0.3 * max(mx)] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(rows)}


# ---------------------------------------------------------------- native arm
def run_native(args):
    import numpy as np
    import torch

    import paper_2012_00881_gb300 as qs
    import workloads as W

    rank, world, local = _dist_env()
    parity_job = _start_parity(args, rank, world)  # before the first CUDA call
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    wl = _load_workload(args)
    forms = ["fp64", "fp32r"] if args.form == "both" else [args.form]
    beams_np = [W.sample_beam(b) for b in wl.beams]
    beam_bytes = sum(7 * 8 * len(b["x"]) for b in beams_np)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"

    results = {}
    for form in forms:
        cfg = qs.config_from_workload(wl, precision=form)
        ctx = qs.Context(cfg)
        if wl.profile is None:
            ctx.init_plasma(wl.ppc)
        else:
            ctx.init_plasma(wl.ppc, wl.profile[0], wl.profile[1])
        # the bunches advance from step to step (consecutive 3D steps of the
        # run: deposit, slice loop in their frozen current, driver push)
        beams = [qs.Beam(b, device=dev) for b in beams_np]

        def one_step():
            st = ctx.step3d(beams)
            ctx.push_beam(beams, wl.dt)
            return st

        for _ in range(args.warmup):
            one_step()
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        sampler = ClockSampler(local)
        sampler.start()
        times, engine_ms, slices, pushes, bytes_alg = [], [], 0, 0, 0.0
        vc = [0, 0, 0]
        max_m = 0
        for _ in range(args.steps):
            flush.zero_()  # evict L2 between timed steps (outside the events)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            st = one_step()
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
            engine_ms.append(st["gpu_ms"])
            slices += st["slices"]
            pushes += st["pushes"]
            vc = [a + b for a, b in zip(vc, st["vcycles"])]
            max_m = max(max_m, st["max_m"])
            bytes_alg += algorithmic_bytes(st, wl, form, wl.n_xi)
        clocks = sampler.stop()
        total_ms = max_over_ranks(sum(times), dev)
        # end to end through the public API with host buffers: each step copies
        # the bunches in from pinned host memory and their pushed state back,
        # which the next step starts from
        host = [{k: b.t[k].cpu().pin_memory() for k in qs.Beam.KEYS} for b in beams]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e2e_slices = 0
        for _ in range(args.steps):
            for hb, db in zip(host, beams):
                for k in qs.Beam.KEYS:
                    db.t[k].copy_(hb[k], non_blocking=True)
            st = one_step()
            e2e_slices += st["slices"]
            for hb, db in zip(host, beams):
                for k in qs.Beam.KEYS:
                    hb[k].copy_(db.t[k], non_blocking=True)
            torch.cuda.synchronize()
        e2e_s = time.perf_counter() - t0
        eng_s = sum(engine_ms) / 1e3
        achieved = bytes_alg / eng_s / 1e9
        results[form] = dict(
            value=job_rate(slices, world, total_ms / 1e3),
            pushes_per_s=job_rate(pushes, world, total_ms / 1e3),
            ms_per_step=total_ms / args.steps,
            slices_per_step=slices / args.steps,
            vcycles_per_step=[v / args.steps for v in vc],
            max_m=max_m,
            engine_ms_per_step=eng_s * 1e3 / args.steps,
            roofline={"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                      "frac": achieved / hbm_peak,
                      "traffic": measured_traffic("slice_engine", wl.name, form),
                      "kernel": "slice_engine", "peak_source": peak_src,
                      "bytes_per_launch": bytes_alg / args.steps},
            e2e={"value": e2e_slices * world / e2e_s, "unit": UNIT,
                 "h2d_bytes_per_step": beam_bytes, "d2h_bytes_per_step": beam_bytes},
            clocks=clocks,
            gpu_launches=args.steps * (1 + 2 * len(beams)),
        )
        ctx.close()

    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    main_form = "fp32r" if "fp32r" in results else forms[0]
    r = results[main_form]
    out = {
        "metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if main_form == "fp64" else "f32+f64",
        "data": "synthetic",
        "config": {"workload": _workload_desc(wl), "form": main_form,
                   "parallelism": f"replicas{world}" if world > 1 else "single",
                   "l2": "history and beam grid larger than L2; 256 MB write between steps"},
        "pushes_per_s": r["pushes_per_s"],
        "slices_per_step": r["slices_per_step"],
        "vcycles_per_step": r["vcycles_per_step"],
        "roofline": r["roofline"],
        "e2e": r["e2e"],
        "gpu_launches": r["gpu_launches"],
        "clocks": r["clocks"],
        "forms": {k: {kk: v[kk] for kk in ("value", "pushes_per_s", "ms_per_step",
                                            "slices_per_step", "vcycles_per_step", "max_m")}
                  for k, v in results.items()},
    }
    if not args.no_cpu_baseline and world == 1:
        out["cpu_baseline"] = cpu_baseline(wl, args.cpu_seconds)
    if parity_job is not None:
        out["parity"] = _finish_parity(parity_job, qs, wl, forms)
    print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


# ---------------------------------------------------------------- gradient
GRAD = "grad256"


def run_grad(args):
    """The differentiable form on the 256^2 case: one gradient evaluation is
    the forward (plasma lattice with the density table, driver from its 8
    parameters, one 3D step, witness gain) plus the backward (witness gain
    cotangent, checkpointed reverse slice loop, chain rules).  Reports
    gradient evaluations' slices/s and the grad/forward time ratio."""
    import numpy as np
    import torch

    import paper_2012_00881_gb300 as qs
    import workloads as W

    rank, world, local = _dist_env()
    torch.cuda.set_device(local)
    wl = W.workload(GRAD)
    if args.slices > 0:
        wl = wl.with_(n_xi=args.slices, xi_len=wl.xi_len * args.slices / wl.n_xi)
    drv, wit = wl.beams
    theta = [drv.amplitude, drv.sigma_x, drv.sigma_y, drv.sigma_z, drv.x_c, drv.y_c, drv.xi_c,
             drv.tilt]
    table, r_max = wl.profile
    z = torch.tensor(W.beam_normals(drv.n_particles, drv.seed), dtype=torch.float64,
                     device="cuda")
    witness = qs.Beam(W.sample_beam(wit))
    forms = ["fp64", "fp32r"] if args.form == "both" else [args.form]
    results = {}
    for form in forms:
        # the forward step keeps every slice's state in HBM for the adjoint
        # (checkpoint_every >= n_xi): the backward recomputes nothing
        ctx = qs.Context(qs.config_from_workload(wl, precision=form,
                                                 checkpoint_every=wl.n_xi))
        th = torch.tensor(theta, dtype=torch.float64, requires_grad=True)
        tb = torch.tensor(table, dtype=torch.float64, requires_grad=True)

        def one():
            th.grad = None
            tb.grad = None
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            e0.record()
            L = qs.witness_gain(ctx, th, tb, z, drv.gamma, witness, wl.dt, wl.ppc, r_max)
            e1.record()
            L.backward()
            e2.record()
            torch.cuda.synchronize()
            return float(L.detach()), e0.elapsed_time(e1), e1.elapsed_time(e2)

        for _ in range(args.warmup):
            one()
        sampler = ClockSampler(local)
        sampler.start()
        fwd, bwd = [], []
        for _ in range(args.steps):
            L, f, b = one()
            fwd.append(f)
            bwd.append(b)
        clocks = sampler.stop()
        slices = wl.n_xi
        results[form] = dict(loss=L, fwd_ms=sum(fwd) / len(fwd), bwd_ms=sum(bwd) / len(bwd),
                             grad_theta=th.grad.tolist(), grad_table=tb.grad.tolist(),
                             clocks=clocks)
        results[form]["value"] = slices / ((results[form]["fwd_ms"] + results[form]["bwd_ms"]) / 1e3)
        ctx.close()
    main = "fp32r" if "fp32r" in results else forms[0]
    r = results[main]
    out = {
        "metric": "xi_slices_per_s", "value": r["value"], "unit": "slices/s (gradient evaluations)",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": r["fwd_ms"] + r["bwd_ms"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if main == "fp64" else "f32+f64",
        "data": "synthetic",
        "config": {"workload": _workload_desc(wl) + ", loss = witness mean energy gain, "
                   "gradient w.r.t. 8 driver parameters and a 16-value density table, "
                   "every slice's state kept in HBM by the forward step", "form": main},
        "grad_over_fwd": r["bwd_ms"] / r["fwd_ms"] + 1.0,
        "forms": {k: {kk: v[kk] for kk in ("value", "fwd_ms", "bwd_ms", "loss", "grad_theta",
                                            "grad_table")} for k, v in results.items()},
        "clocks": r["clocks"],
    }
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------------- batched scan
def run_batched(args):
    """The 48-instance parameter scan (16 each of 128^2, 192^2, 256^2 over
    [-8,8]^2, 512 base slices, 4 ppc, n_b in [0.5, 8], sigma_r in [0.3, 0.8])
    as one batched launch per 3D step, refined form, settings per size from the
    autotuner (tuned untimed on 16-slice windows before the timed steps)."""
    import torch

    import paper_2012_00881_gb300 as qs
    import workloads as W
    from paper_2012_00881_gb300 import autotune as AT

    rank, world, local = _dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    insts = W.scan_instances()
    if args.slices > 0:
        insts = [wl.with_(n_xi=args.slices, xi_len=wl.xi_len * args.slices / wl.n_xi)
                 for wl in insts]
    t0 = time.perf_counter()
    tuned = AT.tune(insts, precision="fp32r", n_slices=16,
                    cands=AT.candidates(tiles=((32, 16), (64, 32)),
                                        sweeps=((3, 2), (2, 2), (2, 1)), coarse=(16, 32)))
    team = AT.tune_team(insts, tuned, precision="fp32r", n_slices=16)
    tune_s = time.perf_counter() - t0
    beams_np = [[W.sample_beam(b) for b in wl.beams] for wl in insts]
    ctxs, beams, master = [], [], []
    for wl, bn in zip(insts, beams_np):
        c = qs.Context(qs.config_from_workload(wl, precision="fp32r", **AT.apply(wl, tuned)))
        c.init_plasma(wl.ppc)
        ctxs.append(c)
        master.append([qs.Beam(b, device=dev) for b in bn])
        beams.append([qs.Beam(b, device=dev) for b in bn])

    def reset():
        for ms, bs in zip(master, beams):
            for a, b in zip(ms, bs):
                for k in qs.Beam.KEYS:
                    b.t[k].copy_(a.t[k])

    def one_step():
        st = qs.step3d_batched(ctxs, beams, team_blocks=team)
        for c, b, wl in zip(ctxs, beams, insts):
            c.push_beam(b, wl.dt)
        return st

    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    for _ in range(args.warmup):
        reset()
        one_step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    sampler = ClockSampler(local)
    sampler.start()
    times, slices, pushes, eng_ms, bytes_alg = [], 0, 0, 0.0, 0.0
    for _ in range(args.steps):
        reset()
        flush.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        st = one_step()
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
        eng_ms += st[0]["gpu_ms"]
        for s_, wl in zip(st, insts):
            slices += s_["slices"]
            pushes += s_["pushes"]
            bytes_alg += algorithmic_bytes(s_, wl, "fp32r", wl.n_xi,
                                           sweeps=cycle_sweeps("fp32r", AT.apply(wl, tuned)))
    clocks = sampler.stop()
    total_ms = max_over_ranks(sum(times), dev)
    # end to end: beams from pinned host memory each step, read back after
    host = [[{k: torch.as_tensor(b[k]).pin_memory() for k in qs.Beam.KEYS} for b in bn]
            for bn in beams_np]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_slices = 0
    for _ in range(args.steps):
        for hs, bs in zip(host, beams):
            for h, b in zip(hs, bs):
                for k in qs.Beam.KEYS:
                    b.t[k].copy_(h[k], non_blocking=True)
        st = one_step()
        e2e_slices += sum(s_["slices"] for s_ in st)
        out = [b.t["pz"].to("cpu", non_blocking=True) for bs in beams for b in bs]
        torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    bbytes = sum(7 * 8 * len(b["x"]) for bn in beams_np for b in bn)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    achieved = bytes_alg / (eng_ms / 1e3) / 1e9
    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    out = {
        "metric": METRIC, "value": job_rate(slices, world, total_ms / 1e3), "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": "scan48: 48 independent instances (16 each of 128^2, 192^2, 256^2 "
                               f"over [-8,8]^2), {insts[0].n_xi} base slices over "
                               f"{insts[0].xi_len:g}, 4 ppc, one driver each (n_b 0.5..8, "
                               "sigma_r 0.3..0.8, sigma_z 0.7, 100k), refined form, one batched "
                               "launch per 3D step",
                   "form": "fp32r-batched", "tuned": {str(k): v for k, v in tuned.items()},
                   "team_blocks": team,
                   "tune_seconds": tune_s,
                   "l2": "history and beam grids larger than L2; 256 MB write between steps"},
        "pushes_per_s": job_rate(pushes, world, total_ms / 1e3),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                     "frac": achieved / hbm_peak, "traffic": None,
                     "kernel": "slice_engine_batched", "peak_source": "measured",
                     "bytes_per_launch": bytes_alg / args.steps},
        "e2e": {"value": e2e_slices * world / e2e_s, "unit": UNIT,
                "h2d_bytes_per_step": bbytes,
                "d2h_bytes_per_step": sum(8 * len(b["x"]) for bn in beams_np for b in bn)},
        "gpu_launches": args.steps * (1 + 2 * sum(len(b) for b in beams)),
        "clocks": clocks,
    }
    print(json.dumps(out), flush=True)
    for c in ctxs:
        c.close()
    if world > 1:
        torch.distributed.destroy_process_group()


# ---------------------------------------------------------------- oracle timing
# ---------------------------------------------------------------- nonuniform grid
NONUNI = "nonuni255"
NONUNI_SOURCES = ("qs_nonuniform.cu", "qs_grid_sync.cuh")
# FP64 flops per finest node, field and V-cycle: four Gauss-Seidel sweeps of
# the 9-point corrected operator (65 flops a node), one residual (63) and the
# grid transfers (13), times 4/3 for the coarse levels, plus the residual of
# the convergence test (63).
NONUNI_FLOPS_PER_NODE_CYCLE = 4.0 / 3.0 * (4 * 65 + 63 + 13) + 63
# The five solves of one slice, grouped as the slice advance groups them:
# psi; E_z and B_z (one Poisson pair); B_x and B_y (one screened pair).
NONUNI_GROUPS = ((("psi",), False), (("ez", "bz"), False), (("bx", "by"), True))


def _nonuni_inputs(wl):
    import numpy as np
    from workloads.nonuniform import bubble_sources
    xn = wl.axis()
    src = bubble_sources(xn, xn, wl.bubble_radius)
    groups = [(np.stack([src[k] for k in keys]), src["m"] if screened else None)
              for keys, screened in NONUNI_GROUPS]
    return xn, groups


def _nonuni_desc(wl, xn):
    import numpy as np
    h = np.diff(xn)
    return (f"{wl.name}: {wl.n}x{wl.n} nodes over [-{wl.half_width:g},{wl.half_width:g}]^2, "
            f"three-region spacing {h.min():.4f}..{h.max():.4f}, 9-point operator with the "
            f"third-order correction, the five field solves of one blowout slice "
            f"(psi; E_z+B_z; B_x+B_y screened) from a zero guess to mg_tol={wl.mg_tol:g}")


def run_nonuniform(args):
    """The field solves of one xi-slice on the nonuniform transverse grid of
    the nonuniform-grid section (255^2 nodes, three-region spacing): psi, the
    E_z/B_z pair and the screened B_x/B_y pair, each from a zero initial guess.
    A step is that set of five solves.  Both forms run (FP64 and the
    float32-refined one, which stops on the same float64 residual); the line
    reports the refined form, the faster."""
    import torch

    import paper_2012_00881_gb300 as qs
    from workloads.nonuniform import nonuniform_workload

    rank, world, local = _dist_env()
    torch.cuda.set_device(local)
    if world > 1 and not torch.distributed.is_initialized():
        torch.distributed.init_process_group("nccl")
    wl = nonuniform_workload(NONUNI)
    xn, groups = _nonuni_inputs(wl)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        dev = [(torch.tensor(j, device="cuda"), None if m is None else torch.tensor(m, device="cuda"))
               for j, m in groups]
        outs = [torch.zeros_like(j) for j, _ in dev]
    n_fields = sum(int(j.shape[0]) for j, _ in dev)
    forms = ["fp64", "fp32r"] if args.form == "both" else [args.form]
    fp64_peak = 1250.0  # GFLOP/s: 152 SMs x 2.07 GHz x 2 FP64 FMA per clock per SM (nominal)
    results = {}
    for form in forms:
        with torch.cuda.stream(stream):
            solver = qs.NonuniformSolver(xn, xn, correction=True, precision=form, stream=stream)
        launches = []

        def step(record):
            for (j, m), u in zip(dev, outs):
                u.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                _, cyc, _ = solver.solve(j, u=u, m=m, tol=wl.mg_tol, max_cycles=100)
                e1.record(stream)
                if record:
                    launches.append((e0, e1, int(j.shape[0]), cyc))

        with torch.cuda.stream(stream):
            for _ in range(args.warmup):
                step(False)
            stream.synchronize()
            if world > 1:
                torch.distributed.barrier()
            sampler = ClockSampler(local)
            sampler.start()
            t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            t0.record(stream)
            for _ in range(args.steps):
                step(True)
            t1.record(stream)
            stream.synchronize()
            clocks = sampler.stop()
        ms = max_over_ranks(t0.elapsed_time(t1), f"cuda:{local}") / args.steps
        dur = sum(a.elapsed_time(b) for a, b, _, _ in launches) / 1e3
        flops = sum(NONUNI_FLOPS_PER_NODE_CYCLE * wl.n * wl.n * nr * cyc
                    for _, _, nr, cyc in launches)
        results[form] = dict(solver=solver, ms=ms, clocks=clocks,
                             value=job_rate(args.steps, world, ms * args.steps / 1e3),
                             cycles=[c for _, _, _, c in launches[:len(dev)]],
                             flops_per_s=flops / dur, launch_ms=dur * 1e3 / len(launches))
    main = "fp32r" if "fp32r" in results else forms[0]
    r = results[main]
    solver = r["solver"]
    # dominant kernel: the solve launch; FP64-equivalent flops counted from
    # the cycles it ran (the refined form's float32 cycles are counted the
    # same way, so its fraction is of the float64 peak)
    achieved = r["flops_per_s"] / 1e9
    traffic = measured_traffic("nu_solve_kernel", NONUNI, main,
                               source_hash=engine_source_hash(NONUNI_SOURCES))

    # end to end through the public API from pinned host buffers
    host_j = [torch.tensor(j).pin_memory() for j, _ in groups]
    host_m = [None if m is None else torch.tensor(m).pin_memory() for _, m in groups]
    host_u = [torch.empty(j.shape, dtype=torch.float64).pin_memory() for j, _ in groups]
    h2d = sum(t.numel() * 8 for t in host_j) + sum(t.numel() * 8 for t in host_m if t is not None)
    d2h = sum(t.numel() * 8 for t in host_u)

    def e2e_step():
        for k, (j, m) in enumerate(dev):
            j.copy_(host_j[k], non_blocking=True)
            if m is not None:
                m.copy_(host_m[k], non_blocking=True)
            outs[k].zero_()
            solver.solve(j, u=outs[k], m=m, tol=wl.mg_tol, max_cycles=100)
            host_u[k].copy_(outs[k], non_blocking=True)
        stream.synchronize()

    with torch.cuda.stream(stream):
        for _ in range(max(1, args.warmup)):
            e2e_step()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            e2e_step()
        e1.record(stream)
        stream.synchronize()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1), f"cuda:{local}") / args.steps
    out = {
        "metric": "nonuniform_slice_field_solves_per_s", "value": r["value"],
        "unit": "slice field sets/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": r["ms"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if main == "fp64" else "f32+f64", "data": "synthetic",
        "config": {"workload": _nonuni_desc(wl, xn), "form": main, "fields_per_step": n_fields,
                   "v_cycles": r["cycles"], "l2": "working set (about 12 MB) is L2-resident; "
                   "every step restarts the solves from zero"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": fp64_peak,
                     "unit": "GFLOP/s (FP64-equivalent, nominal FP64 peak)",
                     "frac": achieved / fp64_peak, "traffic": traffic,
                     "peak_source": FP64_PEAK_SOURCE},
        "e2e": {"value": job_rate(args.steps, world, e2e_ms * args.steps / 1e3),
                "unit": "slice field sets/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": len(dev) * args.steps,  # one solve kernel per qs_nu_solve
        "forms": {k: {"value": v["value"], "ms_per_step": v["ms"], "v_cycles": v["cycles"],
                      "launch_ms": v["launch_ms"]} for k, v in results.items()},
        "clocks": r["clocks"],
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = nonuni_cpu_baseline(wl, args.cpu_seconds)
    for v in results.values():
        v["solver"].close()
    if rank == 0:
        print(json.dumps(out), flush=True)


def nonuni_cpu_baseline(wl, seconds: float):
    """The oracle's sparse-LU solves of the same five fields (one thread)."""
    from oracle import qs_nonuniform as onu
    xn, groups = _nonuni_inputs(wl)
    t0 = time.perf_counter()
    sets = 0
    while True:
        for j, m in groups:
            for c in range(j.shape[0]):
                onu.solve(xn, xn, j[c], m)
        sets += 1
        if time.perf_counter() - t0 > seconds / 3:
            break
    dt = time.perf_counter() - t0
    return {"value": sets / dt, "unit": "slice field sets/s", "cores": 1, "kind": "oracle",
            "sample": f"{sets} full sets of the five solves of {wl.name} with scipy sparse LU "
                      f"(SuperLU), FP64, single thread"}


# ---------------------------------------------------------------- laser envelope
LASER = "laser256"
LASER_SOURCES = ("qs_laser.cu", "qs_grid_sync.cuh")
# FP64 flops per cell and V-cycle of the complex solve: four red-black sweeps
# at 30 flops a cell (complex 5-point Laplacian, kappa u, the update), one
# residual (22) and the transfers (10), times 4/3 for the coarse levels, plus
# the residual of the stopping test (22).
LASER_FLOPS_PER_CELL_CYCLE = 4.0 / 3.0 * (4 * 30 + 22 + 10) + 22


def _laser_desc(wl):
    return (f"{wl.name}: {wl.n}x{wl.n} cells over a {wl.width:g} box, {wl.n_xi} slices of "
            f"{wl.dxi:g}, k0={wl.k0:g}, dt={wl.dt:g}, Gaussian pulse a0={wl.a0:g} w0={wl.w0:g} "
            f"sigma_xi={wl.sigma_xi:g} in a synthetic blowout susceptibility; one time step of "
            f"the envelope per step, slices solved to tol={wl.tol:g}")


def run_laser(args):
    """The laser-envelope advance (Eq. laser_Enve) on laser256: a step is one
    time step of the envelope over all slices (one complex multigrid solve
    per slice, warm-started from the previous time step)."""
    import torch

    import paper_2012_00881_gb300 as qs
    from workloads.laser import bubble_susceptibility, gaussian_pulse, laser_workload

    rank, world, local = _dist_env()
    torch.cuda.set_device(local)
    if world > 1 and not torch.distributed.is_initialized():
        torch.distributed.init_process_group("nccl")
    wl = laser_workload(LASER)
    if args.slices > 0:
        import dataclasses
        wl = dataclasses.replace(wl, n_xi=min(args.slices, wl.n_xi))
    a_host = torch.tensor(gaussian_pulse(wl))
    chi_host = torch.tensor(bubble_susceptibility(wl))
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        lz = qs.LaserEnvelope(wl.n, wl.width, wl.n_xi, wl.k0, wl.dt, wl.dxi, stream=stream)
        chi = chi_host.cuda()
        a = a_host.cuda()
        for _ in range(args.warmup):
            lz.advance(chi, a, steps=1, tol=wl.tol)
        stream.synchronize()
        if world > 1:
            torch.distributed.barrier()
        sampler = ClockSampler(local)
        sampler.start()
        evs = []
        cycles = 0
        for _ in range(args.steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _, c, _ = lz.advance(chi, a, steps=1, tol=wl.tol)
            e1.record(stream)
            evs.append((e0, e1))
            cycles += c
        stream.synchronize()
        clocks = sampler.stop()
    ms = max_over_ranks(sum(x.elapsed_time(y) for x, y in evs), f"cuda:{local}") / args.steps
    slices = wl.n_xi * args.steps
    value = job_rate(slices, world, ms * args.steps / 1e3)
    flops = LASER_FLOPS_PER_CELL_CYCLE * wl.n * wl.n * cycles
    achieved = flops / (ms * args.steps / 1e3) / 1e9
    fp64_peak = 1250.0
    traffic = measured_traffic("laser_kernel", LASER, "fp64",
                               source_hash=engine_source_hash(LASER_SOURCES))
    # end to end: envelope and susceptibility from pinned host memory, the
    # new envelope back, every step
    a_pin = a_host.pin_memory()
    chi_pin = chi_host.pin_memory()
    out_pin = torch.empty_like(a_host).pin_memory()
    with torch.cuda.stream(stream):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            a.copy_(a_pin, non_blocking=True)
            chi.copy_(chi_pin, non_blocking=True)
            lz.advance(chi, a, steps=1, tol=wl.tol)
            out_pin.copy_(a, non_blocking=True)
        e1.record(stream)
        stream.synchronize()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1), f"cuda:{local}") / args.steps
    out = {
        "metric": "laser_xi_slices_per_s", "value": value, "unit": "laser slices/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
        "data": "synthetic",
        "config": {"workload": _laser_desc(wl), "v_cycles_per_slice": cycles / slices,
                   "l2": "working set (about 190 MB: envelope and susceptibility of every "
                         "slice) exceeds L2"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": fp64_peak,
                     "unit": "GFLOP/s (FP64, nominal peak)", "frac": achieved / fp64_peak,
                     "traffic": traffic, "peak_source": FP64_PEAK_SOURCE},
        "e2e": {"value": job_rate(slices, world, e2e_ms * args.steps / 1e3),
                "unit": "laser slices/s", "h2d_bytes_per_step": a_host.numel() * 16 +
                chi_host.numel() * 8, "d2h_bytes_per_step": a_host.numel() * 16},
        "gpu_launches": args.steps,  # one persistent launch per advance
        "clocks": clocks,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = laser_cpu_baseline(wl, args.cpu_seconds)
    lz.close()
    if rank == 0:
        print(json.dumps(out), flush=True)


def laser_cpu_baseline(wl, seconds: float):
    """The oracle's step on the first slices of the same workload (one thread)."""
    import math as _m
    from oracle import qs_laser as OL
    from oracle.qs_oracle import Grid
    from workloads.laser import bubble_susceptibility, gaussian_pulse
    g = Grid.square(wl.n, wl.width / 2)
    a = gaussian_pulse(wl)
    chi = bubble_susceptibility(wl)
    t0 = time.perf_counter()
    k = 4
    while True:
        OL.envelope_advance(g, a[:k], chi[:k], wl.k0, wl.dt, wl.dxi, 1)
        dt = time.perf_counter() - t0
        if dt > seconds / 3 or k >= wl.n_xi:
            break
        k = min(wl.n_xi, 2 * k)
        t0 = time.perf_counter()
    return {"value": k / dt, "unit": "laser slices/s", "cores": 1, "kind": "oracle",
            "sample": f"one time step of the first {k} slices of {wl.name}, scipy sparse LU "
                      f"per slice, FP64, single thread"}


def _oracle_sample(wl, seconds: float):
    """Time the FP64 oracle on the first base slices of one 3D step of the
    workload, growing the slice count until about `seconds` of CPU work."""
    import oracle as O
    import workloads as W

    cfg = O.config_from_workload(wl)
    pl, n_ion = O.plasma_from_workload(wl)
    beams = [W.sample_beam(b) for b in wl.beams]
    t0 = time.perf_counter()
    jzb = O.deposit_beam(cfg, beams)
    t_dep = time.perf_counter() - t0
    n = 2
    while True:
        t0 = time.perf_counter()
        r = O.step3d(cfg, pl, n_ion, beams, jzb=jzb, n_slices=n)
        dt = time.perf_counter() - t0
        if dt > 0.25 * seconds or n >= wl.n_xi:
            break
        n = min(wl.n_xi, max(n + 1, int(n * max(2.0, 0.5 * seconds / max(dt, 1e-3)))))
    return r, dt, n, t_dep


def cpu_baseline(wl, seconds: float):
    r, dt, n, t_dep = _oracle_sample(wl, seconds)
    return {"value": r.slices / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"first {n} base slices ({r.slices} computed slices) of one 3D step of "
                      f"{wl.name}, numpy/scipy FP64, single thread; driver deposit excluded "
                      f"({t_dep:.1f} s)",
            "pushes_per_s": r.pushes / dt}


def run_reference(args):
    rank, world, _ = _dist_env()
    if rank != 0:
        return
    if args.workload == NONUNI:
        return run_reference_nonuniform(args, world)
    if args.workload == LASER:
        return run_reference_laser(args, world)
    wl = _load_workload(args)
    if wl is None:  # the scan: time the oracle on its 256^2 instances
        import workloads as W
        wl = [w for w in W.scan_instances() if w.n == 256][0]
    per_step = max(2.0, args.cpu_seconds / 2)
    vals, slices, secs = [], 0, 0.0
    for i in range(args.warmup + args.steps):
        r, dt, n, _ = _oracle_sample(wl, per_step)
        if i >= args.warmup:
            vals.append(r.slices / dt)
            slices += r.slices
            secs += dt
    v = slices / secs
    sample = (f"first {n} base slices of one 3D step of {wl.name} per step, numpy/scipy FP64, "
              f"single thread")
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs * 1e3 / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": {"workload": _workload_desc(wl), "form": "oracle"},
           "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_reference_nonuniform(args, world):
    from workloads.nonuniform import nonuniform_workload
    wl = nonuniform_workload(NONUNI)
    per_step = max(2.0, args.cpu_seconds / 2)
    vals = []
    for i in range(args.warmup + args.steps):
        b = nonuni_cpu_baseline(wl, per_step)
        if i >= args.warmup:
            vals.append(b["value"])
    v = statistics.mean(vals)
    xn, _ = _nonuni_inputs(wl)
    out = {"impl": "reference", "metric": "nonuniform_slice_field_solves_per_s", "value": v,
           "unit": "slice field sets/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 / v, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": _nonuni_desc(wl, xn), "form": "oracle"},
           "cpu_baseline": {"value": v, "unit": "slice field sets/s", "cores": 1,
                            "kind": "oracle", "sample": b["sample"]},
           "e2e": {"value": v, "unit": "slice field sets/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_reference_laser(args, world):
    from workloads.laser import laser_workload
    wl = laser_workload(LASER)
    vals = []
    for i in range(args.warmup + args.steps):
        b = laser_cpu_baseline(wl, max(2.0, args.cpu_seconds / 2))
        if i >= args.warmup:
            vals.append(b["value"])
    v = statistics.mean(vals)
    out = {"impl": "reference", "metric": "laser_xi_slices_per_s", "value": v,
           "unit": "laser slices/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": wl.n_xi * 1e3 / v, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "c128", "data": "synthetic",
           "config": {"workload": _laser_desc(wl), "form": "oracle"},
           "cpu_baseline": {"value": v, "unit": "laser slices/s", "cores": 1, "kind": "oracle",
                            "sample": b["sample"]},
           "e2e": {"value": v, "unit": "laser slices/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------------- nonuniform slice loop
NUPIC = "nupic255"


def _nupic_inputs():
    """The node-grid slice loop of Sec. "Multigrid Solver with Nonuniform
    Grids" against the uniform grid it replaces: 255^2 nodes on the
    three-region axis over [-12.5, 12.5] (spacing 0.045 on the axis to 0.136
    outside), and 512^2 uniform cells of 0.05 over [-12.8, 12.8]; the driver
    of the 256^2 blowout (n_b = 5, sigma_r = 0.3, sigma_z = 0.7, xi_c = 2.1),
    4 particles per cell, 256 base slices over a 3.0 window (through the
    driver and the front of the bubble)."""
    from workloads.nonuniform import driver_current_nodes, three_region_axis
    import workloads as W
    ax = three_region_axis(255, 12.5)
    n_xi, length = 256, 3.0
    jzb = driver_current_nodes(ax, ax, n_xi, length, 5.0, 0.3, 0.7, 2.1)
    drv = W.workload("blowout256").beams[0]
    uni = W.Workload(name="uniform512", n=512, half_width=12.8, n_xi=n_xi, xi_len=length,
                     ppc=4, beams=(drv,))
    return ax, n_xi, length, jzb, uni


def run_nupic(args):
    import torch

    import paper_2012_00881_gb300 as qs
    import workloads as W

    rank, world, local = _dist_env()
    torch.cuda.set_device(local)
    if world > 1 and not torch.distributed.is_initialized():
        torch.distributed.init_process_group("nccl")
    dev = torch.device("cuda", local)
    ax, n_xi, length, jzb_np, uni = _nupic_inputs()
    form = "fp32r" if args.form == "both" else args.form
    jzb = torch.tensor(jzb_np, device=dev)
    pic = qs.NonuniformPIC(ax, ax, n_xi, length, precision=form)
    pic.init_plasma(4)
    for _ in range(args.warmup):
        pic.step3d(jzb, tol=1e-10)
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    t0 = time.perf_counter()
    slices, ms_dev, vc = 0, 0.0, [0, 0, 0]
    for _ in range(args.steps):
        _, st = pic.step3d(jzb, tol=1e-10)
        slices += st["slices"]
        ms_dev += st["gpu_ms"]
        vc = [a + b for a, b in zip(vc, st["vcycles"])]
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    clocks = sampler.stop()
    total_s = max_over_ranks(ms_dev / 1e3, dev)
    value = job_rate(slices, world, total_s)
    n_nodes = len(ax) - 2
    nu_flops = NONUNI_FLOPS_PER_NODE_CYCLE * n_nodes * n_nodes * (vc[0] + 2 * vc[1] + 2 * vc[2])
    # end to end: the driver current in from pinned host memory, the wake out
    jz_host = torch.tensor(jzb_np).pin_memory()
    hist_host = torch.empty((5,) + tuple(jzb_np.shape), dtype=torch.float64).pin_memory()
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    for _ in range(args.steps):
        jzb.copy_(jz_host, non_blocking=True)
        hist, _ = pic.step3d(jzb, tol=1e-10)
        hist_host.copy_(hist, non_blocking=True)
        torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t1
    pic.close()
    # the uniform 512^2 engine on the same box, driver and window
    ctx = qs.Context(qs.config_from_workload(uni, precision=form))
    ctx.init_plasma(uni.ppc)
    beams = [qs.Beam(W.sample_beam(b), device=dev) for b in uni.beams]
    ctx.step3d(beams)
    u_ms, u_sl = 0.0, 0
    for _ in range(args.steps):
        st = ctx.step3d(beams)
        u_ms += st["gpu_ms"]
        u_sl += st["slices"]
    ctx.close()
    if rank != 0:
        return
    out = {"metric": "nonuniform_xi_slices_per_s", "value": value, "unit": "slices/s",
           "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": total_s * 1e3 / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64 particles, " + form + " solves",
           "data": "synthetic",
           "config": {"workload": f"{NUPIC}: 255^2 nodes, three-region axis on [-12.5,12.5], "
                                  f"{n_xi} slices over {length}, 4 ppc (262,144), bi-Gaussian "
                                  f"driver n_b=5 sigma_r=0.3 sigma_z=0.7 as j_z on the nodes",
                      "form": form, "l2": "history larger than L2"},
           "vcycles_per_step": [v / args.steps for v in vc],
           "wall_ms_per_step": wall * 1e3 / args.steps,
           "uniform_512": {"value": u_sl / (u_ms / 1e3), "unit": "slices/s",
                           "config": "512^2 cells of 0.05 on [-12.8,12.8], same driver "
                                     "(500k particles), window and slices, " + form},
           "e2e": {"value": slices * world / e2e_s, "unit": "slices/s",
                   "h2d_bytes_per_step": jzb_np.nbytes, "d2h_bytes_per_step": 5 * jzb_np.nbytes},
           # the solves' FP64-equivalent flops (the nonuniform solver's count per
           # node, field and V-cycle) over the whole step's device time, which
           # also holds the particle and assembly phases: a lower bound for
           # the solve kernel
           "roofline": {"bound": "alu", "kernel": "nu_solve_kernel",
                        "achieved": nu_flops / (ms_dev / 1e3) / 1e9, "peak": 1250.0,
                        "unit": "GFLOP/s (FP64-equivalent, nominal FP64 peak)",
                        "frac": nu_flops / (ms_dev / 1e3) / 1e9 / 1250.0, "traffic": None,
                        "peak_source": FP64_PEAK_SOURCE,
                        "time": "the whole step's device time"},
           # per computed slice: deposit, psi source, three solves (one
           # persistent launch each), moments, two assemblies, push (none
           # after the last slice)
           "gpu_launches": 9 * slices - args.steps, "clocks": clocks}
    if world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = nupic_cpu_baseline(args.cpu_seconds)
    print(json.dumps(out), flush=True)


def nupic_cpu_baseline(seconds: float):
    """The oracle's node-grid slice loop on the first base slices."""
    import oracle as O  # noqa: F401  (package import)
    from oracle import qs_nonuniform_pic as P
    ax, n_xi, length, jzb, _ = _nupic_inputs()
    G = P.NodeGrid(ax, ax)
    pl, n_ion = P.init_plasma_nodes(G, 4)
    n = 1
    while True:
        t0 = time.perf_counter()
        P.step3d_nodes(G, n, length / n_xi, pl, n_ion, jzb[:n])
        dt = time.perf_counter() - t0
        if dt > 0.25 * seconds or n >= 16:
            break
        n = min(16, max(n + 1, int(n * max(2.0, 0.5 * seconds / max(dt, 1e-3)))))
    return {"value": n / dt, "unit": "slices/s", "cores": 1, "kind": "oracle",
            "sample": f"the first {n} base slices of {NUPIC} (scipy sparse LU per solve), "
                      f"FP64, single thread"}


# ---------------------------------------------------------------- DLA driver push
DLA = "dla256"
DLA_NSUB = 50  # sub-steps per laser time step (the paper's DLA comparison uses 50)


def run_dla(args):
    """The driver push in the laser's own fields (qs_push_beam_dla): a witness
    of 200,000 electrons (gamma = 20, sigma_r = 0.5, 1.0 behind the pulse
    centre) pushed by one laser time step of 5 in 50 sub-steps, in the wake
    and the envelope of one laser-driven step of laserwake256 (the envelope
    at t and after its step)."""
    import torch

    import paper_2012_00881_gb300 as qs
    import workloads as W
    from workloads.laser import gaussian_pulse

    rank, world, local = _dist_env()
    torch.cuda.set_device(local)
    if world > 1 and not torch.distributed.is_initialized():
        torch.distributed.init_process_group("nccl")
    dev = torch.device("cuda", local)
    lw, wl = _laserwake_inputs()
    ctx = qs.Context(qs.config_from_workload(wl, precision="fp32r"))
    ctx.init_plasma(wl.ppc)
    lz = qs.LaserEnvelope(lw.n, lw.width, lw.n_xi, lw.k0, lw.dt, lw.dxi)
    env0 = torch.tensor(gaussian_pulse(lw), device=dev)
    env1 = env0.clone()
    ctx.laser_step3d(lz, env1, tol=lw.tol)  # the wake, and the envelope at t + dt
    spec = W.BeamSpec(amplitude=0.05, sigma_x=0.5, sigma_y=0.5, sigma_z=0.5,
                      xi_c=lw.xi_c + 1.0, n_particles=200_000, seed=11, gamma=20.0)
    wit = W.sample_beam(spec)
    beam = qs.Beam(wit, device=dev)
    master = {k: v.clone() for k, v in beam.t.items()}

    def reset():
        for k in qs.Beam.KEYS:
            beam.t[k].copy_(master[k])

    for _ in range(args.warmup):
        reset()
        ctx.push_beam_dla([beam], lw.dt, env0, env1, lw.k0, DLA_NSUB)
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    times = []
    for _ in range(args.steps):
        reset()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        ctx.push_beam_dla([beam], lw.dt, env0, env1, lw.k0, DLA_NSUB)
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    clocks = sampler.stop()
    ms = max_over_ranks(sum(times), dev) / args.steps
    subs = spec.n_particles * DLA_NSUB
    # float64 work per particle sub-step: two envelope gathers (8 points of
    # A and its three differences, 2 complex values each), the wake gather
    # (8 points, 6 values), the carrier, the fields and the Boris step
    flops_per_sub = 2 * 8 * 4 * 2 * 4 + 8 * 6 * 3 + 60
    achieved = subs * flops_per_sub / (ms / 1e3) / 1e9
    # end to end: the witness in from pinned host memory and back
    host = {k: master[k].cpu().pin_memory() for k in qs.Beam.KEYS}
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for k in qs.Beam.KEYS:
            beam.t[k].copy_(host[k], non_blocking=True)
        ctx.push_beam_dla([beam], lw.dt, env0, env1, lw.k0, DLA_NSUB)
        for k in qs.Beam.KEYS:
            host[k].copy_(beam.t[k], non_blocking=True)
        torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    lz.close()
    ctx.close()
    if rank != 0:
        return
    out = {"metric": "dla_particle_substeps_per_s", "value": job_rate(subs, world, ms / 1e3),
           "unit": "particle sub-steps/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": f"{DLA}: 200,000 witness electrons (gamma 20), one laser "
                                  f"time step of {lw.dt} in {DLA_NSUB} sub-steps, in the wake "
                                  f"and envelopes of one laserwake256 step"},
           "roofline": {"bound": "alu", "achieved": achieved, "peak": 1250.0,
                        "unit": "GFLOP/s (FP64)", "frac": achieved / 1250.0, "traffic": None,
                        "peak_source": FP64_PEAK_SOURCE},
           "e2e": {"value": subs * args.steps / e2e_s, "unit": "particle sub-steps/s",
                   "h2d_bytes_per_step": 7 * 8 * spec.n_particles,
                   "d2h_bytes_per_step": 7 * 8 * spec.n_particles},
           "gpu_launches": args.steps, "clocks": clocks}
    if world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = dla_cpu_baseline(args.cpu_seconds)
    print(json.dumps(out), flush=True)


def dla_cpu_baseline(seconds: float):
    """The oracle's sub-cycled push (qs_dla.push_beam_dla) of a sample of the
    witness in a synthetic wake and the same envelope, on one host core."""
    import numpy as np

    import oracle as O
    from oracle import qs_dla as D
    import workloads as W
    from workloads.laser import gaussian_pulse
    lw, wl = _laserwake_inputs()
    cfg = O.config_from_workload(wl)
    env = gaussian_pulse(lw)
    hist = np.zeros((5, wl.n_xi, wl.n, wl.n))
    n = 200
    while True:
        spec = W.BeamSpec(amplitude=0.05, sigma_x=0.5, sigma_y=0.5, sigma_z=0.5,
                          xi_c=lw.xi_c + 1.0, n_particles=n, seed=11, gamma=20.0)
        b = W.sample_beam(spec)
        t0 = time.perf_counter()
        D.push_beam_dla(cfg, hist, env, env, lw.k0, b, lw.dt, DLA_NSUB)
        dt = time.perf_counter() - t0
        if dt > 0.25 * seconds or n >= 200_000:
            break
        n = min(200_000, int(n * max(2.0, 0.5 * seconds / max(dt, 1e-3))))
    return {"value": n * DLA_NSUB / dt, "unit": "particle sub-steps/s", "cores": 1,
            "kind": "oracle", "sample": f"{n} particles, {DLA_NSUB} sub-steps, numpy FP64, "
                                        f"single thread"}


# ---------------------------------------------------------------- laser-driven step
LASERWAKE = "laserwake256"


def _laserwake_inputs():
    """The laser-driven 3D step: the 256^2 laser geometry (box 24, 256 slices
    of 0.08, k0 = 20, dt = 5) with a uniform plasma of 4 particles per cell,
    driven by the Gaussian envelope a0 = 2, w0 = 3, sigma_xi = 2 centred 4
    behind the head (the laser blowout of the paper's Table 1 scaled to this
    grid) and no beam."""
    import workloads as W
    from workloads.laser import laser_workload
    lw = laser_workload(LASER)
    wl = W.Workload(name=LASERWAKE, n=lw.n, half_width=lw.width / 2, n_xi=lw.n_xi,
                    xi_len=lw.n_xi * lw.dxi, ppc=4, beams=())
    return lw, wl


def run_laserwake(args):
    """One laser-driven 3D step per bench step (qs_laser_step3d): the slice
    loop with the laser terms (|A|^2 in gamma, the ponderomotive force, the
    source term, chi out), then one time step of the envelope with that chi;
    the envelope carries over from step to step."""
    import torch

    import paper_2012_00881_gb300 as qs
    from workloads.laser import gaussian_pulse

    rank, world, local = _dist_env()
    torch.cuda.set_device(local)
    if world > 1 and not torch.distributed.is_initialized():
        torch.distributed.init_process_group("nccl")
    dev = torch.device("cuda", local)
    lw, wl = _laserwake_inputs()
    env0 = torch.tensor(gaussian_pulse(lw))
    forms = ["fp64", "fp32r"] if args.form == "both" else [args.form]
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    results = {}
    for form in forms:
        ctx = qs.Context(qs.config_from_workload(wl, precision=form))
        ctx.init_plasma(wl.ppc)
        lz = qs.LaserEnvelope(lw.n, lw.width, lw.n_xi, lw.k0, lw.dt, lw.dxi)
        a = env0.to(dev)
        for _ in range(args.warmup):
            ctx.laser_step3d(lz, a, tol=lw.tol)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        sampler = ClockSampler(local)
        sampler.start()
        times, wake_ms, slices, bytes_alg, env_cycles = [], 0.0, 0, 0.0, 0
        for _ in range(args.steps):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            st = ctx.laser_step3d(lz, a, tol=lw.tol)
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
            wake_ms += st["gpu_ms"]
            slices += st["slices"]
            env_cycles += st["env_cycles"]
            bytes_alg += algorithmic_bytes(st, wl, form, wl.n_xi)
        clocks = sampler.stop()
        total_ms = max_over_ranks(sum(times), dev)
        # end to end: the envelope from pinned host memory and back every step
        host = a.cpu().pin_memory()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e2e_slices = 0
        for _ in range(args.steps):
            a.copy_(host, non_blocking=True)
            st = ctx.laser_step3d(lz, a, tol=lw.tol)
            host.copy_(a, non_blocking=True)
            torch.cuda.synchronize()
            e2e_slices += st["slices"]
        e2e_s = time.perf_counter() - t0
        achieved = bytes_alg / (wake_ms / 1e3) / 1e9
        results[form] = dict(
            value=job_rate(slices, world, total_ms / 1e3), ms_per_step=total_ms / args.steps,
            wake_ms_per_step=wake_ms / args.steps,
            envelope_ms_per_step=(total_ms - wake_ms) / args.steps,
            env_cycles_per_step=env_cycles / args.steps,
            roofline={"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                      "frac": achieved / hbm_peak, "traffic": None, "kernel": "slice_engine",
                      "peak_source": "measured" if "hbm_gbs" in peaks else "fallback"},
            e2e={"value": e2e_slices * world / e2e_s, "unit": "slices/s",
                 "h2d_bytes_per_step": env0.numel() * 16,
                 "d2h_bytes_per_step": env0.numel() * 16},
            clocks=clocks)
        lz.close()
        ctx.close()
    if rank != 0:
        return
    main = "fp32r" if "fp32r" in results else forms[0]
    r = results[main]
    out = {"metric": "laser_driven_xi_slices_per_s", "value": r["value"], "unit": "slices/s",
           "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": r["ms_per_step"], "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64" if main == "fp64" else "f32+f64",
           "data": "synthetic",
           "config": {"workload": f"{LASERWAKE}: 256^2 on [-12,12]^2, 256 slices of 0.08, "
                                  f"4 ppc (262,144), laser a0=2 w0=3 sigma_xi=2 xi_c=4, "
                                  f"k0=20, dt=5; a step = the wake with the laser terms, "
                                  f"then one envelope time step",
                      "form": main, "l2": "history and envelope larger than L2"},
           "roofline": r["roofline"], "e2e": r["e2e"], "gpu_launches": args.steps * 3,
           "clocks": r["clocks"],
           "forms": {k: {kk: v[kk] for kk in ("value", "ms_per_step", "wake_ms_per_step",
                                               "envelope_ms_per_step", "env_cycles_per_step")}
                     for k, v in results.items()}}
    if world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = laserwake_cpu_baseline(args.cpu_seconds)
    print(json.dumps(out), flush=True)


def laserwake_cpu_baseline(seconds: float):
    """The oracle's laser-driven wake (step3d with laser_a2) on the first base
    slices, grown until about `seconds` of one host core."""
    import numpy as np

    import oracle as O
    from workloads.laser import gaussian_pulse
    lw, wl = _laserwake_inputs()
    a2 = np.abs(gaussian_pulse(lw)) ** 2
    cfg = O.config_from_workload(wl)
    pl, n_ion = O.plasma_from_workload(wl)
    n = 2
    while True:
        t0 = time.perf_counter()
        r = O.step3d(cfg, pl, n_ion, [], jzb=np.zeros((n + 1, wl.n, wl.n)), n_slices=n,
                     laser_a2=a2)
        dt = time.perf_counter() - t0
        if dt > 0.25 * seconds or n >= wl.n_xi:
            break
        n = min(wl.n_xi, max(n + 1, int(n * max(2.0, 0.5 * seconds / max(dt, 1e-3)))))
    return {"value": r.slices / dt, "unit": "slices/s", "cores": 1, "kind": "oracle",
            "sample": f"the laser-driven wake of the first {n} base slices of {LASERWAKE}, "
                      f"numpy/scipy FP64, single thread (the envelope step excluded)"}


def _reference_line(metric: str, workload: str, b: dict, ms_per_step: float, world: int,
                    args) -> str:
    return json.dumps({"impl": "reference", "metric": metric, "value": b["value"],
                       "unit": b["unit"], "n_gpus": world, "steps": args.steps,
                       "warmup": args.warmup, "ms_per_step": ms_per_step,
                       "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                       "dtype": "f64", "data": "synthetic",
                       "config": {"workload": workload, "form": "oracle"}, "cpu_baseline": b,
                       "e2e": {"value": b["value"], "unit": b["unit"], "h2d_bytes_per_step": 0,
                               "d2h_bytes_per_step": 0}})


if __name__ == "__main__":
    a = _args()
    if a.impl == "reference" and a.workload == DLA:
        rank, world, _ = _dist_env()
        if rank == 0:
            b = dla_cpu_baseline(a.cpu_seconds)
            print(_reference_line("dla_particle_substeps_per_s", DLA, b,
                                  200_000 * DLA_NSUB * 1e3 / b["value"], world, a), flush=True)
    elif a.impl == "reference" and a.workload in (LASERWAKE, NUPIC):
        rank, world, _ = _dist_env()
        if rank == 0:
            if a.workload == LASERWAKE:
                b = laserwake_cpu_baseline(a.cpu_seconds)
                print(_reference_line("laser_driven_xi_slices_per_s", LASERWAKE, b,
                                      256e3 / b["value"], world, a), flush=True)
            else:
                b = nupic_cpu_baseline(a.cpu_seconds)
                print(_reference_line("nonuniform_xi_slices_per_s", NUPIC, b,
                                      256e3 / b["value"], world, a), flush=True)
    elif a.impl == "reference":
        run_reference(a)
    elif a.workload == LASERWAKE:
        run_laserwake(a)
    elif a.workload == NUPIC:
        run_nupic(a)
    elif a.workload == DLA:
        run_dla(a)
    elif a.workload == SCAN:
        run_batched(a)
    elif a.workload == GRAD:
        run_grad(a)
    elif a.workload == NONUNI:
        run_nonuniform(a)
    elif a.workload == LASER:
        run_laser(a)
    else:
        run_native(a)
