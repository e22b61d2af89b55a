"""Autotuner of the batched slice engine.

For each transverse size in a batch it times candidate engine settings and
keeps the fastest:

* the output tile of the grid-wide multigrid levels staged in shared memory
  (tile_x, tile_y; both forms stage their grid levels),
* the red-black sweeps before and after the coarse correction (pre_sweeps,
  post_sweeps) and their over-relaxation factor (omega_pct),
* the side below which a level is relaxed by one thread block
  (coarse_block_n),

and, for the whole batch, the number of thread blocks per team
(tune_team).

Every candidate solves to the same residual tolerance, so the choice changes
only the time, not the result.  A candidate is timed on a batch of the
instances of that size with the xi window truncated to a few slices, through
qs_step3d_batched; device time per computed slice is the score.  Settings
that do not fit in shared memory are skipped.
"""
from __future__ import annotations

import itertools
import json
import os
from typing import Dict, List, Sequence

from . import _binding as B

DEFAULT_TILES = ((32, 16), (32, 32), (64, 32))
DEFAULT_SWEEPS = ((3, 2), (2, 2), (3, 3))
DEFAULT_COARSE = (16, 32)
DEFAULT_OMEGAS = (0,)  # 0: the library default


def candidates(tiles=DEFAULT_TILES, sweeps=DEFAULT_SWEEPS, coarse=DEFAULT_COARSE,
               omegas=DEFAULT_OMEGAS) -> List[Dict]:
    return [dict(tile_x=t[0], tile_y=t[1], pre_sweeps=s[0], post_sweeps=s[1], coarse_block_n=c,
                 omega_pct=o)
            for t, s, c, o in itertools.product(tiles, sweeps, coarse, omegas)]


def _truncated(wl, n_slices: int):
    if wl.n_xi <= n_slices:
        return wl
    return wl.with_(n_xi=n_slices, xi_len=wl.xi_len * n_slices / wl.n_xi)


def time_candidate(wls: Sequence, cand: Dict, n_slices: int, precision: str,
                   beams_cache: Dict, repeats: int = 2, team_blocks: int = 0,
                   per_size: Dict = None) -> float:
    """Device milliseconds per computed slice of a truncated batched step
    (settings `cand` for every instance, or per size from `per_size`)."""
    ctxs, beams = [], []
    try:
        for wl in wls:
            w2 = _truncated(wl, n_slices)
            over = apply(wl, per_size) if per_size else cand
            cfg = B.config_from_workload(w2, precision=precision, **over)
            ctx = B.Context(cfg)
            if w2.profile is None:
                ctx.init_plasma(w2.ppc)
            else:
                ctx.init_plasma(w2.ppc, w2.profile[0], w2.profile[1])
            ctxs.append(ctx)
            key = (wl.name, n_slices)
            if key not in beams_cache:
                import workloads as W
                beams_cache[key] = [B.Beam(W.sample_beam(b)) for b in w2.beams]
            beams.append(beams_cache[key])
    except B.QsError:
        for c in ctxs:
            c.close()
        return float("inf")
    best = float("inf")
    B.step3d_batched(ctxs, beams, team_blocks=team_blocks)  # warm-up
    for _ in range(repeats):
        st = B.step3d_batched(ctxs, beams, team_blocks=team_blocks)
        slices = sum(s["slices"] for s in st)
        best = min(best, st[0]["gpu_ms"] / max(slices, 1))
    for c in ctxs:
        c.close()
    return best


def tune(wls: Sequence, precision: str = "fp32r", n_slices: int = 16,
         cands: Sequence[Dict] = None, max_per_size: int = 16, verbose: bool = False) -> Dict:
    """Best settings per transverse size: {n: settings dict (with 'ms_per_slice')}."""
    cands = list(cands or candidates())
    by_size: Dict[int, list] = {}
    for wl in wls:
        by_size.setdefault(wl.n, []).append(wl)
    beams_cache: Dict = {}
    result = {}
    for n, group in sorted(by_size.items()):
        group = group[:max_per_size]
        scored = []
        for cand in cands:
            t = time_candidate(group, cand, n_slices, precision, beams_cache)
            scored.append((t, cand))
            if verbose:
                print(f"n={n} {cand} -> {t:.4f} ms/slice", flush=True)
        t, best = min(scored, key=lambda x: x[0])
        result[n] = dict(best, ms_per_slice=t)
    return result


def tune_team(wls: Sequence, per_size: Dict, precision: str = "fp32r", n_slices: int = 16,
              teams: Sequence[int] = (0, 4, 6, 8, 12, 19), verbose: bool = False) -> int:
    """Blocks per team (0 = one team per instance) that minimise the time of
    the whole truncated batch with the per-size settings `per_size`."""
    beams_cache: Dict = {}
    scored = []
    for tb in teams:
        t = time_candidate(wls, {}, n_slices, precision, beams_cache, team_blocks=tb,
                           per_size=per_size)
        scored.append((t, tb))
        if verbose:
            print(f"team_blocks={tb} -> {t:.4f} ms/slice", flush=True)
    return min(scored)[1]


def apply(wl, tuned: Dict) -> Dict:
    """Config overrides for workload `wl` from a tune() result."""
    s = tuned.get(wl.n) or tuned.get(str(wl.n))
    if not s:
        return {}
    return {k: v for k, v in s.items() if k != "ms_per_slice"}


def save(tuned: Dict, path: str):
    with open(path, "w") as f:
        json.dump({str(k): v for k, v in tuned.items()}, f, indent=1)


def load(path: str) -> Dict:
    if not os.path.exists(path):
        return {}
    with open(path) as f:
        return {int(k): v for k, v in json.load(f).items()}
