"""Host logic of the autotuner (CPU): the candidate grid and how a tuned
result maps onto a workload's configuration overrides."""
import json

import workloads as W
from paper_2012_00881_gb300 import autotune as AT


def test_candidates_are_the_full_product():
    c = AT.candidates(tiles=((32, 16), (64, 32)), sweeps=((2, 2), (2, 1)), coarse=(16, 32),
                      omegas=(0, 115))
    assert len(c) == 2 * 2 * 2 * 2
    assert len({json.dumps(x, sort_keys=True) for x in c}) == len(c)
    assert all(set(x) == {"tile_x", "tile_y", "pre_sweeps", "post_sweeps", "coarse_block_n",
                          "omega_pct"} for x in c)


def test_apply_picks_the_settings_of_the_instance_size(tmp_path):
    tuned = {128: dict(tile_x=64, tile_y=32, pre_sweeps=2, post_sweeps=2, coarse_block_n=32,
                       omega_pct=0, ms_per_slice=0.2),
             256: dict(tile_x=32, tile_y=16, pre_sweeps=2, post_sweeps=1, coarse_block_n=16,
                       omega_pct=0, ms_per_slice=0.5)}
    insts = W.scan_instances()
    over = AT.apply(insts[2], tuned)          # a 256^2 instance
    assert insts[2].n == 256 and over["tile_x"] == 32 and over["post_sweeps"] == 1
    assert "ms_per_slice" not in over
    assert AT.apply(insts[1], tuned) == {}    # 192^2 not tuned: library defaults
    path = tmp_path / "tuned.json"
    AT.save(tuned, str(path))
    back = AT.load(str(path))
    assert back == tuned
    assert AT.load(str(tmp_path / "missing.json")) == {}
