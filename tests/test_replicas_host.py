"""Host logic of the replicas-only multi-GPU bench (CPU, gloo, world size 2).

One instance of the slice advance does not shard (the xi loop is serial), so
N GPUs run N replicas with no data-path collective; the only cross-rank step
is the timing: the job takes the slowest rank's time, and the whole-job rate
is the units all ranks processed over that time."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    os.environ["RANK"] = str(rank)
    os.environ["WORLD_SIZE"] = str(world)
    os.environ["LOCAL_RANK"] = str(rank)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    r, w, loc = bench._dist_env()
    ms = [1500.0, 1800.0][rank]          # the second replica is slower
    slowest = bench.max_over_ranks(ms, "cpu")
    rate = bench.job_rate(1024, w, slowest / 1e3)
    out[rank] = (r, w, loc, slowest, rate)
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_report_the_slowest_time_and_the_summed_rate():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for rank in range(world):
        r, w, loc, slowest, rate = out[rank]
        assert (r, w, loc) == (rank, world, rank)
        assert slowest == 1800.0
        assert rate == pytest.approx(2 * 1024 / 1.8)


def test_single_process_needs_no_group():
    import bench
    assert not dist.is_initialized()
    assert bench.max_over_ranks(12.5) == 12.5
    assert bench.job_rate(100, 1, 2.0) == 50.0


def test_traffic_lines_are_matched_per_line_and_source(tmp_path):
    """The roofline's measured traffic comes from a `<!-- traffic ... -->`
    line of a profile summary whose source hash matches the engine's; every
    line of a file is a candidate."""
    import bench
    (tmp_path / "a.md").write_text(
        "text\n"
        "<!-- traffic kernel=k workload=w form=fp32r source_sha256=abc bytes_per_launch=10 -->\n"
        "<!-- traffic kernel=k workload=w form=fp64 source_sha256=abc bytes_per_launch=20 -->\n")
    d = str(tmp_path)
    assert bench.measured_traffic("k", "w", "fp32r", d, "abc") == 10.0
    assert bench.measured_traffic("k", "w", "fp64", d, "abc") == 20.0
    assert bench.measured_traffic("k", "w", "fp64", d, "other") is None
    assert bench.measured_traffic("k", "x", "fp64", d, "abc") is None
    assert len(bench.engine_source_hash()) == 16
