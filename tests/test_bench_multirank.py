"""bench.py's N > 1 path on CPU: gloo ranks agree on the slowest time and the summed pixels."""
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


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    ms, px = bench.reduce_over_ranks(10.0 + 5.0 * rank, 1000 * (rank + 1), world, torch.device("cpu"))
    out[rank] = (ms, px)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_time_and_pixels():
    world = 2
    port = _free_port()
    out = mp.Manager().dict()
    mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        assert out[r] == (15.0, 3000.0)  # max of 10/15 ms, sum of 1000/2000 pixels


def test_reference_arm_other_ranks_exit_without_work(monkeypatch):
    import bench

    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        steps, warmup, gpus, seed = 1, 0, 2, 0

    assert bench.run_reference(A()) is None  # returns at once, prints nothing


def test_pass_throughput_from_traced_kernels():
    """Forward and backward Mpix/s come from the traced time of their kernels only."""
    import bench

    trace = {"k_project": (2, 0.1), "k_tile_totals": (2, 0.02), "k_scan_tiles": (2, 0.02), "k_scatter": (2, 0.06),
             "k_sort_tiles": (2, 0.1), "k_render<20>": (2, 1.5), "k_backward<20>": (2, 1.4),
             "k_grad_finalize": (2, 0.08), "k_pose_grad_shared": (2, 0.02), "k_mse": (2, 0.04), "k_adam": (2, 0.02)}
    out = bench.pass_throughput(trace, 1_000_000, 2)
    assert abs(out["fwd"]["ms_per_step"] - 0.9) < 1e-12
    assert abs(out["bwd"]["ms_per_step"] - 0.75) < 1e-12
    assert abs(out["fwd"]["mpix_s"] - 1e6 / 0.9e-3 / 1e6) < 1e-6
    assert bench.pass_throughput({}, 10, 1) is None


def test_oracle_timings_of_the_smaller_workloads():
    """The CPU baseline also times the oracle on the whole 64x64 dense frame
    and on a pixel sample of the 256x256 feature scene."""
    import bench

    out = bench.oracle_configs(2)
    assert out["plain_64"]["pixels"] == 64 * 64 and out["posefit_256"]["pixels"] == 8192
    assert all(v["value"] > 0 and v["seconds"] > 0 for v in out.values())
