"""Replica plumbing of bench.py on CPU: two gloo ranks take the slowest
rank's time, report whole-job throughput, and only rank 0 runs the oracle
reference arm."""
import json
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, lr = bench.dist_env()
        bench.barrier(w)
        my_ms = 100.0 + 50.0 * rank          # rank 1 is the slow one
        ms_max = bench.max_over_ranks(my_ms, w)
        value = bench.job_value(1000, 4, w, ms_max)
        with open(os.path.join(out_dir, f"r{rank}.json"), "w") as fh:
            json.dump({"env": [w, r, lr], "ms_max": ms_max, "value": value}, fh)
        bench.barrier(w)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank(tmp_path):
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    res = [json.load(open(tmp_path / f"r{r}.json")) for r in range(world)]
    for r, x in enumerate(res):
        assert x["env"] == [world, r, r]
        assert x["ms_max"] == 150.0
        # 1000 units x 4 steps on each of 2 ranks over the slowest 0.15 s
        assert x["value"] == pytest.approx(1000 * 4 * 2 / 0.150)


def test_single_process_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(12.5, 1) == 12.5
    assert bench.job_value(10, 2, 1, 1000.0) == pytest.approx(20.0)


def _ref_rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import contextlib
    import io

    import bench

    class Args:
        workload = "linear_landau_16"
        precision = None
        steps = 1
        warmup = 0
        gpus = world

    buf = io.StringIO()
    # only rank 0 may touch the oracle; rank 1 must return without work
    if rank == 1:
        import builtins

        real_import = builtins.__import__

        def guard(name, *a, **k):
            if name == "oracle" or name.startswith("oracle."):
                raise AssertionError("rank 1 imported the oracle")
            return real_import(name, *a, **k)

        builtins.__import__ = guard
    with contextlib.redirect_stdout(buf):
        bench.run_reference(Args, world, rank)
    with open(os.path.join(out_dir, f"ref{rank}.txt"), "w") as fh:
        fh.write(buf.getvalue())


def test_reference_arm_runs_on_rank0_only(tmp_path):
    world = 2
    mp.spawn(_ref_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    out0 = (tmp_path / "ref0.txt").read_text().strip().splitlines()
    out1 = (tmp_path / "ref1.txt").read_text()
    assert out1 == ""
    line = json.loads(out0[-1])
    assert line["impl"] == "reference"
    assert line["unit"] == "dof-updates/s" and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"
