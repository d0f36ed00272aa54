"""The multi-GPU path of bench.py is replicas only (the step does not shard): every rank runs its
own lattice, the job's time is the slowest rank's, and only rank 0 prints.  Its host logic runs
here on CPU with world_size 2 over gloo."""
import json
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      LOCAL_RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, local, w = bench.dist_env()
    # rank-dependent step times: every rank must see the slowest one
    ms = bench.max_over_ranks(10.0 + 7.5 * rank, w, device="cpu")
    dist.barrier()
    with open(os.path.join(out_dir, "rank%d.json" % rank), "w") as f:
        json.dump({"rank": r, "local": local, "world": w, "ms": ms}, f)
    dist.destroy_process_group()


def test_max_over_ranks_and_env_with_two_gloo_ranks(tmp_path):
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    got = [json.load(open(tmp_path / ("rank%d.json" % r))) for r in range(2)]
    assert [g["rank"] for g in got] == [0, 1] and all(g["world"] == 2 for g in got)
    assert all(g["ms"] == 17.5 for g in got)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.25, 1) == 3.25


def test_reference_arm_runs_on_rank_zero_only(capsys):
    # under torchrun the other ranks of the reference arm exit without work or output
    sys.path.insert(0, ROOT)
    import argparse
    import bench
    args = argparse.Namespace(steps=1, warmup=0)
    assert bench.run_reference(args, 1, 2) is None
    assert capsys.readouterr().out == ""
