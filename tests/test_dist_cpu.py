"""The N > 1 path of bench.py on CPU: world_size-2 gloo process groups.

Each rank solves its own replica (no collective on the data path); the only
collectives are the barrier around the timed region and the max-over-ranks
of the measured time.  Checked here: every rank receives the slowest
rank's time, the whole-job value is the DOFs all ranks solved over that
time, and the reference arm does no work and prints nothing on other
ranks.
"""
import io
import json
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = 100.0 + 25.0 * rank                 # rank 1 is the slow one
    dist.barrier()
    got = bench.max_over_ranks(local_ms, dist, "cpu")
    value = bench.job_value(world, 1000, 5, got / 1e3)
    # the reference arm: ranks other than 0 return at once and print nothing
    # (rank 0 would time the oracle; not run here)
    printed = io.StringIO()
    if rank != 0:
        with redirect_stdout(printed):
            bench.run_reference(bench.parse_args([]))
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump({"max": got, "value": value, "printed": printed.getvalue()}, f)


def test_two_rank_gloo_timing(tmp_path):
    import torch.multiprocessing as mp
    world, port = 2, _free_port()
    mp.start_processes(_rank_main, args=(world, port, str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    res = [json.load(open(tmp_path / f"r{r}.json")) for r in range(world)]
    assert all(r["max"] == 125.0 for r in res)
    assert all(r["value"] == pytest.approx(2 * 1000 * 5 / 0.125) for r in res)
    assert res[1]["printed"] == ""


def test_single_process_path():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5
    assert bench.job_value(1, 10, 2, 0.5) == 40.0
