"""The multi-process plumbing of bench.py on CPU: two gloo ranks (replicas only: the path does not shard,
so the only cross-rank operations are the barrier and the max-over-ranks timing reduction)."""
import json
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, world: int, port: int, out: str):
    os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import io
    from contextlib import redirect_stdout

    import bench
    import torch.distributed as dist

    w, r, local = bench.dist_setup()
    bench.barrier(w)
    m = bench.max_over_ranks(1.5 + rank, w)          # the slowest rank's time is the job's
    buf = io.StringIO()
    with redirect_stdout(buf):                       # only rank 0 runs and prints the reference arm
        if r != 0:
            bench.run_reference(None, w, r)           # returns before reading its arguments
    bench.barrier(w)
    dist.destroy_process_group()
    with open(f"{out}.{rank}", "w") as f:
        json.dump({"world": w, "rank": r, "max": m, "printed": buf.getvalue()}, f)


def test_two_gloo_ranks_agree_on_the_max_time(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    out = str(tmp_path / "r")
    mp.start_processes(_rank, args=(2, _free_port(), out), nprocs=2, start_method="spawn", join=True)
    res = [json.load(open(f"{out}.{i}")) for i in range(2)]
    assert [r["rank"] for r in res] == [0, 1] and all(r["world"] == 2 for r in res)
    assert all(r["max"] == 2.5 for r in res)
    assert res[1]["printed"] == ""
