"""The N > 1 path of bench.py on CPU: two ranks over gloo (127.0.0.1).

Checks the pieces the multi-GPU run uses besides the kernels: the process
group and barrier, the max-over-ranks time and the sum-over-ranks work, and the
round-robin deal of the batch workload's independent problems (every problem
on exactly one rank, 64 per rank, the single-GPU batch as rank 0's stream
prefix).  No GPU and no data-path collective are involved.
"""
import json
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out_dir):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(ws), "LOCAL_RANK": str(rank)})
    sys.path.insert(0, ROOT)
    import bench
    w, r, local = bench.dist_env()
    barrier = bench.dist_init(w, local, backend="gloo")
    barrier()
    res = {
        "env": [w, r, local],
        "max": bench.dist_reduce(10.0 + rank, "max"),
        "sum": bench.dist_reduce(1.0 + rank, "sum"),
        "shard": bench.shard(range(11), rank, ws),
        "units": [[i, x.N, x.M, x.g] for i, x in bench.shard(bench.batch_units(ws), rank, ws)],
    }
    barrier()
    bench.dist_finish()
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump(res, f)


def test_two_ranks_over_gloo(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ws = 2
    mp.start_processes(_rank_main, args=(ws, _free_port(), str(tmp_path)), nprocs=ws, start_method="spawn")
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(ws)]
    for r in range(ws):
        assert res[r]["env"] == [ws, r, r]
        assert res[r]["max"] == 11.0
        assert res[r]["sum"] == 3.0
    # every item on exactly one rank
    assert sorted(res[0]["shard"] + res[1]["shard"]) == list(range(11))
    units = res[0]["units"] + res[1]["units"]
    assert len(res[0]["units"]) == len(res[1]["units"]) == 64
    assert sorted(u[0] for u in units) == list(range(128))
    # the global stream's first 64 problems are the single-GPU batch
    import bench
    from paper_2005_13679_gb300 import inputs
    single = inputs.uneven_ll_batch()
    stream = sorted(units)
    assert [(u[1], u[2], u[3]) for u in stream[:64]] == [(x.N, x.M, x.g) for x in single]
    assert [i for i, _ in bench.shard(bench.batch_units(1), 0, 1)] == list(range(64))
