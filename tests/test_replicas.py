"""The multi-process path of bench.py on CPU: two gloo ranks (replicas of the
workload, no data-path exchange) agree on the max-over-ranks time, the summed
work, the barrier, and the reference arm running on rank 0 only."""
import json
import os
import socket
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    r, w, local = bench.dist_setup()
    bench.barrier(w)
    ms = 10.0 * (r + 1)                      # rank-dependent step time
    work = 1000.0 * (r + 1)                  # rank-dependent units
    res = {"rank": r, "world": w, "local": local, "max_ms": bench.max_over_ranks(ms, w),
           "sum_work": bench.sum_over_ranks(work, w)}
    # the reference arm: ranks other than 0 return without work
    if r != 0:
        class A:
            config = "uniform3d-64x128x256"
        res["reference_other_rank"] = bench.run_reference(A(), r, w)
    bench.barrier(w)
    import torch.distributed as dist
    dist.destroy_process_group()
    with open(os.path.join(out_dir, "rank%d.json" % r), "w") as f:
        json.dump(res, f)


def test_two_gloo_replicas(tmp_path):
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, start_method="spawn")
    res = [json.load(open(tmp_path / ("rank%d.json" % r))) for r in range(world)]
    for r, d in enumerate(res):
        assert d["rank"] == r and d["world"] == world and d["local"] == r
        assert d["max_ms"] == 20.0 and d["sum_work"] == 3000.0
    assert res[1]["reference_other_rank"] is None
