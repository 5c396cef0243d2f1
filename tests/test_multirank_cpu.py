"""The multi-rank bench path on CPU (gloo, world size 2, no GPU): every rank times its own
replica, the job time is the maximum over ranks, and the whole-job value counts the work of
all ranks; the reference arm runs on rank 0 only.  The batched workload shards: every rank
computes the same partition of the 4096 blocks (tri_batched_partition, host only) and keeps
its own share; together the shares cover every block exactly once, with balanced loads."""
import json
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = 10.0 + 5.0 * rank                  # rank 1 is the slow one
    got = bench.max_over_ranks(torch, dist, local_ms, world, "cpu")
    value = bench.aggregate_value(world, 1.0e12, 4, got)
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump({"max_ms": got, "value": value}, f)


def test_max_over_ranks_and_whole_job_value(tmp_path):
    import torch.multiprocessing as mp
    world, port = 2, _free_port()
    mp.start_processes(_worker, args=(world, port, str(tmp_path)), nprocs=world, join=True, start_method="spawn")
    res = [json.load(open(tmp_path / f"r{r}.json")) for r in range(world)]
    for r in res:
        assert r["max_ms"] == 15.0                # the slowest rank's timed region
        # 2 ranks x 1e12 flops x 4 steps in 15 ms
        assert r["value"] == pytest.approx(2 * 1.0e12 * 4 / 15e-3 / 1e12)


def test_single_rank_value():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(torch, None, 7.5, 1, "cpu") == 7.5
    assert bench.aggregate_value(1, 2.0e12, 3, 6.0) == pytest.approx(1.0e3)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import argparse
    import bench
    args = argparse.Namespace(n=64, steps=1, warmup=0, gpus=2)
    monkeypatch.setenv("RANK", "1")
    assert bench.run_reference(args) == 0
    assert capsys.readouterr().out == ""          # no work and no line on other ranks
    monkeypatch.setenv("RANK", "0")
    assert bench.run_reference(args) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"


def _partition_worker(rank, world, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import numpy as np
    from paper_2307_07611_gb300 import inputs, lib
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sizes = inputs.batched_sizes(4096, seed=0)
    mine = bench.owned_blocks(lib, sizes, rank, world)
    gathered = [None] * world
    dist.all_gather_object(gathered, {"rank": rank, "blocks": mine,
                                      "load": float(sum(float(sizes[i]) ** 3 for i in mine))})
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"p{rank}.json"), "w") as f:
        json.dump(gathered, f)


@pytest.mark.parametrize("world", [2, 3])
def test_batched_partition_over_ranks(tmp_path, world):
    import numpy as np
    import torch.multiprocessing as mp
    sys.path.insert(0, ROOT)
    from paper_2307_07611_gb300 import build as cuda_build
    from paper_2307_07611_gb300 import inputs
    cuda_build.build()
    port = _free_port()
    mp.start_processes(_partition_worker, args=(world, port, str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    views = [json.load(open(tmp_path / f"p{r}.json")) for r in range(world)]
    assert all(v == views[0] for v in views)          # every rank saw the same shares
    shares = views[0]
    blocks = sorted(b for sh in shares for b in sh["blocks"])
    assert blocks == list(range(4096))                # every block exactly once
    loads = np.array([sh["load"] for sh in shares])
    assert loads.max() <= 1.05 * loads.mean()         # rank loads within 5 %
    sizes = inputs.batched_sizes(4096, seed=0)
    assert loads.sum() == pytest.approx(float(np.sum(np.asarray(sizes, dtype=np.float64) ** 3)))

