"""bench.py's multi-GPU host logic on two gloo ranks (CPU): every rank owns a
disjoint range of one global argument stream, the timed region is the
slowest rank's, the reported value is the whole job's, and the reference arm
runs on rank 0 only.  The GPU kernels themselves are not needed for this."""
import json
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, outdir):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    n = 4096
    x = bench.rank_arguments(n, rank)
    np.save(os.path.join(outdir, f"x{rank}.npy"), x)
    my_ms = 10.0 + 2.5 * rank          # the ranks' own timed regions
    total = bench.max_over_ranks(my_ms, dist, torch.device("cpu"))
    value = bench.job_value(world, n, 32, 7, total)
    # the reference arm: rank 1 returns at once and prints nothing
    ref_rc = bench.run_reference(type("A", (), {})()) if rank != 0 else None
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(outdir, f"r{rank}.json"), "w") as f:
        json.dump({"total": total, "value": value, "ref_rc": ref_rc}, f)


def test_two_ranks_gloo(tmp_path):
    world, n = 2, 4096
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       start_method="spawn", join=True)
    from paper_2512_10059_gb300 import workloads as W
    x0, x1 = (np.load(tmp_path / f"x{r}.npy") for r in range(world))
    assert np.array_equal(np.concatenate([x0, x1]), W.mixture_c2(world * n, seed=1))
    assert np.array_equal(x0, W.mixture_c2(n, seed=1))        # rank 0 = the single-GPU workload
    res = [json.loads((tmp_path / f"r{r}.json").read_text()) for r in range(world)]
    assert res[0]["total"] == res[1]["total"] == 12.5            # the slowest rank's time
    assert res[0]["value"] == pytest.approx(world * n * 33 * 7 / 12.5e-3)
    assert res[1]["ref_rc"] == 0
