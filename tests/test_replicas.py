"""Multi-GPU runs are replicas: every rank computes its own product with no
collective on the data path; the benchmark takes the slowest rank's time and
reports the work of all ranks.  These checks run the host side of that path
as two gloo ranks on the CPU: the rank helpers of bench.py (max over ranks,
barrier) and the planner's determinism across processes (every replica
builds the identical plan for the same shape).
"""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    import bench
    import paper_1902_02104_gb300 as ata
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w, r, local = bench.dist_setup()
    assert (w, r, local) == (world, rank, rank)
    # the slowest replica sets the time
    t = bench.max_over_ranks(torch, 1.0 + rank * 0.25, w)
    bench.barrier(w)
    # every replica plans the same product identically
    info = ata.ata_plan_query(10000, 10000, ata.ATA_F64_OZAKI, 0)
    gemm = ata.ata_gemm_query(10000, 5000, 5000, ata.ATA_F64, 0)
    key = (info["cutoff"], info["mults"], info["n_leaf_products"], info["workspace_bytes"], gemm["cutoff"],
           gemm["mults"])
    keys = [None] * world
    dist.all_gather_object(keys, key)
    with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as f:
        f.write(f"{t} {int(all(k == keys[0] for k in keys))}\n")
    dist.destroy_process_group()


def test_two_gloo_replicas(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    port = _free_port()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, str(tmp_path))) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(2):
        t, same = open(tmp_path / f"rank{r}.txt").read().split()
        assert float(t) == 1.25  # max over ranks of 1.0 and 1.25
        assert same == "1"
