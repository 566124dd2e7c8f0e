"""The replica path of bench.py on CPU: two gloo ranks combine their timings (max) and work
(sum) the way the GPU ranks do; the reference arm does its work on rank 0 only."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r = bench.combine_ranks(1.0 + rank, 10.0 * (2 - rank), 100.0 * (rank + 1), torch.device("cpu"))
        out[rank] = r
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_combine_ranks_gloo_world_2():
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(2, _free_port(), out), nprocs=2, join=True)
        res = dict(out)
    for rank in (0, 1):
        assert res[rank] == (2.0, 20.0, 300.0)


def test_combine_ranks_single_process_is_identity():
    import torch
    import bench
    assert bench.combine_ranks(1.5, 2.5, 3.5, torch.device("cpu")) == (1.5, 2.5, 3.5)


def test_reference_arm_non_zero_rank_does_nothing(capsys):
    import bench
    args = bench.argparse.Namespace(operator="elasticity", workload="prefractured", steps=1,
                                    warmup=0)
    assert bench.run_reference(args, rank=1, world=2) is None
    assert capsys.readouterr().out == ""
