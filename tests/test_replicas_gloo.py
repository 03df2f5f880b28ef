"""Host-side logic of the N-replica bench path, on CPU with gloo (world size 2)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2503_00253_gb300 import replicas
    ws, r, local = replicas.rank_info()
    replicas.barrier()
    elapsed = [120.0, 150.0][rank]          # rank 1 is the slowest
    slowest = replicas.max_over_ranks(elapsed)
    out[rank] = (ws, r, local, slowest, replicas.whole_job_rate(10, ws, slowest))
    dist.destroy_process_group()


def test_two_replicas_report_slowest_rank_and_whole_job_rate():
    world = 2
    port = _free_port()
    manager = mp.get_context("spawn").Manager()
    out = manager.dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
    for rank in range(world):
        ws, r, local, slowest, rate = out[rank]
        assert (ws, r, local) == (world, rank, rank)
        assert slowest == 150.0
        assert rate == pytest.approx(2 * 10 / 0.150)


def test_single_process_needs_no_group():
    from paper_2503_00253_gb300 import replicas
    assert replicas.max_over_ranks(3.5) == 3.5
    assert replicas.whole_job_rate(4, 1, 2000.0) == pytest.approx(2.0)
    with pytest.raises(ValueError):
        replicas.whole_job_rate(1, 1, 0.0)
