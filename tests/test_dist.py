"""The multi-GPU path of bench.py is replicas only (one independent problem
per rank, no data-path collective): its rank plumbing -- process-group set-up,
the barrier around the timed region and the max over ranks of the time --
runs here as two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(ws), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import bench
    w, r, local = bench.dist_setup()
    assert (w, r, local) == (ws, rank, rank)
    bench.barrier(w)
    ms = 10.0 + 5.0 * rank          # a rank's timed region
    out[rank] = bench.max_over_ranks(w, ms)
    bench.barrier(w)
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    ws, port = 2, _free_port()
    out = mp.Manager().dict()
    mp.start_processes(_rank, args=(ws, port, out), nprocs=ws, start_method="spawn", join=True)
    # every rank reports the slowest rank's time; the bench divides all ranks' steps by it
    assert dict(out) == {0: 15.0, 1: 15.0}
