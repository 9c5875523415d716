"""Host logic of the multi-process bench line on CPU (gloo, world size 2):
each rank contributes its own time, the line uses the slowest rank's time,
and the whole-job throughput counts every replica's work."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    local = [12.5, 20.0][rank]
    ms = bench.max_over_ranks(local, "cpu")
    out[rank] = (ms, bench.replica_throughput(ws, 1000, 50, ms))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_timing_and_throughput_two_ranks():
    ws, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(ws, port, out), nprocs=ws, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 20.0
    assert res[0][1] == res[1][1] == pytest.approx(2 * 1000 * 50 / 0.020)


def test_single_process_is_local_time():
    import bench
    assert bench.max_over_ranks(7.0, "cpu") == 7.0
