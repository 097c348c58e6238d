"""The N > 1 host logic of the benchmark (replicas only: every rank runs its own workload, no data
collective) on two CPU processes with the gloo backend: the max-over-ranks timing, the barrier, the
per-rank seeds, and the reference arm running on rank 0 only."""
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


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_2506_21804_gb300 import inputs as I
    r, local, w = bench.dist_info()
    bench.barrier(w)
    t = bench.max_over_ranks(1.0 + rank, w)          # per-rank "times" 1.0, 2.0
    # replicas: each rank's channel differs (seed 550 + rank), per-rank work is fixed (weak scaling)
    ch = I.channel(nx=8, ny=10, nz=4, seed=550 + r)
    # the reference arm prints on rank 0 only; other ranks return without work
    class A:
        steps, warmup, gpus = 1, 1, w
    import io, contextlib
    buf = io.StringIO()
    if r != 0:
        with contextlib.redirect_stdout(buf):
            bench.run_reference(A)
    out[rank] = (r, local, w, t, float(abs(ch.u0).sum()), buf.getvalue())
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_replica_logic():
    world, port = 2, _free_port()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.start_processes(_worker, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
        res = dict(out)
    assert sorted(res) == [0, 1]
    for rank in (0, 1):
        r, local, w, t, u0sum, printed = res[rank]
        assert (r, local, w) == (rank, rank, 2)
        assert t == 2.0                                 # max over ranks
    assert res[0][4] != res[1][4]                       # different seeds per replica
    assert res[1][5] == ""                              # rank 1 of the reference arm does nothing
