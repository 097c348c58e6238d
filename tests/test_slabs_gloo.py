"""The slab decomposition across processes: two CPU ranks (gloo backend), each holding one z-slab of
a periodic box with every feature (wall model, porosity, body force, Smagorinsky) on an oracle
sub-domain, exchange their halo buffers with torch.distributed point-to-point messages every step
(post-collision populations leaving through each cut, reference velocities of the wall model), and
after the run rank 0 gathers the slabs: they equal the single-domain oracle bit for bit. With two
ranks and a periodic z axis both cuts of a rank lead to the other rank; the message tag names the
cut."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _workload(q):
    from paper_2506_21804_gb300 import inputs as I
    from tests.helpers import with_features
    return with_features(I.random_box(7, 6, 10, seed=43, q=q, solid_frac=0.15, tau=0.62, cs=0.12))


def _exchange(o, rank, world, side_lists):
    """One halo exchange: for both sides, send this rank's packed list and receive the neighbour's."""
    reqs, recv = [], []
    for side in (0, 1):
        peer = (rank - 1) % world if side == 0 else (rank + 1) % world
        send_list, recv_list = side_lists
        out = torch.from_numpy(np.ascontiguousarray(o.halo_pack(side, send_list)))
        n = len(o.halo_list(side, recv_list)) * (1 if recv_list == 1 else 3)
        buf = torch.zeros(n, dtype=torch.float64)
        # the message crossing the cut below a rank carries tag 0 going down, 1 going up
        reqs.append(dist.isend(out, peer, tag=10 * send_list + side))
        reqs.append(dist.irecv(buf, peer, tag=10 * send_list + (1 - side)))
        recv.append((side, recv_list, buf))
    for r in reqs:
        r.wait()
    for side, recv_list, buf in recv:
        o.halo_unpack(side, recv_list, buf.numpy())


def _worker(rank, world, port, q, steps, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2506_21804_gb300 import inputs as I
    from tests.helpers import oracle_from
    w = _workload(q)
    sub, z0, z1, lo, hi = I.slab(w, world, rank)
    o = oracle_from(sub)
    o.set_ghost(lo, hi)
    for _ in range(steps):
        o.step_collide()
        _exchange(o, rank, world, (0, 1))   # populations
        _exchange(o, rank, world, (2, 3))   # reference velocities
        o.step_stream()
    nxy = w.nx * w.ny
    mine = torch.from_numpy(np.ascontiguousarray(o.populations()[:, lo * nxy:(lo + z1 - z0) * nxy]))
    if rank == 0:
        parts = [mine]
        for r in range(1, world):
            _, a0, a1, _, _ = I.slab(w, world, r)
            buf = torch.zeros((w.q, (a1 - a0) * nxy), dtype=torch.float64)
            dist.recv(buf, r, tag=99)
            parts.append(buf)
        out[0] = np.concatenate([p.numpy() for p in parts], axis=1)
    else:
        dist.send(mine, 0, tag=99)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("q", [19, 27])
def test_two_rank_slabs_reproduce_single_domain(q):
    from tests.helpers import oracle_from
    world, port, steps = 2, _free_port(), 6
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.start_processes(_worker, args=(world, port, q, steps, out), nprocs=world, join=True,
                           start_method="spawn")
        got = out[0]
    g = oracle_from(_workload(q))
    g.step(steps)
    assert np.array_equal(got, g.populations())
