"""Slab decomposition along z (the paper's domain decomposition, Sec. 3.1) over sub-domain lattices.

Each sub-domain is a `lbm.Lattice` of one z-slab with two ghost planes per cut (`inputs.slab`,
`lbm_set_ghost_planes`). This module only moves halo buffers between sub-domains in the order the
C ABI prescribes (include/lbm.h, lbm_halo_*): before a step that starts at an odd step count, the
real-plane slots of every cut go to the neighbour's ghost plane; after it the ghost-plane slots go
back; after every step the wall-model reference velocities that cross a cut. All packing and unpacking
runs in the library's kernels; the buffers are torch tensors on the device.

`LocalSlabs` keeps every sub-domain in this process (one device: the exchange is a device copy);
`RankSlab` holds one sub-domain per torch.distributed rank and exchanges with point-to-point messages.
"""
import numpy as np
import torch

from . import inputs as I
from . import lbm

_STORE = {lbm.F64: torch.float64, lbm.F32: torch.float32, lbm.F16: torch.int16, lbm.BF16: torch.int16}


def _buffers(lat, storage, side, which, device):
    """An empty buffer for halo list `which` of `side` (raw storage values or 3 compute values)."""
    n = lat.halo_count(side, which)
    if which in (0, 1):
        return torch.empty(max(n, 1), dtype=_STORE[storage], device=device)[:n]
    dt = torch.float64 if storage == lbm.F64 else torch.float32
    return torch.empty(max(3 * n, 1), dtype=dt, device=device)[:3 * n]


class _SlabBase:
    """The exchange schedule: before an odd step lists 0 -> 1, after it 1 -> 0, after every step 2 -> 3.

    After an even step the state is stored swapped: the incoming populations of a boundary cell sit in
    its neighbours' slots, for the cells next to a cut in the ghost plane. Reading the state out then
    needs the ghost slots current, i.e. the 0 -> 1 exchange of the coming odd step, done early
    (`_ready`); the step does not repeat it."""

    _fresh = False

    def _ready(self):
        if (self.t & 1) and not self._fresh:
            self._exchange(0, 1)
            self._fresh = True

    def _schedule(self, n):
        for _ in range(n):
            odd = self.t & 1
            self._ready()
            self._step_all()
            self._fresh = False
            if odd:
                self._exchange(1, 0)
            self._exchange(2, 3)
            self.t += 1


class LocalSlabs(_SlabBase):
    """Every slab of workload w in this process, on the current device."""

    def __init__(self, w, parts, storage=lbm.F32):
        self.w, self.parts, self.storage, self.t = w, parts, storage, 0
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.subs = [I.slab(w, parts, k) for k in range(parts)]
        self.lats = []
        stream = torch.cuda.current_stream()
        for sub, z0, z1, lo, hi in self.subs:
            lat = lbm.Lattice.from_workload(sub, storage=storage, ghost=(lo, hi))
            lat.set_stream(stream)
            self.lats.append(lat)
        self.periodic = w.faces[4] == I.FACE_PERIODIC

    def _cuts(self):
        for k in range(self.parts):
            if k + 1 < self.parts:
                yield k, k + 1
            elif self.periodic and self.parts > 1:
                yield k, 0

    def _exchange(self, send, recv):
        for k, kn in self._cuts():
            a, b = self.lats[k], self.lats[kn]   # a below the cut (its side 1), b above (its side 0)
            ba = a.halo_pack(1, send, _buffers(a, self.storage, 1, send, self.device))
            bb = b.halo_pack(0, send, _buffers(b, self.storage, 0, send, self.device))
            b.halo_unpack(0, recv, ba)
            a.halo_unpack(1, recv, bb)

    def _step_all(self):
        for lat in self.lats:
            lat.step(1)

    def step(self, n=1):
        self._schedule(n)

    def sync(self):
        for lat in self.lats:
            lat.sync()

    def populations(self, dtype=np.float64):
        """Populations of the whole domain (q, N) assembled from the real planes of every slab."""
        self._ready()
        nxy = self.w.nx * self.w.ny
        parts = []
        for (sub, z0, z1, lo, hi), lat in zip(self.subs, self.lats):
            parts.append(lat.get_populations(dtype)[:, lo * nxy:(lo + z1 - z0) * nxy])
        return np.concatenate(parts, axis=1)

    def moments(self, dtype=np.float64):
        self._ready()
        nxy = self.w.nx * self.w.ny
        rs, us = [], []
        for (sub, z0, z1, lo, hi), lat in zip(self.subs, self.lats):
            r, u = lat.moments(dtype)
            rs.append(r[lo * nxy:(lo + z1 - z0) * nxy])
            us.append(u[:, lo * nxy:(lo + z1 - z0) * nxy])
        return np.concatenate(rs), np.concatenate(us, axis=1)

    def reduce(self):
        self._ready()
        m, p = 0.0, np.zeros(3)
        for lat in self.lats:
            mi, pi = lat.reduce()
            m += mi
            p += pi
        return m, p

    def close(self):
        for lat in self.lats:
            lat.close()


class RankSlab(_SlabBase):
    """Slab `rank` of `world` slabs of workload w on this rank's device; the neighbours are the ranks
    holding the adjacent slabs (a ring when z is periodic)."""

    def __init__(self, w, rank, world, storage=lbm.F32):
        import torch.distributed as dist
        self.dist = dist
        self.w, self.rank, self.world, self.storage, self.t = w, rank, world, storage, 0
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.sub, self.z0, self.z1, self.lo, self.hi = I.slab(w, world, rank)
        self.lat = lbm.Lattice.from_workload(self.sub, storage=storage, ghost=(self.lo, self.hi))
        self.lat.set_stream(torch.cuda.current_stream())
        periodic = w.faces[4] == I.FACE_PERIODIC
        self.peer = [None, None]
        if self.lo:
            self.peer[0] = (rank - 1) % world
        if self.hi:
            self.peer[1] = (rank + 1) % world
        if not periodic:
            self.peer[0] = rank - 1 if rank > 0 else None
            self.peer[1] = rank + 1 if rank < world - 1 else None

    def _exchange(self, send, recv):
        # Messages between one pair of ranks pair up in posting order: sends go out side 0 then side 1,
        # receives are posted side 1 then side 0, so that with two ranks on a periodic axis (both cuts
        # lead to the same peer) the message crossing a cut meets the receive of that cut.
        sends, recvs, inbox = [], [], []
        for side in (0, 1):
            if self.peer[side] is None:
                continue
            out = self.lat.halo_pack(side, send, _buffers(self.lat, self.storage, side, send, self.device))
            sends.append(self.dist.P2POp(self.dist.isend, out, self.peer[side]))
        for side in (1, 0):
            if self.peer[side] is None:
                continue
            buf = _buffers(self.lat, self.storage, side, recv, self.device)
            recvs.append(self.dist.P2POp(self.dist.irecv, buf, self.peer[side]))
            inbox.append((side, buf))
        ops = sends + recvs
        if ops:
            for r in self.dist.batch_isend_irecv(ops):
                r.wait()
        for side, buf in inbox:
            self.lat.halo_unpack(side, recv, buf)

    def _step_all(self):
        self.lat.step(1)

    def step(self, n=1):
        self._schedule(n)

    def sync(self):
        self.lat.sync()
