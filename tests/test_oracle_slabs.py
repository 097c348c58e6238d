"""The z-slab decomposition of the paper's domain decomposition (Sec. 3.1), on the CPU oracle: the
domain split into slabs with two ghost planes per cut, each step collide -> halo exchange -> stream,
reproduces the single-domain oracle exactly (bit for bit in FP64: the same operations run on the same
values), with the wall model's reference velocities crossing the cuts. The halo lists of the two sides
of every cut agree entry by entry, and the sub-domains classify their own cells exactly as the single
domain does."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2506_21804_gb300 import inputs as I
from tests.helpers import oracle_from, with_features


def run_slabs(w, parts, steps):
    subs = [I.slab(w, parts, k) for k in range(parts)]
    orcs = []
    for sub, z0, z1, lo, hi in subs:
        o = oracle_from(sub)
        o.set_ghost(lo, hi)
        orcs.append(o)
    periodic = w.faces[4] == I.FACE_PERIODIC
    for _ in range(steps):
        for o in orcs:
            o.step_collide()
        for k in range(parts):
            kn = k + 1
            if kn == parts:
                if not periodic:
                    continue
                kn = 0
            a, b = orcs[k], orcs[kn]            # a below the cut (its side 1), b above (its side 0)
            pa, pb = a.halo_pack(1, 0), b.halo_pack(0, 0)
            ra, rb = a.halo_pack(1, 2), b.halo_pack(0, 2)
            b.halo_unpack(0, 1, pa)
            a.halo_unpack(1, 1, pb)
            b.halo_unpack(0, 3, ra)
            a.halo_unpack(1, 3, rb)
        for o in orcs:
            o.step_stream()
    return subs, orcs


def cases(q):
    rb = with_features(I.random_box(7, 6, 9, seed=41, q=q, solid_frac=0.15, tau=0.62, cs=0.12))
    ch = I.channel(nx=6, ny=12, nz=8, q=q, noise=0.3, seed=5, dtype=np.float64)
    cp = I.canopy(nx=40, ny=24, nz=20, q=q, n_buildings=6, seed=2506, domain=(200, 24, 60), crop=(64, 0, 0),
                  dtype=np.float64)
    return [(rb, 3), (rb, 4), (ch, 2), (ch, 4), (cp, 2), (cp, 3), (cp, 5)]


@pytest.mark.parametrize("q", [19, 27])
def test_slabs_reproduce_single_domain(q):
    steps = 7
    for w, parts in cases(q):
        g = oracle_from(w)
        g.step(steps)
        fg = g.populations()
        subs, orcs = run_slabs(w, parts, steps)
        nxy = w.nx * w.ny
        for (sub, z0, z1, lo, hi), o in zip(subs, orcs):
            fl = o.populations()
            got = fl[:, lo * nxy:(lo + z1 - z0) * nxy]
            want = fg[:, z0 * nxy:z1 * nxy]
            assert np.array_equal(got, want), (w.name, parts, z0, np.abs(got - want).max())


@pytest.mark.parametrize("q", [19, 27])
def test_slab_halo_lists_agree_and_classification_is_global(q):
    for w, parts in cases(q):
        g = oracle_from(w)
        kind, isref, nsum, ref = g.classification()
        subs, orcs = run_slabs(w, parts, 0)
        nxy = w.nx * w.ny
        periodic = w.faces[4] == I.FACE_PERIODIC
        for k, ((sub, z0, z1, lo, hi), o) in enumerate(zip(subs, orcs)):
            lk, li, _, _ = o.classification()
            sl = slice(lo * nxy, (lo + z1 - z0) * nxy)
            assert np.array_equal(lk[sl], kind[z0 * nxy:z1 * nxy]), (w.name, k)
            assert np.array_equal(li[sl], isref[z0 * nxy:z1 * nxy]), (w.name, k)
            kn = k + 1
            if kn == parts and not periodic:
                continue
            b = orcs[kn % parts]
            for send, recv in ((0, 1), (2, 3)):
                assert np.array_equal(o.halo_list(1, send), b.halo_list(0, recv)), (w.name, k, send)
                assert np.array_equal(b.halo_list(0, send), o.halo_list(1, recv)), (w.name, k, send)
        # populations cross each cut in the 5 (D3Q19) or 9 (D3Q27) directions with c_z across it
        o = orcs[0]
        lst = o.halo_list(1, 0)
        if len(lst):
            dirs = np.unique(lst // nxy)
            assert len(dirs) == (5 if q == 19 else 9)
