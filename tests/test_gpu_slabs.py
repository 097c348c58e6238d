"""GPU slab decomposition (the paper's domain decomposition along z, Sec. 3.1) through the C ABI:
the halo lists of every sub-domain equal the oracle's entry by entry, the sub-domains classify their
real cells as the whole domain does, and sub-domains stepped with the exchange schedule of
include/lbm.h (here all in one process on one device) reproduce the whole-domain run: FP64 within
1e-12 of the single-domain oracle and bit-identical to the single-domain GPU run, FP32 within 1e-6."""
import numpy as np
import pytest

from paper_2506_21804_gb300 import inputs as I
from tests.helpers import oracle_from, with_features

pytestmark = pytest.mark.gpu
lbm = pytest.importorskip("paper_2506_21804_gb300.lbm")
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    lbm.lib()


def cases(q):
    rb = with_features(I.random_box(7, 6, 10, seed=43, q=q, solid_frac=0.15, tau=0.62, cs=0.12))
    ch = I.channel(nx=6, ny=12, nz=8, q=q, noise=0.3, seed=5, dtype=np.float64)
    cp = I.canopy(nx=40, ny=24, nz=20, q=q, n_buildings=6, seed=2506, domain=(200, 24, 60), crop=(64, 0, 0),
                  dtype=np.float64)
    return [(rb, 3), (rb, 2), (ch, 4), (cp, 3)]


@pytest.mark.parametrize("q", [19, 27])
def test_halo_lists_and_classification_match_oracle(q):
    for w, parts in cases(q):
        kind_g = oracle_from(w).classification()[0]
        nxy = w.nx * w.ny
        for k in range(parts):
            sub, z0, z1, lo, hi = I.slab(w, parts, k)
            o = oracle_from(sub)
            o.set_ghost(lo, hi)
            g = lbm.Lattice.from_workload(sub, storage=lbm.F64, ghost=(lo, hi))
            for side in (0, 1):
                for lst in range(4):
                    assert np.array_equal(g.debug_dump(6 + 4 * side + lst), o.halo_list(side, lst)), (w.name, k, side, lst)
            t = g.debug_dump(0)
            real = slice(lo * nxy, (lo + z1 - z0) * nxy)
            assert np.array_equal(t[real] & 7, kind_g[z0 * nxy:z1 * nxy]), (w.name, k)
            assert not (t[real] & 128).any() and (t[:lo * nxy] & 128).all() and (t[(lo + z1 - z0) * nxy:] & 128).all()
            g.close()


@pytest.mark.parametrize("q", [19, 27])
def test_fp64_slabs_match_oracle_and_whole_domain(q):
    from paper_2506_21804_gb300.shard import LocalSlabs
    steps = 7
    for w, parts in cases(q):
        o = oracle_from(w)
        o.step(steps)
        whole = lbm.Lattice.from_workload(w, storage=lbm.F64)
        whole.step(steps)
        fw = whole.get_populations()
        sl = LocalSlabs(w, parts, storage=lbm.F64)
        sl.step(steps)
        fs = sl.populations()
        fl = np.tile(w.mask != 1, 1)
        assert np.abs(fs[:, fl] - o.populations()[:, fl]).max() < 1e-12, w.name
        assert np.array_equal(fs, fw), (w.name, np.abs(fs - fw).max())
        mo, po = o.reduce()
        ms, ps = sl.reduce()
        assert abs(ms - mo) < 1e-12 * mo and np.abs(ps - po).max() < 1e-12 * mo
        sl.close()
        whole.close()


def test_fp32_canopy_slabs_100_steps():
    from paper_2506_21804_gb300.shard import LocalSlabs
    w = I.canopy(nx=64, ny=48, nz=40, n_buildings=12, seed=2506, domain=(256, 48, 60), crop=(64, 0, 0),
                 dtype=np.float32)
    whole = lbm.Lattice.from_workload(w, storage=lbm.F32)
    whole.step(100)
    rw, uw = whole.moments(np.float64)
    sl = LocalSlabs(w, 4, storage=lbm.F32)
    sl.step(100)
    rs, us = sl.moments(np.float64)
    fl = w.mask != 1
    assert np.abs(rs[fl] - rw[fl]).max() < 1e-6
    assert np.abs(us[:, fl] - uw[:, fl]).max() < 1e-6
    sl.close()
    whole.close()


def test_slab_refusals():
    w = I.channel(nx=8, ny=10, nz=8, seed=1, dtype=np.float32)
    sub, z0, z1, lo, hi = I.slab(w, 2, 0)
    g = lbm.Lattice.from_workload(sub, storage=lbm.F32, ghost=(lo, hi))
    with pytest.raises(lbm.LBMError) as e:
        g.set_collision(lbm.HRR, 0.5)
    assert e.value.code == lbm.ESTATE
    with pytest.raises(lbm.LBMError):
        g.set_ghost_planes(1, 2)
    with pytest.raises(lbm.LBMError):
        g.halo_pack(0, 3, np.zeros(4, np.float32))
