"""Parity of the hybrid recursive regularised (HRR) collision of the CUDA path with the FP64 oracle:
FP64 storage to roundoff on small cases with every boundary kind (sigma = 1, 1/2, 0), the channel
and canopy crops with the wall model, FP32 storage after 100 steps, 16-bit storage on the
Taylor-Green vortex, checkpoint restart, and the calls that must refuse the HRR form."""
import numpy as np
import pytest

from paper_2506_21804_gb300 import inputs as I
from tests.helpers import oracle_from, rel_l2, small_cases, with_features

pytestmark = pytest.mark.gpu

lbm = pytest.importorskip("paper_2506_21804_gb300.lbm")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    lbm.lib()


def _hrr(w, sigma):
    w.model, w.sigma = 1, sigma
    return w


@pytest.mark.parametrize("q", [19, 27])
@pytest.mark.parametrize("sigma", [1.0, 0.5, 0.0])
def test_hrr_fp64_step_parity(q, sigma):
    for w in small_cases(q):
        w = _hrr(with_features(w), sigma)
        o = oracle_from(w)
        g = lbm.Lattice.from_workload(w, storage=lbm.F64)
        for steps in (1, 1, 5):
            o.step(steps)
            g.step(steps)
            fo = o.populations()
            fg = g.get_populations()
            fl = w.mask != 1
            assert np.abs(fg[:, fl] - fo[:, fl]).max() < 1e-12, (w.name, steps)
        ro, uo = o.moments()
        rg, ug = g.moments()
        assert np.abs(rg - ro).max() < 1e-12, w.name
        assert np.abs(ug - uo).max() < 1e-12, w.name


@pytest.mark.parametrize("sigma", [1.0, 0.3])
def test_hrr_fp32_parity_100_steps(sigma):
    cases = [I.channel(nx=32, ny=34, nz=16, seed=550, dtype=np.float64),
             I.canopy(nx=128, ny=64, nz=64, seed=2506, crop=(64, 0, 0), domain=(1024, 512, 256), dtype=np.float64),
             with_features(small_cases(27)[1])]
    for w in cases:
        w = _hrr(w, sigma)
        o = oracle_from(w, cast32=True)
        g = lbm.Lattice.from_workload(w, storage=lbm.F32)
        o.step(100)
        g.step(100)
        ro, uo = o.moments()
        rg, ug = g.moments()
        fl = w.mask != 1
        assert np.abs(rg[fl] - ro[fl]).max() / np.abs(ro[fl]).max() < 1e-5, w.name
        assert rel_l2(ug[:, fl], uo[:, fl]) < 1e-5, w.name


def test_hrr_fp32_taylor_green_32cube():
    w = _hrr(I.taylor_green(n=32, u0=0.05, tau=0.6), 0.5)
    o = oracle_from(w, cast32=True)
    g = lbm.Lattice.from_workload(w, storage=lbm.F32)
    o.step(200)
    g.step(200)
    _, uo = o.moments()
    _, ug = g.moments()
    assert rel_l2(ug, uo) < 1e-5
    shape = w.u0 / 0.05
    A = (ug * shape).sum() / (shape * shape).sum()
    exact = 0.05 * np.exp(-2 * w.meta["nu"] * w.meta["k"] ** 2 * 200)
    assert abs(A / exact - 1) < 0.01


@pytest.mark.parametrize("storage,bound", [(lbm.F16, 1e-3), (lbm.BF16, 2e-2)])
def test_hrr_16bit_taylor_green_error(storage, bound):
    w = _hrr(I.taylor_green(n=32, u0=0.05, tau=0.6), 1.0)
    g = lbm.Lattice.from_workload(w, storage=storage)
    o = oracle_from(w)
    g.step(200)
    o.step(200)
    _, ug = g.moments()
    _, uo = o.moments()
    assert rel_l2(ug, uo) < bound


def test_hrr_save_load_resume_is_bit_identical():
    w = _hrr(with_features(small_cases()[4]), 0.5)
    g = lbm.Lattice.from_workload(w, storage=lbm.F32)
    g.step(5)
    buf = g.save()
    g.step(8)
    a = g.get_populations(np.float32)
    g.load(buf)
    g.step(8)
    b = g.get_populations(np.float32)
    assert np.array_equal(a, b)
    # a BGK context does not accept an HRR checkpoint
    g.set_collision(lbm.BGK)
    with pytest.raises(lbm.LBMError):
        g.load(buf)


def test_hrr_refusals_and_switching():
    w = I.duct(n=10, u_in=0.03, tau=0.7, sigma=2.0, cs=0.1, dtype=np.float64)
    g = lbm.Lattice.from_workload(w, storage=lbm.F64)
    for bad in ((2, 1.0), (1, -0.1), (1, 1.5)):
        with pytest.raises(lbm.LBMError):
            g.set_collision(*bad)
    g.set_collision(lbm.HRR, 0.5)
    with pytest.raises(lbm.LBMError):
        g.objective_forward(4, 2, 1, w.nx - 2, ckpt=2)
    # switching back to BGK reproduces the BGK oracle
    g.set_collision(lbm.BGK)
    o = oracle_from(w)
    g.init_equilibrium(np.asarray(w.rho0), np.asarray(w.u0))
    g.step(3)
    o.step(3)
    assert np.abs(g.get_populations() - o.populations()).max() < 1e-12
