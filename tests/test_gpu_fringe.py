"""GPU parity of the outlet fringe zone (Sec. 3.2 reading: the last L planes relax the
post-collision populations towards f^eq(rho_out, u)) against the oracle, through the C ABI: FP64 to
roundoff on the small cases with every feature (including the wall model, inlet/outlet planes,
slip faces and the HRR collision), FP32 on the canopy crop for 100 steps, the interior kernel the
library then runs, and the refusals."""
import numpy as np
import pytest

from paper_2506_21804_gb300 import inputs as I
from tests.helpers import oracle_from, rel_l2, small_cases, with_features

pytestmark = pytest.mark.gpu
lbm = pytest.importorskip("paper_2506_21804_gb300.lbm")
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    lbm.lib()


@pytest.mark.parametrize("q", [19, 27])
@pytest.mark.parametrize("model", [0, 1])
def test_fringe_fp64_parity(q, model):
    for w in small_cases(q):
        w = with_features(w)
        w.fringe = (min(4, w.nx - 1), 0.25, 2.0)
        if model == 1:
            w.model, w.sigma = 1, 0.5
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
        assert np.abs(rg - ro).max() < 1e-12 and np.abs(ug - uo).max() < 1e-12, w.name
        g.close()


def test_fringe_fp32_canopy_crop_100_steps():
    w = I.canopy(nx=128, ny=64, nz=64, seed=2506, crop=(64, 0, 0), domain=(1024, 512, 256), dtype=np.float64)
    w.fringe = (16, 0.1, 2.0)
    o = oracle_from(w, cast32=True)
    g = lbm.Lattice.from_workload(w, storage=lbm.F32)
    assert g.interior_kernel() == 0
    o.step(100)
    g.step(100)
    ro, uo = o.moments()
    rg, ug = g.moments()
    fl = w.mask != 1
    assert np.abs(rg[fl] - ro[fl]).max() < 1e-5
    assert rel_l2(ug[:, fl], uo[:, fl]) < 1e-5


def test_fringe_switches_off_the_pair_kernel_and_refuses_the_adjoint():
    w = I.channel(nx=32, ny=18, nz=8, seed=3, dtype=np.float32)
    g = lbm.Lattice.from_workload(w, storage=lbm.F32)
    assert g.interior_kernel() == 1
    g.set_fringe(8, 0.2)
    assert g.interior_kernel() == 0
    g.set_fringe(0, 0.0)
    assert g.interior_kernel() == 1
    for bad in ((33, 0.1, 2.0), (4, 1.5, 2.0), (4, 0.1, -1.0)):
        with pytest.raises(lbm.LBMError):
            g.set_fringe(*bad)
    d = I.duct(n=8, u_in=0.03, tau=0.7, sigma=1.5, dtype=np.float32)
    h = lbm.Lattice.from_workload(d, storage=lbm.F32)
    h.set_fringe(3, 0.1)
    with pytest.raises(lbm.LBMError) as e:
        h.objective_forward(4, 2, 1, d.nx - 2, ckpt=2)
    assert e.value.code == lbm.ESTATE
