"""Parity of the vortex-method inlet (Sec. 2.2.2) of the CUDA path with the FP64 oracle: FP64 storage
to roundoff over several steps (the inlet field changes every step and feeds the regularised inlet),
FP32 storage on the canopy crop, reproducibility from the seed, checkpoint restart, refusals."""
import numpy as np
import pytest

from paper_2506_21804_gb300 import inputs as I
from tests.helpers import oracle_from, rel_l2

pytestmark = pytest.mark.gpu

lbm = pytest.importorskip("paper_2506_21804_gb300.lbm")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    lbm.lib()


def _box(q, seed=2):
    w = I.random_box(12, 18, 14, seed=seed, q=q, solid_frac=0.05, tau=0.6, cs=0.1, faces=(3, 3, 2, 2, 1, 2),
                     inflow=True, outflow=True)
    w.vortex = (40, 2.5, 0.2, 1804)
    return w


@pytest.mark.parametrize("q", [19, 27])
def test_vortex_inlet_fp64_parity(q):
    w = _box(q)
    o = oracle_from(w)
    g = lbm.Lattice.from_workload(w, storage=lbm.F64)
    for steps in (1, 1, 5):
        o.step(steps)
        g.step(steps)
        fo, fg = o.populations(), g.get_populations()
        fl = w.mask != 1
        assert np.abs(fg[:, fl] - fo[:, fl]).max() < 1e-12, steps
    ro, uo = o.moments()
    rg, ug = g.moments()
    assert np.abs(ug - uo).max() < 1e-12
    # the inlet field of the last step differs from the mean profile
    fo_in = o.inflow_field()
    assert np.abs(fo_in - w.uin).max() > 1e-4


def test_vortex_inlet_with_hrr_fp64_parity():
    w = _box(19, seed=3)
    w.model, w.sigma = 1, 0.5
    o = oracle_from(w)
    g = lbm.Lattice.from_workload(w, storage=lbm.F64)
    o.step(6)
    g.step(6)
    fl = w.mask != 1
    assert np.abs(g.get_populations()[:, fl] - o.populations()[:, fl]).max() < 1e-12


def test_vortex_inlet_fp32_canopy_crop():
    """FP32 against the FP64 oracle on a canopy crop. The streamwise term takes its direction from
    the gradient of the previous step's perturbed inlet field, which makes the inlet map sensitive
    (a 1e-8 difference grows about 1e6-fold in 50 steps): pointwise parity over 5 steps; after 50
    steps the in-plane components at the inlet (set by the vortices alone) pointwise and the
    streamwise fluctuation by its r.m.s."""
    w = I.canopy(nx=96, ny=48, nz=40, seed=2506, crop=(64, 0, 0), domain=(1024, 512, 256), dtype=np.float64)
    w.vortex = (120, 3.0, 0.15, 7)
    o = oracle_from(w, cast32=True)
    g = lbm.Lattice.from_workload(w, storage=lbm.F32)
    o.step(5)
    g.step(5)
    ro, uo = o.moments()
    rg, ug = g.moments()
    fl = w.mask != 1
    assert np.abs(rg[fl] - ro[fl]).max() < 1e-5
    assert rel_l2(ug[:, fl], uo[:, fl]) < 1e-5
    o.step(45)
    g.step(45)
    inl = w.mask == 3
    _, uo = o.moments()
    _, ug = g.moments()
    assert np.abs(ug[1:, inl] - uo[1:, inl]).max() < 1e-5
    mean = np.asarray(w.uin)[0]
    yz = np.nonzero(inl)[0] // w.nx
    ro_x = np.sqrt(np.mean((uo[0, inl] - mean[yz]) ** 2))
    rg_x = np.sqrt(np.mean((ug[0, inl] - mean[yz]) ** 2))
    assert ro_x > 1e-4 and abs(rg_x / ro_x - 1) < 0.1


def test_vortex_inlet_reproducible_and_restartable():
    w = _box(19, seed=4)
    a = lbm.Lattice.from_workload(w, storage=lbm.F32)
    b = lbm.Lattice.from_workload(w, storage=lbm.F32)
    a.step(4)
    buf = a.save()
    a.step(6)
    b.step(10)
    fa = a.get_populations(np.float32)
    assert np.array_equal(fa, b.get_populations(np.float32))
    b.load(buf)
    b.step(6)
    assert np.array_equal(fa, b.get_populations(np.float32))
    # another seed gives another inlet
    w2 = _box(19, seed=4)
    w2.vortex = (40, 2.5, 0.2, 1805)
    c = lbm.Lattice.from_workload(w2, storage=lbm.F32)
    c.step(10)
    assert not np.array_equal(fa, c.get_populations(np.float32))


def test_vortex_inlet_refusals():
    w = I.duct(n=10, u_in=0.03, tau=0.7, sigma=2.0, cs=0.1, dtype=np.float64)
    g = lbm.Lattice.from_workload(w, storage=lbm.F64)
    for bad in ((-1, 2.0, 0.1, 0), (10, 0.0, 0.1, 0), (10, 2.0, -0.1, 0)):
        with pytest.raises(lbm.LBMError):
            g.set_vortex_inlet(*bad)
    g.set_vortex_inlet(10, 2.0, 0.1, 3)
    with pytest.raises(lbm.LBMError):
        g.objective_forward(4, 2, 1, w.nx - 2, ckpt=2)
    g.set_vortex_inlet(0)
    g.objective_forward(4, 2, 1, w.nx - 2, ckpt=2)


# ---- porous-medium inputs (Sec. 2.1, Eq. lattice_porosity) -------------------------------------------------
def test_permeability_field_matches_oracle_fp64():
    w = I.duct(n=12, u_in=0.03, tau=0.7, sigma=2.0, cs=0.1, dtype=np.float64)
    nu_tau = (w.tau - 0.5) / 3 * w.tau
    rng = np.random.default_rng(5)
    K = nu_tau / (1e-3 + rng.random(w.N))       # gamma spans [0, 1) with clamping below nu tau
    K[rng.random(w.N) < 0.3] = np.inf
    K[:3] = (-1.0, 0.0, np.nan)                 # no valid permeability: impermeable on both sides
    w.gamma = None
    o = oracle_from(w)
    o.set_permeability(K)
    g = lbm.Lattice.from_workload(w, storage=lbm.F64)
    g.set_permeability(K)
    o.step(5)
    g.step(5)
    fl = w.mask != 1
    assert np.abs(g.get_populations()[:, fl] - o.populations()[:, fl]).max() < 1e-12


def test_forchheimer_permeability_matches_oracle():
    from oracle import oracle as O
    for args in ((1.8e-5, 2e-3, 0.5, 0.3, 4.0, 1.2, float("inf")), (1.8e-5, 2e-3, 0.5, 0.3, 4.0, 1.2, 3e-4)):
        assert abs(lbm.forchheimer_permeability(*args) / O.forchheimer_k(*args) - 1) < 1e-15
    assert np.isnan(lbm.forchheimer_permeability(1.8e-5, 2e-3, 0.5, 0.3, 1e-9, 1.2, 3e-4))
