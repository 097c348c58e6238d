"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Integer work (classification, boundary list, wall normals, reference cells, propagation map) is
compared bit-exactly; FP64 storage within 1e-12 on populations; FP32 storage within 1e-5 relative on
rho and u after 100 steps; 16-bit storage against the FP64 oracle with its stated error; the adjoint
against the oracle's transpose; full-size workloads on sampled cells recomputed by the oracle on
crops around them.
"""
import numpy as np
import pytest

from oracle import oracle as O
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


def gpu_from(w, storage):
    return lbm.Lattice.from_workload(w, storage=storage)


# ---- integer work: bit-exact ------------------------------------------------------------------------------
@pytest.mark.parametrize("q", [19, 27])
def test_classification_lists_and_source_map_bit_exact(q):
    for w in small_cases(q):
        o = oracle_from(w)
        g = gpu_from(w, lbm.F32)
        kind, isref, nsum, ref = o.classification()
        t = g.debug_dump(0)
        assert np.array_equal(t & 7, kind), w.name
        assert np.array_equal((t & 8) != 0, isref == 1), w.name
        on = (kind == 2) | (kind == 3) | (kind == 4) | (isref == 1)
        assert np.array_equal((t & 32) != 0, on), w.name
        cells, refpos = o.boundary_list()
        assert np.array_equal(g.debug_dump(1), cells), w.name
        assert np.array_equal(g.debug_dump(2), refpos), w.name
        assert np.array_equal(g.debug_dump(3).reshape(-1, 3), nsum[cells]), w.name
        sd, sc = o.source_map()
        assert np.array_equal(g.debug_dump(4).reshape(q, -1), sd), w.name
        assert np.array_equal(g.debug_dump(5).reshape(q, -1), sc), w.name
        info = g.info()
        assert info["n_list"] == len(cells) and info["n_wall"] == int((kind == 2).sum())


# ---- FP64 storage: parity to roundoff ------------------------------------------------------------------------
@pytest.mark.parametrize("q", [19, 27])
@pytest.mark.parametrize("steps", [1, 2, 7])
def test_fp64_step_parity(q, steps):
    for w in small_cases(q):
        w = with_features(w)
        o = oracle_from(w)
        g = gpu_from(w, lbm.F64)
        o.step(steps)
        g.step(steps)
        fo = o.populations()
        fg = g.get_populations()
        fl = w.mask != 1
        assert np.abs(fg[:, fl] - fo[:, fl]).max() < 1e-12, w.name
        ro, uo = o.moments()
        rg, ug = g.moments()
        assert np.abs(rg - ro).max() < 1e-12, w.name
        assert np.abs(ug - uo).max() < 1e-12, w.name
        mo, po = o.reduce()
        mg, pg = g.reduce()
        assert abs(mg - mo) < 1e-13 * mo and np.abs(pg - po).max() < 1e-13 * mo


def test_fp64_taylor_green_32cube_200_steps():
    """Config: D3Q19 BGK FP64, 32^3 periodic TGV (u0 = 0.05, tau = 0.6), 200 steps: parity with the
    oracle, the analytic amplitude decay exp(-2 nu k^2 t) within 1 %, and exact mass conservation."""
    w = I.taylor_green(n=32, u0=0.05, tau=0.6)
    g = gpu_from(w, lbm.F64)
    o = oracle_from(w)
    m0, _ = g.reduce()
    g.step(200)
    o.step(200)
    rg, ug = g.moments()
    ro, uo = o.moments()
    assert np.abs(rg - ro).max() < 1e-12
    assert np.abs(ug - uo).max() < 1e-12
    shape = w.u0 / 0.05
    A = (ug * shape).sum() / (shape * shape).sum()
    exact = 0.05 * np.exp(-2 * w.meta["nu"] * w.meta["k"] ** 2 * 200)
    assert abs(A / exact - 1) < 0.01
    m1, _ = g.reduce()
    assert abs(m1 - m0) / m0 < 1e-13


# ---- FP32 storage -------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("q", [19, 27])
def test_fp32_parity_100_steps(q):
    for w in small_cases(q):
        w = with_features(w)
        o = oracle_from(w, cast32=True)
        g = gpu_from(w, lbm.F32)
        o.step(100)
        g.step(100)
        ro, uo = o.moments()
        rg, ug = g.moments()
        fl = w.mask != 1
        assert np.abs(rg[fl] - ro[fl]).max() / np.abs(ro[fl]).max() < 1e-5, w.name
        assert rel_l2(ug[:, fl], uo[:, fl]) < 1e-5, w.name


def test_fp32_channel_and_canopy_crops_100_steps():
    """Channel (wall function, force, Smagorinsky) and an urban-canopy crop 128x64x64 of the seeded
    1024x512x256 geometry, 100 steps, FP32 vs the FP64 oracle."""
    cases = [I.channel(nx=32, ny=34, nz=16, seed=550, dtype=np.float64),
             I.canopy(nx=128, ny=64, nz=64, seed=2506, crop=(64, 0, 0), domain=(1024, 512, 256), dtype=np.float64)]
    for w in cases:
        o = oracle_from(w, cast32=True)
        g = gpu_from(w, lbm.F32)
        o.step(100)
        g.step(100)
        ro, uo = o.moments()
        rg, ug = g.moments()
        fl = w.mask != 1
        assert np.abs(rg[fl] - ro[fl]).max() < 1e-5, w.name
        assert rel_l2(ug[:, fl], uo[:, fl]) < 1e-5, w.name
        assert g.info()["n_wall"] > 0


# ---- 16-bit storage ---------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("storage,mode", [(lbm.F16, 2), (lbm.BF16, 3)])
def test_16bit_canopy_crop_vs_fp64_oracle(storage, mode):
    """The precision form on the 128x64x64 crop x in [64,192), y, z in [0,64) of the seeded
    1024x512x256 urban canopy (wall function, log-law inlet, pressure outlet, slip faces), 100 steps,
    16-bit storage against the FP64 oracle. The bound per result is twice the error that the storage
    rounding alone causes: the oracle run with the same round-to-nearest-even 16-bit stores and FP64
    arithmetic, computed here (on this crop: FP16 u 8.5e-4 relative L2, rho 1.5e-4 max; BF16 6.6e-3,
    1.0e-3)."""
    w = I.canopy(nx=128, ny=64, nz=64, seed=2506, crop=(64, 0, 0), domain=(1024, 512, 256), dtype=np.float64)
    fl = w.mask != 1
    o = oracle_from(w, cast32=True)
    o.step(100)
    ro, uo = o.moments()
    e = oracle_from(w, storage=mode, cast32=True)
    e.step(100)
    re_, ue = e.moments()
    bound_u = 2.0 * rel_l2(ue[:, fl], uo[:, fl])
    bound_r = 2.0 * np.abs(re_[fl] - ro[fl]).max()
    g = gpu_from(w, storage)
    g.step(100)
    rg, ug = g.moments()
    err_u = rel_l2(ug[:, fl], uo[:, fl])
    err_r = np.abs(rg[fl] - ro[fl]).max()
    assert err_u <= bound_u, (err_u, bound_u)
    assert err_r <= bound_r, (err_r, bound_r)
    assert bound_u < (2e-3 if storage == lbm.F16 else 1.5e-2)


@pytest.mark.parametrize("storage,bound", [(lbm.F16, 1e-3), (lbm.BF16, 2e-2)])
def test_16bit_taylor_green_error(storage, bound):
    w = I.taylor_green(n=32, u0=0.05, tau=0.6)
    g = gpu_from(w, storage)
    o = oracle_from(w)
    g.step(200)
    o.step(200)
    _, ug = g.moments()
    _, uo = o.moments()
    assert rel_l2(ug, uo) < bound


@pytest.mark.parametrize("storage,bound", [(lbm.F16, 0.01), (lbm.BF16, 0.05)])
def test_16bit_channel_mean_profile_vs_fp32(storage, bound):
    """Turbulent-channel configuration (wall function, Smagorinsky, body force) on 128x130x32:
    the streamwise mean-velocity profile <u_x>(y) of 16-bit storage against FP32 after 300 steps,
    within 1 % (FP16) and 5 % (BF16) of the profile's maximum."""
    w = I.channel(nx=128, ny=130, nz=32, seed=550, dtype=np.float32)
    prof = []
    for st in (lbm.F32, storage):
        g = gpu_from(w, st)
        g.step(300)
        _, u = g.moments(np.float32)
        prof.append(u[0].reshape(w.nz, w.ny, w.nx).mean(axis=(0, 2)))
    ref, got = prof
    assert np.abs(got - ref).max() < bound * np.abs(ref).max()


@pytest.mark.parametrize("model,sigma", [(0, 1.0), (1, 1.0), (1, 0.5)])
def test_16bit_matches_oracle_storage_emulation_one_step(model, sigma):
    """One step of FP16 storage equals the oracle's FP16-rounded storage to within a few units in
    the last place of the stored deviation: FP32 (GPU) and FP64 (oracle) arithmetic can round the
    initial state and the stored result to neighbouring FP16 values. BGK and the HRR collision (with
    and without the finite-difference strain). Solids in most rows make the library run the
    one-cell-per-thread kernel here; the kernels over several cells are checked by the next test."""
    w = I.random_box(12, 8, 6, seed=9, q=19, solid_frac=0.1, tau=0.7, cs=0.1)
    w.model, w.sigma = model, sigma
    g = gpu_from(w, lbm.F16)
    o = oracle_from(w, storage=2)
    g.step(1)
    o.step(1)
    fg = g.get_populations()
    fo = o.populations()
    fl = w.mask != 1
    c, wts, *_ = O.lattice(19)
    dev = np.abs(fo[:, fl] - wts[:, None])
    assert (np.abs(fg[:, fl] - fo[:, fl]) <= 4 * np.maximum(dev, 6.1e-5) * 2.0 ** -10 + 1e-12).all()


@pytest.mark.parametrize("storage", [lbm.F16, lbm.BF16])
def test_16bit_multi_cell_kernels_match_oracle_storage_emulation(storage):
    """The interior kernels that update several cells per thread against the oracle's 16-bit-rounded
    storage, over even and odd steps, on shapes where the library selects them (no warp mixes cell
    kinds): four cells per thread on even steps (nx a multiple of 4; a solid-free periodic box and a
    wall-modelled channel with whole wall rows) and cell pairs (nx = 14, and every odd step).
    Tolerance: GPU (FP32) and oracle (FP64) arithmetic can round a stored input to neighbouring
    16-bit values, one unit in the last place of that input. The collision mixes every population of
    a cell, so an output can differ by a few such units of the cell's largest deviation, not of its
    own (a small rest-population deviation then differs by many of its own units). The bound is
    K units of the largest stored deviation max_i |f_i - w_i| of the cells a population can come
    from (the cell and its 26 neighbours): K = 4 after one step, 8 after two and three (differences
    of a step feed the next). A wrong neighbour or slot gives errors of the size of the
    deviations themselves, orders of magnitude above it."""
    mant = 10 if storage == lbm.F16 else 7
    cases = [(I.random_box(16, 6, 5, seed=21, q=19, solid_frac=0.0, tau=0.7, cs=0.1), 3),
             (I.channel(nx=16, ny=10, nz=4, seed=550, dtype=np.float64), 3),
             (I.random_box(14, 6, 5, seed=22, q=19, solid_frac=0.0, tau=0.7, cs=0.1), 1)]
    for w, kernel in cases:
        g = gpu_from(w, storage)
        assert g.interior_kernel() == kernel, w.name
        o = oracle_from(w, storage=int(storage))
        _check_16bit_steps(g, o, w, mant)


def _check_16bit_steps(g, o, w, mant, steps=3):
    """Each stored population within K units in the last place of the largest stored deviation
    max_i |f_i - w_i| of the cells it can come from (its own cell and the 26 around it, periodic
    wrap: streaming brings a population from a neighbour's collision); K = 4 after one step, 8 after
    two and three."""
    from scipy.ndimage import maximum_filter
    c, wts, *_ = O.lattice(19)
    fl = w.mask != 1
    for t in range(1, steps + 1):
        g.step(1)
        o.step(1)
        fo_all = o.populations()
        hdev = np.where(fl, np.abs(fo_all - wts[:, None]).max(axis=0), 0.0)  # solid cells send nothing
        hgrid = hdev.reshape(w.nz, w.ny, w.nx)
        hnb = maximum_filter(hgrid, size=3, mode="wrap").reshape(-1)[fl]
        fg = g.get_populations()[:, fl]
        fo = fo_all[:, fl]
        k = 4 if t == 1 else 8
        excess = np.abs(fg - fo) - k * 2.0 ** -mant * hnb[None, :]
        assert excess.max() <= 1e-12, (w.name, t, float(excess.max()))


@pytest.mark.parametrize("nx", [520, 544])
def test_row_form_kernels_several_ctas_per_row(nx):
    """Rows wider than one CTA of the row-form interior kernels, so that a row spans several CTAs and
    the last one is partial (nx = 520: 260 pairs, 130 quads per row; nx = 544 also runs the 16-bit L2
    prefetch ahead of the later CTAs, which needs nx a multiple of 16). FP32 cell pairs against the
    FP64 oracle after 20 steps (1e-5), and the 16-bit kernels (four cells per thread on even steps,
    pairs on odd steps) against the oracle's 16-bit storage emulation over three steps, with the bound
    of the multi-cell test above."""
    w = I.random_box(nx, 3, 4, seed=nx, q=19, solid_frac=0.0, tau=0.7, cs=0.1)
    fl = w.mask != 1
    g = gpu_from(w, lbm.F32)
    assert g.interior_kernel() == 1
    o = oracle_from(w, cast32=True)
    g.step(20)
    o.step(20)
    ro, uo = o.moments()
    rg, ug = g.moments()
    assert np.abs(rg[fl] - ro[fl]).max() < 1e-5
    assert rel_l2(ug[:, fl], uo[:, fl]) < 1e-5
    for storage, mant in ((lbm.F16, 10), (lbm.BF16, 7)):
        g = gpu_from(w, storage)
        assert g.interior_kernel() == 3
        o = oracle_from(w, storage=int(storage))
        _check_16bit_steps(g, o, w, mant)


def test_page_locked_host_fields_match_pageable():
    """Initial fields and moments through page-locked host buffers (read and written by the kernels in
    place) give the same bits as through pageable host arrays (staged through device memory), for
    FP32 and FP64 fields."""
    torch = pytest.importorskip("torch")
    w = I.channel(nx=32, ny=12, nz=8, seed=550, dtype=np.float64)
    for dt, tdt in ((np.float32, torch.float32), (np.float64, torch.float64)):
        a = gpu_from(w, lbm.F32)
        a.init_equilibrium(np.asarray(w.rho0, dt), np.asarray(w.u0, dt))
        a.step(5)
        ra, ua = a.moments(dt)
        b = gpu_from(w, lbm.F32)
        rho_h = torch.from_numpy(np.ascontiguousarray(w.rho0, dt)).pin_memory()
        u_h = torch.from_numpy(np.ascontiguousarray(w.u0, dt)).pin_memory()
        b.init_equilibrium(rho_h, u_h)
        b.step(5)
        rho_o = torch.full((w.N,), float("nan"), dtype=tdt).pin_memory()
        u_o = torch.full((3, w.N), float("nan"), dtype=tdt).pin_memory()
        b.moments(dt, rho_o, u_o)
        assert np.array_equal(rho_o.numpy(), ra)
        assert np.array_equal(u_o.numpy(), ua)


def test_interior_kernel_selection():
    """The library's choice of interior kernel: pairs for the FP32 channel, four cells per thread
    (even steps) for its 16-bit forms, pairs for 16-bit D3Q27 and for the HRR collision, one cell per
    thread on the urban canopy (most x-groups mix cell kinds)."""
    ch = I.channel(nx=32, ny=12, nz=4, seed=550, dtype=np.float32)
    assert gpu_from(ch, lbm.F32).interior_kernel() == 1
    assert gpu_from(ch, lbm.F16).interior_kernel() == 3
    assert gpu_from(ch, lbm.BF16).interior_kernel() == 3
    g = gpu_from(ch, lbm.F16)
    g.set_collision(lbm.HRR, 1.0)
    assert g.interior_kernel() == 1
    ch27 = I.channel(nx=32, ny=12, nz=4, seed=550, q=27, dtype=np.float32)
    assert gpu_from(ch27, lbm.F16).interior_kernel() == 1
    cw = I.canopy(nx=64, ny=48, nz=40, n_buildings=8, seed=2506, domain=(256, 48, 60), crop=(64, 0, 0),
                  dtype=np.float32)
    assert gpu_from(cw, lbm.F16).interior_kernel() == 0


# ---- adjoint -------------------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("storage,tol", [(lbm.F64, 1e-11), (lbm.F32, 2e-4)])
def test_reverse_step_matches_oracle_transpose(storage, tol):
    for w in [I.duct(n=8, u_in=0.03, tau=0.7, sigma=1.5, cs=0.12, dtype=np.float64),
              I.random_box(9, 7, 6, seed=1, q=19, solid_frac=0.15, tau=0.62, cs=0.12),
              I.random_box(10, 7, 5, seed=2, q=19, solid_frac=0.1, tau=0.55, cs=0.1, faces=(3, 3, 2, 2, 1, 2),
                           inflow=True, outflow=True),
              I.duct(n=6, q=27, u_in=0.02, tau=0.8, sigma=1.5, cs=0.0, dtype=np.float64)]:
        if w.gamma is None:
            w.gamma = 0.6 + 0.4 * np.random.default_rng(3).random(w.N)
        o = oracle_from(w, cast32=storage == lbm.F32)
        g = gpu_from(w, storage)
        o.step(2)
        g.step(2)
        lam = np.random.default_rng(5).standard_normal((w.q, w.N))
        lam[:, w.mask == 1] = 0
        gl, gg, gu = g.adjoint_step(lam)
        ol, og, ou = o.vjp_step(lam)
        s = np.abs(ol).max()
        assert np.abs(gl - ol).max() < tol * s, w.name
        assert np.abs(gg - og).max() < tol * max(np.abs(og).max(), 1e-30), w.name
        assert np.abs(gu.reshape(-1) - ou).max() <= tol * max(np.abs(ou).max(), 1e-30), w.name


@pytest.mark.parametrize("ckpt", [4, 1])
def test_objective_gradient_fp64_matches_oracle(ckpt):
    """Checkpoints every 4 steps (segments recomputed) and every state kept (ckpt = 1, no
    recomputation) give the oracle's objective and gradients."""
    w = I.duct(n=12, u_in=0.03, tau=0.7, sigma=2.0, cs=0.1, dtype=np.float64)
    T, W = 26, 6
    o = oracle_from(w)
    Jo = o.objective_run(T, W, 1, w.nx - 2)
    go, uo = o.adjoint()
    g = gpu_from(w, lbm.F64)
    Jg = g.objective_forward(T, W, 1, w.nx - 2, ckpt=ckpt)
    gg, ug = g.objective_backward()
    assert abs(Jg - Jo) < 1e-12 * max(1.0, abs(Jo))
    assert rel_l2(gg, go) < 1e-10
    assert rel_l2(ug, uo) < 1e-10
    # the state after backward is the one after the forward run
    assert g.info()["t"] == T
    ro, _ = o.moments()
    rg, _ = g.moments()
    assert np.abs(rg - ro).max() < 1e-12
    if ckpt == 1:
        with pytest.raises(lbm.LBMError):
            g.objective_forward(25, 5, 1, w.nx - 2, ckpt=1)  # odd T with every state kept


def test_objective_gradient_fp32_32cube_vs_fp64_oracle():
    """Differentiation config at 32^3 (sigma = 2 cells, 250 steps, objective over the last 25,
    checkpoint interval 32): GPU FP32 adjoint vs FP64 oracle adjoint within 1e-4 (L2 over gamma)."""
    w = I.duct(n=32, u_in=0.04, tau=0.6, sigma=2.0, dtype=np.float64)
    T, W = 250, 25
    o = oracle_from(w, cast32=True)
    Jo = o.objective_run(T, W, 1, w.nx - 2)
    go, uo = o.adjoint()
    g = gpu_from(w, lbm.F32)
    Jg = g.objective_forward(T, W, 1, w.nx - 2, ckpt=32)
    gg, ug = g.objective_backward()
    assert abs(Jg - Jo) < 1e-4 * abs(Jo)
    assert rel_l2(gg, go) < 1e-4
    prof = w.uin[0] / 0.04
    assert abs((ug[0] * prof).sum() - (uo[0] * prof).sum()) < 1e-4 * abs((uo[0] * prof).sum())


def test_objective_gradient_fp64_central_differences():
    w = I.duct(n=10, u_in=0.03, tau=0.7, sigma=1.5, cs=0.1, dtype=np.float64)
    T, W = 20, 5
    g = gpu_from(w, lbm.F64)
    g.objective_forward(T, W, 1, w.nx - 2, ckpt=6)
    dg, _ = g.objective_backward()
    rng = np.random.default_rng(8)
    cells = rng.choice(np.nonzero(w.mask != 1)[0], 16, replace=False)
    h = 1e-5
    for n in cells:
        vals = []
        for s in (1, -1):
            gam = w.gamma.copy()
            gam[n] += s * h
            g2 = gpu_from(w, lbm.F64)
            g2.set_porosity(gam)
            vals.append(g2.objective_forward(T, W, 1, w.nx - 2, ckpt=6))
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(fd - dg[n]) <= 1e-3 * max(abs(fd), 1e-3 * np.abs(dg).max())


# ---- state handling, checkpoints, failure paths --------------------------------------------------------------
def test_save_load_resume_is_bit_identical():
    w = with_features(small_cases()[4])
    g = gpu_from(w, lbm.F32)
    g.step(5)
    buf = g.save()
    g.step(8)
    a = g.get_populations(np.float32)
    g.load(buf)
    assert g.info()["t"] == 5
    g.step(8)
    b = g.get_populations(np.float32)
    assert np.array_equal(a, b)


def test_populations_round_trip_both_layouts():
    w = small_cases()[1]
    g = gpu_from(w, lbm.F64)
    for steps in (0, 1):
        g.step(steps)
        f = g.get_populations()
        f2 = f * (1 + 1e-3 * np.random.default_rng(1).standard_normal(f.shape))
        f2[:, w.mask == 1] = 0
        g.set_populations(f2)
        assert np.abs(g.get_populations() - f2).max() < 1e-15


def test_nan_is_reported_and_context_recovers():
    w = small_cases()[0]
    g = gpu_from(w, lbm.F32)
    f = g.get_populations()
    n = int(np.nonzero(w.mask != 1)[0][3])
    f[5, n] = np.nan
    g.set_populations(f)
    g.step(2)
    with pytest.raises(lbm.LBMError) as e:
        g.sync()
    assert e.value.code == lbm.ENAN
    g.init_equilibrium(np.asarray(w.rho0, np.float32), np.asarray(w.u0, np.float32))
    g.step(2)
    g.sync()


def test_invalid_arguments_are_rejected():
    g = lbm.Lattice(19, 8, 6, 4, 0.6)
    bad = np.zeros(8 * 6 * 4, np.uint8)
    bad[7] = 9
    with pytest.raises(lbm.LBMError) as e:
        g.set_geometry(bad)
    assert e.value.code == lbm.EINVAL
    with pytest.raises(lbm.LBMError):
        g.set_faces([0, 1, 0, 0, 0, 0])
    with pytest.raises(lbm.LBMError):
        lbm.Lattice(19, 8, 8, 8, 0.5)
    with pytest.raises(lbm.LBMError):
        lbm.Lattice(21, 8, 8, 8, 0.6)
    g.set_wall_model(0.41, 9.52)
    with pytest.raises(lbm.LBMError) as e:
        g.objective_forward(4, 2, 1, 6)
    assert e.value.code == lbm.ESTATE


def test_device_buffers_through_torch():
    import torch
    w = small_cases()[0]
    g = gpu_from(w, lbm.F32)
    s = torch.cuda.Stream()
    g.set_stream(s)
    with torch.cuda.stream(s):
        g.step(3)
        rho = torch.empty(w.N, dtype=torch.float32, device="cuda")
        u = torch.empty(3, w.N, dtype=torch.float32, device="cuda")
        g.moments(np.float32, rho, u)
    s.synchronize()
    rh, uh = g.moments(np.float32)
    assert np.array_equal(rho.cpu().numpy(), rh)
    assert np.array_equal(u.cpu().numpy(), uh)
    g.set_stream(0)


# ---- full-size workloads in the benchmark's launch configuration, sampled --------------------------------------
def _crop_oracle(w, centre, R):
    """Oracle on the (2R+1)^3 neighbourhood of `centre` of workload w: coordinates wrap on periodic
    axes; positions beyond a bounce-back face become solid cells; a crop face on the domain's own
    face keeps its kind; other crop faces are bounce-back (their effect stays > R - 2*steps away)."""
    dims = (w.nx, w.ny, w.nz)
    rng_ax, faces, solid_pad = [], [], []
    for a in range(3):
        per = w.faces[2 * a] == 0
        lo, hi = centre[a] - R, centre[a] + R
        if per:
            if dims[a] <= 2 * R + 1:
                idx = np.arange(dims[a]); f = (0, 0)
            else:
                idx = np.arange(lo, hi + 1) % dims[a]; f = (1, 1)
            pad = np.zeros(len(idx), bool)
        else:
            l2, h2 = max(lo, 0), min(hi, dims[a] - 1)
            fl = w.faces[2 * a] if lo <= 0 else 1
            fh = w.faces[2 * a + 1] if hi >= dims[a] - 1 else 1
            idx = np.arange(l2, h2 + 1)
            pad = np.zeros(len(idx), bool)
            f = (fl, fh)
        rng_ax.append(idx)
        faces += list(f)
        solid_pad.append(pad)
    xs, ys, zs = rng_ax
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    gidx = (X + w.nx * (Y + w.ny * Z)).reshape(-1)
    nx, ny, nz = len(xs), len(ys), len(zs)
    sub = I.Workload(name="crop", q=w.q, nx=nx, ny=ny, nz=nz, tau=w.tau, cs=w.cs, faces=tuple(faces),
                     mask=w.mask[gidx].copy(), force=w.force, rho_out=w.rho_out, wall_model=w.wall_model,
                     kappa=w.kappa, E=w.E, rho0=np.asarray(w.rho0)[gidx], u0=np.asarray(w.u0)[:, gidx])
    sub.model, sub.sigma = getattr(w, "model", 0), getattr(w, "sigma", 1.0)
    if w.ywall is not None:
        sub.ywall = np.asarray(w.ywall)[gidx]
    if w.gamma is not None:
        sub.gamma = np.asarray(w.gamma)[gidx]
    if getattr(w, "fringe", None):
        L, s_max, p = w.fringe[:3]
        first = w.fringe[3] if len(w.fringe) > 3 else w.nx - L
        sub.fringe = (L, s_max, p, first - int(xs[0]))  # the domain's layer in crop coordinates
    if w.uin is not None:
        YY, ZZ = np.meshgrid(ys, zs, indexing="xy")
        pidx = (YY + w.ny * ZZ).reshape(-1)
        sub.uin = np.asarray(w.uin)[:, pidx]
    # open faces keep their inlet/outlet cells only where the crop touches the domain face
    m = sub.mask.reshape(nz, ny, nx)
    if faces[0] != 3:
        m[:, :, 0][m[:, :, 0] == 3] = 0
    if faces[1] != 3:
        m[:, :, -1][m[:, :, -1] == 4] = 0
    sub.mask = m.reshape(-1)
    local = [int(np.nonzero(rng_ax[a] == centre[a])[0][0]) for a in range(3)]
    return sub, local[0] + nx * (local[1] + ny * local[2])


def _sampled_full_size(w, storage, steps, samples, R, seed):
    g = gpu_from(w, storage)
    g.step(steps)
    rg, ug = g.moments(np.float32)
    rng = np.random.default_rng(seed)
    kind = (g.debug_dump(0) & 7)
    cand_wall = np.nonzero(kind == 2)[0]
    cand_bc = np.nonzero((kind == 3) | (kind == 4))[0]
    cand_f = np.nonzero(kind == 0)[0]
    picks = list(rng.choice(cand_f, samples // 2, replace=False))
    if len(cand_wall):
        picks += list(rng.choice(cand_wall, samples // 4, replace=False))
    if len(cand_bc):
        picks += list(rng.choice(cand_bc, samples // 4, replace=False))
    worst_r = worst_u = 0.0
    for n in picks:
        c = (n % w.nx, (n // w.nx) % w.ny, n // (w.nx * w.ny))
        sub, ln = _crop_oracle(w, c, R)
        o = oracle_from(sub, cast32=True)
        o.step(steps)
        ro, uo = o.moments()
        worst_r = max(worst_r, abs(float(rg[n]) - ro[ln]))
        worst_u = max(worst_u, float(np.abs(ug[:, n] - uo[:, ln]).max()) / 0.05)
    return worst_r, worst_u


def test_full_size_channel_256_sampled():
    """256^3 turbulent channel (D3Q19, Smagorinsky C_S = 0.1, wall function, body force), FP32, in the
    benchmark's launch shape: 4 steps (both parities twice), 48 sampled cells recomputed by the oracle
    on 15^3 crops (dependency radius 2 per step including the lagged reference velocity)."""
    w = I.channel(nx=256, ny=256, nz=256, seed=550, dtype=np.float32)
    er, eu = _sampled_full_size(w, lbm.F32, steps=4, samples=48, R=7, seed=1)
    assert er < 1e-6 and eu < 1e-5, (er, eu)


def test_full_size_channel_256_every_cell_100_steps():
    """The 256^3 turbulent channel of the benchmark (D3Q19, Smagorinsky C_S = 0.1, wall function,
    body force), FP32 in the benchmark's launch shape, against the FP64 oracle on the full grid after
    100 steps: every non-solid cell, rho within 1e-5 and u within 1e-5 relative L2 (the oracle runs on
    all host cores, about a minute)."""
    w = I.channel(nx=256, ny=256, nz=256, seed=550, dtype=np.float64)
    g = gpu_from(w, lbm.F32)
    assert g.interior_kernel() == 1
    g.step(100)
    rg, ug = g.moments()
    g.close()
    o = oracle_from(w, cast32=True)
    o.step(100)
    ro, uo = o.moments()
    del o
    fl = w.mask != 1
    assert np.abs(rg[fl] - ro[fl]).max() < 1e-5
    assert rel_l2(ug[:, fl], uo[:, fl]) < 1e-5


@pytest.mark.parametrize("q", [19, 27])
def test_full_size_canopy_512_sampled(q):
    w = I.canopy(nx=512, ny=512, nz=256, q=q, seed=2506, dtype=np.float32)
    er, eu = _sampled_full_size(w, lbm.F32, steps=2, samples=32, R=5, seed=2)
    assert er < 1e-6 and eu < 1e-5, (er, eu)


def test_full_size_channel_256_hrr_sampled():
    """The HRR collision (sigma = 1/2: the strain of the previous step's velocity field from the
    neighbours) on the 256^3 channel in the benchmark's launch shape: 3 steps, 24 sampled cells
    recomputed by the oracle on 15^3 crops."""
    w = I.channel(nx=256, ny=256, nz=256, seed=550, dtype=np.float32)
    w.model, w.sigma = 1, 0.5
    er, eu = _sampled_full_size(w, lbm.F32, steps=3, samples=24, R=7, seed=3)
    assert er < 1e-6 and eu < 1e-5, (er, eu)


def test_full_size_canopy_512_hrr_sampled():
    w = I.canopy(nx=512, ny=512, nz=256, q=19, seed=2506, dtype=np.float32)
    w.model, w.sigma = 1, 0.5
    er, eu = _sampled_full_size(w, lbm.F32, steps=2, samples=24, R=6, seed=4)
    assert er < 1e-6 and eu < 1e-5, (er, eu)


# ---- staged interior kernel (bulk copies into shared memory) -----------------------------------------------
@pytest.mark.parametrize("q,storage", [(19, lbm.F32), (27, lbm.F32), (19, lbm.F16), (19, lbm.BF16)])
def test_staged_kernel_matches_plain_kernel(q, storage):
    """nx a multiple of 128 selects the staged kernel; it must give the plain kernel's results."""
    cases = [I.channel(nx=256, ny=34, nz=6, q=q, seed=5, dtype=np.float64),
             I.canopy(nx=128, ny=64, nz=40, q=q, seed=2506, crop=(64, 0, 0), domain=(1024, 512, 256), dtype=np.float64),
             with_features(I.random_box(128, 9, 7, seed=6, q=q, solid_frac=0.1, tau=0.6, cs=0.1, faces=(0, 0, 2, 2, 1, 2)))]
    for w in cases:
        a = gpu_from(w, storage)
        a.set_option(lbm.OPT_KERNEL, lbm.KERNEL_STAGED)
        b = gpu_from(w, storage)
        for steps in (1, 2, 9):
            a.step(steps)
            b.step(steps)
            fa = a.get_populations()
            fb = b.get_populations()
            tol = {lbm.F32: 2e-7, lbm.F16: 2e-3, lbm.BF16: 2e-2}[storage]
            assert np.abs(fa - fb).max() <= tol, (w.name, steps, np.abs(fa - fb).max())
        a.sync()
        b.sync()


@pytest.mark.parametrize("nx,storage", [(128, lbm.F32), (256, lbm.F16)])
def test_staged_kernel_bounded_wait_reports_timeout_and_recovers(nx, storage):
    """The staged kernels' waits are bounded (per-cell FP32 kernel; paired 16-bit kernel): with a
    barrier that nothing completes, the step ends after the one-second limit, the status reads
    LBM_ETIMEOUT, and the context stays usable."""
    w = I.channel(nx=nx, ny=18, nz=8, seed=5, dtype=np.float32)
    g = gpu_from(w, storage)
    g.set_option(lbm.OPT_KERNEL, lbm.KERNEL_STAGED)
    g.set_option(lbm.OPT_DEBUG_STALL, 1)
    g.step(1)
    with pytest.raises(lbm.LBMError) as e:
        g.sync()
    assert e.value.code == lbm.ETIMEOUT
    g.set_option(lbm.OPT_DEBUG_STALL, 0)
    g.init_equilibrium(np.asarray(w.rho0, np.float32), np.asarray(w.u0, np.float32))
    g.step(4)
    g.sync()
    o = oracle_from(w, cast32=True)
    o.step(4)
    rg, _ = g.moments()
    ro, _ = o.moments()
    assert np.abs(rg - ro).max() < (1e-6 if storage == lbm.F32 else 1e-3)
