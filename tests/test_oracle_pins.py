"""Pins of the FP64 CPU oracle against facts fixed by the paper and by mathematics, independent of
the oracle's own code: exact lattice identities, closed-form flows (Taylor-Green decay, Poiseuille
at the magic relaxation time), conservation laws, brute-force re-implementations on tiny grids,
the Smagorinsky fixed point, Spalding's law limits, IEEE codecs against library conversions, and
finite differences of the discrete adjoint."""
from fractions import Fraction

import numpy as np
import pytest

from oracle import oracle as O
from paper_2506_21804_gb300 import inputs as I
from tests.helpers import oracle_from


# ---- lattice tables (Sec. 2.2, Fig. "lattice") --------------------------------------------------
@pytest.mark.parametrize("q", [19, 27])
def test_lattice_isotropy_exact(q):
    c, w, opp, W, den = O.lattice(q)
    wf = [Fraction(int(Wi), den) for Wi in W]
    assert sum(wf) == 1
    cs2 = Fraction(1, 3)
    d = np.eye(3, dtype=int)
    for a in range(3):
        assert sum(wf[i] * int(c[i, a]) for i in range(q)) == 0
        for b in range(3):
            assert sum(wf[i] * int(c[i, a] * c[i, b]) for i in range(q)) == cs2 * int(d[a, b])
            for g in range(3):
                assert sum(wf[i] * int(c[i, a] * c[i, b] * c[i, g]) for i in range(q)) == 0
                for e in range(3):
                    lhs = sum(wf[i] * int(c[i, a] * c[i, b] * c[i, g] * c[i, e]) for i in range(q))
                    rhs = cs2 * cs2 * (d[a, b] * d[g, e] + d[a, g] * d[b, e] + d[a, e] * d[b, g])
                    assert lhs == rhs
    # opposite pairs and the documented ordering
    assert (c[opp] == -c).all()
    h = (q - 1) // 2
    assert (c[1 + h:] == -c[1:1 + h]).all()
    assert len({tuple(v) for v in c}) == q


@pytest.mark.parametrize("q", [19, 27])
def test_equilibrium_moments(q):
    c, w, *_ = O.lattice(q)
    rng = np.random.default_rng(1)
    for _ in range(5):
        rho = 1 + 0.1 * rng.standard_normal()
        u = 0.05 * rng.standard_normal(3)
        f = O.feq(q, rho, u)
        assert abs(f.sum() - rho) < 1e-15
        assert np.allclose(c.T @ f, rho * u, atol=1e-15)
        P = np.einsum("i,ia,ib->ab", f, c, c)
        assert np.allclose(P, rho / 3 * np.eye(3) + rho * np.outer(u, u), atol=1e-15)


# ---- brute force on a 4^3 grid: plain push-streaming BGK with bounce-back -----------------------
def _bgk_push_step(f, c, w, opp, solid, tau, shape):
    """Independent plain-Python restatement of one BGK step (collide at x, push to x + c_i,
    half-way bounce-back into the opposite population of x when x + c_i is solid)."""
    nz, ny, nx = shape
    q = len(w)
    new = np.zeros_like(f)
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                if solid[z, y, x]:
                    continue
                fl = f[:, z, y, x]
                rho = fl.sum()
                u = (c.T @ fl) / rho
                for i in range(q):
                    cu = c[i] @ u
                    fe = w[i] * rho * (1 + 3 * cu + 4.5 * cu * cu - 1.5 * u @ u)
                    post = fl[i] - (fl[i] - fe) / tau
                    X, Y, Z = (x + c[i, 0]) % nx, (y + c[i, 1]) % ny, (z + c[i, 2]) % nz
                    if solid[Z, Y, X]:
                        new[opp[i], z, y, x] = post
                    else:
                        new[i, Z, Y, X] = post
    return new


@pytest.mark.parametrize("q", [19, 27])
def test_bruteforce_step_4cube(q):
    w_ = I.random_box(4, 4, 4, seed=7, q=q, solid_frac=0.15, tau=0.8, cs=0.0)
    o = oracle_from(w_)
    c, w, opp, *_ = O.lattice(q)
    f0 = o.populations().reshape(q, 4, 4, 4)
    solid = (w_.mask == 1).reshape(4, 4, 4)
    # Oracle output of one step
    o.step(1)
    f1 = o.populations().reshape(q, 4, 4, 4)
    ref = _bgk_push_step(f0, c, w, opp, solid, 0.8, (4, 4, 4))
    fl = ~solid
    assert np.abs(f1[:, fl] - ref[:, fl]).max() < 1e-15
    # brute-force moments
    rho, u = o.moments()
    fr = f1.reshape(q, -1)
    r = fr.sum(0)
    assert np.allclose(rho[fl.reshape(-1)], r[fl.reshape(-1)], atol=1e-15)
    uu = (c.T @ fr) / np.where(r == 0, 1, r)
    assert np.allclose(u[:, fl.reshape(-1)], uu[:, fl.reshape(-1)], atol=1e-15)


# ---- conservation ----------------------------------------------------------------------------------
@pytest.mark.parametrize("q", [19, 27])
def test_periodic_mass_conservation_smagorinsky_bounceback(q):
    w = I.random_box(8, 6, 5, seed=11, q=q, solid_frac=0.12, tau=0.55, cs=0.17)
    o = oracle_from(w)
    m0, _ = o.reduce()
    o.step(40)
    m1, _ = o.reduce()
    assert abs(m1 - m0) / m0 < 1e-13


def test_mass_conservation_with_wall_model_and_slip():
    w = I.random_box(8, 7, 6, seed=12, q=19, solid_frac=0.1, tau=0.52, cs=0.1, faces=(0, 0, 2, 2, 1, 2))
    w.wall_model = True
    o = oracle_from(w)
    m0, _ = o.reduce()
    o.step(30)
    m1, _ = o.reduce()
    assert abs(m1 - m0) / m0 < 1e-13


def test_momentum_gain_equals_body_force():
    w = I.random_box(6, 5, 4, seed=13, q=19, solid_frac=0.0, tau=0.7, cs=0.1)
    F = (1e-5, -2e-5, 3e-6)
    w.force = F
    o = oracle_from(w)
    # total j = sum rho u_rep - N F / 2 (reported velocity carries F/(2 rho)); j gains N F per step
    N = w.N
    _, p0 = o.reduce()
    o.step(10)
    _, p1 = o.reduce()
    assert np.allclose(p1 - p0, 10 * N * np.array(F), rtol=1e-10, atol=1e-14)


# ---- closed-form flows ---------------------------------------------------------------------------------
def test_taylor_green_decay_and_second_order():
    errs = []
    for n in (16, 32):
        u0 = 0.05 * 32 / n
        w = I.taylor_green(n=n, u0=u0, tau=0.6, nz=1)
        o = oracle_from(w)
        T = int(200 * (n / 32) ** 2)
        o.step(T)
        _, u = o.moments()
        shape = w.u0 / u0
        A = (u * shape).sum() / (shape * shape).sum()
        exact = u0 * np.exp(-2 * w.meta["nu"] * w.meta["k"] ** 2 * T)
        errs.append(abs(A / exact - 1))
    assert errs[1] < 0.01          # amplitude within 1% at t = 200 on the 32 grid
    assert 3.0 < errs[0] / errs[1] < 5.0   # second order in space (Sec. 2.2)


def test_poiseuille_exact_at_magic_tau():
    """BGK with half-way bounce-back reproduces the parabola exactly when (tau - 1/2)^2 = 3/16."""
    H = 8
    ny = H + 2
    tau = 0.5 + np.sqrt(3 / 16)
    nu = (tau - 0.5) / 3
    F = 1e-5
    mask = np.zeros((1, ny, 4), np.uint8)
    mask[:, 0, :] = 1
    mask[:, -1, :] = 1
    o = O.Oracle(19, 4, ny, 1, tau, 0.0)
    o.set_faces([0, 0, 1, 1, 0, 0])
    o.set_geometry(mask.reshape(-1))
    o.set_force(F, 0, 0)
    N = 4 * ny
    o.init_equilibrium(np.ones(N), np.zeros((3, N)))
    o.step(6000)
    _, u = o.moments()
    y = np.arange(ny)
    ux = u[0].reshape(ny, 4)[:, 0]
    exact = F / (2 * nu) * (y - 0.5) * (ny - 1.5 - y)
    assert np.abs(ux[1:-1] - exact[1:-1]).max() / exact.max() < 1e-10
    # off the magic value the same channel has a wall slip of the known sign and size O((tau-1/2)^2)
    o2 = O.Oracle(19, 4, ny, 1, 1.2, 0.0)
    o2.set_faces([0, 0, 1, 1, 0, 0])
    o2.set_geometry(mask.reshape(-1))
    o2.set_force(F, 0, 0)
    o2.init_equilibrium(np.ones(N), np.zeros((3, N)))
    o2.step(4000)
    _, u2 = o2.moments()
    nu2 = 0.7 / 3
    ex2 = F / (2 * nu2) * (y - 0.5) * (ny - 1.5 - y)
    slip = u2[0].reshape(ny, 4)[1:-1, 0] - ex2[1:-1]
    # Bounce-back Poiseuille with BGK: the parabola of effective width^2 = H^2 + (16 L - 3)/3,
    # L = (tau - 1/2)^2, i.e. a uniform slip u_s = F (16 L - 3) / (24 nu).
    us = F * (16 * 0.7 ** 2 - 3) / (24 * nu2)
    assert np.allclose(slip, us, rtol=1e-6)


# ---- Smagorinsky, Eq. (tauEff) ---------------------------------------------------------------------------
def test_smagorinsky_fixed_point_and_bgk_limit():
    rng = np.random.default_rng(3)
    for _ in range(20):
        A = rng.standard_normal((3, 3)) * 1e-3
        Pi = A + A.T
        rho = 1 + 0.05 * rng.standard_normal()
        tau0 = 0.5 + rng.uniform(1e-3, 0.5)
        cs = rng.uniform(0.05, 0.2)
        tau = O.tau_smagorinsky(tau0, cs, Pi, rho)
        # Definition: tau = nu_eff/cs^2 + 1/2 with nu_eff = nu0 + (C_S)^2 |S|, |S| = sqrt(2 S:S),
        # S = -Pi / (2 rho cs^2 tau).
        S = -Pi / (2 * rho * (1 / 3) * tau)
        absS = np.sqrt(2 * (S * S).sum())
        nu_eff = (tau0 - 0.5) / 3 + cs * cs * absS
        assert abs(tau - (3 * nu_eff + 0.5)) < 1e-14
        assert tau >= tau0
        assert O.tau_smagorinsky(tau0, 0.0, Pi, rho) == tau0


def test_smagorinsky_zero_constant_is_bitwise_bgk():
    w1 = I.random_box(6, 5, 4, seed=21, q=19, solid_frac=0.1, tau=0.7, cs=0.0)
    o1 = oracle_from(w1)
    w2 = I.random_box(6, 5, 4, seed=21, q=19, solid_frac=0.1, tau=0.7, cs=0.0)
    w2.gamma = np.ones(w2.N)
    o2 = oracle_from(w2)
    o1.step(5)
    o2.step(5)
    assert np.array_equal(o1.populations(), o2.populations())   # gamma = 1 is plain BGK, bitwise


# ---- Spalding's law, Eq. (spaldingfunct) ------------------------------------------------------------------
def test_spalding_limits_and_inverse():
    k, E = 0.41, 9.52
    # viscous sublayer: y+ = u+ + O(u+^4)
    for up in (1e-3, 1e-2):
        assert abs(O.spalding_yplus(up, k, E) - up) < (k * up) ** 4 / 24 / E * 1.01 + 1e-18
    # log region: u+ -> (1/kappa) ln(E y+) as y+ grows (the polynomial terms become negligible)
    for yp in (1e4, 1e5):
        up, it = O.solve_uplus_yplus(yp, k, E)
        assert abs(up - np.log(E * yp) / k) < 0.05
        assert it <= 20
    # round trips and Newton residuals
    for yp in (0.1, 1.0, 5.0, 11.0, 30.0, 100.0, 1000.0):
        up, it = O.solve_uplus_yplus(yp, k, E)
        assert abs(O.spalding_yplus(up, k, E) - yp) <= 1e-12 * yp
        assert it <= 20
    for Re in (1e-3, 1.0, 50.0, 750.0, 22300.0, 1e6):
        up, it = O.solve_uplus_re(Re, k, E)
        assert abs(up * O.spalding_yplus(up, k, E) - Re) <= 1e-12 * Re
        assert it <= 20
    # derivative is the derivative
    for up in (0.5, 5.0, 20.0):
        h = 1e-6
        fd = (O.spalding_yplus(up + h, k, E) - O.spalding_yplus(up - h, k, E)) / (2 * h)
        assert abs(fd - O.spalding_dyplus(up, k, E)) < 1e-6 * fd


def test_wall_model_state_on_channel_wall():
    """A channel wall cell with a known reference velocity: u^B is tangential, u_tau solves Spalding
    at the reference distance, and the modelled shear follows from dy+/du+ at the wall cell."""
    w = I.channel(nx=4, ny=12, nz=4, noise=0.0, seed=1)
    o = oracle_from(w)
    kind, isref, nsum, ref = o.classification()
    n = int(np.nonzero(kind == O.KIND_WALL)[0][0])
    assert ref[n] >= 0 and isref[ref[n]] == 1
    uB, dudn = o.wall_state(n)
    ur = o.refbuf()[ref[n]]
    nu = w.meta["nu"]
    # bottom wall, D3Q19: solid neighbours (0,-1,0) (weight 2) and four diagonals (weight 1), so
    # v = (0, -6, 0), n = +y and u_t = (u_x, 0, u_z)
    assert (nsum[n] == [0, -6, 0]).all()
    U = np.hypot(ur[0], ur[2])
    up_r, _ = O.solve_uplus_re(U * 1.5 / nu)
    utau = U / up_r
    up_w, _ = O.solve_uplus_yplus(0.5 * utau / nu)
    assert abs(np.linalg.norm(uB) - utau * up_w) < 1e-14
    assert abs(uB[1]) == 0.0
    assert abs(dudn - utau * utau / nu / O.spalding_dyplus(up_w)) < 1e-12 * dudn


# ---- boundary reconstruction (Sec. 2.2.2, Sec. 3.2) ----------------------------------------------------
@pytest.mark.parametrize("q", [19, 27])
def test_regularised_boundaries(q):
    c, w, *_ = O.lattice(q)
    rng = np.random.default_rng(5)
    ub = np.array([0.04, 0.01, -0.005])
    f = O.feq(q, 1.01, ub + 0.003 * rng.standard_normal(3)) + 1e-4 * rng.standard_normal(q)
    g = O.bc(q, 3, f, ub)
    rho = g.sum()
    assert np.allclose(c.T @ g / rho, ub, atol=1e-15)
    # mass formula uses only the known populations (c_x <= 0)
    known0 = f[c[:, 0] == 0].sum() + 2 * f[c[:, 0] < 0].sum()
    assert abs(rho - known0 / (1 - ub[0])) < 1e-14
    # a distribution already of regularised form is a fixed point
    assert np.allclose(O.bc(q, 3, g, ub), g, atol=1e-15)
    # pressure outlet: prescribed density, tangential velocity zero
    h = O.bc(q, 4, f, rho_out=1.0)
    assert abs(h.sum() - 1.0) < 1e-14
    uo = c.T @ h
    assert abs(uo[1]) < 1e-15 and abs(uo[2]) < 1e-15


def test_duct_mass_flux_in_equals_out():
    """Straight duct with uniform inlet velocity and a pressure outlet: at steady state the mass flux
    through every cross-section is the same."""
    n = 6
    w = I.duct(n=n, u_in=0.02, tau=0.8, q=19)
    w.nx = 16
    x, y, z = np.meshgrid(np.arange(16), np.arange(n), np.arange(n), indexing="ij")
    x, y, z = x.transpose(2, 1, 0).reshape(-1), y.transpose(2, 1, 0).reshape(-1), z.transpose(2, 1, 0).reshape(-1)
    solid = (y == 0) | (y == n - 1) | (z == 0) | (z == n - 1)
    mask = np.zeros(x.size, np.uint8)
    mask[solid] = 1
    mask[(x == 0) & ~solid] = 3
    mask[(x == 15) & ~solid] = 4
    w.mask = mask
    w.gamma = None
    w.rho0 = np.ones(x.size)
    w.u0 = np.zeros((3, x.size))
    o = oracle_from(w)
    o.step(12000)   # the longitudinal acoustic mode decays like exp(-(2/3) nu k^2 t)
    rho, u = o.moments()
    flux = (rho * u[0]).reshape(n, n, 16).sum(axis=(0, 1))
    assert np.abs(flux - flux[0]).max() < 1e-8 * abs(flux[0])
    assert flux[0] > 0


def test_porosity_uniform_closed_form():
    """Eq. (convexVelocity) with u^B = 0: a uniform state keeps uniform, and each step multiplies the
    velocity by gamma exactly (u_t = gamma^t u_0); gamma = 0 leaves no momentum after one step."""
    n = 4
    N = n ** 3
    u0 = np.array([0.03, -0.02, 0.01])
    for g, T in ((0.9, 10), (0.0, 1)):
        o = O.Oracle(19, n, n, n, 0.7, 0.1)
        o.set_porosity(np.full(N, g))
        o.init_equilibrium(np.ones(N), np.tile(u0[:, None], (1, N)))
        o.step(T)
        rho, u = o.moments()
        assert np.allclose(rho, 1.0, atol=1e-15)
        assert np.allclose(u, (g ** T) * u0[:, None], atol=1e-16)


# ---- geometry and propagation maps ---------------------------------------------------------------------------
def test_classification_single_solid_cell():
    nx = ny = nz = 5
    mask = np.zeros(125, np.uint8)
    centre = 2 + 5 * (2 + 5 * 2)
    mask[centre] = 1
    o = O.Oracle(19, nx, ny, nz, 0.6)
    o.set_geometry(mask)
    kind, isref, nsum, ref = o.classification()
    c, *_ = O.lattice(19)
    walls = np.nonzero(kind == O.KIND_WALL)[0]
    assert len(walls) == 18
    for n in walls:
        x, y, z = n % 5, (n // 5) % 5, n // 25
        d = np.array([2 - x, 2 - y, 2 - z])     # direction towards the solid cell
        # the solid neighbour is the only one, so v = W_i c_i with c_i = d and n = -v/|v|
        W = 2 if (np.abs(d).sum() == 1) else 1
        assert (nsum[n] == W * d).all()
        a = int(np.argmax(np.abs(d)))
        r = np.array([x, y, z])
        r[a] -= d[a]
        assert ref[n] == r[0] + 5 * (r[1] + 5 * r[2])
    assert kind[centre] == O.KIND_SOLID


@pytest.mark.parametrize("faces", [(0, 0, 0, 0, 0, 0), (3, 3, 2, 2, 1, 2), (2, 2, 2, 2, 2, 2), (1, 1, 2, 2, 0, 0)])
@pytest.mark.parametrize("q", [19, 27])
def test_source_map_is_a_slot_bijection(q, faces):
    """Every post-collision population feeds at most one destination, so streaming is a partial
    permutation; interior fluid cells pull from x - c_i; specular sources reverse only the crossed
    components."""
    w = I.random_box(7, 6, 5, seed=41, q=q, solid_frac=0.15, faces=faces, inflow=faces[0] == 3, outflow=faces[1] == 3)
    o = oracle_from(w)
    c, _, opp, *_ = O.lattice(q)
    d, m = o.source_map()
    kind = o.classification()[0]
    fl = kind != O.KIND_SOLID
    pairs = d[:, fl].astype(np.int64) * w.N + m[:, fl]
    assert len(np.unique(pairs)) == pairs.size
    assert (kind[m[:, fl]] != O.KIND_SOLID).all()
    dims = np.array([7, 6, 5])
    for n in np.nonzero(fl)[0][:60]:
        xs = np.array([n % 7, (n // 7) % 6, n // 42])
        for i in range(q):
            s = xs - c[i]
            inside = ((s >= 0) & (s < dims)) | (np.array([faces[0], faces[2], faces[4]]) == 0)
            s = s % dims
            sn = s[0] + 7 * (s[1] + 6 * s[2])
            if inside.all() and w.mask[sn] != 1:
                assert d[i, n] == i and m[i, n] == sn
            elif inside.all():
                assert d[i, n] == opp[i] and m[i, n] == n
            else:
                j = d[i, n]
                flip = c[j] != c[i]
                assert ((c[j][flip] == -c[i][flip])).all()


# ---- IEEE binary16 and bfloat16 codecs (storage form) -----------------------------------------------------
def test_f16_codec_exhaustive():
    bits = np.arange(65536, dtype=np.uint16)
    lib_vals = bits.view(np.float16).astype(np.float64)
    for b in range(0, 65536, 1):
        v = O.f16_decode(b)
        lv = lib_vals[b]
        if np.isnan(lv):
            assert np.isnan(v)
        else:
            assert v == lv
    # encode: every finite value, and the midpoints between neighbours (ties to even)
    fin = np.nonzero(np.isfinite(lib_vals))[0]
    for b in fin[::7]:
        assert O.f16_encode(lib_vals[b]) == np.float64(lib_vals[b]).astype(np.float16).view(np.uint16) or lib_vals[b] == 0
    pos = np.sort(lib_vals[(lib_vals > 0) & np.isfinite(lib_vals)])
    mids = (pos[:-1] + pos[1:]) / 2
    for m in mids[::5]:
        assert O.f16_encode(m) == np.float64(m).astype(np.float16).view(np.uint16)
    assert O.f16_encode(65520.0) == 0x7C00 and O.f16_encode(65519.99) == 0x7BFF


def test_bf16_codec_against_torch():
    torch = pytest.importorskip("torch")
    bits = torch.arange(0, 65536, dtype=torch.int32).to(torch.int16).view(torch.bfloat16)
    vals = bits.to(torch.float64).numpy()
    for b in range(0, 65536, 3):
        v = O.bf16_decode(b)
        if np.isnan(vals[b]):
            assert np.isnan(v)
        else:
            assert v == vals[b]
    rng = np.random.default_rng(9)
    xs = np.concatenate([rng.standard_normal(2000) * 10.0 ** rng.integers(-40, 38, 2000),
                         (vals[1:200] + vals[2:201]) / 2])
    xs = xs[np.isfinite(xs)].astype(np.float32).astype(np.float64)  # representable in fp32: no double rounding
    ref = torch.from_numpy(xs.astype(np.float32)).to(torch.bfloat16).view(torch.int16).numpy().astype(np.uint16)
    for x, r in zip(xs, ref):
        assert O.bf16_encode(x) == r


# ---- discrete adjoint -------------------------------------------------------------------------------------------
def _adj_case(n=6, T=12, W=4, cs=0.1):
    w = I.duct(n=n, u_in=0.03, tau=0.7, sigma=1.5, cs=cs)
    w.u0 = np.zeros((3, w.N))
    w.u0[0] = 0.01
    return w, T, W


def test_adjoint_dot_product():
    w, *_ = _adj_case()
    o = oracle_from(w)
    o.step(3)
    rng = np.random.default_rng(2)
    v = rng.standard_normal((w.q, w.N))
    vg = rng.standard_normal(w.N)
    vu = rng.standard_normal((3, w.ny * w.nz))
    wv = rng.standard_normal((w.q, w.N))
    kind = o.classification()[0]
    v[:, kind == O.KIND_SOLID] = 0
    wv[:, kind == O.KIND_SOLID] = 0
    Jv = o.jvp_step(v, vg, vu)
    JTw, gT, uT = o.vjp_step(wv)
    lhs = (wv * Jv).sum()
    rhs = (JTw * v).sum() + (gT * vg).sum() + (uT * vu.reshape(-1)).sum()
    assert abs(lhs - rhs) < 1e-12 * max(1.0, abs(lhs))


@pytest.mark.parametrize("cs", [0.0, 0.15])
def test_adjoint_matches_central_differences(cs):
    w, T, W = _adj_case(cs=cs)
    xa, xb = 1, w.nx - 2
    o = oracle_from(w)
    o.objective_run(T, W, xa, xb)
    dg, du = o.adjoint()
    rng = np.random.default_rng(4)
    kind = o.classification()[0]
    cand = np.nonzero(kind != O.KIND_SOLID)[0]
    cells = rng.choice(cand, 16, replace=False)
    h = 1e-5
    for n in cells:
        vals = []
        for s in (+1, -1):
            g = w.gamma.copy()
            g[n] += s * h
            w2 = I.duct(n=w.nx, u_in=0.03, tau=0.7, sigma=1.5, cs=cs)
            w2.u0 = w.u0
            w2.gamma = g
            o2 = oracle_from(w2)
            vals.append(o2.objective_run(T, W, xa, xb))
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(fd - dg[n]) <= 1e-3 * max(abs(fd), 1e-3 * np.abs(dg).max()), (n, fd, dg[n])
    # inflow speed: u_in = U * profile
    prof = w.uin[0] / 0.03
    dU = (du[0] * prof).sum()
    vals = []
    for s in (+1, -1):
        w2 = I.duct(n=w.nx, u_in=0.03 + s * h, tau=0.7, sigma=1.5, cs=cs)
        w2.u0 = w.u0
        vals.append(oracle_from(w2).objective_run(T, W, xa, xb))
    fd = (vals[0] - vals[1]) / (2 * h)
    assert abs(fd - dU) <= 1e-3 * abs(fd)
