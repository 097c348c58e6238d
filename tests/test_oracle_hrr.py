"""Pins of the oracle's hybrid recursive regularised (HRR) collision of Sec. 2.2 against facts fixed
by the Hermite expansion and by closed-form flows: the third-order term is the Hermite contraction
H^(3) : a / (6 cs^6) where the velocity set carries it (D3Q27) and reproduces every third moment
the velocity set supports (D3Q19); the equilibrium and the update have the prescribed moments up to
third order; with zero velocity the update is the textbook regularised BGK; the finite-difference
strain is exact on linear fields; the full step conserves mass; Taylor-Green vortices decay at the
viscous rate."""
import itertools

import numpy as np
import pytest

from oracle import oracle as O
from paper_2506_21804_gb300 import inputs as I
from tests.helpers import oracle_from

CS2 = 1.0 / 3.0
MIXED = [(0, 0, 1), (0, 0, 2), (1, 1, 0), (1, 1, 2), (2, 2, 0), (2, 2, 1)]


def _h3(c, a, b, g):
    """Third Hermite polynomial of the velocity c, written out from its definition."""
    return c[a] * c[b] * c[g] - CS2 * (c[a] * (b == g) + c[b] * (a == g) + c[g] * (a == b))


def _h2(c):
    return np.outer(c, c) - CS2 * np.eye(3)


def _sym3(rng):
    a = rng.normal(size=(3, 3, 3))
    return sum(a.transpose(p) for p in itertools.permutations(range(3))) / 6.0


def _third_moment(f, c, trip):
    return sum(f[i] * _h3(c[i], *trip) for i in range(len(f)))


def test_third_order_d3q27_is_hermite_contraction():
    c, w, *_ = O.lattice(27)
    rng = np.random.default_rng(3)
    for _ in range(5):
        a = _sym3(rng)
        got = O.third_order(27, a)
        want = np.array([w[i] * sum(_h3(c[i], al, be, ga) * a[al, be, ga]
                                    for al, be, ga in itertools.product(range(3), repeat=3)) / (6 * CS2 ** 3)
                         for i in range(27)])
        assert np.allclose(got, want, rtol=0, atol=1e-14)


@pytest.mark.parametrize("q", [19, 27])
def test_third_order_moments(q):
    """The term carries exactly the third moments of the tensor that the velocity set supports and
    no moment of order 0, 1 or 2."""
    c, w, *_ = O.lattice(q)
    rng = np.random.default_rng(4)
    a = _sym3(rng)
    t = O.third_order(q, a)
    for trip in MIXED + ([(0, 1, 2)] if q == 27 else []):
        assert abs(_third_moment(t, c, trip) - a[trip]) < 1e-14
    if q == 19:   # H_xyz vanishes on D3Q19: that moment is not carried
        assert abs(_third_moment(t, c, (0, 1, 2))) < 1e-15
    assert abs(t.sum()) < 1e-15
    assert np.allclose(c.T @ t, 0, atol=1e-15)
    assert np.allclose(np.einsum("i,ia,ib->ab", t, c, c), 0, atol=1e-15)


@pytest.mark.parametrize("q", [19, 27])
def test_third_order_equilibrium_moments(q):
    c, w, *_ = O.lattice(q)
    rho, u = 1.07, np.array([0.05, -0.03, 0.02])
    f = O.feq3(q, rho, u)
    assert abs(f.sum() - rho) < 1e-14
    assert np.allclose(c.T @ f, rho * u, atol=1e-15)
    assert np.allclose(np.einsum("i,ia,ib->ab", f, c, c), rho * (CS2 * np.eye(3) + np.outer(u, u)), atol=1e-15)
    for trip in MIXED:
        assert abs(_third_moment(f, c, trip) - rho * u[trip[0]] * u[trip[1]] * u[trip[2]]) < 1e-15
    # the second-order equilibrium differs only by third-order terms
    assert np.allclose(f - O.feq(q, rho, u), O.third_order(q, rho * np.einsum("a,b,c->abc", u, u, u)), atol=1e-16)


@pytest.mark.parametrize("q", [19, 27])
def test_hrr_update_moments(q):
    """f* has rho, rho u_eq, the equilibrium stress plus (1 - 1/tau) A2, and the third moments of
    the equilibrium plus (1 - 1/tau) times the recursive A3 = sym(u_h A2)."""
    c, w, *_ = O.lattice(q)
    rng = np.random.default_rng(5)
    rho, tau = 0.97, 0.58
    ueq, uh = np.array([0.04, 0.01, -0.02]), np.array([0.035, 0.012, -0.018])
    A2 = rng.normal(scale=1e-3, size=(3, 3))
    A2 = A2 + A2.T
    fs = O.collide_hrr(q, rho, ueq, uh, tau, A2)
    k = 1 - 1 / tau
    assert abs(fs.sum() - rho) < 1e-14
    assert np.allclose(c.T @ fs, rho * ueq, atol=1e-15)
    second = np.einsum("i,iab->ab", fs, np.array([_h2(ci) for ci in c]))
    assert np.allclose(second, rho * np.outer(ueq, ueq) + k * A2, atol=1e-15)
    A3 = np.einsum("a,bc->abc", uh, A2) + np.einsum("b,ac->abc", uh, A2) + np.einsum("c,ab->abc", uh, A2)
    for trip in MIXED:
        want = rho * ueq[trip[0]] * ueq[trip[1]] * ueq[trip[2]] + k * A3[trip]
        assert abs(_third_moment(fs, c, trip) - want) < 1e-15


@pytest.mark.parametrize("q", [19, 27])
def test_hrr_at_rest_is_regularised_bgk(q):
    """u = 0: f*_i = w_i (rho + (1 - 1/tau) Q_i : Pi / (2 cs^4)) (regularised BGK)."""
    c, w, *_ = O.lattice(q)
    rho, tau = 1.02, 0.71
    Pi = np.array([[2e-3, 5e-4, -1e-4], [5e-4, -1e-3, 3e-4], [-1e-4, 3e-4, 4e-4]])
    fs = O.collide_hrr(q, rho, np.zeros(3), np.zeros(3), tau, Pi)
    want = np.array([w[i] * (rho + (1 - 1 / tau) * np.sum(_h2(c[i]) * Pi) / (2 * CS2 ** 2)) for i in range(q)])
    assert np.allclose(fs, want, rtol=0, atol=1e-16)


def test_strain_fd_exact_on_linear_fields():
    """Central and one-sided differences are exact for a linear velocity field, at interior cells,
    next to a solid cell, and at non-periodic faces; a direction with no usable neighbour gives 0."""
    nx, ny, nz = 6, 5, 5
    w = I.random_box(nx, ny, nz, seed=21, q=19, solid_frac=0.0, tau=0.6, cs=0.0, faces=(1, 1, 1, 1, 2, 2))
    mask = np.zeros(w.N, np.uint8)
    mask[2 + nx * (2 + ny * 2)] = O.MASK_SOLID
    w.mask = mask
    w.model = 1
    o = oracle_from(w)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    x, y, z = x.reshape(-1), y.reshape(-1), z.reshape(-1)
    G = np.array([[0.0, 2e-3, -1e-3], [5e-4, 1e-3, 0.0], [3e-4, -7e-4, 2e-4]])   # du_a/dx_b
    u = G @ np.stack([x, y, z]).astype(float)
    o.set_velocity_field(u)
    S = 0.5 * (G + G.T)
    kind = o.classification()[0]
    for n in range(w.N):
        if kind[n] == O.KIND_SOLID:
            continue
        assert np.allclose(o.strain_fd(n), S, atol=1e-15), n
    # one cell thick in y between walls: no usable y neighbour -> d/dy terms vanish
    w1 = I.random_box(4, 1, 3, seed=22, q=19, solid_frac=0.0, tau=0.6, cs=0.0, faces=(0, 0, 1, 1, 0, 0))
    w1.model = 1
    o1 = oracle_from(w1)
    z, y, x = np.meshgrid(np.arange(3), np.arange(1), np.arange(4), indexing="ij")
    o1.set_velocity_field(np.stack([0.01 * y.reshape(-1), 0 * x.reshape(-1), 0 * x.reshape(-1)]).astype(float))
    assert np.allclose(o1.strain_fd(0), 0, atol=1e-18)


@pytest.mark.parametrize("sigma", [1.0, 0.5, 0.0])
def test_hrr_step_conserves_mass(sigma):
    w = I.random_box(8, 6, 5, seed=23, q=19, solid_frac=0.1, tau=0.56, cs=0.15)
    w.model, w.sigma = 1, sigma
    o = oracle_from(w)
    m0, _ = o.reduce()
    o.step(30)
    m1, _ = o.reduce()
    assert abs(m1 - m0) / m0 < 1e-13


@pytest.mark.parametrize("sigma,tol", [(1.0, 0.01), (0.5, 0.01), (0.0, 0.015)])
def test_hrr_taylor_green_decay(sigma, tol):
    """The viscous decay rate exp(-2 nu k^2 t) of the vortex amplitude at t = 200 on 32^2 and
    second-order convergence (16^2 -> 32^2), with the local stress (sigma = 1), the blend, and the
    finite-difference strain alone (sigma = 0; the strain of the previous step adds a lag error,
    whence the looser amplitude bound)."""
    errs = []
    for n in (16, 32):
        u0 = 0.05 * 32 / n
        w = I.taylor_green(n=n, u0=u0, tau=0.6, nz=1)
        w.model, w.sigma = 1, sigma
        o = oracle_from(w)
        T = int(200 * (n / 32) ** 2)
        o.step(T)
        _, u = o.moments()
        shape = w.u0 / u0
        A = (u * shape).sum() / (shape * shape).sum()
        exact = u0 * np.exp(-2 * w.meta["nu"] * w.meta["k"] ** 2 * T)
        errs.append(abs(A / exact - 1))
    assert errs[1] < tol
    assert 3.0 < errs[0] / errs[1] < 5.0


def test_hrr_sigma_one_without_velocity_gradients_matches_bgk_at_equilibrium():
    """A uniform flow at equilibrium is a fixed point of both collisions."""
    w = I.random_box(5, 4, 3, seed=24, q=27, solid_frac=0.0, tau=0.7, cs=0.1)
    w.rho0 = np.full(w.N, 1.01)
    w.u0 = np.tile(np.array([[0.03], [-0.01], [0.02]]), (1, w.N))
    w.model = 1
    o = oracle_from(w)
    f0 = o.populations().copy()
    o.step(1)
    # the initial state is the second-order equilibrium; after one HRR step the cells hold the
    # third-order one (the update adds only the third-order equilibrium terms)
    f3 = O.feq3(27, 1.01, np.array([0.03, -0.01, 0.02]))
    assert np.allclose(o.populations(), f3[:, None], atol=1e-15)
    assert not np.allclose(f0, o.populations(), atol=1e-12)
