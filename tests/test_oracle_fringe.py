"""Pins of the oracle's outlet fringe zone (Sec. 3.2: a fixed-pressure outlet with a fringe zone in
front of it; the paper gives no parameters). The reading: in the last L planes the post-collision
populations relax towards f^eq(rho_out, u) with strength s(x) = s_max xi^p, xi = (x - (nx - L) + 1)/L.

* With p = 0 and the layer covering a periodic box, a uniform state (rho0, u0) stays uniform and its
  density perturbation decays exactly as (1 - s_max)^t while the velocity stays u0 (f^eq is linear in
  rho at fixed u, and the BGK collision leaves an equilibrium unchanged).
* The strength profile is the formula, restated here.
* One step on a random box: every post-collision population of every cell equals the plain BGK
  update written out in this file, relaxed by s(x) in the layer and untouched before it.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2506_21804_gb300 import inputs as I
from tests.helpers import oracle_from


@pytest.mark.parametrize("q", [19, 27])
def test_fringe_uniform_perturbation_decays_in_closed_form(q):
    nx, ny, nz = 6, 5, 4
    N = nx * ny * nz
    rho0, u0, s_max, rho_out = 1.02, np.array([0.03, -0.01, 0.02]), 0.1, 0.995
    o = O.Oracle(q, nx, ny, nz, 0.7, 0.1)
    o.set_geometry(np.zeros(N, np.uint8))
    o.set_outflow(rho_out)
    o.set_fringe(nx, s_max, 0.0)
    o.init_equilibrium(np.full(N, rho0), np.tile(u0[:, None], (1, N)))
    for t in range(1, 11):
        o.step(1)
        rho, u = o.moments()
        want = rho_out + (1.0 - s_max) ** t * (rho0 - rho_out)
        assert np.abs(rho - want).max() < 1e-14, t
        assert np.abs(u - u0[:, None]).max() < 1e-15, t


def test_fringe_strength_profile():
    nx, L, s_max, p = 20, 6, 0.4, 2.0
    o = O.Oracle(19, nx, 3, 3, 0.6, 0.0)
    o.set_fringe(L, s_max, p)
    for x in range(nx):
        want = 0.0 if x < nx - L else s_max * ((x - (nx - L) + 1) / L) ** p
        assert o.fringe_strength(x) == pytest.approx(want, rel=0, abs=1e-16)
    assert o.fringe_strength(nx - 1) == s_max
    with pytest.raises(ValueError):
        o.set_fringe(-1, 0.1, 2.0)
    with pytest.raises(ValueError):
        o.set_fringe(3, 1.5, 2.0)


def _feq(c, w, rho, u):
    cu = c @ u
    return w * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * (u @ u))


@pytest.mark.parametrize("q", [19, 27])
def test_fringe_one_step_every_population(q):
    c, w, opp, *_ = O.lattice(q)
    c = c.astype(np.float64)
    ci = c.astype(int)
    wk = I.random_box(10, 6, 5, seed=31, q=q, solid_frac=0.1, tau=0.65, cs=0.0, faces=(0, 0, 0, 0, 0, 0))
    L, s_max, p, rho_out = 4, 0.3, 2.0, 1.01
    wk.rho_out = rho_out
    wk.fringe = (L, s_max, p)
    o = oracle_from(wk)
    f0 = o.populations()
    o.step(1)
    f1 = o.populations()
    nx, ny, nz = wk.nx, wk.ny, wk.nz
    solid = wk.mask == I.MASK_SOLID
    relaxed = 0
    for n in np.nonzero(~solid)[0]:
        x, y, z = n % nx, (n // nx) % ny, n // (nx * ny)
        rho = f0[:, n].sum()
        u = (c.T @ f0[:, n]) / rho
        fs = _feq(c, w, rho, u) + (1.0 - 1.0 / wk.tau) * (f0[:, n] - _feq(c, w, rho, u))
        s = 0.0 if x < nx - L else s_max * ((x - (nx - L) + 1) / L) ** p
        if s > 0:
            fs = fs - s * (fs - _feq(c, w, rho_out, u))
            relaxed += 1
        got = np.zeros(q)
        for i in range(q):
            tx, ty, tz = (x + ci[i, 0]) % nx, (y + ci[i, 1]) % ny, (z + ci[i, 2]) % nz
            m = tx + nx * (ty + ny * tz)
            got[i] = f1[opp[i], n] if solid[m] else f1[i, m]
        assert np.abs(got - fs).max() < 1e-15, (n, x)
    assert relaxed > 50
