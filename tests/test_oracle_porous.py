"""Pins of the oracle's porous-medium inputs (Sec. 2.1, Eq. lattice_porosity): the Forchheimer
permeability reduces to Darcy's law without the inertial term and satisfies the Forchheimer
pressure-drop law it inverts; the lattice porosity from K is 1 for K = inf (bitwise the plain
collision), 0 at and below K = nu tau, and a uniform porous box decays as gamma(K)^t."""
import numpy as np

from oracle import oracle as O


def test_forchheimer_darcy_limit_and_pressure_law():
    mu, Q, A, L, dP, rho = 1.8e-5, 2.0e-3, 0.5, 0.3, 4.0, 1.2
    # Darcy: Q = K A dP / (mu L)
    K0 = O.forchheimer_k(mu, Q, A, L, dP, rho)
    assert abs(Q - K0 * A * dP / (mu * L)) < 1e-15 * Q
    # with the inertial term the Forchheimer law dP/L = mu Q/(K A) + rho Q^2/(K_beta A^2) holds
    Kb = 3.0e-4
    K = O.forchheimer_k(mu, Q, A, L, dP, rho, Kb)
    assert K > K0
    assert abs(mu * Q / (K * A) + rho * Q * Q / (Kb * A * A) - dP / L) < 1e-12 * dP / L
    assert np.isnan(O.forchheimer_k(mu, Q, A, L, 1e-9, rho, Kb))


def test_porosity_from_permeability_limits():
    n, tau = 4, 0.7
    nu = (tau - 0.5) / 3
    o = O.Oracle(19, n, n, n, tau, 0.1)
    K = np.full(n ** 3, np.inf)
    K[:8] = nu * tau            # at the threshold: solid-like
    K[8:16] = 0.5 * nu * tau    # below it: clamped
    K[16:24] = 10 * nu * tau    # gamma = 0.9
    K[24] = -1.0                # invalid permeabilities are impermeable
    K[25] = np.nan
    o.set_permeability(K)
    g = o.porosity()
    assert np.all(g[:16] == 0.0) and g[24] == 0.0 and g[25] == 0.0
    g[24:26] = 1.0
    assert np.allclose(g[16:24], 0.9, atol=1e-15)
    assert np.all(g[24:] == 1.0)


def test_uniform_porous_box_decay_from_permeability():
    """Uniform K: every step multiplies the velocity by gamma(K) = 1 - nu tau / K."""
    n, tau = 4, 0.7
    nu = (tau - 0.5) / 3
    N = n ** 3
    u0 = np.array([0.03, -0.02, 0.01])
    K = 4 * nu * tau
    o = O.Oracle(19, n, n, n, tau, 0.1)
    o.set_permeability(np.full(N, K))
    o.init_equilibrium(np.ones(N), np.tile(u0[:, None], (1, N)))
    o.step(6)
    _, u = o.moments()
    assert np.allclose(u, 0.75 ** 6 * u0[:, None], atol=1e-16)
    # K = inf everywhere is bitwise the fluid collision
    a = O.Oracle(19, n, n, n, tau, 0.1)
    b = O.Oracle(19, n, n, n, tau, 0.1)
    a.set_permeability(np.full(N, np.inf))
    for o_ in (a, b):
        o_.init_equilibrium(np.ones(N), np.tile(u0[:, None], (1, N)))
        o_.step(3)
    assert np.array_equal(a.populations(), b.populations())
