"""Pins of the oracle's vortex-method inlet (Sec. 2.2.2) against facts fixed outside its code: the
published SplitMix64 output sequence, uniformity of the counter-based draws, the 2D vortex field
being divergence free with the closed-form circulation of one vortex, the in-plane kinetic energy
of many random vortices equal to 2/3 of the prescribed k (which fixes the constant 6 ln 3 - 9 ln 2
of the circulation together with the vortex profile), and the sign and size of the streamwise
(Langevin) fluctuation on a linear mean profile."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2506_21804_gb300 import inputs as I


def test_splitmix64_published_sequence():
    """First three outputs of SplitMix64 started from state 0 (state advances by 0x9E3779B97F4A7C15)."""
    g = 0x9E3779B97F4A7C15
    want = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    got = [O.splitmix64((k * g) & 0xFFFFFFFFFFFFFFFF) for k in (1, 2, 3)]
    assert got == want


def test_counter_uniforms_are_uniform():
    u = np.array([O.vm_uniform(1804, c) for c in range(40000)])
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 4 * np.sqrt(1 / 12 / u.size)
    assert abs(u.var() - 1 / 12) < 0.003
    h, _ = np.histogram(u, bins=20, range=(0, 1))
    assert h.min() > 0.9 * u.size / 20 and h.max() < 1.1 * u.size / 20


def test_single_vortex_circulation_and_divergence():
    """Circulation around a circle of radius R about one vortex: Gamma (1 - e^{-a}) e^{-a},
    a = R^2/(2 sigma^2) (Stokes on the profile); the field of several vortices is divergence free."""
    sigma, gam = 3.0, 0.7
    v = np.array([[10.3, 7.9, gam]])
    for R in (0.5, 2.0, 3.0, 7.5):
        th = np.linspace(0, 2 * np.pi, 721)[:-1]
        circ = 0.0
        for t in th:
            y, z = 10.3 + R * np.cos(t), 7.9 + R * np.sin(t)
            u = O.vm_field(v, sigma, y, z)
            circ += (u[0] * -np.sin(t) + u[1] * np.cos(t)) * R * (2 * np.pi / th.size)
        a = R * R / (2 * sigma * sigma)
        assert abs(circ - gam * (1 - np.exp(-a)) * np.exp(-a)) < 1e-9
    vs = np.array([[3.1, 4.2, 0.5], [8.7, 2.2, -0.9], [5.5, 9.9, 0.3]])
    h = 1e-4
    for (y, z) in [(4.0, 5.0), (7.3, 3.1), (6.6, 8.8)]:
        div = ((O.vm_field(vs, 2.0, y + h, z)[0] - O.vm_field(vs, 2.0, y - h, z)[0]) +
               (O.vm_field(vs, 2.0, y, z + h)[1] - O.vm_field(vs, 2.0, y, z - h)[1])) / (2 * h)
        scale = np.abs(O.vm_field(vs, 2.0, y, z)).max()
        assert abs(div) < 1e-7 * max(scale, 1e-3)


def _inlet_box(ny, nz, U, I_t, sigma, n_v, seed, mean=None):
    w = I.random_box(3, ny, nz, seed=7, q=19, solid_frac=0.0, tau=0.8, cs=0.0, faces=(3, 3, 0, 0, 0, 0),
                     inflow=True, outflow=True)
    uin = np.zeros((3, ny * nz))
    uin[0] = U if mean is None else mean
    o = O.Oracle(19, 3, ny, nz, 0.8, 0.0)
    o.set_faces(w.faces)
    o.set_geometry(w.mask)
    o.set_inflow(uin)
    o.set_vortex_inlet(n_v, sigma, I_t, seed)
    o.init_equilibrium(np.ones(w.N), np.zeros((3, w.N)))
    return o, uin


def test_vortex_energy_is_two_thirds_of_k():
    """Uniform mean U, intensity I: k = 3/2 (U I)^2 and the mean in-plane kinetic energy of the
    vortex field, away from the plane edges, is 2/3 k = (U I)^2."""
    ny = nz = 120
    U, It, sigma = 0.05, 0.1, 2.5
    o, uin = _inlet_box(ny, nz, U, It, sigma, 600, 2506)
    m = int(5 * sigma)
    E = []
    for _ in range(12):
        o.step(1)
        f = o.inflow_field().reshape(3, nz, ny)
        E.append(0.5 * (f[1, m:-m, m:-m] ** 2 + f[2, m:-m, m:-m] ** 2).mean())
    assert abs(np.mean(E) / (U * It) ** 2 - 1) < 0.06


def test_streamwise_fluctuation_on_linear_mean_profile():
    """Mean U = a z: on the first step grad U = (0, a) at interior positions, so u'_x = -u_z."""
    ny, nz, a = 24, 20, 2e-3
    zz = np.repeat(np.arange(nz), ny).astype(float)
    mean = a * zz + 0.01
    o, uin = _inlet_box(ny, nz, None, 0.2, 2.0, 30, 11, mean=mean)
    o.step(1)
    f = o.inflow_field().reshape(3, nz, ny)
    ux = f[0] - mean.reshape(nz, ny)
    assert np.abs(f[2]).max() > 1e-5
    assert np.allclose(ux[1:-1, :], -f[2][1:-1, :], atol=1e-15)
    # second step: the gradient is taken from the perturbed field of step 1
    o.step(1)
    g = o.inflow_field().reshape(3, nz, ny)
    assert not np.allclose(g[0] - mean.reshape(nz, ny), -g[2], atol=1e-12)


def test_inlet_restarts_from_the_mean_and_steps_are_reproducible():
    o, uin = _inlet_box(16, 12, 0.04, 0.1, 2.0, 20, 5)
    o.step(3)
    a = o.inflow_field().copy()
    assert not np.allclose(a, uin)
    o.init_equilibrium(np.ones(3 * 16 * 12), np.zeros((3, 3 * 16 * 12)))
    assert np.array_equal(o.inflow_field(), uin)
    o.step(3)
    assert np.array_equal(o.inflow_field(), a)
