"""Pins of the oracle's sigma = 0 wall-cell update (Sec. 2.2.1 turbulent wall model with Sec. 2.2's
finite-difference non-equilibrium part f^(1,FD)) against quantities this file computes itself.

Nothing here goes through the oracle's wall-model functions. For every WALL cell the test derives,
from the mask and the oracle's populations alone:
  * the wall normal n = -sum_{solid i} w_i c_i / |...| and the reference cell one step along the
    dominant axis of n, used only when it is a FLUID cell away from every boundary (no solid or
    outside streaming source: the reference point lies in the flow);
  * the reference velocity (the reported velocity j/rho + F/(2 rho) of that cell in the state the
    step starts from) and its tangential part u_t = u_r - (u_r . n) n, t = u_t/|u_t|;
  * u+ at the reference distance y_r = y_w + 1 from u+ y+(u+) = |u_t| y_r / nu, u_tau = |u_t|/u+,
    u+_w from y+(u+_w) = y_w u_tau / nu, with Spalding's law (Eq. spaldingfunct) written out below
    and inverted by bracketing (scipy's brentq), not by the oracle's Newton iteration;
  * u^B = u_tau u+_w t, du/dn = (u_tau^2/nu) / y+'(u+_w), S = (du/dn)/2 (t n^T + n t^T) and
    tau_eff = tau0 + 3 C_S^2 |du/dn|.
It then recovers the cell's post-collision populations f*_i from the next state (f*_i(x) arrives at
x + c_i, or returns to x in the opposite direction when x + c_i is solid) and checks them.

A plausible mistake in the oracle's wall branch fails here. Flipping the sign of f^(1,FD) (or of the
HRR branch's A2 = -2 rho cs^2 tau S) in oracle/lbm_oracle.cpp makes both the moment test and the
per-population test fail. So does dropping the weight w_i, losing the factor 1/2 of S, using tau0
instead of tau_eff, or taking u instead of u^B. Each of these mistakes was planted in the oracle's
source in turn, rebuilt and run against this file. (Writing S as (du/dn) t n^T without the
symmetric half is not a mistake: Q_i : S sees only the symmetric part, and t . n = 0.) The bulk test fixes the sign and weights of the reading f^(1,FD)_i =
-(w_i rho tau / cs^2) Q_i : S independently, against the BGK bulk's own Chapman-Enskog
non-equilibrium in a steady Poiseuille flow.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2506_21804_gb300 import inputs as I
from tests.helpers import oracle_from

scipy_opt = pytest.importorskip("scipy.optimize")

CS2 = 1.0 / 3.0


def spalding_y(up, k, E):
    """Spalding's law y+(u+) (Eq. spaldingfunct)."""
    x = k * up
    return up + (np.exp(x) - 1.0 - x - x * x / 2.0 - x ** 3 / 6.0) / E


def spalding_dy(up, k, E):
    x = k * up
    return 1.0 + k * (np.exp(x) - 1.0 - x - x * x / 2.0) / E


def solve_bracket(fun, target):
    """Root of fun(u) = target for an increasing fun with fun(0) = 0."""
    hi = 1.0
    while fun(hi) < target:
        hi *= 2.0
    return scipy_opt.brentq(lambda u: fun(u) - target, 0.0, hi, xtol=1e-15, rtol=1e-15, maxiter=500)


def feq(c, w, rho, u):
    cu = c @ u
    return w * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * (u @ u))


def qcontract(c, S):
    """Q_i : S with Q_i = c_i c_i - cs^2 I, for every i."""
    return np.einsum("ia,ib,ab->i", c, c, S) - CS2 * np.trace(S)


def _wrap(w, p):
    """Periodic wrap of position p on the periodic axes; None when p leaves through another face."""
    dims = (w.nx, w.ny, w.nz)
    out = []
    for a in range(3):
        v = int(p[a])
        if v < 0 or v >= dims[a]:
            if w.faces[2 * a + (0 if v < 0 else 1)] != I.FACE_PERIODIC:
                return None
            v %= dims[a]
        out.append(v)
    return out


def _solid_at(w, p):
    """True where position p is a solid cell or lies beyond a bounce-back face."""
    q = _wrap(w, p)
    if q is None:
        return True
    return w.mask[q[0] + w.nx * (q[1] + w.ny * q[2])] == I.MASK_SOLID


def _plain_fluid(w, c, r):
    """Fluid cell with no solid or outside streaming source (the only admissible reference cell)."""
    if w.mask[r] != I.MASK_FLUID:
        return False
    x, y, z = r % w.nx, (r // w.nx) % w.ny, r // (w.nx * w.ny)
    for i in range(1, len(c)):
        q = _wrap(w, (x - c[i, 0], y - c[i, 1], z - c[i, 2]))
        if q is None or w.mask[q[0] + w.nx * (q[1] + w.ny * q[2])] == I.MASK_SOLID:
            return False
    return True


def expected_wall_update(w, c, wts, f0, n, meta_nu):
    """The sigma = 0 update of WALL cell n, derived in the test: (rho, u_hat, tau, S). A cell whose
    weighted solid-neighbour sum vanishes (solids on opposite sides) has no normal and gets u^B = 0,
    S = 0; so does a cell whose reference position is not a plain fluid cell, or whose tangential
    reference velocity is below 1e-12."""
    x, y, z = n % w.nx, (n // w.nx) % w.ny, n // (w.nx * w.ny)
    # integer sum of W_i c_i (W_i = w_i times the common denominator), so that ties between axes
    # are exact
    Wint = np.rint(wts * (36 if len(wts) == 19 else 216)).astype(np.int64)
    v = np.zeros(3, np.int64)
    for i in range(len(wts)):
        if _solid_at(w, (x + c[i, 0], y + c[i, 1], z + c[i, 2])):
            v += Wint[i] * c[i].astype(np.int64)
    rho = f0[:, n].sum()
    F = np.asarray(w.force, np.float64)
    if not v.any():
        return rho, F / rho, w.tau, np.zeros((3, 3))
    nrm = -v / np.linalg.norm(v.astype(np.float64))
    a = int(np.argmax(np.abs(v)))  # ties: lowest axis (argmax returns the first)
    step = np.zeros(3, int)
    step[a] = 1 if nrm[a] > 0 else -1
    rp = _wrap(w, (x + step[0], y + step[1], z + step[2]))
    tau0 = w.tau
    uB = np.zeros(3)
    S = np.zeros((3, 3))
    dudn = 0.0
    if rp is not None:
        r = rp[0] + w.nx * (rp[1] + w.ny * rp[2])
        if _plain_fluid(w, c, r):
            rho_r = f0[:, r].sum()
            u_r = (c.T @ f0[:, r]) / rho_r + F / (2.0 * rho_r)
            u_t = u_r - (u_r @ nrm) * nrm
            U = np.linalg.norm(u_t)
            if U >= 1e-12:
                t = u_t / U
                # the wall distances reach the oracle rounded to FP32 (the GPU's input precision)
                yw = 0.5 if w.ywall is None else float(np.float32(w.ywall[n]))
                k, E, nu = w.kappa, w.E, meta_nu
                up_r = solve_bracket(lambda u: u * spalding_y(u, k, E), U * (yw + 1.0) / nu)
                utau = U / up_r
                up_w = solve_bracket(lambda u: spalding_y(u, k, E), yw * utau / nu)
                uB = utau * up_w * t
                dudn = (utau * utau / nu) / spalding_dy(up_w, k, E)
                S = 0.5 * dudn * (np.outer(t, nrm) + np.outer(nrm, t))
    tau = tau0 + 3.0 * w.cs * w.cs * abs(dudn)
    u_hat = uB + F / rho
    return rho, u_hat, tau, S


def post_collision(w, c, opp, f1, n):
    """f*_i(x) recovered from the state after the step (push streaming with half-way bounce-back)."""
    x, y, z = n % w.nx, (n // w.nx) % w.ny, n // (w.nx * w.ny)
    out = np.zeros(len(opp))
    for i in range(len(opp)):
        p = (x + c[i, 0], y + c[i, 1], z + c[i, 2])
        if _solid_at(w, p):
            out[i] = f1[opp[i], n]
        else:
            q = _wrap(w, p)
            out[i] = f1[i, q[0] + w.nx * (q[1] + w.ny * q[2])]
    return out


def wall_cases(q):
    ch = I.channel(nx=6, ny=12, nz=5, q=q, noise=0.4, seed=3, dtype=np.float64)
    rb = I.random_box(9, 8, 7, seed=11, q=q, solid_frac=0.15, tau=0.62, cs=0.14, faces=(0, 0, 0, 0, 0, 0))
    rb.wall_model = True
    rb.force = (3e-6, -2e-6, 1e-6)
    return [ch, rb]


def _nu(w):
    return (w.tau - 0.5) / 3.0


@pytest.mark.parametrize("q", [19, 27])
@pytest.mark.parametrize("model", [0, 1])
def test_wall_cell_moments_from_spalding(q, model):
    """Moments of the sigma = 0 update at every WALL cell: sum f* = rho, sum f* c = rho u_hat and
    sum f* c c = rho cs^2 I + rho u_hat u_hat + (1 - 1/tau_eff)(-2 rho cs^2 tau_eff S), with u_hat =
    u^B + F/rho and S, tau_eff from the hand-derived wall law. Holds for the BGK form and for the
    HRR form (whose f^(1) is rebuilt from A2 = -2 rho cs^2 tau_eff S)."""
    c, wts, opp, *_ = O.lattice(q)
    c = c.astype(np.float64)
    checked = 0
    strained = 0
    for w in wall_cases(q):
        o = oracle_from(w)
        if model == 1:
            o.set_collision(1, 0.5)
        f0 = o.populations()
        kind = o.classification()[0]
        o.step(1)
        f1 = o.populations()
        for n in np.nonzero(kind == O.KIND_WALL)[0]:
            rho, uh, tau, S = expected_wall_update(w, c, wts, f0, int(n), _nu(w))
            fs = post_collision(w, c, opp, f1, int(n))
            M2 = rho * CS2 * np.eye(3) + rho * np.outer(uh, uh) + (1.0 - 1.0 / tau) * (-2.0 * rho * CS2 * tau * S)
            assert abs(fs.sum() - rho) < 1e-13
            assert np.abs(c.T @ fs - rho * uh).max() < 1e-13
            got2 = np.einsum("i,ia,ib->ab", fs, c, c)
            assert np.abs(got2 - M2).max() < 1e-13 * max(1.0, np.abs(M2).max()), (w.name, n, got2 - M2)
            checked += 1
            strained += np.abs(S).max() > 1e-6
    assert checked > 40 and strained > 20


@pytest.mark.parametrize("q", [19, 27])
def test_wall_cell_populations_from_spalding(q):
    """Every population of the BGK sigma = 0 update: f*_i = f^eq_i(rho, u_hat) + (1 - 1/tau_eff)
    f^(1,FD)_i with f^(1,FD)_i = -(w_i rho tau_eff / cs^2) Q_i : S."""
    c, wts, opp, *_ = O.lattice(q)
    c = c.astype(np.float64)
    for w in wall_cases(q):
        o = oracle_from(w)
        f0 = o.populations()
        kind = o.classification()[0]
        o.step(1)
        f1 = o.populations()
        for n in np.nonzero(kind == O.KIND_WALL)[0]:
            rho, uh, tau, S = expected_wall_update(w, c, wts, f0, int(n), _nu(w))
            f1fd = -(wts * rho * tau / CS2) * qcontract(c, S)
            want = feq(c, wts, rho, uh) + (1.0 - 1.0 / tau) * f1fd
            got = post_collision(w, c, opp, f1, int(n))
            assert np.abs(got - want).max() < 1e-14, (w.name, n)


def _poiseuille_fneq_deviation(umax):
    """Steady body-force Poiseuille flow (BGK, half-way bounce-back walls between y = 0.5 and
    y = ny - 1.5, tau = 1/2 + sqrt(3/16) where the lattice profile is the exact parabola): the largest
    deviation of the even part of f - f^eq(rho, u) from -(w_i rho tau / cs^2) Q_i : S over all fluid
    cells and populations, relative to the largest value of the formula."""
    q = 19
    c, wts, opp, *_ = O.lattice(q)
    c = c.astype(np.float64)
    nx, ny, nz = 2, 34, 2
    tau = 0.5 + np.sqrt(3.0 / 16.0)
    nu = (tau - 0.5) / 3.0
    H = ny - 2.0
    Fx = 8.0 * nu * umax / (H * H)
    y0, y1 = 0.5, ny - 1.5
    yy = np.tile(np.arange(ny)[None, :, None], (nz, 1, nx)).reshape(-1)
    mask = np.zeros(nx * ny * nz, np.uint8)
    mask[(yy == 0) | (yy == ny - 1)] = 1
    o = O.Oracle(q, nx, ny, nz, tau, 0.0)
    o.set_faces((0, 0, 1, 1, 0, 0))
    o.set_geometry(mask)
    o.set_force(Fx, 0.0, 0.0)
    u0 = np.zeros((3, mask.size))
    u0[0] = np.where(mask == 0, Fx / (2 * nu) * (yy - y0) * (y1 - yy), 0.0)
    o.init_equilibrium(np.ones(mask.size), u0)
    o.step(4000)
    f = o.populations()
    worst = scale = 0.0
    for n in np.nonzero(mask == 0)[0]:
        rho = f[:, n].sum()
        u = (c.T @ f[:, n]) / rho
        fneq = f[:, n] - feq(c, wts, rho, u)
        even = 0.5 * (fneq + fneq[opp])
        S = np.zeros((3, 3))
        S[0, 1] = S[1, 0] = 0.5 * Fx / (2 * nu) * (y0 + y1 - 2.0 * yy[n])
        want = -(wts * rho * tau / CS2) * qcontract(c, S)
        worst = max(worst, np.abs(even - want).max())
        scale = max(scale, np.abs(want).max())
    return worst / scale


def test_fneq_reading_matches_bgk_bulk_in_poiseuille():
    """The reading f^(1,FD)_i = -(w_i rho tau / cs^2) Q_i : S (weights w_i, minus sign) is the
    Chapman-Enskog non-equilibrium part that the BGK bulk itself carries: in steady Poiseuille flow
    the even part of f - f^eq(rho, u) equals the formula with the exact strain S_xy = (du/dy)/2 up to
    a relative deviation that halves with the velocity (an O(Ma^2) correction). A flipped sign is off
    by 200 %, a dropped weight by a factor of up to 36."""
    r1 = _poiseuille_fneq_deviation(0.01)
    r2 = _poiseuille_fneq_deviation(0.005)
    assert r1 < 5e-3 and r2 < 5e-3, (r1, r2)
    assert 1.7 < r1 / r2 < 2.3, (r1, r2)
