"""Seeded synthetic inputs for the LBM workloads (geometry masks, initial fields, inlet profiles,
porosity fields).

This module holds no lattice Boltzmann arithmetic: it only draws numbers and lays out arrays. Both
the CUDA path and the CPU oracle receive their inputs from here. Random numbers come from a
counter-based generator, SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) applied to
(seed, stream, index), so any element can be regenerated on its own.

Array conventions: cell index n = x + nx*(y + ny*z); masks uint8 of length N with codes
0 fluid, 1 solid, 3 inflow, 4 outflow; velocity fields (3, N); inlet velocity (3, ny*nz) indexed
y + ny*z; face kinds ordered (x-, x+, y-, y+, z-, z+) with 0 periodic, 1 bounce-back wall,
2 full slip, 3 open (inflow/outflow).
"""
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

MASK = 0xFFFFFFFFFFFFFFFF
FACE_PERIODIC, FACE_WALL, FACE_SLIP, FACE_OPEN = 0, 1, 2, 3
MASK_FLUID, MASK_SOLID, MASK_INFLOW, MASK_OUTFLOW = 0, 1, 3, 4


def splitmix64(x):
    """SplitMix64 finaliser on a uint64 array (wrapping arithmetic)."""
    x = np.asarray(x, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = x + np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def counter_bits(seed, stream, index):
    """64 random bits for each (seed, stream, index)."""
    with np.errstate(over="ignore"):
        key = splitmix64(np.uint64(seed & MASK) ^ (np.uint64(stream) * np.uint64(0xD1B54A32D192ED03)))
        return splitmix64(key + np.asarray(index, dtype=np.uint64))


def uniform(seed, stream, index):
    """Uniform doubles in [0, 1)."""
    return (counter_bits(seed, stream, index) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(seed, stream, index):
    """Standard normal doubles by the Box-Muller transform of two counter streams."""
    u1 = uniform(seed, 2 * stream + 1000003, index)
    u2 = uniform(seed, 2 * stream + 1000004, index)
    return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * np.pi * u2)


@dataclass
class Workload:
    """Everything a run needs, in the C ABI's layouts."""
    name: str
    q: int
    nx: int
    ny: int
    nz: int
    tau: float
    cs: float
    faces: tuple = (0, 0, 0, 0, 0, 0)
    mask: Optional[np.ndarray] = None      # uint8 (N,)
    ywall: Optional[np.ndarray] = None     # float (N,) or None (0.5 everywhere)
    force: tuple = (0.0, 0.0, 0.0)
    uin: Optional[np.ndarray] = None       # (3, ny*nz)
    rho_out: float = 1.0
    gamma: Optional[np.ndarray] = None     # (N,)
    wall_model: bool = False
    kappa: float = 0.41
    E: float = 9.52
    rho0: Optional[np.ndarray] = None      # (N,)
    u0: Optional[np.ndarray] = None        # (3, N)
    model: int = 0                         # collision: 0 BGK, 1 hybrid recursive regularised
    sigma: float = 1.0                     # hybridisation factor of the HRR collision
    vortex: Optional[tuple] = None         # vortex-method inlet (n, sigma, intensity, seed) or None
    fringe: Optional[tuple] = None         # outlet fringe zone (L, s_max, p[, first plane]) or None
    meta: dict = field(default_factory=dict)

    @property
    def N(self):
        return self.nx * self.ny * self.nz


def _grid(nx, ny, nz):
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return x.reshape(-1), y.reshape(-1), z.reshape(-1)


def taylor_green(n=32, u0=0.05, tau=0.6, q=19, nz=None, dtype=np.float64):
    """z-invariant 2D Taylor-Green vortex in a periodic n x n x nz box:
    u = u0 cos(kx) sin(ky), v = -u0 sin(kx) cos(ky), w = 0, k = 2 pi / n,
    rho = 1 - (3 u0^2 / 4)(cos 2kx + cos 2ky) (the vortex's pressure field over cs^2)."""
    nz = n if nz is None else nz
    x, y, z = _grid(n, n, nz)
    k = 2.0 * np.pi / n
    u = np.zeros((3, x.size), dtype)
    u[0] = u0 * np.cos(k * x) * np.sin(k * y)
    u[1] = -u0 * np.sin(k * x) * np.cos(k * y)
    rho = (1.0 - 0.75 * u0 * u0 * (np.cos(2 * k * x) + np.cos(2 * k * y))).astype(dtype)
    return Workload(name=f"tgv{n}", q=q, nx=n, ny=n, nz=nz, tau=tau, cs=0.0,
                    mask=np.zeros(x.size, np.uint8), rho0=rho, u0=u,
                    meta=dict(u0=u0, k=k, nu=(tau - 0.5) / 3.0))


def channel(nx=256, ny=256, nz=256, re_tau=550.0, u_tau=0.0025, u_bulk=0.05, noise=0.05, seed=550,
            cs=0.1, q=19, wall_model=True, dtype=np.float32):
    """Plane channel: periodic in x and z, solid rows y = 0 and y = ny-1 (walls half-way between the
    solid rows and the first fluid rows), half height h = (ny-2)/2, viscosity nu = u_tau h / Re_tau,
    body force F_x = u_tau^2 / h, initial laminar-shaped profile 1.5 U_b (1 - eta^2) plus uniform
    noise of +-noise*U_b per component."""
    h = (ny - 2) / 2.0
    nu = u_tau * h / re_tau
    tau = 0.5 + 3.0 * nu
    x, y, z = _grid(nx, ny, nz)
    mask = np.zeros(x.size, np.uint8)
    mask[(y == 0) | (y == ny - 1)] = MASK_SOLID
    eta = (y - (ny - 1) / 2.0) / h
    u = np.zeros((3, x.size), dtype)
    idx = np.arange(x.size, dtype=np.uint64)
    prof = 1.5 * u_bulk * np.clip(1.0 - eta * eta, 0.0, None)
    for a in range(3):
        r = uniform(seed, a, idx) * 2.0 - 1.0
        u[a] = (prof if a == 0 else 0.0) + noise * u_bulk * r
    u[:, mask == MASK_SOLID] = 0.0
    rho = np.ones(x.size, dtype)
    return Workload(name=f"channel{nx}x{ny}x{nz}", q=q, nx=nx, ny=ny, nz=nz, tau=tau, cs=cs,
                    faces=(FACE_PERIODIC, FACE_PERIODIC, FACE_WALL, FACE_WALL, FACE_PERIODIC, FACE_PERIODIC),
                    mask=mask, force=(u_tau * u_tau / h, 0.0, 0.0), wall_model=wall_model,
                    rho0=rho, u0=u, meta=dict(h=h, nu=nu, re_tau=re_tau, u_tau=u_tau))


def canopy_buildings(nx, ny, nz, n_buildings=200, seed=2506, wmin=8, wmax=32, h_median=40.0, h_sigma=0.5):
    """Axis-aligned box buildings: footprints w_x, w_y uniform in {wmin..wmax}, positions uniform in
    x in [64, nx-64-w_x), y in [0, ny-w_y), heights round(exp(ln h_median + h_sigma N(0,1))) clamped
    to [4, nz-32]. Returns an int array (n, 5): x0, y0, wx, wy, height."""
    b = np.arange(n_buildings, dtype=np.uint64)
    span = wmax - wmin + 1
    wx = wmin + np.floor(uniform(seed, 10, b) * span).astype(np.int64)
    wy = wmin + np.floor(uniform(seed, 11, b) * span).astype(np.int64)
    x0 = 64 + np.floor(uniform(seed, 12, b) * (nx - 128 - wx)).astype(np.int64)
    y0 = np.floor(uniform(seed, 13, b) * (ny - wy)).astype(np.int64)
    hh = np.rint(np.exp(np.log(h_median) + h_sigma * normal(seed, 14, b))).astype(np.int64)
    hh = np.clip(hh, 4, nz - 32)
    return np.stack([x0, y0, wx, wy, hh], axis=1)


def loglaw_profile(z, u_ref=0.05, z_ref=200.0, z0=0.5):
    """u(z) = u_ref ln(z_w/z0)/ln(z_ref/z0) with z_w = z - 0.5 the height above the ground face,
    clamped at 0."""
    zw = np.asarray(z, np.float64) - 0.5
    with np.errstate(divide="ignore", invalid="ignore"):
        u = u_ref * np.log(np.maximum(zw, 1e-30) / z0) / np.log(z_ref / z0)
    return np.clip(u, 0.0, None)


def canopy(nx=512, ny=512, nz=256, q=19, n_buildings=200, seed=2506, cs=0.1, nu=1e-4, crop=None,
           domain=None, wall_model=True, fringe=True, dtype=np.float32):
    """Urban canopy: solid ground z = 0, seeded box buildings, log-law inlet at x = 0, pressure outlet
    at x = nx-1 with a fringe zone over the last NX/8 planes (strength 0.2 xi^2), full-slip faces
    y = 0, y = ny-1, z = nz-1. Every fluid cell next to a solid gets the wall function. `domain` =
    (NX, NY, NZ) of the seeded geometry when it differs from the grid and `crop` = (x0, y0, z0)
    selects the sub-box that is simulated (the crop keeps the same face conditions and the domain's
    fringe layer: fringe = (L, s_max, p, first layer plane in crop coordinates))."""
    NX, NY, NZ = domain if domain is not None else (nx, ny, nz)
    ox, oy, oz = crop if crop is not None else (0, 0, 0)
    bl = canopy_buildings(NX, NY, NZ, n_buildings=n_buildings, seed=seed)
    x, y, z = _grid(nx, ny, nz)
    gx, gy, gz = x + ox, y + oy, z + oz
    solid3 = np.zeros((nz, ny, nx), bool)
    solid3[(gz.reshape(nz, ny, nx) == 0)] = True
    zs = np.arange(nz) + oz
    ys = np.arange(ny) + oy
    xs = np.arange(nx) + ox
    for (bx, by, wx, wy, hh) in bl:
        xm = (xs >= bx) & (xs < bx + wx)
        ym = (ys >= by) & (ys < by + wy)
        zm = (zs >= 0) & (zs < hh)
        if xm.any() and ym.any() and zm.any():
            solid3[np.ix_(zm, ym, xm)] = True
    mask = np.zeros(x.size, np.uint8)
    solid = solid3.reshape(-1)
    mask[solid] = MASK_SOLID
    mask[(x == 0) & ~solid] = MASK_INFLOW
    mask[(x == nx - 1) & ~solid] = MASK_OUTFLOW
    prof = loglaw_profile(zs)
    uin = np.zeros((3, ny * nz), np.float64)
    uin[0] = np.tile(prof[:, None], (1, ny)).reshape(-1)
    u = np.zeros((3, x.size), dtype)
    u[0] = prof[z]
    u[:, solid] = 0.0
    rho = np.ones(x.size, dtype)
    tau = 0.5 + 3.0 * nu
    fr = None
    if fringe:
        L = max(1, NX // 8)
        if NX - L - ox < nx:  # the layer reaches into the simulated box
            fr = (L, 0.2, 2.0, NX - L - ox)
    return Workload(name=f"canopy{nx}x{ny}x{nz}q{q}", q=q, nx=nx, ny=ny, nz=nz, tau=tau, cs=cs,
                    faces=(FACE_OPEN, FACE_OPEN, FACE_SLIP, FACE_SLIP, FACE_WALL, FACE_SLIP),
                    mask=mask, uin=uin, rho_out=1.0, wall_model=wall_model, rho0=rho, u0=u, fringe=fr,
                    meta=dict(buildings=bl, nu=nu, crop=crop, domain=(NX, NY, NZ)))


def smooth_field(shape, sigma, seed, stream=0):
    """White normal noise on a periodic grid (nz, ny, nx), Gaussian-blurred with standard deviation
    sigma cells (spectral multiplication by exp(-sigma^2 |k|^2 / 2)) and standardised."""
    nz, ny, nx = shape
    idx = np.arange(nx * ny * nz, dtype=np.uint64)
    w = normal(seed, stream, idx).reshape(shape)
    kz = np.fft.fftfreq(nz) * 2 * np.pi
    ky = np.fft.fftfreq(ny) * 2 * np.pi
    kx = np.fft.rfftfreq(nx) * 2 * np.pi
    K2 = kz[:, None, None] ** 2 + ky[None, :, None] ** 2 + kx[None, None, :] ** 2
    s = np.fft.irfftn(np.fft.rfftn(w) * np.exp(-0.5 * sigma * sigma * K2), s=shape, axes=(0, 1, 2))
    s = (s - s.mean()) / s.std()
    return s


def duct(n=128, u_in=0.04, tau=0.6, seed=1804, sigma=8.0, q=19, cs=0.0, dtype=np.float32):
    """Square duct for the differentiation workload: solid walls y, z in {0, n-1}, uniform inlet
    u_in at x = 0, pressure outlet rho = 1 at x = n-1, porosity gamma = sigmoid(2 + 2 s) with s a
    standardised smooth random field (correlation length sigma cells); starts at rest."""
    x, y, z = _grid(n, n, n)
    mask = np.zeros(x.size, np.uint8)
    solid = (y == 0) | (y == n - 1) | (z == 0) | (z == n - 1)
    mask[solid] = MASK_SOLID
    mask[(x == 0) & ~solid] = MASK_INFLOW
    mask[(x == n - 1) & ~solid] = MASK_OUTFLOW
    s = smooth_field((n, n, n), sigma, seed).reshape(-1)
    gamma = 1.0 / (1.0 + np.exp(-(2.0 + 2.0 * s)))
    uin = np.zeros((3, n * n), np.float64)
    ys = np.arange(n)
    inner = ((ys > 0) & (ys < n - 1))
    prof = np.outer(inner, inner).astype(np.float64).T.reshape(-1)  # index y + n*z
    uin[0] = u_in * prof
    rho = np.ones(x.size, dtype)
    u = np.zeros((3, x.size), dtype)
    return Workload(name=f"duct{n}", q=q, nx=n, ny=n, nz=n, tau=tau, cs=cs,
                    faces=(FACE_OPEN, FACE_OPEN, FACE_WALL, FACE_WALL, FACE_WALL, FACE_WALL),
                    mask=mask, uin=uin, rho_out=1.0, gamma=gamma.astype(np.float64), rho0=rho, u0=u,
                    meta=dict(u_in=u_in, inlet_profile=prof))


def random_box(nx, ny, nz, seed, q=19, solid_frac=0.1, tau=0.7, cs=0.1, faces=(0, 0, 0, 0, 0, 0), u_amp=0.03,
               inflow=False, outflow=False, dtype=np.float64):
    """Small randomised parity case: random solid cells, random velocity and density perturbations,
    optional inlet/outlet planes on x faces."""
    x, y, z = _grid(nx, ny, nz)
    N = x.size
    idx = np.arange(N, dtype=np.uint64)
    mask = np.where(uniform(seed, 20, idx) < solid_frac, MASK_SOLID, MASK_FLUID).astype(np.uint8)
    if inflow:
        mask[(x == 0) & (mask != MASK_SOLID)] = MASK_INFLOW
    if outflow:
        mask[(x == nx - 1) & (mask != MASK_SOLID)] = MASK_OUTFLOW
    u = np.stack([u_amp * (2 * uniform(seed, 21 + a, idx) - 1) for a in range(3)]).astype(dtype)
    rho = (1.0 + 0.01 * (2 * uniform(seed, 24, idx) - 1)).astype(dtype)
    u[:, mask == MASK_SOLID] = 0.0
    uin = np.zeros((3, ny * nz))
    uin[0] = 0.02 + 0.01 * uniform(seed, 25, np.arange(ny * nz, dtype=np.uint64))
    ywall = 0.3 + 0.4 * uniform(seed, 26, idx)
    return Workload(name=f"random{nx}x{ny}x{nz}", q=q, nx=nx, ny=ny, nz=nz, tau=tau, cs=cs, faces=tuple(faces),
                    mask=mask, ywall=ywall, uin=uin, rho_out=1.0, rho0=rho, u0=u)


GHOST = 2  # ghost planes per cut of a z-slab decomposition


def slab(w, parts, k):
    """Sub-domain k of a decomposition of workload w into `parts` z-slabs (layout only, no LB
    arithmetic). Slab k owns the planes [z0, z1), z0 = k nz // parts; every side that is a cut (both
    sides when z is periodic and parts > 1, else the inner ones) gets GHOST extra planes holding the
    neighbour's mask, wall distance, porosity, inlet velocity and initial state, with the z face of the
    sub-domain beyond them a bounce-back wall (it only shapes the classification of the outer ghost
    plane). Returns (workload, z0, z1, lo, hi), lo/hi the ghost planes below/above."""
    import dataclasses
    nz = w.nz
    z0, z1 = k * nz // parts, (k + 1) * nz // parts
    if z1 - z0 < GHOST:
        raise ValueError("every slab needs at least %d planes" % GHOST)
    periodic = w.faces[4] == FACE_PERIODIC
    if parts == 1:
        return w, 0, nz, 0, 0
    lo = GHOST if (periodic or k > 0) else 0
    hi = GHOST if (periodic or k < parts - 1) else 0
    zs = np.arange(z0 - lo, z1 + hi) % nz
    nxy = w.nx * w.ny
    cells = (zs[:, None] * nxy + np.arange(nxy)[None, :]).reshape(-1)
    faces = list(w.faces)
    faces[4] = FACE_WALL if lo else w.faces[4]
    faces[5] = FACE_WALL if hi else w.faces[5]
    if faces[4] == FACE_PERIODIC and faces[5] != FACE_PERIODIC:
        faces[4] = FACE_WALL
    if faces[5] == FACE_PERIODIC and faces[4] != FACE_PERIODIC:
        faces[5] = FACE_WALL

    def cut(a):
        return None if a is None else np.asarray(a)[..., cells].copy()

    uin = None
    if w.uin is not None:
        cols = (zs[:, None] * w.ny + np.arange(w.ny)[None, :]).reshape(-1)
        uin = np.asarray(w.uin)[:, cols].copy()
    sub = dataclasses.replace(w, name=f"{w.name}_slab{k}of{parts}", nz=len(zs), faces=tuple(faces),
                              mask=cut(w.mask), ywall=cut(w.ywall), gamma=cut(w.gamma), uin=uin,
                              rho0=cut(w.rho0), u0=cut(w.u0), meta=dict(w.meta, slab=(k, parts, z0, z1, lo, hi)))
    return sub, z0, z1, lo, hi
