"""Shared test helpers: oracle and GPU lattices built from the same seeded workload."""
import numpy as np

from oracle import oracle as O
from paper_2506_21804_gb300 import inputs as I


def _arr(a, cast32):
    if a is None:
        return None
    a = np.asarray(a, np.float64)
    return a.astype(np.float32).astype(np.float64) if cast32 else a


def oracle_from(w, storage=0, cast32=False):
    """Oracle instance for workload w. cast32 rounds every real input through float32 first, so
    that an FP32 GPU run and the oracle start from identical numbers."""
    o = O.Oracle(w.q, w.nx, w.ny, w.nz, w.tau, w.cs)
    o.set_faces(w.faces)
    o.set_geometry(w.mask, None if w.ywall is None else _arr(w.ywall, True))
    o.set_force(*w.force)
    if w.uin is not None:
        o.set_inflow(_arr(w.uin, cast32))
    o.set_outflow(w.rho_out)
    if w.gamma is not None:
        o.set_porosity(_arr(w.gamma, cast32))
    o.set_wall_model(w.wall_model, w.kappa, w.E)
    o.set_storage(storage)
    if getattr(w, "model", 0):
        o.set_collision(w.model, w.sigma)
    if getattr(w, "vortex", None):
        o.set_vortex_inlet(*w.vortex)
    if getattr(w, "fringe", None):
        o.set_fringe(*w.fringe)
    o.init_equilibrium(_arr(w.rho0, cast32), _arr(w.u0, cast32))
    return o


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300))


def small_cases(q=19):
    return [
        I.random_box(9, 7, 6, seed=1, q=q, solid_frac=0.15, tau=0.62, cs=0.12, faces=(0, 0, 0, 0, 0, 0)),
        I.random_box(10, 7, 5, seed=2, q=q, solid_frac=0.1, tau=0.55, cs=0.1, faces=(3, 3, 2, 2, 1, 2),
                     inflow=True, outflow=True),
        I.random_box(8, 6, 7, seed=3, q=q, solid_frac=0.2, tau=0.8, cs=0.0, faces=(2, 2, 2, 2, 2, 2)),
        I.random_box(33, 5, 4, seed=4, q=q, solid_frac=0.05, tau=0.7, cs=0.15, faces=(1, 1, 2, 2, 0, 0)),
        I.canopy(nx=40, ny=24, nz=20, q=q, n_buildings=6, seed=2506, domain=(200, 24, 60), crop=(64, 0, 0),
                 dtype=np.float64),
        I.channel(nx=16, ny=14, nz=6, q=q, noise=0.05, seed=5, dtype=np.float64),
        I.duct(n=10, q=q, u_in=0.03, tau=0.7, sigma=2.0, cs=0.1, dtype=np.float64),
    ]


def with_features(w):
    """Switch on force, porosity and the wall model where the case has room for them."""
    rng = np.random.default_rng(w.nx * 7 + w.ny)
    if w.gamma is None and w.name.startswith("random"):
        w.gamma = 0.7 + 0.3 * rng.random(w.N)
    if w.name.startswith("random") and w.faces[0] != 3:
        w.force = (2e-6, -1e-6, 5e-7)
    w.wall_model = True
    return w
