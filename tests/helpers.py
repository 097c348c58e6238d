"""Shared test helpers: oracle and GPU lattices built from the same seeded workload."""
import numpy as np

from oracle import oracle as O


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
    o.init_equilibrium(_arr(w.rho0, cast32), _arr(w.u0, cast32))
    return o


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300))
