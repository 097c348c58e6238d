"""Shared test helpers: build an oracle instance from a seeded workload."""
import numpy as np

from oracle import oracle as O


def oracle_from(w, storage=0):
    o = O.Oracle(w.q, w.nx, w.ny, w.nz, w.tau, w.cs)
    o.set_faces(w.faces)
    o.set_geometry(w.mask, w.ywall)
    o.set_force(*w.force)
    if w.uin is not None:
        o.set_inflow(w.uin)
    o.set_outflow(w.rho_out)
    if w.gamma is not None:
        o.set_porosity(w.gamma)
    o.set_wall_model(w.wall_model, w.kappa, w.E)
    o.set_storage(storage)
    o.init_equilibrium(np.asarray(w.rho0, np.float64), np.asarray(w.u0, np.float64))
    return o
