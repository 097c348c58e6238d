"""ctypes binding of the FP64 CPU oracle (lbm_oracle.cpp).

TEST INFRASTRUCTURE ONLY: imported by tests/, by the smoke check and by the benchmark's CPU
baseline leg. It never imports the CUDA package and the CUDA package never imports it.

Array conventions (same as the C ABI of the CUDA library, but implemented independently):
  cell index n = x + nx*(y + ny*z); populations f[i*N + n]; velocities u[a*N + n];
  inlet velocity uin[a*ny*nz + y + ny*z].
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None

FACE_PERIODIC, FACE_WALL, FACE_SLIP, FACE_OPEN = 0, 1, 2, 3
MASK_FLUID, MASK_SOLID, MASK_INFLOW, MASK_OUTFLOW = 0, 1, 3, 4
KIND_FLUID, KIND_SOLID, KIND_WALL, KIND_INFLOW, KIND_OUTFLOW = 0, 1, 2, 3, 4

_d = ctypes.c_double
_i = ctypes.c_int
_p = ctypes.c_void_p


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        sig = {
            "orc_create": (_p, [_i, _i, _i, _i, _d, _d]),
            "orc_destroy": (None, [_p]),
            "orc_last_error": (ctypes.c_char_p, []),
            "orc_lattice": (_i, [_i, _p, _p, _p, _p, _p]),
            "orc_set_faces": (_i, [_p, _p]),
            "orc_set_geometry": (_i, [_p, _p, _p]),
            "orc_set_force": (None, [_p, _d, _d, _d]),
            "orc_set_inflow": (None, [_p, _p]),
            "orc_set_outflow": (None, [_p, _d]),
            "orc_set_fringe": (_i, [_p, _i, _d, _d, _i]),
            "orc_fringe_strength": (_d, [_p, _i]),
            "orc_set_porosity": (None, [_p, _p]),
            "orc_set_wall_model": (None, [_p, _i, _d, _d]),
            "orc_set_storage": (None, [_p, _i]),
            "orc_set_collision": (_i, [_p, _i, _d]),
            "orc_get_collision": (_i, [_p, _p]),
            "orc_third_order": (_i, [_i, _p, _p]),
            "orc_feq3": (_i, [_i, _d, _p, _p]),
            "orc_collide_hrr": (_i, [_i, _d, _p, _p, _d, _p, _p]),
            "orc_strain_fd": (None, [_p, ctypes.c_longlong, _p]),
            "orc_get_velocity_field": (None, [_p, _p]),
            "orc_set_velocity_field": (None, [_p, _p]),
            "orc_set_vortex_inlet": (_i, [_p, _i, _d, _d, ctypes.c_ulonglong]),
            "orc_forchheimer_k": (_d, [_d, _d, _d, _d, _d, _d, _d]),
            "orc_set_permeability": (None, [_p, _p]),
            "orc_get_porosity": (None, [_p, _p]),
            "orc_vm_vortices": (None, [_p, ctypes.c_longlong, _p]),
            "orc_vm_field": (None, [_i, _p, _d, _d, _d, _p]),
            "orc_inflow_field": (None, [_p, _p]),
            "orc_splitmix64": (ctypes.c_ulonglong, [ctypes.c_ulonglong]),
            "orc_vm_uniform": (_d, [ctypes.c_ulonglong, ctypes.c_ulonglong]),
            "orc_init_equilibrium": (None, [_p, _p, _p]),
            "orc_set_populations": (None, [_p, _p]),
            "orc_get_populations": (None, [_p, _p]),
            "orc_get_refbuf": (None, [_p, _p]),
            "orc_step": (None, [_p, _i]),
            "orc_moments": (None, [_p, _p, _p]),
            "orc_reduce": (None, [_p, _p, _p]),
            "orc_classification": (None, [_p, _p, _p, _p, _p]),
            "orc_source_map": (None, [_p, _p, _p]),
            "orc_spalding_yplus": (_d, [_d, _d, _d]),
            "orc_spalding_dyplus": (_d, [_d, _d, _d]),
            "orc_solve_uplus_re": (_d, [_d, _d, _d, _p]),
            "orc_solve_uplus_yplus": (_d, [_d, _d, _d, _p]),
            "orc_tau_smagorinsky": (_d, [_d, _d, _p, _d]),
            "orc_feq": (None, [_i, _d, _p, _p]),
            "orc_bc": (None, [_i, _i, _p, _p, _d]),
            "orc_wall_state": (_i, [_p, ctypes.c_longlong, _p, _p]),
            "orc_f16_encode": (ctypes.c_uint16, [_d]),
            "orc_f16_decode": (_d, [ctypes.c_uint16]),
            "orc_bf16_encode": (ctypes.c_uint16, [_d]),
            "orc_bf16_decode": (_d, [ctypes.c_uint16]),
            "orc_jvp_step": (None, [_p, _p, _p, _p, _p]),
            "orc_vjp_step": (None, [_p, _p, _p, _p, _p]),
            "orc_objective_run": (_i, [_p, _i, _i, _i, _i, _p]),
            "orc_adjoint": (_i, [_p, _p, _p]),
            "orc_set_threads": (None, [_i]),
            "orc_set_ghost": (_i, [_p, _i, _i]),
            "orc_step_collide": (None, [_p]),
            "orc_step_stream": (None, [_p]),
            "orc_halo_count": (ctypes.c_longlong, [_p, _i, _i]),
            "orc_halo_list": (None, [_p, _i, _i, _p]),
            "orc_halo_pack": (None, [_p, _i, _i, _p]),
            "orc_halo_unpack": (None, [_p, _i, _i, _p]),
            "orc_get_threads": (_i, []),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def lattice(q):
    """Velocity set of the oracle: c (q,3) int, w (q,), opp (q,), integer weights W, denominator."""
    c = np.zeros((q, 3), np.int32)
    w = np.zeros(q)
    opp = np.zeros(q, np.int32)
    W = np.zeros(q, np.int32)
    den = ctypes.c_int()
    if lib().orc_lattice(q, _ptr(c), _ptr(w), _ptr(opp), _ptr(W), ctypes.byref(den)):
        raise ValueError("lattice must be 19 or 27")
    return c, w, opp, W, den.value


def third_order(q, a):
    """Third-order Hermite term of every population for the symmetric 3x3x3 tensor a."""
    a = _f64(np.asarray(a).reshape(27))
    out = np.zeros(q)
    if lib().orc_third_order(q, _ptr(a), _ptr(out)):
        raise ValueError("lattice must be 19 or 27")
    return out


def feq3(q, rho, u):
    """Third-order equilibrium f^eq_i(rho, u)."""
    uu = _f64(np.asarray(u).reshape(3))
    out = np.zeros(q)
    if lib().orc_feq3(q, float(rho), _ptr(uu), _ptr(out)):
        raise ValueError("lattice must be 19 or 27")
    return out


def collide_hrr(q, rho, ueq, uh, tau, A2):
    """One HRR update from (rho, equilibrium velocity, expansion velocity, tau, A2)."""
    ue = _f64(np.asarray(ueq).reshape(3))
    uh = _f64(np.asarray(uh).reshape(3))
    A = _f64(np.asarray(A2).reshape(9))
    out = np.zeros(q)
    if lib().orc_collide_hrr(q, float(rho), _ptr(ue), _ptr(uh), float(tau), _ptr(A), _ptr(out)):
        raise ValueError("lattice must be 19 or 27")
    return out


def forchheimer_k(mu, Q, A, L, dP, rho, Kbeta=float("inf")):
    return lib().orc_forchheimer_k(mu, Q, A, L, dP, rho, Kbeta)


def splitmix64(z):
    return lib().orc_splitmix64(int(z) & 0xFFFFFFFFFFFFFFFF)


def vm_uniform(seed, counter):
    return lib().orc_vm_uniform(int(seed), int(counter))


def vm_field(vortices, sigma, y, z):
    """In-plane velocity (u_y, u_z) of vortices (rows y, z, Gamma) at plane position (y, z)."""
    v = _f64(np.asarray(vortices).reshape(-1))
    out = np.zeros(2)
    lib().orc_vm_field(len(v) // 3, _ptr(v), float(sigma), float(y), float(z), _ptr(out))
    return out


def set_threads(n):
    lib().orc_set_threads(int(n))


def get_threads():
    return lib().orc_get_threads()


def spalding_yplus(up, kappa=0.41, E=9.52):
    return lib().orc_spalding_yplus(up, kappa, E)


def spalding_dyplus(up, kappa=0.41, E=9.52):
    return lib().orc_spalding_dyplus(up, kappa, E)


def solve_uplus_re(Re, kappa=0.41, E=9.52):
    it = ctypes.c_int()
    u = lib().orc_solve_uplus_re(Re, kappa, E, ctypes.byref(it))
    return u, it.value


def solve_uplus_yplus(yp, kappa=0.41, E=9.52):
    it = ctypes.c_int()
    u = lib().orc_solve_uplus_yplus(yp, kappa, E, ctypes.byref(it))
    return u, it.value


def tau_smagorinsky(tau0, cs, Pi, rho):
    Pi = _f64(np.asarray(Pi).reshape(9))
    return lib().orc_tau_smagorinsky(tau0, cs, _ptr(Pi), rho)


def feq(q, rho, u):
    u = _f64(u)
    out = np.zeros(q)
    lib().orc_feq(q, rho, _ptr(u), _ptr(out))
    return out


def bc(q, kind, f, ub=(0.0, 0.0, 0.0), rho_out=1.0):
    f = _f64(f).copy()
    ub = _f64(ub)
    lib().orc_bc(q, kind, _ptr(f), _ptr(ub), rho_out)
    return f


def f16_encode(x):
    return lib().orc_f16_encode(float(x))


def f16_decode(b):
    return lib().orc_f16_decode(int(b))


def bf16_encode(x):
    return lib().orc_bf16_encode(float(x))


def bf16_decode(b):
    return lib().orc_bf16_decode(int(b))


class Oracle:
    """One FP64 lattice: populations, geometry and boundary settings."""

    def __init__(self, q, nx, ny, nz, tau, cs=0.0):
        self.q, self.nx, self.ny, self.nz = q, nx, ny, nz
        self.N = nx * ny * nz
        self.h = lib().orc_create(q, nx, ny, nz, tau, cs)
        if not self.h:
            raise ValueError(lib().orc_last_error().decode())

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_destroy(self.h)
            self.h = None

    def _chk(self, rc):
        if rc:
            raise ValueError(lib().orc_last_error().decode())

    def set_faces(self, kinds):
        k = np.ascontiguousarray(kinds, dtype=np.int32)
        assert k.size == 6
        self._chk(lib().orc_set_faces(self.h, _ptr(k)))

    def set_geometry(self, mask, ywall=None):
        m = np.ascontiguousarray(mask, dtype=np.uint8).reshape(-1)
        assert m.size == self.N
        y = _f64(None if ywall is None else np.asarray(ywall).reshape(-1))
        self._chk(lib().orc_set_geometry(self.h, _ptr(m), _ptr(y)))

    def set_force(self, fx, fy, fz):
        lib().orc_set_force(self.h, fx, fy, fz)

    def set_inflow(self, uin):
        u = _f64(np.asarray(uin).reshape(-1))
        assert u.size == 3 * self.ny * self.nz
        lib().orc_set_inflow(self.h, _ptr(u))

    def set_outflow(self, rho):
        lib().orc_set_outflow(self.h, rho)

    def set_fringe(self, L, s_max, p=2.0, x0=None):
        """Outlet fringe zone over the last L planes (L = 0: off), strength s_max xi^p with
        xi = (x - x0 + 1)/L; x0 = nx - L unless given (a crop keeps its domain's layer)."""
        x0 = self.nx - int(L) if x0 is None else int(x0)
        self._chk(lib().orc_set_fringe(self.h, int(L), float(s_max), float(p), x0))

    def fringe_strength(self, x):
        return lib().orc_fringe_strength(self.h, int(x))

    def set_porosity(self, gamma):
        g = _f64(None if gamma is None else np.asarray(gamma).reshape(-1))
        lib().orc_set_porosity(self.h, _ptr(g))

    def set_permeability(self, K):
        """Porosity from the per-cell permeability K (lattice units; inf = fluid)."""
        k = _f64(np.asarray(K).reshape(-1))
        lib().orc_set_permeability(self.h, _ptr(k))

    def porosity(self):
        g = np.zeros(self.N)
        lib().orc_get_porosity(self.h, _ptr(g))
        return g

    def set_wall_model(self, on=True, kappa=0.41, E=9.52):
        lib().orc_set_wall_model(self.h, int(on), kappa, E)

    def set_storage(self, mode):
        lib().orc_set_storage(self.h, int(mode))

    def set_collision(self, model, sigma=1.0):
        """model 0: BGK; 1: hybrid recursive regularised with hybridisation factor sigma."""
        self._chk(lib().orc_set_collision(self.h, int(model), float(sigma)))

    def collision(self):
        s = np.zeros(1)
        return lib().orc_get_collision(self.h, _ptr(s)), s[0]

    def strain_fd(self, n):
        S = np.zeros(9)
        lib().orc_strain_fd(self.h, int(n), _ptr(S))
        return S.reshape(3, 3)

    def velocity_field(self):
        u = np.zeros(3 * self.N)
        lib().orc_get_velocity_field(self.h, _ptr(u))
        return u.reshape(3, self.N)

    def set_velocity_field(self, u):
        u = _f64(np.asarray(u).reshape(-1))
        lib().orc_set_velocity_field(self.h, _ptr(u))

    def set_vortex_inlet(self, n, sigma=4.0, intensity=0.1, seed=0):
        """Vortex-method inlet with n vortices per step (0: off)."""
        self._chk(lib().orc_set_vortex_inlet(self.h, int(n), float(sigma), float(intensity), int(seed)))
        self.vm_n = int(n)

    def vortices(self, t):
        """Vortices of step t, rows (y, z, Gamma)."""
        n = getattr(self, "vm_n", 0)
        out = np.zeros(3 * max(n, 1))
        lib().orc_vm_vortices(self.h, int(t), _ptr(out))
        return out.reshape(-1, 3)[:n]

    def inflow_field(self):
        out = np.zeros(3 * self.ny * self.nz)
        lib().orc_inflow_field(self.h, _ptr(out))
        return out.reshape(3, self.ny * self.nz)

    def _bgk_only(self):
        if self.collision()[0] != 0:
            raise RuntimeError("the adjoint is defined for the BGK collision only")

    def init_equilibrium(self, rho, u):
        r = _f64(np.asarray(rho).reshape(-1))
        uu = _f64(np.asarray(u).reshape(-1))
        lib().orc_init_equilibrium(self.h, _ptr(r), _ptr(uu))

    def set_populations(self, f):
        f = _f64(np.asarray(f).reshape(-1))
        lib().orc_set_populations(self.h, _ptr(f))

    def populations(self):
        f = np.zeros(self.q * self.N)
        lib().orc_get_populations(self.h, _ptr(f))
        return f.reshape(self.q, self.N)

    def refbuf(self):
        u = np.zeros(3 * self.N)
        lib().orc_get_refbuf(self.h, _ptr(u))
        return u.reshape(self.N, 3)

    def step(self, n=1):
        lib().orc_step(self.h, int(n))

    # ---- slab sub-domain (z decomposition) -------------------------------------------------------
    def set_ghost(self, lo, hi):
        """First lo and last hi z-planes are ghost planes (0 or 2 each)."""
        self._chk(lib().orc_set_ghost(self.h, int(lo), int(hi)))

    def step_collide(self):
        lib().orc_step_collide(self.h)

    def step_stream(self):
        lib().orc_step_stream(self.h)

    def halo_list(self, side, which):
        n = lib().orc_halo_count(self.h, int(side), int(which))
        out = np.zeros(max(n, 1), np.int64)
        lib().orc_halo_list(self.h, int(side), int(which), _ptr(out))
        return out[:n]

    def halo_pack(self, side, which):
        n = lib().orc_halo_count(self.h, int(side), int(which))
        buf = np.zeros(max(n, 1) * (1 if which == 0 else 3))
        lib().orc_halo_pack(self.h, int(side), int(which), _ptr(buf))
        return buf[: n * (1 if which == 0 else 3)]

    def halo_unpack(self, side, which, buf):
        b = _f64(np.asarray(buf).reshape(-1))
        lib().orc_halo_unpack(self.h, int(side), int(which), _ptr(b))

    def moments(self):
        rho = np.zeros(self.N)
        u = np.zeros(3 * self.N)
        lib().orc_moments(self.h, _ptr(rho), _ptr(u))
        return rho, u.reshape(3, self.N)

    def reduce(self):
        m = np.zeros(1)
        p = np.zeros(3)
        lib().orc_reduce(self.h, _ptr(m), _ptr(p))
        return m[0], p

    def classification(self):
        kind = np.zeros(self.N, np.uint8)
        isref = np.zeros(self.N, np.uint8)
        nsum = np.zeros(3 * self.N, np.int32)
        ref = np.zeros(self.N, np.int64)
        lib().orc_classification(self.h, _ptr(kind), _ptr(isref), _ptr(nsum), _ptr(ref))
        return kind, isref, nsum.reshape(self.N, 3), ref

    def boundary_list(self):
        """Sorted cell indices handled by the boundary-cell pass: WALL, INFLOW, OUTFLOW or reference
        cells; and for each entry the list position of its reference cell (-1 if none)."""
        kind, isref, _, ref = self.classification()
        sel = (kind == KIND_WALL) | (kind == KIND_INFLOW) | (kind == KIND_OUTFLOW) | (isref == 1)
        cells = np.nonzero(sel)[0].astype(np.int64)
        pos = {int(c): k for k, c in enumerate(cells)}
        refpos = np.array([pos[int(ref[c])] if ref[c] >= 0 else -1 for c in cells], dtype=np.int64)
        return cells, refpos

    def source_map(self):
        d = np.zeros(self.q * self.N, np.int32)
        c = np.zeros(self.q * self.N, np.int64)
        lib().orc_source_map(self.h, _ptr(d), _ptr(c))
        return d.reshape(self.q, self.N), c.reshape(self.q, self.N)

    def wall_state(self, n):
        uB = np.zeros(3)
        d = np.zeros(1)
        self._chk(lib().orc_wall_state(self.h, int(n), _ptr(uB), _ptr(d)))
        return uB, d[0]

    def jvp_step(self, vf, vg=None, vu=None):
        self._bgk_only()
        vf = _f64(np.asarray(vf).reshape(-1))
        vg = _f64(None if vg is None else np.asarray(vg).reshape(-1))
        vu = _f64(None if vu is None else np.asarray(vu).reshape(-1))
        out = np.zeros(self.q * self.N)
        lib().orc_jvp_step(self.h, _ptr(vf), _ptr(vg), _ptr(vu), _ptr(out))
        return out.reshape(self.q, self.N)

    def vjp_step(self, w):
        self._bgk_only()
        w = _f64(np.asarray(w).reshape(-1))
        of = np.zeros(self.q * self.N)
        og = np.zeros(self.N)
        ou = np.zeros(3 * self.ny * self.nz)
        lib().orc_vjp_step(self.h, _ptr(w), _ptr(of), _ptr(og), _ptr(ou))
        return of.reshape(self.q, self.N), og, ou

    def objective_run(self, T, W, xa, xb):
        J = np.zeros(1)
        self._chk(lib().orc_objective_run(self.h, int(T), int(W), int(xa), int(xb), _ptr(J)))
        return J[0]

    def adjoint(self):
        g = np.zeros(self.N)
        u = np.zeros(3 * self.ny * self.nz)
        self._chk(lib().orc_adjoint(self.h, _ptr(g), _ptr(u)))
        return g, u.reshape(3, self.ny * self.nz)
