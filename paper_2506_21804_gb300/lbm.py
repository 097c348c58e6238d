"""Python binding of liblbm.so (include/lbm.h): argument marshalling only.

Every computation runs in the library's CUDA kernels. Arrays may be numpy arrays (host) or torch
tensors (host or CUDA); outputs default to new numpy arrays. The library must have been built
(`paper_2506_21804_gb300.build.build()` or `__graft_entry__.build()`); importing this module on a
machine without it raises instead of falling back to anything else.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "liblbm.so")

D3Q19, D3Q27 = 19, 27
F64, F32, F16, BF16 = 0, 1, 2, 3
OK, EINVAL, ENOMEM, ECUDA, ENAN, ETIMEOUT, ESTATE = range(7)
DTYPE_F64, DTYPE_F32 = 0, 1
FACE_PERIODIC, FACE_WALL, FACE_SLIP, FACE_OPEN = 0, 1, 2, 3
KIND_FLUID, KIND_SOLID, KIND_WALL, KIND_INFLOW, KIND_OUTFLOW = 0, 1, 2, 3, 4
T_KIND, T_REF, T_NEAR, T_LIST = 7, 8, 16, 32
OPT_KERNEL, OPT_DEBUG_STALL = 1, 2
KERNEL_PLAIN, KERNEL_STAGED = 0, 2
BGK, HRR = 0, 1
STORAGE_NAMES = {"f64": F64, "f32": F32, "f16": F16, "bf16": BF16}

_ERR_NAMES = {EINVAL: "LBM_EINVAL", ENOMEM: "LBM_ENOMEM", ECUDA: "LBM_ECUDA", ENAN: "LBM_ENAN",
              ETIMEOUT: "LBM_ETIMEOUT", ESTATE: "LBM_ESTATE"}


class LBMError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_ERR_NAMES.get(code, code)}: {msg}")
        self.code = code


_lib = None
_p = ctypes.c_void_p
_i = ctypes.c_int
_d = ctypes.c_double

SIGNATURES = {
    "lbm_create": (_p, [_i, _i, _i, _i, _d, _d]),
    "lbm_destroy": (None, [_p]),
    "lbm_last_error": (ctypes.c_char_p, []),
    "lbm_set_precision": (_i, [_p, _i]),
    "lbm_set_collision": (_i, [_p, _i, _d]),
    "lbm_interior_kernel": (_i, [_p]),
    "lbm_set_vortex_inlet": (_i, [_p, _i, _d, _d, ctypes.c_ulonglong]),
    "lbm_set_permeability": (_i, [_p, _p]),
    "lbm_set_permeability_ex": (_i, [_p, _p, _i]),
    "lbm_forchheimer_permeability": (_d, [_d, _d, _d, _d, _d, _d, _d]),
    "lbm_set_periodic": (_i, [_p, _i, _i, _i]),
    "lbm_set_faces": (_i, [_p, _p]),
    "lbm_set_geometry": (_i, [_p, _p, _p]),
    "lbm_set_force": (_i, [_p, _d, _d, _d]),
    "lbm_set_inflow": (_i, [_p, _p]),
    "lbm_set_inflow_ex": (_i, [_p, _p, _i]),
    "lbm_set_outflow": (_i, [_p, _d]),
    "lbm_set_porosity": (_i, [_p, _p]),
    "lbm_set_porosity_ex": (_i, [_p, _p, _i]),
    "lbm_set_wall_model": (_i, [_p, _d, _d]),
    "lbm_init_equilibrium": (_i, [_p, _p, _p]),
    "lbm_init_equilibrium_ex": (_i, [_p, _p, _p, _i]),
    "lbm_step": (_i, [_p, _i]),
    "lbm_step_timed": (_i, [_p, _i, _p]),
    "lbm_sync": (_i, [_p]),
    "lbm_moments": (_i, [_p, _p, _p]),
    "lbm_moments_ex": (_i, [_p, _p, _p, _i]),
    "lbm_reduce": (_i, [_p, _p, _p]),
    "lbm_get_populations": (_i, [_p, _p, _i]),
    "lbm_set_populations": (_i, [_p, _p, _i]),
    "lbm_objective_forward": (_i, [_p, _i, _i, _i, _i, _i, _p]),
    "lbm_objective_backward": (_i, [_p, _p, _p]),
    "lbm_adjoint_step": (_i, [_p, _p, _p, _i, _p, _p]),
    "lbm_adjoint_timing": (_i, [_p, _p]),
    "lbm_save": (_i, [_p, _p, _p]),
    "lbm_load": (_i, [_p, _p, ctypes.c_size_t]),
    "lbm_set_stream": (_i, [_p, _p]),
    "lbm_info": (_i, [_p, _p]),
    "lbm_set_option": (_i, [_p, _i, _i]),
    "lbm_reduce_static": (_i, [_i, _p, _i, _p, ctypes.c_int64, _p, _p]),
    "lbm_launch_count": (_i, [_p, _p]),
    "lbm_set_fringe": (_i, [_p, _i, _d, _d]),
    "lbm_set_ghost_planes": (_i, [_p, _i, _i]),
    "lbm_halo_count": (_i, [_p, _i, _i, _p]),
    "lbm_halo_pack": (_i, [_p, _i, _i, _p]),
    "lbm_halo_unpack": (_i, [_p, _i, _i, _p]),
    "lbm_reduce_static_error": (ctypes.c_char_p, []),
    "lbm_debug_dump": (_i, [_p, _i, _p, ctypes.c_size_t]),
}


def lib():
    """Load liblbm.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(rc):
    if rc != OK:
        raise LBMError(rc, lib().lbm_last_error().decode())


def _is_torch(x):
    return type(x).__module__.startswith("torch")


class _Arr:
    """Pointer + dtype code of an input array, keeping the owner alive."""

    def __init__(self, x, dtype=None, default=np.float32):
        if _is_torch(x):
            t = x.contiguous()
            if dtype is not None:
                import torch
                t = t.to({np.float32: torch.float32, np.float64: torch.float64, np.uint8: torch.uint8}[dtype])
            self.obj = t
            self.ptr = ctypes.c_void_p(t.data_ptr())
            name = str(t.dtype)
            self.code = DTYPE_F64 if name == "torch.float64" else DTYPE_F32
            self.nbytes = t.numel() * t.element_size()
        else:
            a = np.asarray(x)
            want = dtype if dtype is not None else (a.dtype if a.dtype in (np.float32, np.float64) else default)
            a = np.ascontiguousarray(a, dtype=want)
            self.obj = a
            self.ptr = a.ctypes.data_as(ctypes.c_void_p)
            self.code = DTYPE_F64 if a.dtype == np.float64 else DTYPE_F32
            self.nbytes = a.nbytes


def forchheimer_permeability(mu, Q, A, L, dP, rho, K_beta=float("inf")):
    """Forchheimer permeability of a sample (K_beta = inf: Darcy's law)."""
    return lib().lbm_forchheimer_permeability(float(mu), float(Q), float(A), float(L), float(dP), float(rho),
                                              float(K_beta))


class Lattice:
    """One lattice on the current CUDA device (owns its device memory through liblbm)."""

    def __init__(self, q, nx, ny, nz, tau, c_smag=0.0, storage=F32):
        self.q, self.nx, self.ny, self.nz = q, nx, ny, nz
        self.N = nx * ny * nz
        h = lib().lbm_create(q, nx, ny, nz, float(tau), float(c_smag))
        if not h:
            raise LBMError(EINVAL, lib().lbm_last_error().decode())
        self.h = h
        self.storage = F32
        if storage != F32:
            self.set_precision(storage)

    def close(self):
        if getattr(self, "h", None):
            lib().lbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- configuration -------------------------------------------------------------------------------
    def set_precision(self, storage):
        _check(lib().lbm_set_precision(self.h, int(storage)))
        self.storage = int(storage)

    def set_periodic(self, px, py, pz):
        _check(lib().lbm_set_periodic(self.h, int(px), int(py), int(pz)))

    def set_faces(self, kinds):
        k = np.ascontiguousarray(kinds, dtype=np.int32)
        _check(lib().lbm_set_faces(self.h, k.ctypes.data_as(_p)))

    def set_geometry(self, mask, wall_dist=None):
        m = _Arr(mask, dtype=np.uint8)
        w = None if wall_dist is None else _Arr(wall_dist, dtype=np.float32)
        _check(lib().lbm_set_geometry(self.h, m.ptr, None if w is None else w.ptr))

    def set_force(self, fx, fy, fz):
        _check(lib().lbm_set_force(self.h, float(fx), float(fy), float(fz)))

    def set_inflow(self, u_in):
        a = _Arr(u_in)
        _check(lib().lbm_set_inflow_ex(self.h, a.ptr, a.code))

    def set_outflow(self, rho_out):
        _check(lib().lbm_set_outflow(self.h, float(rho_out)))

    def set_fringe(self, L, s_max, p=2.0):
        """Outlet fringe zone over the last L planes (L = 0: off), strength s_max xi^p."""
        _check(lib().lbm_set_fringe(self.h, int(L), float(s_max), float(p)))

    def set_ghost_planes(self, lo, hi):
        """Slab sub-domain: the first lo and last hi z-planes (0 or 2) are ghost planes."""
        _check(lib().lbm_set_ghost_planes(self.h, int(lo), int(hi)))

    def halo_count(self, side, which):
        n = np.zeros(1, np.int64)
        _check(lib().lbm_halo_count(self.h, int(side), int(which), n.ctypes.data_as(_p)))
        return int(n[0])

    def halo_pack(self, side, which, buf):
        """Pack halo list `which` of `side` into buf (a torch tensor or numpy array of the right size)."""
        ptr = ctypes.c_void_p(buf.data_ptr()) if _is_torch(buf) else buf.ctypes.data_as(_p)
        _check(lib().lbm_halo_pack(self.h, int(side), int(which), ptr))
        return buf

    def halo_unpack(self, side, which, buf):
        ptr = ctypes.c_void_p(buf.data_ptr()) if _is_torch(buf) else np.ascontiguousarray(buf).ctypes.data_as(_p)
        _check(lib().lbm_halo_unpack(self.h, int(side), int(which), ptr))

    def set_porosity(self, gamma):
        if gamma is None:
            _check(lib().lbm_set_porosity_ex(self.h, None, DTYPE_F32))
            return
        a = _Arr(gamma)
        _check(lib().lbm_set_porosity_ex(self.h, a.ptr, a.code))

    def set_permeability(self, K):
        """Porosity from the per-cell permeability K (lattice units; inf = fluid)."""
        a = _Arr(K)
        _check(lib().lbm_set_permeability_ex(self.h, a.ptr, a.code))

    def set_wall_model(self, kappa=0.41, E=9.52):
        _check(lib().lbm_set_wall_model(self.h, float(kappa), float(E)))

    def interior_kernel(self):
        """0: one cell per thread, 1: cell pairs, 2: staged, 3: four cells per thread on even steps,
        pairs on odd steps (16-bit D3Q19)."""
        k = lib().lbm_interior_kernel(self.h)
        if k < 0:
            raise LBMError(EINVAL, lib().lbm_last_error().decode())
        return k

    def set_vortex_inlet(self, n, sigma=4.0, intensity=0.1, seed=0):
        """Vortex-method inlet with n vortices per step (0: off)."""
        _check(lib().lbm_set_vortex_inlet(self.h, int(n), float(sigma), float(intensity), int(seed)))

    def set_collision(self, model, sigma=1.0):
        """BGK (model 0) or the hybrid recursive regularised collision (model 1, HRR) with
        hybridisation factor sigma."""
        _check(lib().lbm_set_collision(self.h, int(model), float(sigma)))

    def set_stream(self, stream):
        ptr = stream if isinstance(stream, int) else getattr(stream, "cuda_stream", 0)
        _check(lib().lbm_set_stream(self.h, ctypes.c_void_p(ptr)))

    def init_equilibrium(self, rho, u):
        r = _Arr(rho)
        v = _Arr(u, dtype=np.float64 if r.code == DTYPE_F64 else np.float32) if not _is_torch(u) else _Arr(u)
        if r.code != v.code:
            raise ValueError("rho and u must have the same dtype")
        _check(lib().lbm_init_equilibrium_ex(self.h, r.ptr, v.ptr, r.code))

    # ---- stepping ------------------------------------------------------------------------------------------
    def step(self, n=1):
        _check(lib().lbm_step(self.h, int(n)))

    def step_timed(self, n=1):
        """Returns [interior-kernel ms, boundary-kernel ms, first-to-last ms] over the n steps."""
        ms = np.zeros(3)
        _check(lib().lbm_step_timed(self.h, int(n), ms.ctypes.data_as(_p)))
        return ms

    def sync(self):
        _check(lib().lbm_sync(self.h))

    # ---- state access ----------------------------------------------------------------------------------------
    def moments(self, dtype=np.float64, rho=None, u=None):
        code = DTYPE_F64 if dtype == np.float64 else DTYPE_F32
        if rho is None:
            rho = np.zeros(self.N, dtype)
            u = np.zeros((3, self.N), dtype)
            _check(lib().lbm_moments_ex(self.h, rho.ctypes.data_as(_p), u.ctypes.data_as(_p), code))
            return rho, u
        _check(lib().lbm_moments_ex(self.h, ctypes.c_void_p(rho.data_ptr()), ctypes.c_void_p(u.data_ptr()), code))
        return rho, u

    def reduce(self):
        m = np.zeros(1)
        p = np.zeros(3)
        _check(lib().lbm_reduce(self.h, m.ctypes.data_as(_p), p.ctypes.data_as(_p)))
        return m[0], p

    def get_populations(self, dtype=np.float64):
        f = np.zeros((self.q, self.N), dtype)
        _check(lib().lbm_get_populations(self.h, f.ctypes.data_as(_p), DTYPE_F64 if dtype == np.float64 else DTYPE_F32))
        return f

    def set_populations(self, f):
        a = _Arr(f)
        _check(lib().lbm_set_populations(self.h, a.ptr, a.code))

    def set_option(self, option, value):
        _check(lib().lbm_set_option(self.h, int(option), int(value)))

    def info(self):
        out = np.zeros(10, np.int64)
        _check(lib().lbm_info(self.h, out.ctypes.data_as(_p)))
        keys = ["N", "n_list", "n_wall", "n_ref", "n_inflow", "n_outflow", "n_solid", "t", "storage", "q"]
        return dict(zip(keys, (int(v) for v in out)))

    def launch_count(self):
        """Kernels launched by the step calls of this lattice so far."""
        n = np.zeros(1, np.int64)
        _check(lib().lbm_launch_count(self.h, n.ctypes.data_as(_p)))
        return int(n[0])

    def debug_dump(self, which):
        info = self.info()
        if which >= 6:
            count = self.halo_count((which - 6) // 4, (which - 6) % 4)
        else:
            count = {0: self.N, 1: info["n_list"], 2: info["n_list"], 3: 3 * info["n_list"],
                     4: self.q * self.N, 5: self.q * self.N}[which]
        out = np.zeros(max(count, 1), np.int64)
        _check(lib().lbm_debug_dump(self.h, int(which), out.ctypes.data_as(_p), ctypes.c_size_t(out.size)))
        return out[:count]

    def save(self):
        n = ctypes.c_size_t(0)
        _check(lib().lbm_save(self.h, None, ctypes.byref(n)))
        buf = np.zeros(n.value, np.uint8)
        _check(lib().lbm_save(self.h, buf.ctypes.data_as(_p), ctypes.byref(n)))
        return buf

    def load(self, buf):
        b = np.ascontiguousarray(buf, dtype=np.uint8)
        _check(lib().lbm_load(self.h, b.ctypes.data_as(_p), ctypes.c_size_t(b.size)))

    # ---- differentiation -------------------------------------------------------------------------------------
    def objective_forward(self, T, W, xa, xb, ckpt=32):
        J = np.zeros(1)
        _check(lib().lbm_objective_forward(self.h, int(T), int(W), int(xa), int(xb), int(ckpt), J.ctypes.data_as(_p)))
        return J[0]

    def objective_backward(self, dgamma=None, duin=None):
        """dJ/dgamma (N) and dJ/du_in (3, ny*nz) in FP64. Without arguments they come back as host
        arrays; given FP64 torch tensors (device or host) of those sizes, the library writes them."""
        if dgamma is None and duin is None:
            g = np.zeros(self.N)
            u = np.zeros(3 * self.ny * self.nz)
            _check(lib().lbm_objective_backward(self.h, g.ctypes.data_as(_p), u.ctypes.data_as(_p)))
            return g, u.reshape(3, self.ny * self.nz)
        for t, n in ((dgamma, self.N), (duin, 3 * self.ny * self.nz)):
            if t is not None and (str(t.dtype) != "torch.float64" or t.numel() != n or not t.is_contiguous()):
                raise ValueError("gradient outputs must be contiguous float64 tensors of N and 3*ny*nz values")
        gp = None if dgamma is None else ctypes.c_void_p(dgamma.data_ptr())
        up = None if duin is None else ctypes.c_void_p(duin.data_ptr())
        _check(lib().lbm_objective_backward(self.h, gp, up))
        return dgamma, duin

    def adjoint_step(self, lam_in):
        a = _Arr(lam_in, dtype=np.float64)
        out = np.zeros((self.q, self.N))
        g = np.zeros(self.N)
        u = np.zeros(3 * self.ny * self.nz)
        _check(lib().lbm_adjoint_step(self.h, a.ptr, out.ctypes.data_as(_p), DTYPE_F64, g.ctypes.data_as(_p),
                                      u.ctypes.data_as(_p)))
        return out, g, u.reshape(3, self.ny * self.nz)

    def adjoint_timing(self):
        """[recompute ms, reverse ms, forward ms] of the last objective forward/backward."""
        ms = np.zeros(3)
        _check(lib().lbm_adjoint_timing(self.h, ms.ctypes.data_as(_p)))
        return ms

    # ---- convenience ---------------------------------------------------------------------------------------------
    @classmethod
    def from_workload(cls, w, storage=F32, init=True, ghost=(0, 0)):
        """Lattice configured from a seeded `inputs.Workload` (faces, geometry, force, inlet,
        outlet, porosity, wall model, initial equilibrium); ghost = (lo, hi) ghost z-planes of a slab
        sub-domain (inputs.slab)."""
        lat = cls(w.q, w.nx, w.ny, w.nz, w.tau, w.cs, storage=storage)
        lat.set_faces(w.faces)
        if ghost != (0, 0):
            lat.set_ghost_planes(*ghost)
        lat.set_geometry(w.mask, None if w.ywall is None else np.asarray(w.ywall, np.float32))
        lat.set_force(*w.force)
        if w.uin is not None:
            lat.set_inflow(np.asarray(w.uin, np.float64 if storage == F64 else np.float32))
        lat.set_outflow(w.rho_out)
        if w.gamma is not None:
            lat.set_porosity(np.asarray(w.gamma, np.float64 if storage == F64 else np.float32))
        if w.wall_model:
            lat.set_wall_model(w.kappa, w.E)
        if getattr(w, "model", 0):
            lat.set_collision(w.model, w.sigma)
        if getattr(w, "vortex", None):
            lat.set_vortex_inlet(*w.vortex)
        if getattr(w, "fringe", None):
            fr = w.fringe
            if len(fr) > 3 and fr[3] != w.nx - fr[0]:
                raise ValueError("the library's fringe layer ends at the outlet plane (a crop of it is oracle-only)")
            lat.set_fringe(*fr[:3])
        if init:
            dt = np.float64 if storage == F64 else np.float32
            lat.init_equilibrium(np.asarray(w.rho0, dt), np.asarray(w.u0, dt))
        return lat
