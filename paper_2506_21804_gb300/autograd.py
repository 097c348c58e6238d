"""PyTorch autograd wrapper of the checkpointed objective (forward = T steps of the lattice with the
time-averaged pressure-drop objective, backward = the discrete adjoint): porosity gamma and inlet
velocity u_in are the differentiable inputs. All arithmetic runs in the CUDA library through its C
ABI (`lbm_objective_forward`, `lbm_objective_backward`); this module only moves arrays.
"""
import numpy as np
import torch

from . import lbm


class PressureDropObjective(torch.autograd.Function):
    """J(gamma, u_in) = (1/W) sum over the last W of T steps of cs^2 (<rho>_{x=xa} - <rho>_{x=xb}),
    plane means over non-solid cells, starting from the equilibrium state (rho0, u0).

    forward(gamma (N,), u_in (3, ny*nz), lattice, rho0, u0, T, W, xa, xb, ckpt) -> J (0-d tensor)
    backward -> dJ/dgamma, dJ/du_in (scaled by the incoming gradient)
    """

    @staticmethod
    def forward(ctx, gamma, u_in, lattice, rho0, u0, T, W, xa, xb, ckpt=32):
        dt = np.float64 if lattice.storage == lbm.F64 else np.float32
        lattice.set_porosity(gamma.detach().to("cpu", torch.float64).numpy().astype(dt))
        lattice.set_inflow(u_in.detach().to("cpu", torch.float64).numpy().astype(dt))
        lattice.init_equilibrium(np.asarray(rho0, dt), np.asarray(u0, dt))
        J = lattice.objective_forward(int(T), int(W), int(xa), int(xb), ckpt=int(ckpt))
        ctx.lattice = lattice
        ctx.like = (gamma, u_in)
        return torch.tensor(J, dtype=gamma.dtype, device=gamma.device)

    @staticmethod
    def backward(ctx, gJ):
        g, gu = ctx.lattice.objective_backward()
        gamma, u_in = ctx.like
        s = gJ.detach().to("cpu", torch.float64).item()
        dg = torch.from_numpy(g * s).to(gamma.device, gamma.dtype)
        du = torch.from_numpy(gu * s).to(u_in.device, u_in.dtype).reshape(u_in.shape)
        return dg, du, None, None, None, None, None, None, None, None


def pressure_drop(gamma, u_in, lattice, rho0, u0, T, W, xa, xb, ckpt=32):
    """Differentiable J(gamma, u_in); see PressureDropObjective."""
    return PressureDropObjective.apply(gamma, u_in, lattice, rho0, u0, T, W, xa, xb, ckpt)
