"""PyTorch autograd wrapper of the checkpointed objective (forward = T steps of the lattice with the
time-averaged pressure-drop objective, backward = the discrete adjoint): porosity gamma and inlet
velocity u_in are the differentiable inputs. All arithmetic of the method runs in the CUDA library
through its C ABI (`lbm_set_porosity_ex`, `lbm_set_inflow_ex`, `lbm_objective_forward`,
`lbm_objective_backward`); tensors are handed over by pointer where they live (CUDA tensors stay on
the device), and the gradients come back as FP64 tensors on the inputs' device. The only torch
arithmetic is the chain rule's product with the incoming gradient.
"""
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
        lattice.set_porosity(gamma.detach().contiguous())
        lattice.set_inflow(u_in.detach().reshape(3, -1).contiguous())
        lattice.init_equilibrium(rho0, u0)
        J = lattice.objective_forward(int(T), int(W), int(xa), int(xb), ckpt=int(ckpt))
        ctx.lattice = lattice
        ctx.like = (gamma, u_in)
        return torch.tensor(J, dtype=gamma.dtype, device=gamma.device)

    @staticmethod
    def backward(ctx, gJ):
        gamma, u_in = ctx.like
        lat = ctx.lattice
        g = torch.empty(lat.N, dtype=torch.float64, device=gamma.device)
        gu = torch.empty((3, lat.ny * lat.nz), dtype=torch.float64, device=u_in.device)
        lat.objective_backward(g, gu)
        s = gJ.detach().to(torch.float64)
        dg = (g * s.to(g.device)).to(gamma.dtype)
        du = (gu * s.to(gu.device)).to(u_in.dtype).reshape(u_in.shape)
        return dg, du, None, None, None, None, None, None, None, None


def pressure_drop(gamma, u_in, lattice, rho0, u0, T, W, xa, xb, ckpt=32):
    """Differentiable J(gamma, u_in); see PressureDropObjective."""
    return PressureDropObjective.apply(gamma, u_in, lattice, rho0, u0, T, W, xa, xb, ckpt)
